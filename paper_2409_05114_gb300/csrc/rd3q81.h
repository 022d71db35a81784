// RD3Q81 velocity set and the constants derived from it.
//
// Paper: Atif et al., "Lattice Boltzmann Model for Transonic Flows" (arXiv 2409.05114),
// Sec. III and Table "tab:weights": ten energy shells (SC-1..4, FCC-1,2, BCC-1/2, 1, 3/2,
// 5/2) plus the rest particle, 81 velocities in all; each shell weight is a quintic
// polynomial in theta0, and w_0 = 1 - sum of the other weights.
//
// Velocities are stored in half units h = 2c so that every component is an integer.
// Directions come in +/- pairs: for i >= 1, direction i+1 (i odd) is -c_i.
// This header is used by the device kernels (compile-time direction data) and by the host
// code that fills the constant-memory tables.
#pragma once

#ifdef __CUDACC__
#define RD3Q81_HD __host__ __device__
#else
#define RD3Q81_HD
#endif

namespace rd3q81 {

constexpr int kQ = 81;       // number of velocities
constexpr int kShells = 11;  // shell 0 = rest, 1..10 as in Table "tab:weights"
constexpr int kPairs = 40;   // (kQ - 1) / 2
constexpr int kReach = 4;    // largest |index displacement| of a pull (SC-4)

// theta0 as printed below Table "tab:weights".
constexpr double kTheta0 = 0.821035006329447750282591763;

struct Dir {
  int hx, hy, hz;  // 2 c_i
  int shell;       // 0 .. 10
};

// The library's direction order (rest first, then each shell as +v, -v pairs).
constexpr Dir kDirs[kQ] = {
    {0, 0, 0, 0},   //  0 rest
    { 2,  0,  0,  1},  //  1 SC-1
    {-2,  0,  0,  1},  //  2 SC-1
    { 0,  2,  0,  1},  //  3 SC-1
    { 0, -2,  0,  1},  //  4 SC-1
    { 0,  0,  2,  1},  //  5 SC-1
    { 0,  0, -2,  1},  //  6 SC-1
    { 4,  0,  0,  2},  //  7 SC-2
    {-4,  0,  0,  2},  //  8 SC-2
    { 0,  4,  0,  2},  //  9 SC-2
    { 0, -4,  0,  2},  // 10 SC-2
    { 0,  0,  4,  2},  // 11 SC-2
    { 0,  0, -4,  2},  // 12 SC-2
    { 6,  0,  0,  3},  // 13 SC-3
    {-6,  0,  0,  3},  // 14 SC-3
    { 0,  6,  0,  3},  // 15 SC-3
    { 0, -6,  0,  3},  // 16 SC-3
    { 0,  0,  6,  3},  // 17 SC-3
    { 0,  0, -6,  3},  // 18 SC-3
    { 8,  0,  0,  4},  // 19 SC-4
    {-8,  0,  0,  4},  // 20 SC-4
    { 0,  8,  0,  4},  // 21 SC-4
    { 0, -8,  0,  4},  // 22 SC-4
    { 0,  0,  8,  4},  // 23 SC-4
    { 0,  0, -8,  4},  // 24 SC-4
    { 2,  2,  0,  5},  // 25 FCC-1
    {-2, -2,  0,  5},  // 26 FCC-1
    { 2, -2,  0,  5},  // 27 FCC-1
    {-2,  2,  0,  5},  // 28 FCC-1
    { 2,  0,  2,  5},  // 29 FCC-1
    {-2,  0, -2,  5},  // 30 FCC-1
    { 2,  0, -2,  5},  // 31 FCC-1
    {-2,  0,  2,  5},  // 32 FCC-1
    { 0,  2,  2,  5},  // 33 FCC-1
    { 0, -2, -2,  5},  // 34 FCC-1
    { 0,  2, -2,  5},  // 35 FCC-1
    { 0, -2,  2,  5},  // 36 FCC-1
    { 4,  4,  0,  6},  // 37 FCC-2
    {-4, -4,  0,  6},  // 38 FCC-2
    { 4, -4,  0,  6},  // 39 FCC-2
    {-4,  4,  0,  6},  // 40 FCC-2
    { 4,  0,  4,  6},  // 41 FCC-2
    {-4,  0, -4,  6},  // 42 FCC-2
    { 4,  0, -4,  6},  // 43 FCC-2
    {-4,  0,  4,  6},  // 44 FCC-2
    { 0,  4,  4,  6},  // 45 FCC-2
    { 0, -4, -4,  6},  // 46 FCC-2
    { 0,  4, -4,  6},  // 47 FCC-2
    { 0, -4,  4,  6},  // 48 FCC-2
    { 1,  1,  1,  7},  // 49 BCC-1/2
    {-1, -1, -1,  7},  // 50 BCC-1/2
    { 1,  1, -1,  7},  // 51 BCC-1/2
    {-1, -1,  1,  7},  // 52 BCC-1/2
    { 1, -1,  1,  7},  // 53 BCC-1/2
    {-1,  1, -1,  7},  // 54 BCC-1/2
    {-1,  1,  1,  7},  // 55 BCC-1/2
    { 1, -1, -1,  7},  // 56 BCC-1/2
    { 2,  2,  2,  8},  // 57 BCC-1
    {-2, -2, -2,  8},  // 58 BCC-1
    { 2,  2, -2,  8},  // 59 BCC-1
    {-2, -2,  2,  8},  // 60 BCC-1
    { 2, -2,  2,  8},  // 61 BCC-1
    {-2,  2, -2,  8},  // 62 BCC-1
    {-2,  2,  2,  8},  // 63 BCC-1
    { 2, -2, -2,  8},  // 64 BCC-1
    { 3,  3,  3,  9},  // 65 BCC-3/2
    {-3, -3, -3,  9},  // 66 BCC-3/2
    { 3,  3, -3,  9},  // 67 BCC-3/2
    {-3, -3,  3,  9},  // 68 BCC-3/2
    { 3, -3,  3,  9},  // 69 BCC-3/2
    {-3,  3, -3,  9},  // 70 BCC-3/2
    {-3,  3,  3,  9},  // 71 BCC-3/2
    { 3, -3, -3,  9},  // 72 BCC-3/2
    { 5,  5,  5, 10},  // 73 BCC-5/2
    {-5, -5, -5, 10},  // 74 BCC-5/2
    { 5,  5, -5, 10},  // 75 BCC-5/2
    {-5, -5,  5, 10},  // 76 BCC-5/2
    { 5, -5,  5, 10},  // 77 BCC-5/2
    {-5,  5, -5, 10},  // 78 BCC-5/2
    {-5,  5,  5, 10},  // 79 BCC-5/2
    { 5, -5, -5, 10},  // 80 BCC-5/2
};

// |c|^2 of each shell: SC-k: k^2, FCC-1: 2, FCC-2: 8, BCC-b: 3 b^2 (b = 1/2, 1, 3/2, 5/2).
constexpr double kShellC2[kShells] = {0.0, 1.0, 4.0, 9.0, 16.0, 2.0, 8.0, 0.75, 3.0, 6.75, 18.75};
constexpr int kShellCount[kShells] = {1, 6, 6, 6, 6, 12, 12, 8, 8, 8, 8};

// Table "tab:weights": w_shell = (sum_{k=1..5} num[k] * theta0^k) / den, shells 1..10.
struct WeightPoly {
  double num[6];  // index = power of theta0 (index 0 unused, always 0)
  double den;
};
constexpr WeightPoly kWeightPoly[kShells] = {
    {{0, 0, 0, 0, 0, 0}, 1},                                                   // rest: 1 - sum
    {{0, 388800, -2508408, 7033852, -7856469, 2838528}, 486000},               // SC-1
    {{0, -388800, 3091608, -8269102, 8694819, -2838528}, 3888000},             // SC-2
    {{0, 388800, -3199608, 8977852, -9120069, 2838528}, 30618000},             // SC-3
    {{0, -97200, 809352, -2315338, 2396961, -709632}, 108864000},              // SC-4
    {{0, 0, 0, 8, -9, 0}, 12},                                                 // FCC-1
    {{0, 0, 0, -2, 9, 0}, 768},                                                // FCC-2
    {{0, 0, 24300, -103834, 126963, -44352}, 7776},                            // BCC-1/2
    {{0, 0, -24300, 189022, -328275, 177408}, 272160},                         // BCC-1
    {{0, 0, 2700, -24778, 67995, -44352}, 699840},                             // BCC-3/2
    {{0, 0, -972, 11818, -43371, 44352}, 68040000},                            // BCC-5/2
};

// Index displacement d of a pull (the population arriving at target index n left
// index n - d one step earlier) and whether it comes from the other sublattice.
// Primary sites P sit at integer positions n, replica sites R at n + (1/2, 1/2, 1/2).
// Integer links (h even) stay on the sublattice: d = h/2.  Half links (h odd) cross it:
// into P from R at n - (h+1)/2, into R from P at n - (h-1)/2.
RD3Q81_HD constexpr int pull_disp(int h, int target_sub) {
  return (h % 2 == 0) ? h / 2 : (target_sub == 0 ? (h + 1) / 2 : (h - 1) / 2);
}
RD3Q81_HD constexpr bool crosses_sublattice(const Dir& d) { return (d.hx % 2) != 0; }

// Shape of a moving shell (s = 1..10): every member has |h_a| in {0, k} for each axis a, and
// `kind` components are nonzero (1: SC, 2: FCC, 3: BCC), with all sign choices and axis
// permutations present.  Sums of exp(zeta.c) over a shell therefore factor into per-axis
// cosh / sinh of zeta_a k / 2.
struct ShellShape {
  int kind, k;
};
RD3Q81_HD constexpr int iabs(int a) { return a < 0 ? -a : a; }
RD3Q81_HD constexpr ShellShape shell_shape(int s) {
  for (int i = 1; i < kQ; ++i)
    if (kDirs[i].shell == s) {
      const int ax = iabs(kDirs[i].hx), ay = iabs(kDirs[i].hy), az = iabs(kDirs[i].hz);
      const int k = ax > ay ? (ax > az ? ax : az) : (ay > az ? ay : az);
      return {(ax != 0) + (ay != 0) + (az != 0), k};
    }
  return {0, 0};
}
constexpr int kMaxShellK = 8;  // SC-4
RD3Q81_HD constexpr bool shells_are_uniform() {
  for (int i = 1; i < kQ; ++i) {
    const ShellShape sh = shell_shape(kDirs[i].shell);
    const int h[3] = {kDirs[i].hx, kDirs[i].hy, kDirs[i].hz};
    int nz = 0;
    for (int a = 0; a < 3; ++a) {
      if (h[a] != 0 && iabs(h[a]) != sh.k) return false;
      nz += h[a] != 0;
    }
    if (nz != sh.kind || sh.k > kMaxShellK || kShellCount[kDirs[i].shell] != (sh.kind == 2 ? 12 : sh.kind == 1 ? 6 : 8))
      return false;
  }
  return true;
}
static_assert(shells_are_uniform(), "shell shapes");

}  // namespace rd3q81
