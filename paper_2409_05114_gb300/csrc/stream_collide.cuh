// Fused pull-stream + collide step of the RD3Q81 model (one thread per lattice site).
//
// Paper: Sec. II, Eq. (discretelbm)  f_i(x + c_i, t + 1) = f_i + alpha beta (f~eq_i - f_i),
// alpha = 2, beta = 1 / (2 tau + 1); moments by Eq. (conslaws); f~eq by App. B (series
// temperature weights W~ to eta^4, f^(2), f^(3), R-bar).  The physical lattice is the
// primary + replica (body-centred cubic) lattice: half-integer links (BCC-1/2, 3/2, 5/2)
// join the two sublattices (Sec. I, replica grid).
//
// Per site: 81 pulled loads (structure-of-arrays, consecutive threads read consecutive x),
// the moment sums, theta, the per-shell W~ polynomials and the per-site equilibrium
// scalars, then for each +/- velocity pair the even/odd parts of f~eq, the BGK update and
// 81 coalesced stores into the other buffer (ping-pong).  The update is a per-site
// nonlinear map of 81 values read once and written once: HBM-bound, no tensor-core work.
#pragma once

#include <cfloat>

#include "device_common.cuh"

namespace lbm {

constexpr int kScBlock = 128;

template <class R>
__device__ __forceinline__ const R* tab_wp(const LatticeTables& t, int s) {
  if constexpr (std::is_same_v<R, double>) return t.wp[s]; else return t.wpf[s];
}
template <class R>
__device__ __forceinline__ const R* tab_p(const LatticeTables& t, int s) {
  if constexpr (std::is_same_v<R, double>) return t.p[s]; else return t.pf[s];
}
template <class R>
__device__ __forceinline__ R tab_w(const LatticeTables& t, int s) {
  if constexpr (std::is_same_v<R, double>) return t.w[s]; else return t.wf[s];
}
template <class R>
__device__ __forceinline__ const R* tab_na(const LatticeTables& t) {
  if constexpr (std::is_same_v<R, double>) return t.na; else return t.naf;
}
template <class R>
__device__ __forceinline__ const R* tab_nb(const LatticeTables& t) {
  if constexpr (std::is_same_v<R, double>) return t.nb; else return t.nbf;
}

// Source coordinates of site t for index displacements d = -4 .. 4 (slot d + 4): x as an
// element index within a row, y and z as element offsets of the row and plane.
__device__ __forceinline__ void site_coords(const Geometry& g, int t, int* xs, int* ys, int* zs) {
  const int x = t % g.nx;
  const int r = t / g.nx;
  const int y = r % g.ny;
  const int z = r / g.ny;
#pragma unroll
  for (int k = 0; k < 9; ++k) {
    const int d = k - 4;
    xs[k] = (g.x_periodic ? wrap_idx(x - d, g.nx) : x - d) + g.xoff;
    ys[k] = wrap_idx(y - d, g.ny) * g.pitch;
    zs[k] = wrap_idx(z - d, g.nz) * static_cast<int>(g.plane);
  }
}

// Calls fn(i, pointer) with the source element of direction i pulled into a site of
// sublattice SUB whose coordinates are xs/ys/zs.
template <class Store, int SUB, class Fn>
__device__ __forceinline__ void for_each_source(const Geometry& g, const Store* src, const int* xs, const int* ys,
                                                const int* zs, Fn&& fn) {
  const Store* same = src + SUB * g.sub_stride;
  const Store* other = src + (1 - SUB) * g.sub_stride;
  static_for<kQ>([&](auto Ic) {
    constexpr int i = decltype(Ic)::value;
    constexpr rd3q81::Dir d = rd3q81::kDirs[i];
    constexpr int dx = rd3q81::pull_disp(d.hx, SUB);
    constexpr int dy = rd3q81::pull_disp(d.hy, SUB);
    constexpr int dz = rd3q81::pull_disp(d.hz, SUB);
    constexpr bool cross = (d.hx % 2) != 0;
    const Store* base = (cross ? other : same) + static_cast<long long>(i) * g.dir_stride;
    fn(Ic, base + (zs[dz + 4] + ys[dy + 4] + xs[dx + 4]));
  });
}

// Conserved moments of Eq. (conslaws) in arithmetic M.
template <class M>
struct Moments {
  using value_type = M;
  M rho, jx, jy, jz, E;
};

// Offset storage holds d_i = f_i/w_i - 1, so rho = 1 + <w, d>, j = <w, d c>,
// <f, c^2> = 3 theta0 + <w, d c^2> (the weights' own moments are 1, 0, 3 theta0).
// FP32 sums of FP32 populations are also taken over the deviations f_i - w_i: the same
// moments, summed from numbers ~10x smaller than f_i, hence ~10x smaller rounding.
// FP32 storage with FP64-quality moments: exact integer sums.  With h_i = 2 c_i (integers) the
// moments are rho = <f, 1>, j_a = <f, h_a> / 2 and <f, c^2> = <f, h^2> / 4.  Every population is
// scaled by 2^K (exact) and rounded to a 64-bit integer, an error below 2^-(K+1) in f; the
// integer sums are then exact (the conversion is below).  K is the largest exponent with B 2^K < 2^61, B = sum_i |f_i|
// (1 + h_i^2) (taken in FP32 with a margin), so that no partial sum of the rho, h_a or h^2
// weighted integers can leave (-2^62, 2^62).  The roundings add at most 81 2^-(K+1) < 2^-54 B to
// rho and sum_i h_i^2 2^-(K+1) < 2^-49 B to <f, h^2> -- with B about 6 rho near theta0, the
// FP64 level (K is capped at 120, which costs relative precision only below B ~ 2^-59).  Each
// shell's populations (pair sums and differences) are added first and weighted by the shell's
// h^2 and |h_a| once.  The sums return as double words (the rounded integer and its
// remainder, each converted once), scaled back exactly.  A non-finite population makes the
// moments NaN, which the caller flags.
__device__ __forceinline__ Dw fixed_to_dw(long long m, float scale) {
  const float hi = __ll2float_rn(m);
  const float lo = __ll2float_rn(m - __float2ll_rn(hi));
  return Dw{hi * scale, lo * scale};
}

__device__ __forceinline__ Moments<Dw> site_moments_dw(const float* f) {
  float B = fabsf(f[0]);
  static_for<kPairs>([&](auto Pc) {
    constexpr int P = decltype(Pc)::value;
    constexpr float g = 1.0f + static_cast<float>(4.0 * rd3q81::kShellC2[rd3q81::kDirs[1 + 2 * P].shell]);
    B = fmaf(fabsf(f[1 + 2 * P]) + fabsf(f[2 + 2 * P]), g, B);
  });
  // 2^e > B (1 + 2^-10) covers the FP32 rounding of B (below 2^-17 relative)
  const int e = ((__float_as_int(B * 1.0009765625f) >> 23) & 0xff) - 126;
  const int K = min(61 - e, 120);
  const float sc = __int_as_float((K + 127) << 23);
  // two's-complement sums in unsigned arithmetic (wrapping defined even for a non-finite input)
  using U = unsigned long long;
  // rint(t) as a 64-bit integer from two 32-bit conversions: t = a 2^31 + b with a = rint(t 2^-31) and
  // b = t - a 2^31, both exact floats with |a|, |b| <= 2^30 (b has at most 24 significant bits), and
  // rint(t) = a 2^31 + rint(b).  The 64-bit conversion instructions run on this GPU's FP64 pipe: with
  // them the kernel ran at 5475 MLUPS (TGV 512^3, FP64 pipe 77 % busy), with this form at 6920-6956.
  auto to_fixed = [](float t) {
    const float af = rintf(t * 0x1p-31f);
    const float bf = __fmaf_rn(-af, 0x1p31f, t);
    return (static_cast<U>(static_cast<long long>(__float2int_rn(af))) << 31) +
           static_cast<U>(static_cast<long long>(__float2int_rn(bf)));
  };
  U rho = to_fixed(f[0] * sc), e2 = 0, jx = 0, jy = 0, jz = 0;
  U S = 0, X = 0, Y = 0, Z = 0;
  static_for<kPairs>([&](auto Pc) {
    constexpr int P = decltype(Pc)::value;
    constexpr rd3q81::Dir d = rd3q81::kDirs[1 + 2 * P];
    constexpr int s = d.shell;
    constexpr bool first = P == 0 || rd3q81::kDirs[2 * P - 1].shell != s;
    constexpr bool last = P == kPairs - 1 || rd3q81::kDirs[3 + 2 * P].shell != s;
    const U ip = to_fixed(f[1 + 2 * P] * sc), im = to_fixed(f[2 + 2 * P] * sc);
    const U sum = ip + im, dif = ip - im;
    if constexpr (first) S = X = Y = Z = 0;
    S += sum;
    if constexpr (d.hx != 0) X = d.hx > 0 ? X + dif : X - dif;
    if constexpr (d.hy != 0) Y = d.hy > 0 ? Y + dif : Y - dif;
    if constexpr (d.hz != 0) Z = d.hz > 0 ? Z + dif : Z - dif;
    // (empty) ordering point: without it the compiler converts all 81 populations up front and
    // holds 162 registers of integers
    asm volatile("" : "+l"(S), "+l"(X), "+l"(Y), "+l"(Z));
    if constexpr (last) {
      constexpr U h2 = static_cast<U>(4.0 * rd3q81::kShellC2[s] + 0.5);
      constexpr U k = static_cast<U>(rd3q81::shell_shape(s).k);
      rho += S;
      e2 += h2 * S;
      jx += k * X;
      jy += k * Y;
      jz += k * Z;
    }
  });
  const bool ok = B <= FLT_MAX;
  const float s0 = ok ? __int_as_float((127 - K) << 23) : __int_as_float(0x7fc00000);
  const float s1 = 0.5f * s0, s2 = 0.25f * s0;
  auto dw = [](U m, float scale) { return fixed_to_dw(static_cast<long long>(m), scale); };
  return Moments<Dw>{dw(rho, s0), dw(jx, s1), dw(jy, s1), dw(jz, s1), dw(e2, s2)};
}

// Offset storage with FP64-quality moments: rho = 1 + sum_s w_s S_s, <f, c^2> = 3 theta0 + sum_s
// w_s c_s^2 S_s and j_a = sum_s (w_s k_s / 2) J_a,s, where S_s sums the offsets of shell s and
// J_a,s their signed sum over the members with h_a != 0 (every such component is +-k_s / 2).
// The shell sums are cascaded (Sum2: each TwoSum's error collects in a second float), multiplied
// by the shell's weights held as double words, and the products accumulated the same way: the
// double-word scheme of site_moments_dw with the weights' rounding removed too.
__device__ __forceinline__ Moments<Dw> site_moments_dw_offset(const float* d, const LatticeTables& tb) {
  auto acc = [](float& p, float& q, Dw v) {  // p + q += v
    const Dw t = two_sum(p, v.hi);
    p = t.hi;
    q = __fadd_rn(q, __fadd_rn(t.lo, v.lo));
  };
  auto wmul = [](Dw a, const float* w) { return dw_mul(a, Dw{w[0], w[1]}); };
  float pr = 0.0f, qr = 0.0f, pe = 0.0f, qe = 0.0f, px = 0.0f, qx = 0.0f, py = 0.0f, qy = 0.0f, pz = 0.0f, qz = 0.0f;
  acc(pr, qr, wmul(Dw{d[0], 0.0f}, tb.w_dw[0]));
  float sp = 0.0f, sq = 0.0f, xp = 0.0f, xq = 0.0f, yp = 0.0f, yq = 0.0f, zp = 0.0f, zq = 0.0f;
  static_for<kPairs>([&](auto Pc) {
    constexpr int P = decltype(Pc)::value;
    constexpr rd3q81::Dir dd = rd3q81::kDirs[1 + 2 * P];
    constexpr int s = dd.shell;
    constexpr bool last = P == kPairs - 1 || rd3q81::kDirs[3 + 2 * P].shell != s;
    const float fp = d[1 + 2 * P], fm = d[2 + 2 * P];
    const Dw sum = two_sum(fp, fm), dif = two_sum(fp, -fm);
    const Dw ndif{-dif.hi, -dif.lo};
    acc(sp, sq, sum);
    if constexpr (dd.hx != 0) acc(xp, xq, dd.hx > 0 ? dif : ndif);
    if constexpr (dd.hy != 0) acc(yp, yq, dd.hy > 0 ? dif : ndif);
    if constexpr (dd.hz != 0) acc(zp, zq, dd.hz > 0 ? dif : ndif);
    if constexpr (last) {
      const Dw S = two_sum(sp, sq);
      acc(pr, qr, wmul(S, tb.w_dw[s]));
      acc(pe, qe, wmul(S, tb.wc2_dw[s]));
      acc(px, qx, wmul(two_sum(xp, xq), tb.whk_dw[s]));
      acc(py, qy, wmul(two_sum(yp, yq), tb.whk_dw[s]));
      acc(pz, qz, wmul(two_sum(zp, zq), tb.whk_dw[s]));
      sp = sq = xp = xq = yp = yq = zp = zq = 0.0f;
    }
  });
  return Moments<Dw>{dw_add(two_sum(pr, qr), 1.0f), two_sum(px, qx), two_sum(py, qy), two_sum(pz, qz),
                     dw_add(two_sum(pe, qe), Dw{tb.theta0x3_dw[0], tb.theta0x3_dw[1]})};
}

template <class Store, bool kF64Mom>
__device__ __forceinline__ auto site_moments(const typename Codec<Store>::Real* f, const LatticeTables& tb) {
  if constexpr (kF64Mom && std::is_same_v<Store, float>) {
    return site_moments_dw(f);
  } else if constexpr (kF64Mom && Codec<Store>::kOffset) {
    return site_moments_dw_offset(f, tb);
  } else {
  using C = Codec<Store>;
  using R = typename C::Real;
  using M = std::conditional_t<kF64Mom, double, R>;
  constexpr bool kDev = C::kOffset || std::is_same_v<M, float>;
  M rho, jx = M(0), jy = M(0), jz = M(0), E = M(0);
  if constexpr (C::kOffset) rho = tab_w<M>(tb, 0) * M(f[0]);
  else if constexpr (kDev) rho = M(f[0]) - tab_w<M>(tb, 0);
  else rho = M(f[0]);
  static_for<kPairs>([&](auto Pc) {
    constexpr int P = decltype(Pc)::value;
    constexpr rd3q81::Dir d = rd3q81::kDirs[1 + 2 * P];
    constexpr double c2 = rd3q81::kShellC2[d.shell];
    const M fp = M(f[1 + 2 * P]);
    const M fm = M(f[2 + 2 * P]);
    M sum = fp + fm;
    M dif = fp - fm;
    if constexpr (C::kOffset) {
      const M ws = tab_w<M>(tb, d.shell);
      sum *= ws;
      dif *= ws;
    } else if constexpr (kDev) {
      sum -= M(2) * tab_w<M>(tb, d.shell);
    }
    rho += sum;
    E += M(c2) * sum;
    if constexpr (d.hx != 0) jx += M(0.5 * d.hx) * dif;
    if constexpr (d.hy != 0) jy += M(0.5 * d.hy) * dif;
    if constexpr (d.hz != 0) jz += M(0.5 * d.hz) * dif;
  });
  if constexpr (kDev) {
    rho += M(1);
    E += M(3.0 * rd3q81::kTheta0);
  }
  return Moments<M>{rho, jx, jy, jz, E};
  }
}

// ---- entropic alpha (Eq. (delH)) -------------------------------------------------------
// alpha is the nontrivial root of Delta H(alpha) = H[f + alpha D] - H[f], D = feq - f, with feq
// the exact entropic equilibrium of f's conserved moments.  Because log(feq / w) is affine in
// (1, c, c^2) and D carries no mass, momentum or energy, <D, log(f/w)> = -<f, x log(1 + x)>
// with x = D / f, so
//   Delta H(alpha) = <f, (1 + alpha x) log(1 + alpha x) - alpha x> - alpha <f, x log(1 + x)>,
// a sum of terms of order f x^2 without the cancellation between O(1) values of the plain
// definition.  Delta H is convex in alpha, zero at 0 and negative at 1.
// * Every |x_i| <= kX: both brackets expanded in x,
//     Delta H(alpha) / alpha = sum_{n=2..N} (-1)^n a_n [alpha^(n-1) / (n (n-1)) - 1 / (n-1)],
//   a_n = <f, x^n>, solved by three Newton steps from alpha = 2 (its limit as x -> 0).  The
//   first dropped term moves the root by about 2^(N+1) x^(N-1) / (N (N+1)), which moves the
//   update by that times beta x: below 1e-7 relative for FP32 (N = 6, |x| <= 0.05) and 1e-15
//   for FP64 (N = 8, |x| <= 0.01).
// * Otherwise the full expression.  alpha_max = min over x_i < 0 of -1 / x_i is where a
//   population would reach zero; if Delta H(alpha_max) <= 0 there is no root before it and
//   alpha = alpha_max (on coarse grids with omega near 2 this is the common case, set by a
//   tiny outer-shell population).  Else Newton from min(2, 1 + 0.9 (alpha_max - 1)),
//   safeguarded by bisection on [1, alpha_max]; it stops once a Newton step or the bracket is
//   below the tolerance (near equilibrium the rounding of Delta H decides which comes first).
// * A population <= 0 (H undefined) or D = 0: alpha = 2.

template <class R>
__device__ __forceinline__ R ratio(R a, R b) {
  if constexpr (std::is_same_v<R, double>) return a / b; else return __fdividef(a, b);
}

// Calls fn(F, E, wgt) for every direction: F = f_i and E = feq_i (plain storage), or
// F = f_i / w_i and E = feq_i / w_i with wgt = w_i (offset storage; wgt = 1 otherwise), feq the
// exact entropic equilibrium with multipliers lam.
template <class Store, class R, class Fn>
__device__ __forceinline__ void visit_populations(const R* f, const R* lam, R rho, const LatticeTables& tb, Fn&& fn) {
  constexpr bool kOff = Codec<Store>::kOffset;
  fn(kOff ? R(1) + f[0] : f[0], entropic_shell_factor<0, kOff>(lam, rho, tb), kOff ? tab_w<R>(tb, 0) : R(1));
  entropic_pair_values<R, kOff>(lam, rho, tb, [&](auto Pc, R vp, R vm) {
    constexpr int P = decltype(Pc)::value;
    constexpr int s = rd3q81::kDirs[1 + 2 * P].shell;
    const R wg = kOff ? tab_w<R>(tb, s) : R(1);
    fn(kOff ? R(1) + f[1 + 2 * P] : f[1 + 2 * P], vp, wg);
    fn(kOff ? R(1) + f[2 + 2 * P] : f[2 + 2 * P], vm, wg);
  });
}

// log(1 + y) for y > -1, FP32: for |y| < 1/4 from log(1 + y) = 2 atanh(s), s = y / (2 + y)
// (|s| <= 1/7; the odd series to s^9 leaves below 1e-9 relative); otherwise the hardware
// logarithm of u = 1 + y, corrected for the rounding of u by (y - (u - 1)) / u.  Relative error
// below 2e-6 everywhere (the hardware log2 is good to 2^-21 absolute on [1/2, 2]).  Both forms
// are evaluated and one is selected: a branch would split the unrolled direction loops of the
// alpha solve into blocks the compiler cannot interleave (measured 7 % slower for FP32 storage,
// 23 % for FP16).
__device__ __forceinline__ float log1p_alpha(float y) {
  const float u = 1.0f + y;
  const float s = __fdividef(y, 2.0f + y), s2 = s * s;
  const float ser = 2.0f * s * (1.0f + s2 * (1.0f / 3.0f + s2 * (0.2f + s2 * (1.0f / 7.0f + s2 * (1.0f / 9.0f)))));
  const float hw = __logf(u) + __fdividef(y - (u - 1.0f), u);
  return fabsf(y) < 0.25f ? ser : hw;
}
__device__ __forceinline__ double log1p_alpha(double y) { return log1p(y); }

// Per-thread columns of x_i and w_i F_i for the alpha solve.  The walk over the directions runs
// once, to fill them; the sums over directions are then short runtime loops (an unrolled
// evaluation per iterate would not fit the instruction cache).  FP32 keeps the 2 x 81 values
// in dynamic shared memory, one column per thread ([2][81][blockDim.x]: consecutive threads,
// consecutive banks), 648 bytes a thread: in per-thread local memory they overflowed L1 at any
// useful occupancy and every pass went to L2 (1274 DRAM bytes a site against 648).  FP64 keeps
// a local array.
template <class R>
struct AlphaColumns {
  R* xs;
  R* wf;
  int stride;
};

// The full-expression solve on the columns.
// Each pass expands Delta H about a centre a0 exactly in delta = alpha - a0: with u_i = 1 + a0 x_i,
// L_i = log u_i and z_i = x_i / u_i,
//   Delta H(a0 + delta) = F0 + F1 delta + sum_{n>=2} (-1)^n M_n delta^n / (n (n-1)),
//   F0 = <f, u L - a0 x> - a0 b,  F1 = <f, x L> - b,  M_n = <f, u z^n>,
// which converges for q = |delta| max|z| < 1, the terms beyond n = N summing to at most
// |delta|^(N+1) <f, u |z|^(N+1)> / (N (N+1) (1 - q)).  The root of the series truncated at N
// (Newton from 0) is accepted when that bound moves alpha by less than the tolerance (divided
// by the slope F1), or when delta itself is below it; otherwise the root becomes the next centre,
// kept inside the bracket [lo, hi] that the signs of F0 maintain (bisection when it would leave
// it).  One pass usually suffices: populations with large |z| weigh little in the bound.
// The test for a root before alpha_max (Delta H(alpha_max) <= 0: alpha = alpha_max) takes one
// more logarithm per population.  It runs with the first pass when alpha_max < 5/2 (near the
// usual root, where it often decides), and otherwise only once a root estimate reaches
// alpha_max: a root found below alpha_max already implies Delta H(alpha_max) > 0, since Delta H
// is convex, zero at 0 and negative at 1.  The direction loops are unrolled by 3 (81 = 3 x 27)
// so that three populations' dependent chains interleave.
template <class R>
__device__ __forceinline__ R entropic_alpha_full(const AlphaColumns<R>& c, R amax) {
  constexpr bool kDbl = std::is_same_v<R, double>;
  constexpr int N = kDbl ? 10 : 6;
  constexpr int kMaxPass = kDbl ? 40 : 20;
  const R tol = R(kDbl ? 1e-14 : 1e-6);
  const R* xs = c.xs;
  const R* wf = c.wf;
  const int stride = c.stride;
  const bool finite = amax < R(1e30);
  const bool eager = amax < R(2.5);
  // Delta H(alpha_max) + alpha_max b (the limiting population's term is 1 there)
  auto dh_amax = [&]() {
    R Sm = R(0);
#pragma unroll 3
    for (int i = 0; i < kQ; ++i) {
      const R x = xs[i * stride], w = wf[i * stride];
      const R ym = amax * x;
      Sm += w * (ym > R(-1) ? (R(1) + ym) * log1p_alpha(ym) - ym : R(1));
    }
    return Sm;
  };
  R lo = R(1), hi = amax;
  R a0 = fmin(R(2), R(1) + R(0.9) * (amax - R(1)));
  R b = R(0);
  bool checked = false;
  for (int pass = 0; pass < kMaxPass; ++pass) {
    R F0 = R(0), F1 = R(0), zmax = R(0), Mabs = R(0), M[N - 1];  // M[k] = M_{k+2}
#pragma unroll
    for (int k = 0; k < N - 1; ++k) M[k] = R(0);
    auto term = [&](R x, R w) {
      const R y = a0 * x, u = R(1) + y;
      const R L = log1p_alpha(y);
      const R z = ratio(x, u);
      F0 += w * (u * L - y);
      F1 += w * x * L;
      zmax = fmax(zmax, fabs(z));
      R t = w * u * z;
#pragma unroll
      for (int k = 0; k < N - 1; ++k) {
        t *= z;
        M[k] += t;
      }
      Mabs += fabs(t * z);
    };
    if (pass == 0) {
      // the first pass also sums b = <f, x log(1 + x)>, and Delta H(alpha_max) when eager
      R Sm = R(0);
#pragma unroll 3
      for (int i = 0; i < kQ; ++i) {
        const R x = xs[i * stride], w = wf[i * stride];
        b += w * x * log1p_alpha(x);
        if (eager) {
          const R ym = amax * x;
          Sm += w * (ym > R(-1) ? (R(1) + ym) * log1p_alpha(ym) - ym : R(1));
        }
        term(x, w);
      }
      if (eager && finite) {
        checked = true;
        if (Sm - amax * b <= R(0)) return amax;  // no root before the positivity boundary
      }
    } else {
#pragma unroll 3
      for (int i = 0; i < kQ; ++i) term(xs[i * stride], wf[i * stride]);
    }
    F0 -= a0 * b;
    F1 -= b;
    if (F0 < R(0)) lo = a0; else hi = a0;
    // root of the truncated series: Newton in delta from 0
    R d = R(0);
    for (int it = 0; it < 8; ++it) {
      R G = F0 + F1 * d, dG = F1, p = d;             // p = d^(n-1)
#pragma unroll
      for (int k = 0; k < N - 1; ++k) {
        const int nn = k + 2;
        const R cf = ((nn % 2 == 0) ? R(1) : R(-1)) * M[k];
        dG += cf * p * R(1.0 / (nn - 1));
        p *= d;
        G += cf * p * R(1.0 / (nn * (nn - 1)));
      }
      const R step = G / dG;
      d -= step;
      if (!(fabs(step) > tol * a0)) break;
    }
    const R na = a0 + d;
    if (!checked && finite && !(na < hi)) {
      checked = true;
      if (dh_amax() - amax * b <= R(0)) return amax;
    }
    const R q = fabs(d) * zmax;
    R bound = R(1e30);
    if (q < R(1)) {
      bound = Mabs / (R(N * (N + 1)) * (R(1) - q));
#pragma unroll
      for (int k = 0; k <= N; ++k) bound *= fabs(d);
    }
    const bool inside = na > lo && na < hi;
    if (inside && (bound <= tol * fabs(F1) * a0 || fabs(d) <= tol * a0)) return na;
    a0 = inside ? na : R(0.5) * (lo + hi);
    if (hi - lo <= tol * a0) break;
  }
  return a0;
}

// One walk over the populations fills the columns (x_i = feq_i / f_i - 1 and w_i F_i) and
// finds min x, max |x| and min F; then the series form when every |x_i| <= kX (its moments
// a_n = <f, x^n> summed from the columns), else the full expression.
template <class Store, class R>
__device__ __forceinline__ R entropic_alpha(const R* f, const R* lam, R rho, const LatticeTables& tb) {
  constexpr bool kDbl = std::is_same_v<R, double>;
  constexpr int N = kDbl ? 8 : 6;
  const R kX = R(kDbl ? 0.01 : 0.05);
  [[maybe_unused]] R xs_local[kDbl ? kQ : 1], wf_local[kDbl ? kQ : 1];
  AlphaColumns<R> c;
  if constexpr (kDbl) {
    c = AlphaColumns<R>{xs_local, wf_local, 1};
  } else {
    extern __shared__ float alpha_smem[];
    c = AlphaColumns<R>{alpha_smem + threadIdx.x, alpha_smem + kQ * blockDim.x + threadIdx.x,
                        static_cast<int>(blockDim.x)};
  }
  R xmin = R(0), xabs = R(0), Fmin = R(1);
  int n = 0;
  visit_populations<Store>(f, lam, rho, tb, [&](R F, R E, R wg) {
    const R x = ratio(E - F, F);
    Fmin = fmin(Fmin, F);
    xmin = fmin(xmin, x);
    xabs = fmax(xabs, fabs(x));
    c.xs[n * c.stride] = x;
    c.wf[n * c.stride] = wg * F;
    ++n;
  });
  if (!(Fmin > R(0)) || !(xabs > R(0))) return R(2);
  R al = R(2);
  if (xabs <= kX) {
    R an[N - 1];  // a_2 .. a_N
#pragma unroll
    for (int k = 0; k < N - 1; ++k) an[k] = R(0);
#pragma unroll 3
    for (int i = 0; i < kQ; ++i) {
      const R x = c.xs[i * c.stride];
      R pw = c.wf[i * c.stride] * x;
#pragma unroll
      for (int k = 0; k < N - 1; ++k) {
        pw *= x;
        an[k] += pw;
      }
    }
    if (!(an[0] > R(0))) return R(2);
#pragma unroll
    for (int it = 0; it < 3; ++it) {
      R G = R(0), dG = R(0), pw = R(1);  // pw = al^(n-2)
#pragma unroll
      for (int k = 0; k < N - 1; ++k) {
        const int nn = k + 2;
        const R sa = (nn % 2 == 0) ? an[k] : -an[k];
        G += sa * (pw * al * R(1.0 / (nn * (nn - 1))) - R(1.0 / (nn - 1)));
        dG += sa * pw * R(1.0 / nn);
        pw *= al;
      }
      al -= G / dG;
    }
  } else {
    al = entropic_alpha_full<R>(c, xmin < R(0) ? R(-1) / xmin : R(1e30));
  }
  return (al > R(0) && al < R(1e30)) ? al : R(2);
}

// Temperature recovery, equilibrium (App. B series, or the exact one of Sec. III) and the
// collision (alpha = 2, or the entropic alpha) of one site's populations f (in place), given
// their moments.

template <class Store, class M, int kEq = kEqSeries>
__device__ __forceinline__ void site_relax(typename Codec<Store>::Real* f, const Moments<M>& mo, double omega,
                                           unsigned int* flag, const LatticeTables& tb) {
  using C = Codec<Store>;
  using R = typename C::Real;
  R rh, theta, mux, muy, muz;
  if constexpr (std::is_same_v<M, Dw>) {
    // double-word recovery of u and theta (site_moments_dw), rounded once to FP32
    const Dw inv = dw_recip(mo.rho);
    const Dw ux = dw_mul(mo.jx, inv), uy = dw_mul(mo.jy, inv), uz = dw_mul(mo.jz, inv);
    const Dw u2 = dw_add(dw_add(dw_mul(ux, ux), dw_mul(uy, uy)), dw_mul(uz, uz));
    const Dw th3 = dw_add(dw_mul(mo.E, inv), Dw{-u2.hi, -u2.lo});
    rh = dw_to_float(mo.rho);
    theta = dw_to_float(dw_mul(th3, Dw{kThirdHi, kThirdLo}));
    mux = dw_to_float(ux);
    muy = dw_to_float(uy);
    muz = dw_to_float(uz);
  } else {
    const M irho = M(1) / mo.rho;
    const M dux = mo.jx * irho, duy = mo.jy * irho, duz = mo.jz * irho;
    const M mtheta = (mo.E * irho - (dux * dux + duy * duy + duz * duz)) * M(1.0 / 3.0);
    rh = R(mo.rho);
    theta = R(mtheta);
    mux = R(dux);
    muy = R(duy);
    muz = R(duz);
  }
  if (!(rh > R(0) && theta > R(0) && rh < R(FLT_MAX) && theta < R(FLT_MAX))) atomicOr(flag, 1u);
  // ---- equilibrium: App. B series (kEqSeries) or the exact minimiser of Sec. III ---------
  [[maybe_unused]] EqScalars<R> e;
  [[maybe_unused]] R W[kShells];     // series: W~_s (or W~_s / w_s)
  [[maybe_unused]] R lam[5];         // entropic: multipliers (mu, zeta, gamma)
  // <feq, phi phi^T> at lam for the FP32 projection: with the entropic alpha the Newton's last
  // matrix is kept (measured 16 % faster, and the kernel no longer spills); with BGK it is
  // evaluated again at the projection (keeping it live doubled that kernel's spill and cost it
  // 12 %).
  constexpr bool kKeepJ = std::is_same_v<Store, float> && kEq == kEqEntropicAlpha;
  [[maybe_unused]] R Jm[15];
  if constexpr (kEq == kEqSeries) {
    const R eta = theta * R(1.0 / rd3q81::kTheta0) - R(1);
    eq_scalars<R>(mux, muy, muz, theta, eta, tab_na<R>(tb), tab_nb<R>(tb), e);
#pragma unroll
    for (int s = 0; s < kShells; ++s)
      W[s] = rh * poly4(C::kOffset ? tab_p<R>(tb, s) : tab_wp<R>(tb, s), eta);
  } else if constexpr (kEq == kEqSeriesExactW) {
    R An, Bn;
    if (!exact_weights<R>(theta, tb, W, An, Bn)) atomicOr(flag, 1u);
    eq_scalars_ab<R>(mux, muy, muz, theta, An, Bn, e);
#pragma unroll
    for (int s = 0; s < kShells; ++s) W[s] *= C::kOffset ? rh : rh * tab_w<R>(tb, s);
  } else {
    constexpr bool kDbl = std::is_same_v<R, double>;
    const R T[5] = {rh, R(mo.jx), R(mo.jy), R(mo.jz), R(mo.E)};
    if (!entropic_multipliers<R>(T, mux, muy, muz, theta, R(kDbl ? 1e-13 : 1e-6), kDbl ? 30 : 16, tb, lam,
                                 kKeepJ ? Jm : nullptr))
      atomicOr(flag, 1u);
  }

  // ---- entropic alpha (Eq. (delH)) or alpha = 2 --------------------------------------------
  [[maybe_unused]] R alpha = R(2);
  if constexpr (kEq == kEqEntropicAlpha) alpha = entropic_alpha<Store>(f, lam, rh, tb);

  // ---- BGK collision, Eq. (discretelbm) -------------------------------------------------
  // f_i <- f_i + omega D_i with D_i = f~eq_i - f_i.  In exact arithmetic D has zero mass,
  // momentum and energy.  In FP32 it does not quite (f~eq is evaluated at rho, u, theta
  // rounded to FP32), and the defect would accumulate step after step.  For FP32 storage
  // the defects of D are therefore summed (D is small, so the sums are accurate) and removed,
  // for the series equilibria, by subtracting w_i (a + b.c_i + g c_i^2) with a, b, g fixed by
  // the weights' moments
  // <w,1> = 1, <w,c c> = theta0 I, <w,c^2> = 3 theta0, <w,c^4> = 15 theta0^2.  The
  // correction has the shape of an equilibrium perturbation, so it adds no non-equilibrium
  // part (with omega near 2 such a part would hardly decay).  The entropic equilibria take a
  // correction shaped like f~eq itself (below).  The result equals the plain update in exact
  // arithmetic; in FP32 it conserves to the rounding of the defect sums.
  constexpr bool kProject = std::is_same_v<Store, float>;
  R om = R(omega);                   // alpha beta with alpha = 2
  if constexpr (kEq == kEqEntropicAlpha) om = R(0.5) * om * alpha;
  R d1 = R(0), dE = R(0), dx = R(0), dy = R(0), dz = R(0);
  auto relax_rest = [&](R feq0) {
    if constexpr (C::kOffset) feq0 -= R(1);
    const R D0 = feq0 - f[0];
    if constexpr (kProject) d1 += D0;
    f[0] += om * D0;
  };
  auto relax_pair = [&](auto Pc, R fp, R fm) {
    constexpr int P = decltype(Pc)::value;
    constexpr rd3q81::Dir d = rd3q81::kDirs[1 + 2 * P];
    if constexpr (C::kOffset) {
      fp -= R(1);
      fm -= R(1);
    }
    const R Dp = fp - f[1 + 2 * P];
    const R Dm = fm - f[2 + 2 * P];
    if constexpr (kProject) {
      constexpr double c2 = rd3q81::kShellC2[d.shell];
      const R sD = Dp + Dm, dD = Dp - Dm;
      d1 += sD;
      dE += R(c2) * sD;
      if constexpr (d.hx != 0) dx += R(0.5 * d.hx) * dD;
      if constexpr (d.hy != 0) dy += R(0.5 * d.hy) * dD;
      if constexpr (d.hz != 0) dz += R(0.5 * d.hz) * dD;
    }
    f[1 + 2 * P] += om * Dp;
    f[2 + 2 * P] += om * Dm;
  };
  if constexpr (eq_is_series(kEq)) {
    relax_rest(W[0] * (e.c0 + e.k0 * (R(0) - e.t3)));
    static_for<kPairs>([&](auto Pc) {
      constexpr int P = decltype(Pc)::value;
      constexpr int s = rd3q81::kDirs[1 + 2 * P].shell;
      R ev, od;
      eq_pair_parts<P, R>(e, ev, od);
      const R we = W[s] * ev;
      const R wo = W[s] * od;
      relax_pair(Pc, we + wo, we - wo);
    });
  } else {
    // f~eq / w_i for offset storage: the weights cancel against the codec's 1 + d form.
    relax_rest(entropic_shell_factor<0, C::kOffset>(lam, rh, tb));
    entropic_pair_values<R, C::kOffset>(lam, rh, tb, relax_pair);
  }
  if constexpr (kProject && (kEq == kEqEntropic || kEq == kEqEntropicAlpha)) {
    // With the exact entropic equilibrium the correction must be small relative to every
    // population, the smallest included: with the entropic alpha their update decides alpha, and
    // at Mach 2 the upstream outer-shell equilibria are orders of magnitude below w_i, so a
    // w_i-shaped correction of the Newton's residual (up to its tolerance, 1e-6, every step, with
    // the same sign) builds a non-equilibrium part there that omega near 2 hardly damps (the FP32
    // Mach-2 blob failed within 100 steps that way; FP16 storage, which has no projection, ran).
    // The defects are removed by subtracting omega feq_i (k . phi_i), k from
    // <feq, phi phi^T> k = defects (the Newton's 5x5 matrix at the final multipliers), which is
    // the shape of a change of the multipliers.  In exact arithmetic the defects and k are zero.
    if constexpr (!kKeepJ) entropic_moment_matrix<R>(lam, rh, tb, Jm);
    R k[5] = {d1, dx, dy, dz, dE};
    if (solve_spd5<R>(Jm, k)) {
      f[0] -= om * entropic_shell_factor<0, false>(lam, rh, tb) * k[0];
      entropic_pair_values<R, false>(lam, rh, tb, [&](auto Pc, R vp, R vm) {
        constexpr int P = decltype(Pc)::value;
        constexpr rd3q81::Dir d = rd3q81::kDirs[1 + 2 * P];
        constexpr double c2 = rd3q81::kShellC2[d.shell];
        const R ev = k[0] + R(c2) * k[4];
        R od = R(0);
        if constexpr (d.hx != 0) od += R(0.5 * d.hx) * k[1];
        if constexpr (d.hy != 0) od += R(0.5 * d.hy) * k[2];
        if constexpr (d.hz != 0) od += R(0.5 * d.hz) * k[3];
        f[1 + 2 * P] -= om * vp * (ev + od);
        f[2 + 2 * P] -= om * vm * (ev - od);
      });
    }
  } else if constexpr (kProject) {
    constexpr double t0 = rd3q81::kTheta0;
    const R g = (dE - R(3.0 * t0) * d1) * R(1.0 / (6.0 * t0 * t0));
    const R a = d1 - R(3.0 * t0) * g;
    const R oa = om * a, og = om * g, obx = om * dx * R(1.0 / t0), oby = om * dy * R(1.0 / t0),
            obz = om * dz * R(1.0 / t0);
    f[0] -= tab_w<R>(tb, 0) * oa;
    static_for<kPairs>([&](auto Pc) {
      constexpr int P = decltype(Pc)::value;
      constexpr rd3q81::Dir d = rd3q81::kDirs[1 + 2 * P];
      constexpr double c2 = rd3q81::kShellC2[d.shell];
      const R ws = tab_w<R>(tb, d.shell);
      const R ce = ws * (oa + R(c2) * og);
      R co = R(0);
      if constexpr (d.hx != 0) co += R(0.5 * d.hx) * obx;
      if constexpr (d.hy != 0) co += R(0.5 * d.hy) * oby;
      if constexpr (d.hz != 0) co += R(0.5 * d.hz) * obz;
      co *= ws;
      f[1 + 2 * P] -= ce + co;
      f[2 + 2 * P] -= ce - co;
    });
  }
}

template <class Store>
__device__ __forceinline__ void site_store(const Geometry& g, void* dst_buf, int sub, int own,
                                           const typename Codec<Store>::Real* f) {
  Store* dst = static_cast<Store*>(dst_buf) + sub * g.sub_stride + own;
  static_for<kQ>([&](auto Ic) {
    constexpr int i = decltype(Ic)::value;
    Codec<Store>::store(dst + static_cast<long long>(i) * g.dir_stride, f[i]);
  });
}

// Updates interior site t of sublattice SUB: reads `src`, writes `dst` (both whole
// population buffers of geometry g), relaxation omega, instability flag `flag`.
// kF64Mom: the moment sums and the temperature recovery run in FP64 whatever the storage.
// kEq: the equilibrium and collision (Equilibrium).
template <class Store, bool kF64Mom, int SUB, int kEq = kEqSeries>
__device__ __forceinline__ void site_update(const Geometry& g, const void* src_buf, void* dst_buf, double omega,
                                            unsigned int* flag, const LatticeTables& tb, int t) {
  using C = Codec<Store>;
  using R = typename C::Real;
  int xs[9], ys[9], zs[9];
  site_coords(g, t, xs, ys, zs);
  R f[kQ];
  for_each_source<Store, SUB>(g, static_cast<const Store*>(src_buf), xs, ys, zs, [&](auto Ic, const Store* p) {
    f[decltype(Ic)::value] = C::load(p);
  });
  const auto mo = site_moments<Store, kF64Mom>(f, tb);
  site_relax<Store, typename decltype(mo)::value_type, kEq>(f, mo, omega, flag, tb);
  site_store<Store>(g, dst_buf, SUB, zs[4] + ys[4] + xs[4], f);
}

// Where a step finds the base address of each direction slab it reads and writes, per target
// sublattice SUB and direction i (a compile-time constant in the unrolled loops):
//   ParamSlabs   the kernel parameters (StepParams, filled by fill_slab_bases), for one case;
//   SharedSlabs  a block's shared-memory copy of one served case's table (the same values).
template <int SUB>
struct ParamSlabs {
  const StepParams& p;
  __device__ __forceinline__ const void* src(int i) const { return p.src_slab[SUB][i]; }
  __device__ __forceinline__ void* dst(int i) const { return p.dst_slab[SUB][i]; }
};
struct SharedSlabs {
  const void* const* s;
  void* const* d;
  __device__ __forceinline__ const void* src(int i) const { return s[i]; }
  __device__ __forceinline__ void* dst(int i) const { return d[i]; }
};

// The single-case form of site_update: the same phases, with the slab base addresses taken
// from a table (Slabs) instead of being computed per access.  kKind (StepKind) picks where
// population i is read and written; the slab bases (fill_slab_bases) pick the sublattice and
// slot:
//   ping-pong:    read the source of c_i (pull),  write own site;
//   AA neighbour: read the source of c_i (pull),  write the site that pulls c_i next (push);
//   AA own:       read own site,                  write own site.
template <class Store, bool kF64Mom, int SUB, int kEq, int kKind, class Slabs>
__device__ __forceinline__ void site_update_table(const Geometry& g, double omega, unsigned int* flag,
                                                  const LatticeTables& tab, const Slabs& sl, int t) {
  using C = Codec<Store>;
  using R = typename C::Real;
  int xs[9], ys[9], zs[9];
  site_coords(g, t, xs, ys, zs);
  R f[kQ];
  static_for<kQ>([&](auto Ic) {
    constexpr int i = decltype(Ic)::value;
    constexpr rd3q81::Dir d = rd3q81::kDirs[i];
    constexpr bool kPull = kKind != kStepAAOwn;
    constexpr int dx = kPull ? rd3q81::pull_disp(d.hx, SUB) : 0;
    constexpr int dy = kPull ? rd3q81::pull_disp(d.hy, SUB) : 0;
    constexpr int dz = kPull ? rd3q81::pull_disp(d.hz, SUB) : 0;
    f[i] = C::load(static_cast<const Store*>(sl.src(i)) + (zs[dz + 4] + ys[dy + 4] + xs[dx + 4]));
  });
  const auto mo = site_moments<Store, kF64Mom>(f, tab);
  site_relax<Store, typename decltype(mo)::value_type, kEq>(f, mo, omega, flag, tab);
  static_for<kQ>([&](auto Ic) {
    constexpr int i = decltype(Ic)::value;
    constexpr rd3q81::Dir d = rd3q81::kDirs[i];
    constexpr bool kPush = kKind == kStepAANeighbour;
    constexpr int dx = kPush ? rd3q81::pull_disp(-d.hx, SUB) : 0;
    constexpr int dy = kPush ? rd3q81::pull_disp(-d.hy, SUB) : 0;
    constexpr int dz = kPush ? rd3q81::pull_disp(-d.hz, SUB) : 0;
    Store* q = static_cast<Store*>(sl.dst(i)) + (zs[dz + 4] + ys[dy + 4] + xs[dx + 4]);
    // In-place (AA) steps store with the evict-first hint (st.global.cs): FP32 7232 -> 7473 MLUPS at
    // TGV 512^3.  Ping-pong lost with it (FP32 8818 -> 8602, FP16 14940 -> 14668): plain stores.
    if constexpr (kKind != kStepPingPong)
      C::store_evict_first(q, f[i]);
    else
      C::store(q, f[i]);
  });
}

template <class Store, bool kF64Mom, int SUB, int kEq, int kKind = kStepPingPong>
__device__ __forceinline__ void site_update_slabs(const StepParams& p, int t) {
  site_update_table<Store, kF64Mom, SUB, kEq, kKind>(p.g, p.omega, p.flag, p.tab, ParamSlabs<SUB>{p}, t);
}

// Resident blocks per SM the compiler must fit (register budget 65536 / (blocks * 128)):
// 4 for FP32/FP16/BF16 storage (<= 128 registers, 16 warps per SM; with FP64-quality moments
// too: their double-word sums run at FP32 rates, 9 % faster than at 3 blocks for FP32), and no
// bound for FP64 storage (its 81 doubles
// need ~250).  The entropic alpha: 2 blocks, the most its 83 KB of shared memory a block allow
// (255 registers, no spill).
template <class Store, bool kF64Mom, int kEq>
RD3Q81_HD constexpr int sc_min_blocks_128() {
  if constexpr (std::is_same_v<Store, double>) return 1;
  else if constexpr (kEq == kEqEntropicAlpha) return 2;  // shared memory of the alpha solve
  else return 4;
}

// Dynamic shared memory of the fused kernel: the FP32 alpha solve's 2 x 81 values per thread.
template <class Store, int kEq, int kBlock>
constexpr int sc_dyn_smem() {
  return (kEq == kEqEntropicAlpha && !std::is_same_v<Store, double>) ? 2 * kQ * kBlock * static_cast<int>(sizeof(float))
                                                                      : 0;
}

// Threads per block of the fused kernel.  The issue-bound equilibria (exact entropic, exact
// W(theta)) run 4-7 % faster in 256-thread blocks; the series equilibrium, whose FP32 form is
// bandwidth-bound, and FP16 storage run 1-4 % faster in 128-thread blocks.  The register budget
// per thread is the same either way (sc_min_blocks scales with the block).
template <class Store, bool kF64Mom, int kEq>
RD3Q81_HD constexpr int sc_block() {
  return (kEq == kEqEntropic || kEq == kEqSeriesExactW) && !std::is_same_v<Store, double> ? 2 * kScBlock : kScBlock;
}

template <class Store, bool kF64Mom, int kEq>
RD3Q81_HD constexpr int sc_min_blocks() {
  constexpr int b = sc_min_blocks_128<Store, kF64Mom, kEq>() * kScBlock / sc_block<Store, kF64Mom, kEq>();
  return b < 1 ? 1 : b;
}

template <class Store, bool kF64Mom, int kEq, int kKind = kStepPingPong>
__global__ void __launch_bounds__(sc_block<Store, kF64Mom, kEq>(), sc_min_blocks<Store, kF64Mom, kEq>())
    stream_collide_kernel(const StepParams p) {
  const long long nxy = static_cast<long long>(p.g.nx) * p.g.ny;
  constexpr int kBlock = sc_block<Store, kF64Mom, kEq>();
  const long long t = p.z0 * nxy + static_cast<long long>(blockIdx.x) * kBlock + threadIdx.x;
  if (t >= p.z1 * nxy) return;
  if (blockIdx.y == 0)
    site_update_slabs<Store, kF64Mom, 0, kEq, kKind>(p, static_cast<int>(t));
  else
    site_update_slabs<Store, kF64Mom, 1, kEq, kKind>(p, static_cast<int>(t));
}

template <class Store, bool kF64Mom, int kEq = kEqSeries, int kKind = kStepPingPong>
cudaError_t launch_sc(const StepParams& p, cudaStream_t s) {
  const long long n = static_cast<long long>(p.g.nx) * p.g.ny * (p.z1 - p.z0);
  if (n <= 0) return cudaSuccess;
  constexpr int kBlock = sc_block<Store, kF64Mom, kEq>();
  const dim3 grid(static_cast<unsigned>((n + kBlock - 1) / kBlock), 2);
  constexpr int kSmem = sc_dyn_smem<Store, kEq, kBlock>();
  if constexpr (kEq == kEqEntropicAlpha) {
    // the alpha solve keeps 2 x 81 values per thread: in shared memory (FP32; more than the
    // default 48 KB a block, and the most shared memory the carveout gives) or in local memory
    // (FP64; then all of L1 for it).  Set on the direct launches; graphs are captured only after
    // those.
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaError_t e = cudaStreamIsCapturing(s, &cs);
    if (e == cudaSuccess && cs == cudaStreamCaptureStatusNone) {
      e = cudaFuncSetAttribute(stream_collide_kernel<Store, kF64Mom, kEq, kKind>,
                               cudaFuncAttributePreferredSharedMemoryCarveout, kSmem > 0 ? 100 : 0);
      if (e == cudaSuccess && kSmem > 0)
        e = cudaFuncSetAttribute(stream_collide_kernel<Store, kF64Mom, kEq, kKind>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, kSmem);
    }
    if (e != cudaSuccess) return e;
  }
  stream_collide_kernel<Store, kF64Mom, kEq, kKind><<<grid, kBlock, kSmem, s>>>(p);
  return cudaGetLastError();
}

// Both AA kinds of one storage and equilibrium (the sc_aa_*.cu units).
template <class Store, int kEq, bool kF64Mom = false>
cudaError_t launch_sc_aa(int kind, const StepParams& p, cudaStream_t s) {
  return kind == kStepAAOwn ? launch_sc<Store, kF64Mom, kEq, kStepAAOwn>(p, s)
                            : launch_sc<Store, kF64Mom, kEq, kStepAANeighbour>(p, s);
}

// FP64-quality moments are offered with the series equilibrium.
template <class Store>
cudaError_t launch_sc_aa_all(int fp64_moments, int eq, int kind, const StepParams& p, cudaStream_t s) {
  if (fp64_moments) return eq == kEqSeries ? launch_sc_aa<Store, kEqSeries, true>(kind, p, s) : cudaErrorInvalidValue;
  switch (eq) {
    case kEqSeries: return launch_sc_aa<Store, kEqSeries>(kind, p, s);
    case kEqSeriesExactW: return launch_sc_aa<Store, kEqSeriesExactW>(kind, p, s);
    case kEqEntropic: return launch_sc_aa<Store, kEqEntropic>(kind, p, s);
    case kEqEntropicAlpha: return launch_sc_aa<Store, kEqEntropicAlpha>(kind, p, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace lbm
