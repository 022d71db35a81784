// Fused pull-stream + collide for offset storage (FP16 / BF16), two x-adjacent sites per
// thread.  Same step as stream_collide.cuh (Sec. II, Eq. (discretelbm); moments by
// Eq. (conslaws); App. B series equilibrium; BGK, alpha = 2), same storage (d_i = f_i/w_i - 1,
// structure of arrays, x contiguous), same FP32 arithmetic per site; only the work is laid out
// for 2-byte elements:
//
// * one 32-bit register holds direction i of both sites (site x in the low half, x + 1 in the
//   high half), so the 81 populations of two sites take 81 registers;
// * the pull of a direction whose x displacement is even reads both sources as one aligned
//   32-bit word (49 of the 81 directions on either sublattice); an odd displacement reads two
//   16-bit elements and packs them;
// * the stores of the own sites are aligned 32-bit words, converted and packed by one
//   instruction per direction;
// * the address arithmetic of every access serves both sites.
//
// Arithmetic.  Both sites run the same operations, so the moment sums and the BGK update use
// the two-lane FP32 instructions of sm_100 and later (__ffma2_rn, __fadd2_rn, __fmul2_rn: one
// instruction for both sites, each lane rounded as its scalar form).  The moment sums add the
// offsets of a shell first (its members share w_s, |c|^2 and |c_a| = k_s/2), then weight them.
// The equilibrium bracket of App. B is evaluated per lane in scalar FP32, regrouped as in
// eq_pair_parts: for the pair +-c of shell s, xi = u.c = sigma (k/2) l and psi = sum_a u_a^3
// c_a = sigma (k/2) l3, where l = +-u_x +- u_y +- u_z over the nonzero components of c (first
// sign +, sigma = +-1) and l3 the same combination of the u_a^3 -- 13 combinations, each shared
// by every shell with that sign pattern; then
//   ev = a0_s + a2 xi^2,  od = xi (a1_s + a3 xi^2) + a4 psi,
//   bracket(+c) = ev + sigma od,  bracket(-c) = ev - sigma od.
// The BGK update of an offset value is written
//   d' = d + omega (W'_s bracket - 1 - d) = (1 - omega) d + (omega W'_s ev - omega) +- omega W'_s od,
// W'_s = W~_s / w_s.  Requires nx even (pairs never straddle a row) and the ping-pong layout.
#pragma once

#include <cfloat>
#include <cstdint>

#include "device_common.cuh"

namespace lbm {

// Packed pairs of 2-byte storage values (low half: site x, high half: site x + 1).
template <class S>
struct Pack2;
template <>
struct Pack2<__half> {
  static __device__ __forceinline__ float lo(uint32_t v) {
    return __half2float(__ushort_as_half(static_cast<unsigned short>(v & 0xffffu)));
  }
  static __device__ __forceinline__ float hi(uint32_t v) {
    return __half2float(__ushort_as_half(static_cast<unsigned short>(v >> 16)));
  }
  static __device__ __forceinline__ uint32_t pack(float a, float b) {
    const __half2 h = __floats2half2_rn(a, b);
    return *reinterpret_cast<const uint32_t*>(&h);
  }
};
template <>
struct Pack2<__nv_bfloat16> {
  static __device__ __forceinline__ float lo(uint32_t v) { return __uint_as_float(v << 16); }
  static __device__ __forceinline__ float hi(uint32_t v) { return __uint_as_float(v & 0xffff0000u); }
  static __device__ __forceinline__ uint32_t pack(float a, float b) {
    const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
    return *reinterpret_cast<const uint32_t*>(&h);
  }
};

// Signed combination of (x, y, z) with the compile-time signs (SX, SY, SZ) in {-1, 0, 1},
// normalised so that its first nonzero sign is +1; kSigma is the factor taken out.  Every
// shell with the same sign pattern writes the same expression, which the compiler evaluates
// once per site.
template <int SX, int SY, int SZ>
struct SignedCombo {
  static constexpr int first = SX != 0 ? SX : (SY != 0 ? SY : SZ);
  static constexpr int kSigma = first;
  static __device__ __forceinline__ float eval(float x, float y, float z) {
    constexpr int ax = SX * first, ay = SY * first, az = SZ * first;
    float r;
    if constexpr (ax != 0) {
      r = x;
      if constexpr (ay > 0) r = r + y;
      if constexpr (ay < 0) r = r - y;
      if constexpr (az > 0) r = r + z;
      if constexpr (az < 0) r = r - z;
    } else if constexpr (ay != 0) {
      r = y;
      if constexpr (az > 0) r = r + z;
      if constexpr (az < 0) r = r - z;
    } else {
      r = z;
    }
    return r;
  }
};

RD3Q81_HD constexpr int isign(int a) { return (a > 0) - (a < 0); }

// ---- two-lane FP32 arithmetic (x: site x, y: site x + 1) ---------------------------------
// The packed FP32 instructions of sm_100 and later: one instruction does the operation for
// both sites, each lane rounded exactly as its scalar form (__fmaf_rn, __fadd_rn, __fmul_rn).
__device__ __forceinline__ float2 f2(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __fadd2_rn(a, make_float2(-b.x, -b.y)); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }

// Per-site scalars of the pair relax, both sites in the lanes: EqScalars with 3 theta folded
// into the shell terms (a0_s = c0 + k0 c_s^2, a1_s = c1 + k1 c_s^2), eta and omega rho, from
// which each shell's omega W~_s / w_s is formed where that shell is relaxed (fewer live
// registers than holding all eleven).
struct PairSiteEq {
  float2 ux, uy, uz, ux3, uy3, uz3, a2, a3, a4, c0, k0, c1, k1;
  float2 eta, rom;
  // omega W~_s / w_s per lane (scalar: the polynomial's coefficients are constant operands)
  template <int s>
  __device__ __forceinline__ float2 wom(const LatticeTables& tb) const {
    return make_float2(rom.x * poly4(tb.pf[s], eta.x), rom.y * poly4(tb.pf[s], eta.y));
  }
};

template <class Store>
__device__ __forceinline__ float2 unpack2(uint32_t v) {
  return make_float2(Pack2<Store>::lo(v), Pack2<Store>::hi(v));
}

// Moments (Eq. (conslaws)) of both sites from their 81 packed offsets: rho = 1 + <w, d>,
// j = <w, d c>, <f, c^2> = 3 theta0 + <w, d c^2>.  Each shell's offsets are summed first (its
// members share w_s and |c|^2, and every nonzero component of c_i is +-k_s/2), then weighted.
template <class Store>
__device__ __forceinline__ void pair_moments(const uint32_t* f, const LatticeTables& tb, Moments<float2>& m) {
  float2 rho = mul2(f2(tb.wf[0]), unpack2<Store>(f[0]));
  float2 jx = f2(0.0f), jy = f2(0.0f), jz = f2(0.0f), E = f2(0.0f);
  float2 S = f2(0.0f), X = f2(0.0f), Y = f2(0.0f), Z = f2(0.0f);
  static_for<kPairs>([&](auto Pc) {
    constexpr int P = decltype(Pc)::value;
    constexpr rd3q81::Dir d = rd3q81::kDirs[1 + 2 * P];
    constexpr int s = d.shell;
    constexpr bool first = P == 0 || rd3q81::kDirs[2 * P - 1].shell != s;
    constexpr bool last = P == kPairs - 1 || rd3q81::kDirs[3 + 2 * P].shell != s;
    const float2 fp = unpack2<Store>(f[1 + 2 * P]), fm = unpack2<Store>(f[2 + 2 * P]);
    const float2 sum = add2(fp, fm), dif = sub2(fp, fm);
    S = first ? sum : add2(S, sum);
    if constexpr (d.hx != 0) X = first ? (d.hx > 0 ? dif : make_float2(-dif.x, -dif.y)) : (d.hx > 0 ? add2(X, dif) : sub2(X, dif));
    if constexpr (d.hy != 0) Y = first ? (d.hy > 0 ? dif : make_float2(-dif.x, -dif.y)) : (d.hy > 0 ? add2(Y, dif) : sub2(Y, dif));
    if constexpr (d.hz != 0) Z = first ? (d.hz > 0 ? dif : make_float2(-dif.x, -dif.y)) : (d.hz > 0 ? add2(Z, dif) : sub2(Z, dif));
    if constexpr (last) {
      rho = fma2(f2(tb.wf[s]), S, rho);
      E = fma2(f2(tb.wc2f[s]), S, E);
      jx = fma2(f2(tb.whkf[s]), X, jx);
      jy = fma2(f2(tb.whkf[s]), Y, jy);
      jz = fma2(f2(tb.whkf[s]), Z, jz);
      X = Y = Z = f2(0.0f);
    }
  });
  m.rho = add2(rho, f2(1.0f));
  m.jx = jx;
  m.jy = jy;
  m.jz = jz;
  m.E = add2(E, f2(static_cast<float>(3.0 * rd3q81::kTheta0)));
}

// Temperature recovery and the per-site equilibrium scalars of one site (lane), FP32; flags
// non-physical states.
__device__ __forceinline__ void pair_site_scalars(float rho, float jx, float jy, float jz, float E, float omega,
                                                  unsigned int* flag, const LatticeTables& tb, float* o) {
  const float irho = 1.0f / rho;
  const float ux = jx * irho, uy = jy * irho, uz = jz * irho;
  const float theta = (E * irho - (ux * ux + uy * uy + uz * uz)) * (1.0f / 3.0f);
  if (!(rho > 0.0f && theta > 0.0f && rho < FLT_MAX && theta < FLT_MAX)) atomicOr(flag, 1u);
  const float eta = theta * static_cast<float>(1.0 / rd3q81::kTheta0) - 1.0f;
  EqScalars<float> e;
  eq_scalars<float>(ux, uy, uz, theta, eta, tb.naf, tb.nbf, e);
  const float v[15] = {e.ux, e.uy, e.uz, e.ux3, e.uy3, e.uz3, e.a2, e.a3, e.a4, fmaf(-e.k0, e.t3, e.c0), e.k0,
                       fmaf(-e.k1, e.t3, e.c1), e.k1, eta, omega * rho};
#pragma unroll
  for (int k = 0; k < 15; ++k) o[k] = v[k];
}

__device__ __forceinline__ void pair_site_eq(const Moments<float2>& m, float omega, unsigned int* flag,
                                             const LatticeTables& tb, PairSiteEq& q) {
  float a[15], b[15];
  pair_site_scalars(m.rho.x, m.jx.x, m.jy.x, m.jz.x, m.E.x, omega, flag, tb, a);
  pair_site_scalars(m.rho.y, m.jx.y, m.jy.y, m.jz.y, m.E.y, omega, flag, tb, b);
  float2* dst[15] = {&q.ux, &q.uy, &q.uz, &q.ux3, &q.uy3, &q.uz3, &q.a2, &q.a3, &q.a4, &q.c0, &q.k0, &q.c1, &q.k1,
                     &q.eta, &q.rom};
#pragma unroll
  for (int k = 0; k < 15; ++k) *dst[k] = make_float2(a[k], b[k]);
}

// Even and odd parts (in c -> -c) of the series bracket of pair P at one site, up to the sign
// SignedCombo::kSigma of the odd part; per lane in scalar FP32, whose constant operands and
// looser register pairing keep the kernel within 128 registers.
template <int P>
__device__ __forceinline__ void pair_eq_lane(float ux, float uy, float uz, float ux3, float uy3, float uz3, float a2,
                                             float a3, float a4, float c0, float k0, float c1, float k1, float& ev,
                                             float& od) {
  constexpr rd3q81::Dir d = rd3q81::kDirs[1 + 2 * P];
  constexpr float hk = 0.5f * rd3q81::shell_shape(d.shell).k;
  constexpr float c2 = static_cast<float>(rd3q81::kShellC2[d.shell]);
  using Cb = SignedCombo<isign(d.hx), isign(d.hy), isign(d.hz)>;
  const float xi = hk * Cb::eval(ux, uy, uz);
  const float psi = hk * Cb::eval(ux3, uy3, uz3);
  const float xi2 = xi * xi;
  ev = fmaf(a2, xi2, fmaf(k0, c2, c0));
  od = fmaf(xi, fmaf(a3, xi2, fmaf(k1, c2, c1)), a4 * psi);
}

// New offsets of the +c and -c members of pair P at both sites (BGK with the series
// equilibrium): the bracket per lane, the update of both lanes in two-lane arithmetic.
template <int P>
__device__ __forceinline__ void pair_relax(const PairSiteEq& q, float om, const LatticeTables& tb, float2 dp,
                                           float2 dm, float2& np, float2& nm) {
  constexpr rd3q81::Dir d = rd3q81::kDirs[1 + 2 * P];
  constexpr int s = d.shell;
  using Cb = SignedCombo<isign(d.hx), isign(d.hy), isign(d.hz)>;
  float2 ev, od;
  pair_eq_lane<P>(q.ux.x, q.uy.x, q.uz.x, q.ux3.x, q.uy3.x, q.uz3.x, q.a2.x, q.a3.x, q.a4.x, q.c0.x, q.k0.x, q.c1.x,
                  q.k1.x, ev.x, od.x);
  pair_eq_lane<P>(q.ux.y, q.uy.y, q.uz.y, q.ux3.y, q.uy3.y, q.uz3.y, q.a2.y, q.a3.y, q.a4.y, q.c0.y, q.k0.y, q.c1.y,
                  q.k1.y, ev.y, od.y);
  const float2 wom = q.wom<s>(tb);
  const float2 Ep = fma2(wom, ev, f2(-om));
  const float2 Op = mul2(wom, od);
  const float2 cm = f2(1.0f - om);
  if constexpr (Cb::kSigma > 0) {
    np = add2(fma2(cm, dp, Ep), Op);
    nm = sub2(fma2(cm, dm, Ep), Op);
  } else {
    np = sub2(fma2(cm, dp, Ep), Op);
    nm = add2(fma2(cm, dm, Ep), Op);
  }
}

// Updates the sites t (x even) and t + 1 of sublattice SUB (ping-pong).
template <class Store, int SUB>
__device__ __forceinline__ void site_pair_update(const StepParams& p, int t) {
  using PK = Pack2<Store>;
  const Geometry& g = p.g;
  const int x = t % g.nx;
  const int r = t / g.nx;
  const int y = r % g.ny;
  const int z = r / g.ny;
  // xe[j]: element index of x + j - 4 (j = 0 .. 9); ys, zs as in site_coords.
  int xe[10], ys[9], zs[9];
#pragma unroll
  for (int j = 0; j < 10; ++j) xe[j] = (g.x_periodic ? wrap_idx(x + j - 4, g.nx) : x + j - 4) + g.xoff;
#pragma unroll
  for (int k = 0; k < 9; ++k) {
    ys[k] = wrap_idx(y - (k - 4), g.ny) * g.pitch;
    zs[k] = wrap_idx(z - (k - 4), g.nz) * static_cast<int>(g.plane);
  }
  uint32_t f[kQ];
  static_for<kQ>([&](auto Ic) {
    constexpr int i = decltype(Ic)::value;
    constexpr rd3q81::Dir d = rd3q81::kDirs[i];
    constexpr int dx = rd3q81::pull_disp(d.hx, SUB);
    constexpr int dy = rd3q81::pull_disp(d.hy, SUB);
    constexpr int dz = rd3q81::pull_disp(d.hz, SUB);
    const Store* row = static_cast<const Store*>(p.src_slab[SUB][i]) + (zs[dz + 4] + ys[dy + 4]);
    if constexpr (dx % 2 == 0) {
      // sources x - dx (even) and x + 1 - dx: one aligned word (no wrap falls between them)
      f[i] = *reinterpret_cast<const uint32_t*>(row + xe[4 - dx]);
    } else {
      const uint32_t a = *reinterpret_cast<const unsigned short*>(row + xe[4 - dx]);
      const uint32_t b = *reinterpret_cast<const unsigned short*>(row + xe[5 - dx]);
      f[i] = __byte_perm(a, b, 0x5410);
    }
  });
  const float omega = static_cast<float>(p.omega);
  PairSiteEq q;
  {
    Moments<float2> m;
    pair_moments<Store>(f, p.tab, m);
    pair_site_eq(m, omega, p.flag, p.tab, q);
  }
  // The relax converts the packed values again: without this (empty) barrier the compiler keeps
  // the 162 floats of the moment sums alive instead of the 81 packed words, and spills.
#pragma unroll
  for (int i = 0; i < kQ; ++i) asm volatile("" : "+r"(f[i]));
  const int own = zs[4] + ys[4] + xe[4];
  {
    const float2 n0 = fma2(f2(1.0f - omega), unpack2<Store>(f[0]), fma2(q.wom<0>(p.tab), q.c0, f2(-omega)));
    *reinterpret_cast<uint32_t*>(static_cast<Store*>(p.dst_slab[SUB][0]) + own) = PK::pack(n0.x, n0.y);
  }
  static_for<kPairs>([&](auto Pc) {
    constexpr int P = decltype(Pc)::value;
    float2 np, nm;
    pair_relax<P>(q, omega, p.tab, unpack2<Store>(f[1 + 2 * P]), unpack2<Store>(f[2 + 2 * P]), np, nm);
    *reinterpret_cast<uint32_t*>(static_cast<Store*>(p.dst_slab[SUB][1 + 2 * P]) + own) = PK::pack(np.x, np.y);
    *reinterpret_cast<uint32_t*>(static_cast<Store*>(p.dst_slab[SUB][2 + 2 * P]) + own) = PK::pack(nm.x, nm.y);
  });
}

// 128 threads, 4 resident blocks per SM (128 registers, a 96-byte spill): 16 warps of 64 sites.
// Measured at TGV 512^3 FP16: 15.1 GLUPS.  All-scalar arithmetic at 4 blocks (16-byte spill):
// 14.2; two-lane moments only: 14.7; two-lane arithmetic throughout (more registers in pairs) at
// 3 blocks: 13.6.
constexpr int kPairBlock = 128;
constexpr int kPairMinBlocks = 4;

template <class Store>
__global__ void __launch_bounds__(kPairBlock, kPairMinBlocks) stream_collide_pair_kernel(const StepParams p) {
  const long long half_nxy = static_cast<long long>(p.g.nx / 2) * p.g.ny;
  const long long t2 = p.z0 * half_nxy + static_cast<long long>(blockIdx.x) * kPairBlock + threadIdx.x;
  if (t2 >= p.z1 * half_nxy) return;
  const int t = static_cast<int>(2 * t2);
  if (blockIdx.y == 0)
    site_pair_update<Store, 0>(p, t);
  else
    site_pair_update<Store, 1>(p, t);
}

// The paired kernel covers offset storage, series equilibrium, FP32 moments, ping-pong, nx even.
inline bool pair_kernel_applies(int fp64_moments, int eq, const StepParams& p) {
  return fp64_moments == 0 && eq == kEqSeries && p.g.nx % 2 == 0 && p.src != p.dst;
}

template <class Store>
cudaError_t launch_sc_pair(const StepParams& p, cudaStream_t s) {
  const long long n = static_cast<long long>(p.g.nx / 2) * p.g.ny * (p.z1 - p.z0);
  if (n <= 0) return cudaSuccess;
  const dim3 grid(static_cast<unsigned>((n + kPairBlock - 1) / kPairBlock), 2);
  stream_collide_pair_kernel<Store><<<grid, kPairBlock, 0, s>>>(p);
  return cudaGetLastError();
}

}  // namespace lbm
