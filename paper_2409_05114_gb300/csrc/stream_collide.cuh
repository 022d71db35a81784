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

// kF64Mom: the moment sums and the temperature recovery run in FP64 whatever the storage.
template <class Store, bool kF64Mom, int SUB>
__device__ __forceinline__ void site_update(const StepParams& p, int t) {
  using C = Codec<Store>;
  using R = typename C::Real;                                  // collide arithmetic
  using M = std::conditional_t<kF64Mom, double, R>;            // moment arithmetic
  const Geometry& g = p.g;

  const int x = t % g.nx;
  const int r = t / g.nx;
  const int y = r % g.ny;
  const int z = r / g.ny;

  // Source coordinates for index displacements d = -4 .. 4 (slot d + 4).
  int xs[9], ys[9], zs[9];
#pragma unroll
  for (int k = 0; k < 9; ++k) {
    const int d = k - 4;
    xs[k] = (g.x_periodic ? wrap_idx(x - d, g.nx) : x - d) + g.xoff;
    ys[k] = wrap_idx(y - d, g.ny) * g.pitch;
    zs[k] = wrap_idx(z - d, g.nz) * static_cast<int>(g.plane);
  }

  // ---- pull -----------------------------------------------------------------------------
  const Store* src = static_cast<const Store*>(p.src);
  const Store* same = src + SUB * g.sub_stride;
  const Store* other = src + (1 - SUB) * g.sub_stride;
  R f[kQ];
  static_for<kQ>([&](auto Ic) {
    constexpr int i = decltype(Ic)::value;
    constexpr rd3q81::Dir d = rd3q81::kDirs[i];
    constexpr int dx = rd3q81::pull_disp(d.hx, SUB);
    constexpr int dy = rd3q81::pull_disp(d.hy, SUB);
    constexpr int dz = rd3q81::pull_disp(d.hz, SUB);
    constexpr bool cross = (d.hx % 2) != 0;
    const Store* base = (cross ? other : same) + static_cast<long long>(i) * g.dir_stride;
    f[i] = C::load(base + (zs[dz + 4] + ys[dy + 4] + xs[dx + 4]));
  });

  // ---- moments, Eq. (conslaws) ----------------------------------------------------------
  // Offset storage holds d_i = f_i/w_i - 1, so rho = 1 + <w, d>, j = <w, d c>,
  // <f, c^2> = 3 theta0 + <w, d c^2> (the weights' own moments are 1, 0, 3 theta0).
  const LatticeTables& tb = p.tab;
  M rho, jx = M(0), jy = M(0), jz = M(0), E = M(0);
  if constexpr (C::kOffset) rho = tab_w<M>(tb, 0) * M(f[0]); else rho = M(f[0]);
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
    }
    rho += sum;
    E += M(c2) * sum;
    if constexpr (d.hx != 0) jx += M(0.5 * d.hx) * dif;
    if constexpr (d.hy != 0) jy += M(0.5 * d.hy) * dif;
    if constexpr (d.hz != 0) jz += M(0.5 * d.hz) * dif;
  });
  if constexpr (C::kOffset) {
    rho += M(1);
    E += M(3.0 * rd3q81::kTheta0);
  }
  const M irho = M(1) / rho;
  const M mux = jx * irho, muy = jy * irho, muz = jz * irho;
  const M mtheta = (E * irho - (mux * mux + muy * muy + muz * muz)) * M(1.0 / 3.0);

  const R rh = R(rho);
  const R theta = R(mtheta);
  if (!(rh > R(0) && theta > R(0) && rh < R(FLT_MAX) && theta < R(FLT_MAX))) atomicOr(p.flag, 1u);

  // ---- equilibrium scalars, App. B ------------------------------------------------------
  const R eta = theta * R(1.0 / rd3q81::kTheta0) - R(1);
  EqScalars<R> e;
  eq_scalars<R>(R(mux), R(muy), R(muz), theta, eta, tab_na<R>(tb), tab_nb<R>(tb), e);
  // W~_s / w_s for offset storage (the collide then works on d = f/w - 1), W~_s otherwise.
  R W[kShells];
#pragma unroll
  for (int s = 0; s < kShells; ++s)
    W[s] = rh * poly4(C::kOffset ? tab_p<R>(tb, s) : tab_wp<R>(tb, s), eta);

  // ---- BGK collision, Eq. (discretelbm) -------------------------------------------------
  const R om = R(p.omega);
  {
    R feq0 = W[0] * (e.c0 + e.k0 * (R(0) - e.t3));
    if constexpr (C::kOffset) feq0 -= R(1);
    f[0] += om * (feq0 - f[0]);
  }
  static_for<kPairs>([&](auto Pc) {
    constexpr int P = decltype(Pc)::value;
    constexpr int s = rd3q81::kDirs[1 + 2 * P].shell;
    R ev, od;
    eq_pair_parts<P, R>(e, ev, od);
    const R we = W[s] * ev;
    const R wo = W[s] * od;
    R fp = we + wo, fm = we - wo;
    if constexpr (C::kOffset) {
      fp -= R(1);
      fm -= R(1);
    }
    f[1 + 2 * P] += om * (fp - f[1 + 2 * P]);
    f[2 + 2 * P] += om * (fm - f[2 + 2 * P]);
  });

  // ---- store (coalesced, same site index in the other buffer) ----------------------------
  Store* dst = static_cast<Store*>(p.dst) + SUB * g.sub_stride + (zs[4] + ys[4] + xs[4]);
  static_for<kQ>([&](auto Ic) {
    constexpr int i = decltype(Ic)::value;
    C::store(dst + static_cast<long long>(i) * g.dir_stride, f[i]);
  });
}

template <class Store, bool kF64Mom>
__global__ void __launch_bounds__(kScBlock) stream_collide_kernel(const StepParams p) {
  const long long n = static_cast<long long>(p.g.nx) * p.g.ny * p.g.nz;
  const long long t = static_cast<long long>(blockIdx.x) * kScBlock + threadIdx.x;
  if (t >= n) return;
  if (blockIdx.y == 0)
    site_update<Store, kF64Mom, 0>(p, static_cast<int>(t));
  else
    site_update<Store, kF64Mom, 1>(p, static_cast<int>(t));
}

template <class Store, bool kF64Mom>
cudaError_t launch_sc(const StepParams& p, cudaStream_t s) {
  const long long n = static_cast<long long>(p.g.nx) * p.g.ny * p.g.nz;
  const dim3 grid(static_cast<unsigned>((n + kScBlock - 1) / kScBlock), 2);
  stream_collide_kernel<Store, kF64Mom><<<grid, kScBlock, 0, s>>>(p);
  return cudaGetLastError();
}

}  // namespace lbm
