// Small device helpers: compile-time loops over the 81 directions / 40 pairs, polynomial
// evaluation, index wrapping, and the App. B equilibrium written once for any real type.
#pragma once

#include <type_traits>
#include <utility>

#include "lbm_internal.h"

namespace lbm {

template <class F, int... Is>
__host__ __device__ __forceinline__ void static_for_impl(F&& f, std::integer_sequence<int, Is...>) {
  (f(std::integral_constant<int, Is>{}), ...);
}
// Calls f(std::integral_constant<int, i>) for i = 0 .. N-1; every i is a compile-time constant.
template <int N, class F>
__host__ __device__ __forceinline__ void static_for(F&& f) {
  static_for_impl(f, std::make_integer_sequence<int, N>());
}

// sum_k c[k] eta^k, k = 0..4 (Horner).
template <class R>
__host__ __device__ __forceinline__ R poly4(const R* c, R eta) {
  return c[0] + eta * (c[1] + eta * (c[2] + eta * (c[3] + eta * c[4])));
}

// Per-site scalars of the series equilibrium (App. B, f~eq with f^(2), f^(3)):
//   f~eq_i = W~_s(i) [a0_s + xi (a1_s + xi (a2 + xi a3)) + a4 psi_i],
//   xi = u.c_i, psi_i = sum_k u_k^3 c_ik, q = u^2, K = Rb / (2 + 5 Rb),
//   a0_s = 1 - q/(2 theta) - (5/6)(q/theta^2) K (c_s^2 - 3 theta),
//   a1_s = 1/theta - q/(2 theta^2) - (5/(6 theta^3)) K q (c_s^2 - 3 theta) + (5 q Rb - 3 B q)/(6 theta^2),
//   a2 = 1/(2 theta^2), a3 = 1/(6 theta^3), a4 = -A/(6 theta^2).
// This is the printed f^(2), f^(3) regrouped by powers of xi, with the cubic contraction
//   u_a u_z u_e c_ix R-bar_{x a z e} = A psi_i + 3 B q xi.
template <class R>
struct EqScalars {
  R ux, uy, uz, ux3, uy3, uz3;
  R a2, a3, a4;
  R c0, k0;  // a0_s = c0 + k0 (c_s^2 - 3 theta)
  R c1, k1;  // a1_s = c1 + k1 (c_s^2 - 3 theta)
  R t3;      // 3 theta
};

template <class R>
__host__ __device__ __forceinline__ void eq_scalars(R ux, R uy, R uz, R theta, R eta, const R* na,
                                                    const R* nb, EqScalars<R>& e) {
  const R q = ux * ux + uy * uy + uz * uz;
  const R ith = R(1) / theta;
  const R ith2 = ith * ith;
  const R ith3 = ith2 * ith;
  const R A = poly4(na, eta) * ith2;
  const R B = poly4(nb, eta) * ith2;
  const R Rb = R(0.2) * A + B;
  const R K = Rb / (R(2) + R(5) * Rb);
  e.ux = ux;
  e.uy = uy;
  e.uz = uz;
  e.ux3 = ux * ux * ux;
  e.uy3 = uy * uy * uy;
  e.uz3 = uz * uz * uz;
  e.a2 = R(0.5) * ith2;
  e.a3 = ith3 * R(1.0 / 6.0);
  e.a4 = -A * ith2 * R(1.0 / 6.0);
  e.c0 = R(1) - R(0.5) * q * ith;
  e.k0 = -R(5.0 / 6.0) * q * ith2 * K;
  e.c1 = ith - R(0.5) * q * ith2 + (R(5) * q * Rb - R(3) * B * q) * ith2 * R(1.0 / 6.0);
  e.k1 = -R(5.0 / 6.0) * ith3 * K * q;
  e.t3 = R(3) * theta;
}

// Even and odd parts (in c -> -c) of the bracket of f~eq for the +c member of pair P:
//   bracket(+c) = ev + od, bracket(-c) = ev - od.
template <int P, class R>
__host__ __device__ __forceinline__ void eq_pair_parts(const EqScalars<R>& e, R& ev, R& od) {
  constexpr rd3q81::Dir d = rd3q81::kDirs[1 + 2 * P];
  constexpr int s = d.shell;
  constexpr double c2 = rd3q81::kShellC2[s];
  R xi = R(0), psi = R(0);
  if constexpr (d.hx != 0) {
    xi = R(0.5 * d.hx) * e.ux;
    psi = R(0.5 * d.hx) * e.ux3;
  }
  if constexpr (d.hy != 0) {
    xi += R(0.5 * d.hy) * e.uy;
    psi += R(0.5 * d.hy) * e.uy3;
  }
  if constexpr (d.hz != 0) {
    xi += R(0.5 * d.hz) * e.uz;
    psi += R(0.5 * d.hz) * e.uz3;
  }
  const R dc = R(c2) - e.t3;
  const R a0 = e.c0 + e.k0 * dc;
  const R a1 = e.c1 + e.k1 * dc;
  const R xi2 = xi * xi;
  ev = a0 + e.a2 * xi2;
  od = xi * (a1 + e.a3 * xi2) + e.a4 * psi;
}

// Full equilibrium of one state in arithmetic R (float or double), feq[i] in the library's
// direction order.  With kOverW it returns feq_i / w_i instead (offset storage).
template <class R, bool kOverW = false>
__host__ __device__ inline void equilibrium_all(R rho, R ux, R uy, R uz, R theta, const LatticeTables& tab,
                                                R* feq) {
  const bool dbl = sizeof(R) == sizeof(double);
  const R eta = theta / R(tab.theta0) - R(1);
  R na[5], nb[5];
  for (int k = 0; k < 5; ++k) {
    na[k] = dbl ? R(tab.na[k]) : R(tab.naf[k]);
    nb[k] = dbl ? R(tab.nb[k]) : R(tab.nbf[k]);
  }
  EqScalars<R> e;
  eq_scalars<R>(ux, uy, uz, theta, eta, na, nb, e);
  R W[kShells];
  for (int s = 0; s < kShells; ++s) {
    R c[5];
    for (int k = 0; k < 5; ++k)
      c[k] = kOverW ? (dbl ? R(tab.p[s][k]) : R(tab.pf[s][k])) : (dbl ? R(tab.wp[s][k]) : R(tab.wpf[s][k]));
    W[s] = rho * poly4(c, eta);
  }
  // rest particle: xi = psi = 0
  feq[0] = W[0] * (e.c0 + e.k0 * (R(0) - e.t3));
  static_for<kPairs>([&](auto Pc) {
    constexpr int P = decltype(Pc)::value;
    constexpr int s = rd3q81::kDirs[1 + 2 * P].shell;
    R ev, od;
    eq_pair_parts<P, R>(e, ev, od);
    feq[1 + 2 * P] = W[s] * (ev + od);
    feq[2 + 2 * P] = W[s] * (ev - od);
  });
}

__host__ __device__ inline void equilibrium_f64(double rho, double ux, double uy, double uz,
                                                double theta, const LatticeTables& tab, double* feq) {
  equilibrium_all<double, false>(rho, ux, uy, uz, theta, tab, feq);
}

// Wrap an index displaced by at most kReach into [0, n).
__device__ __forceinline__ int wrap_idx(int a, int n) {
  if (n >= rd3q81::kReach) {
    a = a < 0 ? a + n : a;
    return a >= n ? a - n : a;
  }
  int m = a % n;
  return m < 0 ? m + n : m;
}

}  // namespace lbm
