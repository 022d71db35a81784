// Small device helpers: compile-time loops over the 81 directions / 40 pairs, polynomial
// evaluation, index wrapping, and the App. B equilibrium written once for any real type.
#pragma once

#include <cmath>
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

// ---- double-word arithmetic: a value hi + lo of two floats, |lo| <= ulp(hi) / 2 -----------------
// About 48 significant bits from FP32 operations, which this part runs some 60 times faster than
// FP64.  The building blocks are the error-free transformations TwoSum (Knuth), Fast2Sum
// (Dekker) and TwoProd through a fused multiply-add; sums, products and the reciprocal combine
// them as in the double-word algorithms analysed by Joldes, Muller and Popescu (ACM TOMS 44,
// 2017), each with a relative error of a few units of 2^-48.  The __f*_rn intrinsics keep the
// compiler from contracting or reassociating any step.
struct Dw {
  float hi, lo;
};

__device__ __forceinline__ Dw two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bv = __fsub_rn(s, a);
  return {s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bv)), __fsub_rn(b, bv))};
}

__device__ __forceinline__ Dw fast_two_sum(float a, float b) {  // needs |a| >= |b| or a = 0
  const float s = __fadd_rn(a, b);
  return {s, __fsub_rn(b, __fsub_rn(s, a))};
}

__device__ __forceinline__ Dw two_prod(float a, float b) {
  const float p = __fmul_rn(a, b);
  return {p, __fmaf_rn(a, b, -p)};
}

__device__ __forceinline__ Dw dw_add(Dw x, float y) {
  const Dw s = two_sum(x.hi, y);
  return fast_two_sum(s.hi, __fadd_rn(x.lo, s.lo));
}

__device__ __forceinline__ Dw dw_add(Dw x, Dw y) {
  const Dw s = two_sum(x.hi, y.hi), t = two_sum(x.lo, y.lo);
  const Dw v = fast_two_sum(s.hi, __fadd_rn(s.lo, t.hi));
  return fast_two_sum(v.hi, __fadd_rn(t.lo, v.lo));
}

__device__ __forceinline__ Dw dw_mul(Dw x, Dw y) {
  const Dw c = two_prod(x.hi, y.hi);
  const float cross = __fmaf_rn(x.lo, y.hi, __fmul_rn(x.hi, y.lo));
  return fast_two_sum(c.hi, __fadd_rn(c.lo, cross));
}

// 1 / y: the rounded FP32 reciprocal t, then one Newton step t + t (1 - y t) with the residual
// formed exactly enough (1 - y.hi t by TwoProd, exact by Sterbenz' lemma).
__device__ __forceinline__ Dw dw_recip(Dw y) {
  const float t = __frcp_rn(y.hi);
  const Dw p = two_prod(y.hi, t);
  const float d = __fsub_rn(__fsub_rn(1.0f, p.hi), __fmaf_rn(y.lo, t, p.lo));
  return fast_two_sum(t, __fmul_rn(d, t));
}

__device__ __forceinline__ double dw_to_double(Dw x) {
  return static_cast<double>(x.hi) + static_cast<double>(x.lo);
}

__device__ __forceinline__ float dw_to_float(Dw x) { return __fadd_rn(x.hi, x.lo); }

constexpr float kThirdHi = static_cast<float>(1.0 / 3.0);  // 1/3 as a double word
constexpr float kThirdLo = static_cast<float>(1.0 / 3.0 - static_cast<double>(kThirdHi));

// exp, log and sqrt in the arithmetic R (float or double).
template <class R>
__host__ __device__ __forceinline__ R eexp(R x) {
  if constexpr (sizeof(R) == sizeof(double)) return exp(x); else return expf(x);
}
template <class R>
__host__ __device__ __forceinline__ R elog(R x) {
  if constexpr (sizeof(R) == sizeof(double)) return log(x); else return logf(x);
}
template <class R>
__host__ __device__ __forceinline__ R esqrt(R x) {
  if constexpr (sizeof(R) == sizeof(double)) return sqrt(x); else return sqrtf(x);
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

// An = <W/rho, c_x^4> - 3 <W/rho, c_x^2 c_y^2> and Bn = <W/rho, c_x^2 c_y^2> - theta^2 (so that
// A = An / theta^2, B = Bn / theta^2 and Rb = A/5 + B).
template <class R>
__host__ __device__ __forceinline__ void eq_scalars_ab(R ux, R uy, R uz, R theta, R An, R Bn, EqScalars<R>& e) {
  const R q = ux * ux + uy * uy + uz * uz;
  const R ith = R(1) / theta;
  const R ith2 = ith * ith;
  const R ith3 = ith2 * ith;
  const R A = An * ith2;
  const R B = Bn * ith2;
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

// With the eta^4 series W~: An, Bn are quartic polynomials in eta (coefficients na, nb).
template <class R>
__host__ __device__ __forceinline__ void eq_scalars(R ux, R uy, R uz, R theta, R eta, const R* na,
                                                    const R* nb, EqScalars<R>& e) {
  eq_scalars_ab<R>(ux, uy, uz, theta, poly4(na, eta), poly4(nb, eta), e);
}

// ---- exact temperature weights (App. B, Eq. (zeroveleq)) -----------------------------------
// W_i(theta) = w_i A G^(4 c_i^2) with A = 1 / F0 and G fixed by theta' = F2 / (3 theta0 F0),
// F0 = <w, G^(4 c^2)>, F2 = <w, c^2 G^(4 c^2)> (Eq. (f0f2geqn)).  In g = 4 ln G the powers are
// exp(g c_s^2), one exponential per shell.  Newton on r(g) = F2/F0 - 3 theta (slope: the
// variance of c^2 under W, positive) from the paper's series multiplier
// g0 = 1/(2 theta0) - 1/(2 theta); stops when a step is below tol (1 + |g|).
// Shell sums of c_x^4 and c_x^2 c_y^2 give <W, c_x^4> and <W, c_x^2 c_y^2> for A and B.
template <int s>
__host__ __device__ constexpr double shell_sum_x4() {
  double a = 0;
  for (int i = 0; i < kQ; ++i)
    if (rd3q81::kDirs[i].shell == s) a += 0.0625 * rd3q81::kDirs[i].hx * rd3q81::kDirs[i].hx * rd3q81::kDirs[i].hx * rd3q81::kDirs[i].hx;
  return a;
}
template <int s>
__host__ __device__ constexpr double shell_sum_x2y2() {
  double a = 0;
  for (int i = 0; i < kQ; ++i)
    if (rd3q81::kDirs[i].shell == s) a += 0.0625 * rd3q81::kDirs[i].hx * rd3q81::kDirs[i].hx * rd3q81::kDirs[i].hy * rd3q81::kDirs[i].hy;
  return a;
}

// Per-shell factors E_s = exp(g c_s^2) / F0 (so W_s = w_s E_s), and the numerators An, Bn of
// eq_scalars_ab for these weights.  Returns false if the iteration did not settle.
template <class R>
__host__ __device__ __forceinline__ bool exact_weights(R theta, const LatticeTables& tb, R* E, R& An, R& Bn) {
  constexpr bool kDbl = sizeof(R) == sizeof(double);
  const R tol = R(kDbl ? 1e-12 : 1e-5);
  constexpr int kMaxIt = kDbl ? 20 : 8;
  const R t0 = R(rd3q81::kTheta0);
  R g = R(0.5) / t0 - R(0.5) / theta;
  bool ok = false;
  for (int it = 0; it < kMaxIt && !ok; ++it) {
    R F0 = R(0), F2 = R(0), F4 = R(0);
    static_for<kShells>([&](auto Sc) {
      constexpr int s = decltype(Sc)::value;
      constexpr double c2 = rd3q81::kShellC2[s];
      constexpr double cnt = rd3q81::kShellCount[s];
      const R ws = R(cnt) * (kDbl ? R(tb.w[s]) : R(tb.wf[s]));
      const R v = s == 0 ? ws : ws * eexp(g * R(c2));
      F0 += v;
      F2 += R(c2) * v;
      F4 += R(c2 * c2) * v;
    });
    const R m2 = F2 / F0;
    const R step = (m2 - R(3) * theta) / (F4 / F0 - m2 * m2);
    g -= step;
    ok = fabs(step) <= tol * (R(1) + fabs(g));
  }
  R F0 = R(0), Mxx = R(0), Mxy = R(0);
  static_for<kShells>([&](auto Sc) {
    constexpr int s = decltype(Sc)::value;
    constexpr double c2 = rd3q81::kShellC2[s];
    E[s] = s == 0 ? R(1) : eexp(g * R(c2));
    const R ws = kDbl ? R(tb.w[s]) : R(tb.wf[s]);
    constexpr double sx4 = shell_sum_x4<s>(), sx2y2 = shell_sum_x2y2<s>();
    constexpr double cnt = rd3q81::kShellCount[s];
    F0 += R(cnt) * ws * E[s];
    Mxx += R(sx4) * ws * E[s];
    Mxy += R(sx2y2) * ws * E[s];
  });
  const R iF0 = R(1) / F0;
#pragma unroll
  for (int s = 0; s < kShells; ++s) E[s] *= iF0;
  Mxx *= iF0;
  Mxy *= iF0;
  An = Mxx - R(3) * Mxy;
  Bn = Mxy - theta * theta;
  return ok && g == g;
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
// kExactW: the exact temperature weights W(theta) in place of the eta^4 series (returns false
// if their 1-D iteration did not settle; always true otherwise).
template <class R, bool kOverW = false, bool kExactW = false>
__host__ __device__ inline bool equilibrium_all(R rho, R ux, R uy, R uz, R theta, const LatticeTables& tab,
                                                R* feq) {
  const bool dbl = sizeof(R) == sizeof(double);
  EqScalars<R> e;
  R W[kShells];
  bool ok = true;
  if constexpr (kExactW) {
    R An, Bn;
    ok = exact_weights<R>(theta, tab, W, An, Bn);
    eq_scalars_ab<R>(ux, uy, uz, theta, An, Bn, e);
    for (int s = 0; s < kShells; ++s) W[s] *= kOverW ? rho : rho * (dbl ? R(tab.w[s]) : R(tab.wf[s]));
  } else {
    const R eta = theta / R(tab.theta0) - R(1);
    R na[5], nb[5];
    for (int k = 0; k < 5; ++k) {
      na[k] = dbl ? R(tab.na[k]) : R(tab.naf[k]);
      nb[k] = dbl ? R(tab.nb[k]) : R(tab.nbf[k]);
    }
    eq_scalars<R>(ux, uy, uz, theta, eta, na, nb, e);
    for (int s = 0; s < kShells; ++s) {
      R c[5];
      for (int k = 0; k < 5; ++k)
        c[k] = kOverW ? (dbl ? R(tab.p[s][k]) : R(tab.pf[s][k])) : (dbl ? R(tab.wp[s][k]) : R(tab.wpf[s][k]));
      W[s] = rho * poly4(c, eta);
    }
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
  return ok;
}

__host__ __device__ inline void equilibrium_f64(double rho, double ux, double uy, double uz,
                                                double theta, const LatticeTables& tab, double* feq) {
  equilibrium_all<double, false>(rho, ux, uy, uz, theta, tab, feq);
}

// ---- exact entropic equilibrium (Sec. III) --------------------------------------------
// f_i = w_i rho exp(mu + zeta.c_i + gamma c_i^2), the minimiser of H = <f, log(f/w) - 1> at the
// given conserved moments T = (rho, j_x, j_y, j_z, <f, c^2>).  The multipliers
// lam = (mu, zeta_x, zeta_y, zeta_z, gamma) follow the paper's iteration: evaluate f at the
// current guess, form the 5x5 matrix <f, phi_a phi_b> and the residual T_a - <f, phi_a>
// (phi = 1, c_x, c_y, c_z, c^2), solve for the correction (Cholesky), add it, repeat.  The
// first guess is the continuous Maxwellian's multipliers relative to w ~ exp(-c^2/(2 theta0)).
//
// Evaluation.  With E_a = exp(zeta_a / 2) and c = h / 2, exp(zeta.c_i) = prod_a E_a^(h_ia).
// The moving shells are walked in order of k, the common |h_a| of their members (1, 2, 3, 4,
// 5, 6, 8), keeping P_a = E_a^k and Q_a = E_a^-k, so six exponentials serve all 80 moving
// directions.  Over a whole shell the sums factor into C_a = P_a + Q_a and S_a = P_a - Q_a
// (a BCC shell, for instance, has sum_i exp(zeta.c_i) = C_x C_y C_z), so the 15 moments cost a
// few operations per shell; the shell factor rho w_s exp(mu + gamma c_s^2) adds one exponential
// per shell.  The result is the same sum as the direction-by-direction one, regrouped.

// Shell factor rho * ws * exp(mu + gamma c_s^2), ws = w_s (kOverW false) or 1.
template <int s, bool kOverW, class R>
__host__ __device__ __forceinline__ R entropic_shell_factor(const R* lam, R rho, const LatticeTables& tb) {
  constexpr double c2 = rd3q81::kShellC2[s];
  const R x = (s == 0) ? lam[0] : lam[0] + lam[4] * R(c2);
  if constexpr (kOverW) {
    return rho * eexp(x);
  } else {
    const R ws = sizeof(R) == sizeof(double) ? R(tb.w[s]) : R(tb.wf[s]);
    return rho * ws * eexp(x);
  }
}

// Calls fn(std::integral_constant<int, K>, P, Q) for K = 1 .. kMaxShellK, with
// P_a = E_a^K and Q_a = E_a^-K, E_a = exp(zeta_a / 2).
template <class R, class F>
__host__ __device__ __forceinline__ void axis_power_walk(const R* lam, F&& fn) {
  R E[3], Ei[3], P[3], Q[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    E[a] = eexp(R(0.5) * lam[1 + a]);
    Ei[a] = eexp(R(-0.5) * lam[1 + a]);
    P[a] = E[a];
    Q[a] = Ei[a];
  }
  static_for<rd3q81::kMaxShellK>([&](auto Kc) {
    constexpr int K = decltype(Kc)::value + 1;
    if constexpr (K > 1) {
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        P[a] *= E[a];
        Q[a] *= Ei[a];
      }
    }
    fn(std::integral_constant<int, K>{}, P, Q);
  });
}

// The 15 distinct entries of <f, phi_a phi_b> (order 00 01 02 03 04 11 12 13 14 22 23 24 33 34
// 44; <f, phi_a> = J[a] for a < 5) of f_i = w_i rho exp(lam . phi_i).
template <class R>
__host__ __device__ __forceinline__ void entropic_moment_matrix(const R* lam, R rho, const LatticeTables& tb, R* J) {
#pragma unroll
  for (int k = 0; k < 15; ++k) J[k] = R(0);
  J[0] = entropic_shell_factor<0, false>(lam, rho, tb);
  axis_power_walk<R>(lam, [&](auto Kc, const R* P, const R* Q) {
    constexpr int K = decltype(Kc)::value;
    static_for<kShells - 1>([&](auto Sc) {
      constexpr int s = decltype(Sc)::value + 1;
      constexpr rd3q81::ShellShape sh = rd3q81::shell_shape(s);
      if constexpr (sh.k == K) {
        constexpr double c2 = rd3q81::kShellC2[s];
        constexpr double hk = 0.5 * K;
        const R e = entropic_shell_factor<s, false>(lam, rho, tb);
        const R C0 = P[0] + Q[0], C1 = P[1] + Q[1], C2 = P[2] + Q[2];
        const R S0 = P[0] - Q[0], S1 = P[1] - Q[1], S2 = P[2] - Q[2];
        // Z = sum exp(zeta.c), M_a = sum c_a exp / (k/2), N_ab = sum c_a c_b exp / (k/2)^2
        R Z, M0, M1, M2, N0, N1, N2, X01 = R(0), X02 = R(0), X12 = R(0);
        if constexpr (sh.kind == 1) {          // SC: (+-k, 0, 0) and permutations
          Z = C0 + C1 + C2;
          M0 = S0; M1 = S1; M2 = S2;
          N0 = C0; N1 = C1; N2 = C2;
        } else if constexpr (sh.kind == 2) {   // FCC: (+-k, +-k, 0) and permutations
          const R Cs = C0 + C1 + C2;
          Z = C0 * C1 + C0 * C2 + C1 * C2;
          const R r0 = Cs - C0, r1 = Cs - C1, r2 = Cs - C2;
          M0 = S0 * r0; M1 = S1 * r1; M2 = S2 * r2;
          N0 = C0 * r0; N1 = C1 * r1; N2 = C2 * r2;
          X01 = S0 * S1; X02 = S0 * S2; X12 = S1 * S2;
        } else {                                // BCC: (+-k, +-k, +-k)
          const R C12 = C1 * C2;
          Z = C0 * C12;
          M0 = S0 * C12; M1 = S1 * (C0 * C2); M2 = S2 * (C0 * C1);
          N0 = Z; N1 = Z; N2 = Z;
          X01 = S0 * S1 * C2; X02 = S0 * S2 * C1; X12 = S1 * S2 * C0;
        }
        const R eZ = e * Z, eh = e * R(hk), eh2 = e * R(hk * hk);
        J[0] += eZ;
        J[4] += R(c2) * eZ;
        J[14] += R(c2 * c2) * eZ;
        const R m0 = eh * M0, m1 = eh * M1, m2 = eh * M2;
        J[1] += m0; J[2] += m1; J[3] += m2;
        J[8] += R(c2) * m0; J[11] += R(c2) * m1; J[13] += R(c2) * m2;
        J[5] += eh2 * N0; J[9] += eh2 * N1; J[12] += eh2 * N2;
        if constexpr (sh.kind > 1) {
          J[6] += eh2 * X01; J[7] += eh2 * X02; J[10] += eh2 * X12;
        }
      }
    });
  });
}

// Calls fn(pair constant P, v_plus, v_minus) for each +/- pair, with
// v = rho ws exp(lam . phi) of its +c and -c members (ws = w, or 1 with kOverW), in the order
// of the shell walk.  The rest value is entropic_shell_factor<0, kOverW>.
template <class R, bool kOverW, class F>
__host__ __device__ __forceinline__ void entropic_pair_values(const R* lam, R rho, const LatticeTables& tb, F&& fn) {
  axis_power_walk<R>(lam, [&](auto Kc, const R* P, const R* Q) {
    constexpr int K = decltype(Kc)::value;
    [[maybe_unused]] R e = R(0);
    static_for<kPairs>([&](auto Pc) {
      constexpr int Pi = decltype(Pc)::value;
      constexpr rd3q81::Dir d = rd3q81::kDirs[1 + 2 * Pi];
      if constexpr (rd3q81::shell_shape(d.shell).k == K) {
        if constexpr (Pi == 0 || rd3q81::kDirs[2 * Pi - 1].shell != d.shell)
          e = entropic_shell_factor<d.shell, kOverW>(lam, rho, tb);
        R vp = e, vm = e;
        if constexpr (d.hx > 0) { vp *= P[0]; vm *= Q[0]; }
        if constexpr (d.hx < 0) { vp *= Q[0]; vm *= P[0]; }
        if constexpr (d.hy > 0) { vp *= P[1]; vm *= Q[1]; }
        if constexpr (d.hy < 0) { vp *= Q[1]; vm *= P[1]; }
        if constexpr (d.hz > 0) { vp *= P[2]; vm *= Q[2]; }
        if constexpr (d.hz < 0) { vp *= Q[2]; vm *= P[2]; }
        fn(Pc, vp, vm);
      }
    });
  });
}

// Solves the symmetric positive definite 5x5 system J x = r in place (Cholesky); J is given
// by its 15 distinct entries in the order 00 01 02 03 04 11 12 13 14 22 23 24 33 34 44.
template <class R>
__host__ __device__ __forceinline__ bool solve_spd5(const R* Jp, R* x) {
  R a[5][5];
  int k = 0;
  for (int i = 0; i < 5; ++i)
    for (int j = i; j < 5; ++j) a[i][j] = a[j][i] = Jp[k++];
  R Lm[5][5];
  for (int j = 0; j < 5; ++j) {
    R d = a[j][j];
    for (int m = 0; m < j; ++m) d -= Lm[j][m] * Lm[j][m];
    if (!(d > R(0))) return false;
    const R ljj = esqrt(d);
    const R il = R(1) / ljj;
    Lm[j][j] = ljj;
    for (int i = j + 1; i < 5; ++i) {
      R v = a[i][j];
      for (int m = 0; m < j; ++m) v -= Lm[i][m] * Lm[j][m];
      Lm[i][j] = v * il;
    }
  }
  for (int i = 0; i < 5; ++i) {
    R v = x[i];
    for (int m = 0; m < i; ++m) v -= Lm[i][m] * x[m];
    x[i] = v / Lm[i][i];
  }
  for (int i = 4; i >= 0; --i) {
    R v = x[i];
    for (int m = i + 1; m < 5; ++m) v -= Lm[m][i] * x[m];
    x[i] = v / Lm[i][i];
  }
  return true;
}

// Newton for the multipliers.  T = conserved moments, (ux, uy, uz, theta) for the first guess.
// The callers allow 30 evaluations in FP64 and 16 in FP32: near Mach 2.6 in a cold vortex core the
// Maxwellian first guess is far from the lattice's minimiser, and 6 FP32 evaluations left a
// Mach-2 blob (128 x 32 x 4) drifting to O(1) errors within 5 steps and failing within 10; with
// 16 it stays within 5e-6 of the FP64 run.  Converged sites exit early, so the cap costs the
// others nothing.
// On return lam holds multipliers whose moments are within tol of T (relative to rho for mass
// and momentum, to <f, c^2> for energy), or the last iterate after max_it evaluations, and Jout
// (if given; element k at Jout[k * jstride]) the 15 entries of <f, phi phi^T> at lam (the last
// evaluation).
// Returns false if the iteration broke down (non-positive pivot or non-finite values).
template <class R>
__host__ __device__ __forceinline__ bool entropic_multipliers(const R* T, R ux, R uy, R uz, R theta, R tol,
                                                              int max_it, const LatticeTables& tb, R* lam,
                                                              R* Jout = nullptr, int jstride = 1) {
  const R q = ux * ux + uy * uy + uz * uz;
  const R t0 = R(rd3q81::kTheta0);
  lam[0] = R(-1.5) * elog(theta / t0) - q / (R(2) * theta);
  lam[1] = ux / theta;
  lam[2] = uy / theta;
  lam[3] = uz / theta;
  lam[4] = R(0.5) / t0 - R(0.5) / theta;
  const R rho = T[0];
  for (int it = 0;; ++it) {
    R J[15];
    entropic_moment_matrix<R>(lam, rho, tb, J);
    R r[5] = {T[0] - J[0], T[1] - J[1], T[2] - J[2], T[3] - J[3], T[4] - J[4]};
    const bool small = fabs(r[0]) <= tol * T[0] && fabs(r[1]) <= tol * T[0] && fabs(r[2]) <= tol * T[0] &&
                       fabs(r[3]) <= tol * T[0] && fabs(r[4]) <= tol * T[4];
    if (small || it + 1 >= max_it) {
      if (Jout)
        for (int k = 0; k < 15; ++k) Jout[k * jstride] = J[k];
      return small || (J[0] == J[0]);
    }
    if (!solve_spd5<R>(J, r)) {
      if (Jout)
        for (int k = 0; k < 15; ++k) Jout[k * jstride] = J[k];
      return false;
    }
    for (int k = 0; k < 5; ++k) lam[k] += r[k];
  }
}

// Full exact entropic equilibrium of one state (feq_i, or feq_i / w_i with kOverW), or false
// if the iteration broke down.
template <class R, bool kOverW = false>
__host__ __device__ inline bool entropic_all(R rho, R ux, R uy, R uz, R theta, const LatticeTables& tab, R* feq) {
  constexpr bool kDbl = sizeof(R) == sizeof(double);
  const R T[5] = {rho, rho * ux, rho * uy, rho * uz, rho * (ux * ux + uy * uy + uz * uz) + R(3) * rho * theta};
  R lam[5];
  const bool ok = entropic_multipliers<R>(T, ux, uy, uz, theta, R(kDbl ? 1e-13 : 1e-6), kDbl ? 30 : 16, tab, lam);
  feq[0] = entropic_shell_factor<0, kOverW>(lam, rho, tab);
  entropic_pair_values<R, kOverW>(lam, rho, tab, [&](auto Pc, R vp, R vm) {
    constexpr int P = decltype(Pc)::value;
    feq[1 + 2 * P] = vp;
    feq[2 + 2 * P] = vm;
  });
  return ok;
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
