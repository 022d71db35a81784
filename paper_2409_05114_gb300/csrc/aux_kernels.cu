// Auxiliary kernels around the fused step: initialisation from macroscopic fields, moment
// read-back, raw population get/set (FP64, dense layout), boundary ghost layers, and the
// deterministic global conservation sums.
#include "device_common.cuh"
#include "reduce.cuh"

namespace lbm {

namespace {

constexpr int kAuxBlock = 256;

// Element offset of interior site t (0 <= t < nx*ny*nz) of sublattice `sub`, direction 0.
__device__ __forceinline__ long long site_offset(const Geometry& g, int sub, long long t) {
  const int x = static_cast<int>(t % g.nx);
  const long long r = t / g.nx;
  const int y = static_cast<int>(r % g.ny);
  const int z = static_cast<int>(r / g.ny);
  return sub * g.sub_stride + z * g.plane + static_cast<long long>(y) * g.pitch + g.xoff + x;
}

// Element offset of population i of interior site t of sublattice sub in the stored state
// (StateLayout): own slot, the slot of -c_i (AA own), or slot i of the site that pulls it
// next (AA pushed; on a non-periodic x face that site may be a ghost).
__device__ __forceinline__ long long pop_offset(const Geometry& g, const LatticeTables& tab, int layout, int sub,
                                                long long t, int i) {
  const int x = static_cast<int>(t % g.nx);
  const long long r = t / g.nx;
  const int y = static_cast<int>(r % g.ny);
  const int z = static_cast<int>(r / g.ny);
  if (layout == kLayoutAAPushed) {
    const signed char* d = tab.push_d[sub][i];
    const int xx = g.x_periodic ? wrap_idx(x - d[0], g.nx) : x - d[0];
    const int yy = wrap_idx(y - d[1], g.ny), zz = wrap_idx(z - d[2], g.nz);
    return d[3] * g.sub_stride + zz * g.plane + static_cast<long long>(yy) * g.pitch + g.xoff + xx +
           i * g.dir_stride;
  }
  const int slot = layout == kLayoutAAOwn ? tab.opp[i] : i;
  return sub * g.sub_stride + z * g.plane + static_cast<long long>(y) * g.pitch + g.xoff + x + slot * g.dir_stride;
}

template <class S>
__device__ __forceinline__ double decode(S v, double w) {
  if constexpr (Codec<S>::kOffset) {
    return w * (1.0 + static_cast<double>(Codec<S>::load(&v)));
  } else {
    return static_cast<double>(v);
  }
}

template <class S>
__device__ __forceinline__ void encode(S* p, double f, double w) {
  if constexpr (Codec<S>::kOffset) {
    Codec<S>::store(p, static_cast<float>(f / w - 1.0));
  } else {
    *p = static_cast<S>(f);
  }
}

template <class S, int kEq>
__global__ void init_kernel(Geometry g, LatticeTables tab, S* buf, const double* rho, const double* u,
                            const double* theta, long long first, long long count, long long us,
                            unsigned int* flag, int own_slots) {
  const long long k = static_cast<long long>(blockIdx.x) * kAuxBlock + threadIdx.x;
  if (k >= count) return;
  const long long n = static_cast<long long>(g.nx) * g.ny * g.nz;
  const long long gs = first + k;
  const int sub = gs >= n ? 1 : 0;
  const long long off = site_offset(g, sub, gs - sub * n);
  // The equilibrium is evaluated in the arithmetic the step kernel uses for this storage:
  // FP64 for FP64 populations, FP32 otherwise (offset storage directly as feq/w - 1).
  using R = typename Codec<S>::Real;
  auto put = [&](int i, R v) {
    const int io = i == 0 ? 0 : (i % 2 == 1 ? i + 1 : i - 1);
    S* q = buf + off + (own_slots ? io : i) * g.dir_stride;  // AA keeps f_i in the slot of -c_i
    if constexpr (Codec<S>::kOffset)
      Codec<S>::store(q, v - R(1));
    else
      Codec<S>::store(q, v);
  };
  if constexpr (kEq == 0) {
    // The series equilibrium of equilibrium_all, with each pair stored as soon as it is
    // evaluated: no array of 81 values stays live, so more warps fit on an SM.
    constexpr bool kOverW = Codec<S>::kOffset;
    constexpr bool dbl = std::is_same_v<R, double>;
    const R rr = R(rho[k]), th = R(theta[k]);
    const R eta = th / R(tab.theta0) - R(1);
    R na[5], nb[5];
    for (int j = 0; j < 5; ++j) {
      na[j] = dbl ? R(tab.na[j]) : R(tab.naf[j]);
      nb[j] = dbl ? R(tab.nb[j]) : R(tab.nbf[j]);
    }
    EqScalars<R> e;
    eq_scalars<R>(R(u[k]), R(u[us + k]), R(u[2 * us + k]), th, eta, na, nb, e);
    R W[kShells];
    for (int sh = 0; sh < kShells; ++sh) {
      R c[5];
      for (int j = 0; j < 5; ++j)
        c[j] = kOverW ? (dbl ? R(tab.p[sh][j]) : R(tab.pf[sh][j])) : (dbl ? R(tab.wp[sh][j]) : R(tab.wpf[sh][j]));
      W[sh] = rr * poly4(c, eta);
    }
    put(0, W[0] * (e.c0 + e.k0 * (R(0) - e.t3)));
    static_for<kPairs>([&](auto Pc) {
      constexpr int P = decltype(Pc)::value;
      constexpr int sh = rd3q81::kDirs[1 + 2 * P].shell;
      R ev, od;
      eq_pair_parts<P, R>(e, ev, od);
      put(1 + 2 * P, W[sh] * (ev + od));
      put(2 + 2 * P, W[sh] * (ev - od));
    });
    return;
  }
  R feq[kQ];
  if constexpr (kEq == 2) {
    if (!equilibrium_all<R, Codec<S>::kOffset, true>(R(rho[k]), R(u[k]), R(u[us + k]), R(u[2 * us + k]),
                                                     R(theta[k]), tab, feq))
      atomicOr(flag, 1u);
  } else {
    if (!entropic_all<R, Codec<S>::kOffset>(R(rho[k]), R(u[k]), R(u[us + k]), R(u[2 * us + k]), R(theta[k]), tab,
                                            feq))
      atomicOr(flag, 1u);
  }
  static_for<kQ>([&](auto Ic) { put(decltype(Ic)::value, feq[decltype(Ic)::value]); });
}

// Moments of the stored populations (Eq. (conslaws)), returned in FP64; for offset storage
// as deviations from the weights' own moments (1, 0, 3 theta0).  Every storage type is summed
// in FP64 (shell by shell, then the 11 shell sums): the stored values are exact in FP64, so
// the result carries FP64 rounding only.  Used by the conservation totals (a diagnostic, off
// the step) and by the FP64-storage read-back; the other read-backs use site_moments_dw.
template <class S>
__device__ __forceinline__ void site_moments(const Geometry& g, const LatticeTables& tab, const S* buf, int layout,
                                             int sub, long long t, double& rho, double& jx, double& jy,
                                             double& jz, double& e) {
  const long long off = site_offset(g, sub, t);
  using R = typename Codec<S>::Real;
  R fv[kQ];
  if (layout == kLayoutPlain) {
    static_for<kQ>([&](auto Ic) {
      constexpr int i = decltype(Ic)::value;
      fv[i] = Codec<S>::load(buf + off + i * g.dir_stride);
    });
  } else {
    static_for<kQ>([&](auto Ic) {
      constexpr int i = decltype(Ic)::value;
      fv[i] = Codec<S>::load(buf + pop_offset(g, tab, layout, sub, t, i));
    });
  }
  double sr[kShells], sx[kShells], sy[kShells], sz[kShells];
#pragma unroll
  for (int s = 0; s < kShells; ++s) sr[s] = sx[s] = sy[s] = sz[s] = 0.0;
  static_for<kQ>([&](auto Ic) {
    constexpr int i = decltype(Ic)::value;
    constexpr rd3q81::Dir d = rd3q81::kDirs[i];
    const double f = static_cast<double>(fv[i]);
    sr[d.shell] += f;
    if constexpr (d.hx != 0) sx[d.shell] += 0.5 * d.hx * f;
    if constexpr (d.hy != 0) sy[d.shell] += 0.5 * d.hy * f;
    if constexpr (d.hz != 0) sz[d.shell] += 0.5 * d.hz * f;
  });
  rho = jx = jy = jz = e = 0.0;
  static_for<kShells>([&](auto Sc) {
    constexpr int s = decltype(Sc)::value;
    constexpr double c2 = rd3q81::kShellC2[s];
    const double ws = Codec<S>::kOffset ? tab.w[s] : 1.0;
    rho += ws * sr[s];
    e += ws * c2 * sr[s];
    jx += ws * sx[s];
    jy += ws * sy[s];
    jz += ws * sz[s];
  });
  if constexpr (Codec<S>::kOffset) {
    rho += 1.0;
    e += 3.0 * tab.theta0;
  }
}

// Moments of one site of FP32 / FP16 / BF16 storage as double words.  The shell sums are FP32 as
// in site_moments; FP32 populations are then combined shell by shell in double words.  Offset
// storage combines the weighted offset sums (deviations from the weights' moments, small) in
// FP32 and adds the reference 1 and 3 theta0 in double words.
template <class S>
__device__ __forceinline__ void site_moments_dw(const Geometry& g, const LatticeTables& tab, const S* buf,
                                                int layout, int sub, long long t, Dw& rho, Dw& jx, Dw& jy, Dw& jz,
                                                Dw& e) {
  const long long off = site_offset(g, sub, t);
  // all 81 loads first, in one branch-free run per layout: the site waits on one round trip
  // to memory, not 81
  float fv[kQ];
  if (layout == kLayoutPlain) {
    static_for<kQ>([&](auto Ic) {
      constexpr int i = decltype(Ic)::value;
      fv[i] = Codec<S>::load(buf + off + i * g.dir_stride);
    });
  } else {
    static_for<kQ>([&](auto Ic) {
      constexpr int i = decltype(Ic)::value;
      fv[i] = Codec<S>::load(buf + pop_offset(g, tab, layout, sub, t, i));
    });
  }
  float sr[kShells], sx[kShells], sy[kShells], sz[kShells];
#pragma unroll
  for (int s = 0; s < kShells; ++s) sr[s] = sx[s] = sy[s] = sz[s] = 0.0f;
  static_for<kQ>([&](auto Ic) {
    constexpr int i = decltype(Ic)::value;
    constexpr rd3q81::Dir d = rd3q81::kDirs[i];
    const float f = fv[i];
    sr[d.shell] += f;
    if constexpr (d.hx != 0) sx[d.shell] += 0.5f * d.hx * f;
    if constexpr (d.hy != 0) sy[d.shell] += 0.5f * d.hy * f;
    if constexpr (d.hz != 0) sz[d.shell] += 0.5f * d.hz * f;
  });
  if constexpr (Codec<S>::kOffset) {
    float dr = 0.0f, dx = 0.0f, dy = 0.0f, dz = 0.0f, de = 0.0f;
    static_for<kShells>([&](auto Sc) {
      constexpr int s = decltype(Sc)::value;
      constexpr float c2 = static_cast<float>(rd3q81::kShellC2[s]);
      const float w = tab.wf[s];
      dr = fmaf(w, sr[s], dr);
      dx = fmaf(w, sx[s], dx);
      dy = fmaf(w, sy[s], dy);
      dz = fmaf(w, sz[s], dz);
      de = fmaf(w * c2, sr[s], de);
    });
    rho = two_sum(1.0f, dr);
    jx = {dx, 0.0f};
    jy = {dy, 0.0f};
    jz = {dz, 0.0f};
    e = dw_add(Dw{tab.theta0x3_dw[0], tab.theta0x3_dw[1]}, de);
  } else {
    // Cascaded sums (Sum2 and Dot2 of Ogita, Rump and Oishi, SIAM J. Sci. Comput. 26, 2005):
    // the running sum stays one float and the rounding error of every addition (TwoSum) and
    // product (TwoProd) collects in a second float; the pair is as accurate as a sum in twice
    // the working precision, at about half the operations of a renormalised double-word sum.
    float pr = sr[0], px = 0.0f, py = 0.0f, pz = 0.0f, pe = 0.0f;
    float qr = 0.0f, qx = 0.0f, qy = 0.0f, qz = 0.0f, qe = 0.0f;
    static_for<kShells - 1>([&](auto Sc) {
      constexpr int s = decltype(Sc)::value + 1;
      constexpr float c2 = static_cast<float>(rd3q81::kShellC2[s]);  // multiples of 1/4: exact
      Dw t = two_sum(pr, sr[s]);
      pr = t.hi;
      qr = __fadd_rn(qr, t.lo);
      t = two_sum(px, sx[s]);
      px = t.hi;
      qx = __fadd_rn(qx, t.lo);
      t = two_sum(py, sy[s]);
      py = t.hi;
      qy = __fadd_rn(qy, t.lo);
      t = two_sum(pz, sz[s]);
      pz = t.hi;
      qz = __fadd_rn(qz, t.lo);
      const Dw h = two_prod(c2, sr[s]);
      t = two_sum(pe, h.hi);
      pe = t.hi;
      qe = __fadd_rn(qe, __fadd_rn(t.lo, h.lo));
    });
    rho = fast_two_sum(pr, qr);
    jx = two_sum(px, qx);  // momenta may cancel to below their error term
    jy = two_sum(py, qy);
    jz = two_sum(pz, qz);
    e = fast_two_sum(pe, qe);
  }
}

// rho, u = j / rho and theta = (e / rho - u.u) / 3 per site (Eq. (conslaws)), returned in FP64.
// FP64 storage sums and divides in FP64.  The narrower storage types carry the shell sums'
// FP32 rounding and otherwise double-word accuracy (relative ~1e-14 beyond the shell sums),
// with 15 FP64 operations a site (the final conversions), not the ~250 of an FP64 combination.
template <class S>
__global__ void moments_kernel(Geometry g, LatticeTables tab, const S* buf, int layout, double* rho, double* u,
                               double* theta, long long first, long long count, long long us) {
  const long long k = static_cast<long long>(blockIdx.x) * kAuxBlock + threadIdx.x;
  if (k >= count) return;
  const long long n = static_cast<long long>(g.nx) * g.ny * g.nz;
  const long long gs = first + k;
  const int sub = gs >= n ? 1 : 0;
  if constexpr (std::is_same_v<S, double>) {
    double r, jx, jy, jz, e;
    site_moments<S>(g, tab, buf, layout, sub, gs - sub * n, r, jx, jy, jz, e);
    const double ux = jx / r, uy = jy / r, uz = jz / r;
    rho[k] = r;
    u[k] = ux;
    u[us + k] = uy;
    u[2 * us + k] = uz;
    theta[k] = (e / r - (ux * ux + uy * uy + uz * uz)) / 3.0;
  } else {
    Dw r, jx, jy, jz, e;
    site_moments_dw<S>(g, tab, buf, layout, sub, gs - sub * n, r, jx, jy, jz, e);
    const Dw inv = dw_recip(r);
    const Dw ux = dw_mul(jx, inv), uy = dw_mul(jy, inv), uz = dw_mul(jz, inv);
    const Dw u2 = dw_add(dw_add(dw_mul(ux, ux), dw_mul(uy, uy)), dw_mul(uz, uz));
    const Dw th3 = dw_add(dw_mul(e, inv), Dw{-u2.hi, -u2.lo});
    rho[k] = dw_to_double(r);
    u[k] = dw_to_double(ux);
    u[us + k] = dw_to_double(uy);
    u[2 * us + k] = dw_to_double(uz);
    theta[k] = dw_to_double(dw_mul(th3, Dw{kThirdHi, kThirdLo}));
  }
}

// Dense FP64 layout f[sub][i][z][y][x] <-> padded storage.
// Dense element k = (sub*81 + i)*n + t; the kernels handle k in [first, first + count)
// with f pointing at element `first`.
template <class S>
__global__ void get_pop_kernel(Geometry g, LatticeTables tab, const S* buf, int layout, double* f, long long first,
                               long long count) {
  const long long n = static_cast<long long>(g.nx) * g.ny * g.nz;
  const long long j = static_cast<long long>(blockIdx.x) * kAuxBlock + threadIdx.x;
  if (j >= count) return;
  const long long k = first + j;
  const long long t = k % n;
  const int i = static_cast<int>((k / n) % kQ);
  const int sub = static_cast<int>(k / (n * kQ));
  f[j] = decode<S>(buf[pop_offset(g, tab, layout, sub, t, i)], tab.wdir[i]);
}

template <class S>
__global__ void set_pop_kernel(Geometry g, LatticeTables tab, S* buf, int layout, const double* f, long long first,
                               long long count) {
  const long long n = static_cast<long long>(g.nx) * g.ny * g.nz;
  const long long j = static_cast<long long>(blockIdx.x) * kAuxBlock + threadIdx.x;
  if (j >= count) return;
  const long long k = first + j;
  const long long t = k % n;
  const int i = static_cast<int>((k / n) % kQ);
  const int sub = static_cast<int>(k / (n * kQ));
  encode<S>(buf + pop_offset(g, tab, layout, sub, t, i), f[j], tab.wdir[i]);
}

// Populations of selected sites: thread per (sample, direction).
template <class S>
__global__ void probe_kernel(Geometry g, LatticeTables tab, const S* buf, int layout, const long long* sites,
                             long long count, double* f) {
  const long long n = static_cast<long long>(g.nx) * g.ny * g.nz;
  const long long j = static_cast<long long>(blockIdx.x) * kAuxBlock + threadIdx.x;
  if (j >= count * kQ) return;
  const long long k = j / kQ;
  const int i = static_cast<int>(j % kQ);
  const long long gs = sites[k];
  const int sub = gs >= n ? 1 : 0;
  f[j] = decode<S>(buf[pop_offset(g, tab, layout, sub, gs - sub * n, i)], tab.wdir[i]);
}

// Ghost layers of one x face: thread per (sub, i, z, y) row.  Zero gradient copies the
// nearest interior site of the same sublattice into all kReach layers; inflow writes feq.
template <class S>
__global__ void zero_gradient_kernel(Geometry g, S* buf, int face, int z0, int nzr) {
  const long long rows = 2LL * kQ * nzr * g.ny;
  const long long k = static_cast<long long>(blockIdx.x) * kAuxBlock + threadIdx.x;
  if (k >= rows) return;
  const int y = static_cast<int>(k % g.ny);
  const long long r = k / g.ny;
  const int z = z0 + static_cast<int>(r % nzr);
  const long long si = r / nzr;  // sub * kQ + i
  const long long row = (si / kQ) * g.sub_stride + (si % kQ) * g.dir_stride + z * g.plane +
                        static_cast<long long>(y) * g.pitch;
  if (face == 0) {
    const S v = buf[row + g.xoff];
    for (int l = 1; l <= rd3q81::kReach; ++l) buf[row + g.xoff - l] = v;
  } else {
    const S v = buf[row + g.xoff + g.nx - 1];
    for (int l = 0; l < rd3q81::kReach; ++l) buf[row + g.xoff + g.nx + l] = v;
  }
}

template <class S>
__global__ void inflow_kernel(Geometry g, LatticeTables tab, S* buf, int face, Feq81 feq) {
  const long long rows = 2LL * kQ * g.nz * g.ny;
  const long long k = static_cast<long long>(blockIdx.x) * kAuxBlock + threadIdx.x;
  if (k >= rows) return;
  const int y = static_cast<int>(k % g.ny);
  const long long r = k / g.ny;
  const int z = static_cast<int>(r % g.nz);
  const long long si = r / g.nz;
  const int i = static_cast<int>(si % kQ);
  const long long row = (si / kQ) * g.sub_stride + i * g.dir_stride + z * g.plane +
                        static_cast<long long>(y) * g.pitch;
  const long long x0 = face == 0 ? g.xoff - rd3q81::kReach : g.xoff + g.nx;
  for (int l = 0; l < rd3q81::kReach; ++l) encode<S>(buf + row + x0 + l, feq.v[i], tab.wdir[i]);
}

// Bounce-back wall on one x face (LBM_BC_BOUNCE_BACK), thread per (sub, i, z, y) ghost row, z in
// [z0, z0 + nzr).  Ghost (s', g) of direction i is pulled by exactly one site p = (push_d[s'][i][3],
// g - push_d[s'][i][0..2]).  Where p is a fluid site (0 <= x < nx), the link p -> g leaves the
// fluid, and the wall returns p's own population of the opposite direction to p:
//   mode 0 (ping-pong, before a step):        ghost slot i      <- p slot opp(i);
//   mode 1 (AA own layout, before a neighbour step, which reads ghost slot opp(i) for f_i):
//                                             ghost slot opp(i) <- p slot i (= f*_opp(i) of p);
//   mode 2 (AA, after that neighbour step, which pushed f*_opp(i) of p into ghost slot opp(i)):
//                                             p slot i          <- ghost slot opp(i).
// A ghost row writes only ghost elements (modes 0, 1) or only the (p, i) slots that no neighbour
// step wrote (mode 2); each such element belongs to one thread.  Offset storage copies the stored
// offsets: i and opp(i) share their weight.
template <class S>
__global__ void bounce_back_kernel(Geometry g, LatticeTables tab, S* buf, int face, int mode, int z0, int nzr) {
  const long long rows = 2LL * kQ * nzr * g.ny;
  const long long k = static_cast<long long>(blockIdx.x) * kAuxBlock + threadIdx.x;
  if (k >= rows) return;
  const int y = static_cast<int>(k % g.ny);
  const long long r = k / g.ny;
  const int z = z0 + static_cast<int>(r % nzr);
  const long long si = r / nzr;
  const int sub = static_cast<int>(si / kQ), i = static_cast<int>(si % kQ);
  const signed char* d = tab.push_d[sub][i];
  const int py = wrap_idx(y - d[1], g.ny), pz = wrap_idx(z - d[2], g.nz);
  const long long grow = sub * g.sub_stride + z * g.plane + static_cast<long long>(y) * g.pitch + g.xoff;
  const long long prow = d[3] * g.sub_stride + pz * g.plane + static_cast<long long>(py) * g.pitch + g.xoff;
  const long long si_i = i * g.dir_stride, si_o = tab.opp[i] * g.dir_stride;
  for (int l = 0; l < rd3q81::kReach; ++l) {
    const int gx = face == 0 ? -1 - l : g.nx + l;
    const int px = gx - d[0];
    if (px < 0 || px >= g.nx) continue;
    if (mode == 0)
      buf[grow + si_i + gx] = buf[prow + si_o + px];
    else if (mode == 1)
      buf[grow + si_o + gx] = buf[prow + si_i + px];
    else
      buf[prow + si_i + px] = buf[grow + si_o + gx];
  }
}

// AA streaming, after a neighbour step: the populations a ghost site of this x face would have
// pushed into the interior (the neighbour step runs on interior sites only).  Thread per
// (sub, z, y, ghost layer).  Zero gradient: the ghost holds the nearest interior site's
// post-collision populations, which that site pushed to the same relative place; inflow: feq.
template <class S>
__global__ void aa_ghost_push_kernel(Geometry g, LatticeTables tab, S* buf, int face, int zero_grad, Feq81 feq) {
  const long long cols = 2LL * g.nz * g.ny * rd3q81::kReach;
  const long long k = static_cast<long long>(blockIdx.x) * kAuxBlock + threadIdx.x;
  if (k >= cols) return;
  const int l = static_cast<int>(k % rd3q81::kReach);
  long long r = k / rd3q81::kReach;
  const int y = static_cast<int>(r % g.ny);
  r /= g.ny;
  const int z = static_cast<int>(r % g.nz);
  const int sub = static_cast<int>(r / g.nz);
  const int gx = face == 0 ? -1 - l : g.nx + l;
  const int xn = face == 0 ? 0 : g.nx - 1;
  static_for<kQ>([&](auto Ic) {
    constexpr int i = decltype(Ic)::value;
    constexpr rd3q81::Dir d = rd3q81::kDirs[i];
    if constexpr (d.hx != 0) {
      if ((face == 0) == (d.hx > 0)) {  // enters the interior through this face
        const int pdx = sub == 0 ? rd3q81::pull_disp(-d.hx, 0) : rd3q81::pull_disp(-d.hx, 1);
        const int pdy = sub == 0 ? rd3q81::pull_disp(-d.hy, 0) : rd3q81::pull_disp(-d.hy, 1);
        const int pdz = sub == 0 ? rd3q81::pull_disp(-d.hz, 0) : rd3q81::pull_disp(-d.hz, 1);
        const int to = (d.hx % 2 != 0) ? 1 - sub : sub;
        const int tx = gx - pdx;
        if (tx >= 0 && tx < g.nx) {
          const int ty = wrap_idx(y - pdy, g.ny), tz = wrap_idx(z - pdz, g.nz);
          const long long base = to * g.sub_stride + tz * g.plane + static_cast<long long>(ty) * g.pitch + g.xoff +
                                 i * g.dir_stride;
          if (zero_grad)
            buf[base + tx] = buf[base + (xn - pdx)];
          else
            encode<S>(buf + base + tx, feq.v[i], tab.wdir[i]);
        }
      }
    }
  });
}

// Global sums (rho, j_x, j_y, j_z, <f, c^2>) over all sites.  Pass 1: per-block partials
// (fixed grid, fixed per-thread order, then warp-shuffle trees); pass 2: one warp sums them
// (fixed lane striding, then a shuffle tree), so the result is bitwise reproducible.
template <class S>
__global__ void totals_pass1(Geometry g, LatticeTables tab, const S* buf, int layout, double* partials) {
  const long long n = static_cast<long long>(g.nx) * g.ny * g.nz;
  double acc[5] = {0, 0, 0, 0, 0};
  for (long long k = static_cast<long long>(blockIdx.x) * kAuxBlock + threadIdx.x; k < 2 * n;
       k += static_cast<long long>(gridDim.x) * kAuxBlock) {
    const int sub = k >= n ? 1 : 0;
    double r, jx, jy, jz, e;
    site_moments<S>(g, tab, buf, layout, sub, k - sub * n, r, jx, jy, jz, e);
    acc[0] += r;
    acc[1] += jx;
    acc[2] += jy;
    acc[3] += jz;
    acc[4] += e;
  }
  block_sum5_fixed<kAuxBlock>(acc);
  if (threadIdx.x == 0)
    for (int q = 0; q < 5; ++q) partials[blockIdx.x * 5 + q] = acc[q];
}

// one warp
__global__ void totals_pass2(const double* partials, int nblocks, double* out) {
  warp_total5_fixed(partials, nblocks, out);
}

unsigned blocks_for(long long n) { return static_cast<unsigned>((n + kAuxBlock - 1) / kAuxBlock); }

}  // namespace

#define LBM_STORAGE_DISPATCH(storage, BODY)            \
  switch (storage) {                                   \
    case kF64: { using S = double; BODY; } break;      \
    case kF32: { using S = float; BODY; } break;       \
    case kF16Off: { using S = __half; BODY; } break;   \
    case kBF16Off: { using S = __nv_bfloat16; BODY; } break; \
    default: return cudaErrorInvalidValue;             \
  }

cudaError_t launch_init(int storage, int eq, const Geometry& g, const LatticeTables& tab, void* buf,
                        const double* rho, const double* u, const double* theta,
                        long long first_site, long long count, long long u_stride, cudaStream_t s,
                        unsigned int* flag, int own_slots) {
  if (count <= 0) return cudaSuccess;
  if (eq == 1) {
    LBM_STORAGE_DISPATCH(storage, (init_kernel<S, 1><<<blocks_for(count), kAuxBlock, 0, s>>>(
                                      g, tab, static_cast<S*>(buf), rho, u, theta, first_site, count, u_stride, flag,
                                      own_slots)));
  } else if (eq == 2) {
    LBM_STORAGE_DISPATCH(storage, (init_kernel<S, 2><<<blocks_for(count), kAuxBlock, 0, s>>>(
                                      g, tab, static_cast<S*>(buf), rho, u, theta, first_site, count, u_stride, flag,
                                      own_slots)));
  } else {
    LBM_STORAGE_DISPATCH(storage, (init_kernel<S, 0><<<blocks_for(count), kAuxBlock, 0, s>>>(
                                      g, tab, static_cast<S*>(buf), rho, u, theta, first_site, count, u_stride, flag,
                                      own_slots)));
  }
  return cudaGetLastError();
}

cudaError_t launch_moments(int storage, const Geometry& g, const LatticeTables& tab, const void* buf,
                           double* rho, double* u, double* theta, long long first_site,
                           long long count, long long u_stride, cudaStream_t s, int layout) {
  if (count <= 0) return cudaSuccess;
  LBM_STORAGE_DISPATCH(storage, (moments_kernel<S><<<blocks_for(count), kAuxBlock, 0, s>>>(
                                    g, tab, static_cast<const S*>(buf), layout, rho, u, theta, first_site, count,
                                    u_stride)));
  return cudaGetLastError();
}

cudaError_t launch_get_populations(int storage, const Geometry& g, const LatticeTables& tab,
                                   const void* buf, double* f, long long first, long long count,
                                   cudaStream_t s, int layout) {
  if (count <= 0) return cudaSuccess;
  LBM_STORAGE_DISPATCH(storage, (get_pop_kernel<S><<<blocks_for(count), kAuxBlock, 0, s>>>(
                                    g, tab, static_cast<const S*>(buf), layout, f, first, count)));
  return cudaGetLastError();
}

cudaError_t launch_set_populations(int storage, const Geometry& g, const LatticeTables& tab, void* buf,
                                   const double* f, long long first, long long count, cudaStream_t s,
                                   int layout) {
  if (count <= 0) return cudaSuccess;
  LBM_STORAGE_DISPATCH(storage, (set_pop_kernel<S><<<blocks_for(count), kAuxBlock, 0, s>>>(
                                    g, tab, static_cast<S*>(buf), layout, f, first, count)));
  return cudaGetLastError();
}

cudaError_t launch_fill_zero_gradient(int storage, const Geometry& g, void* buf, int face, cudaStream_t s,
                                      int z0, int z1) {
  if (z1 < 0) z1 = g.nz;
  if (z0 < 0 || z1 > g.nz) return cudaErrorInvalidValue;
  if (z1 <= z0) return cudaSuccess;
  const long long rows = 2LL * kQ * (z1 - z0) * g.ny;
  LBM_STORAGE_DISPATCH(storage, (zero_gradient_kernel<S><<<blocks_for(rows), kAuxBlock, 0, s>>>(
                                    g, static_cast<S*>(buf), face, z0, z1 - z0)));
  return cudaGetLastError();
}

cudaError_t launch_bounce_back(int storage, const Geometry& g, const LatticeTables& tab, void* buf, int face,
                               int mode, cudaStream_t s, int z0, int z1) {
  if (z1 < 0) z1 = g.nz;
  if (z0 < 0 || z1 > g.nz || mode < 0 || mode > 2) return cudaErrorInvalidValue;
  if (z1 <= z0) return cudaSuccess;
  const long long rows = 2LL * kQ * (z1 - z0) * g.ny;
  LBM_STORAGE_DISPATCH(storage, (bounce_back_kernel<S><<<blocks_for(rows), kAuxBlock, 0, s>>>(
                                    g, tab, static_cast<S*>(buf), face, mode, z0, z1 - z0)));
  return cudaGetLastError();
}

cudaError_t launch_fill_inflow(int storage, const Geometry& g, const LatticeTables& tab, void* buf,
                               int face, const Feq81& feq, cudaStream_t s) {
  const long long rows = 2LL * kQ * g.nz * g.ny;
  LBM_STORAGE_DISPATCH(storage, (inflow_kernel<S><<<blocks_for(rows), kAuxBlock, 0, s>>>(
                                    g, tab, static_cast<S*>(buf), face, feq)));
  return cudaGetLastError();
}

cudaError_t launch_probe(int storage, const Geometry& g, const LatticeTables& tab, const void* buf,
                         const long long* sites, long long count, double* f, cudaStream_t s, int layout) {
  if (count <= 0) return cudaSuccess;
  LBM_STORAGE_DISPATCH(storage, (probe_kernel<S><<<blocks_for(count * kQ), kAuxBlock, 0, s>>>(
                                    g, tab, static_cast<const S*>(buf), layout, sites, count, f)));
  return cudaGetLastError();
}

int totals_blocks(const Geometry& g) {
  const long long n = 2LL * g.nx * g.ny * g.nz;
  const long long b = (n + kAuxBlock - 1) / kAuxBlock;
  return static_cast<int>(b < 1024 ? b : 1024);
}

cudaError_t launch_totals(int storage, const Geometry& g, const LatticeTables& tab, const void* buf,
                          double* partials, int nblocks, double* out5, cudaStream_t s, int layout) {
  LBM_STORAGE_DISPATCH(storage, (totals_pass1<S><<<nblocks, kAuxBlock, 0, s>>>(
                                    g, tab, static_cast<const S*>(buf), layout, partials)));
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  totals_pass2<<<1, 32, 0, s>>>(partials, nblocks, out5);
  return cudaGetLastError();
}

cudaError_t launch_aa_ghost_push(int storage, const Geometry& g, const LatticeTables& tab, void* buf, int face,
                                 int zero_grad, const Feq81& feq, cudaStream_t s) {
  const long long cols = 2LL * g.nz * g.ny * rd3q81::kReach;
  LBM_STORAGE_DISPATCH(storage, (aa_ghost_push_kernel<S><<<blocks_for(cols), kAuxBlock, 0, s>>>(
                                    g, tab, static_cast<S*>(buf), face, zero_grad, feq)));
  return cudaGetLastError();
}

cudaError_t launch_stream_collide(int storage, int fp64_moments, int eq, int kind, const StepParams& p,
                                  cudaStream_t s) {
  if (p.z0 < 0 || p.z1 > p.g.nz) return cudaErrorInvalidValue;
  if (kind != kStepPingPong) {
    if (fp64_moments && eq != kEqSeries) return cudaErrorInvalidValue;
    switch (storage) {
      case kF64: return launch_sc_aa_f64(fp64_moments, eq, kind, p, s);
      case kF32: return launch_sc_aa_f32(fp64_moments, eq, kind, p, s);
      case kF16Off: return launch_sc_aa_f16(fp64_moments, eq, kind, p, s);
      case kBF16Off: return launch_sc_aa_bf16(fp64_moments, eq, kind, p, s);
      default: return cudaErrorInvalidValue;
    }
  }
  switch (storage) {
    case kF64: return launch_sc_f64(fp64_moments, eq, p, s);
    case kF32: return launch_sc_f32(fp64_moments, eq, p, s);
    case kF16Off: return launch_sc_f16(fp64_moments, eq, p, s);
    case kBF16Off: return launch_sc_bf16(fp64_moments, eq, p, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace lbm
