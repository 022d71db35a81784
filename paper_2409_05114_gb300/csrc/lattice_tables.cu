// Host-side construction of the lattice constants (FP64), from Table "tab:weights" and the
// series temperature weights of App. B, Eq. (zeroveleqseries).
#include <algorithm>
#include <cstdlib>

#include "lbm_internal.h"

namespace lbm {

void build_lattice_tables(LatticeTables* t) {
  using namespace rd3q81;
  const double t0 = kTheta0;

  // Shell weights: quintic polynomials in theta0 (Horner), w_0 = 1 - sum of the others.
  double w[kShells];
  double others = 0.0;
  for (int s = 1; s < kShells; ++s) {
    const WeightPoly& wp = kWeightPoly[s];
    double acc = 0.0;
    for (int k = 5; k >= 1; --k) acc = (acc + wp.num[k]) * t0;
    w[s] = acc / wp.den;
    others += kShellCount[s] * w[s];
  }
  w[0] = 1.0 - others;

  // W~_s / (rho w_s) = 1 + eta/2 (y-3) + eta^2/8 (y^2-10y+15) + eta^3/48 (y^3-21y^2+105y-105)
  //                    + eta^4/384 (y^4-36y^3+378y^2-1260y+945),   y = c_s^2 / theta0.
  for (int s = 0; s < kShells; ++s) {
    const double y = kShellC2[s] / t0;
    const double y2 = y * y, y3 = y2 * y, y4 = y3 * y;
    t->p[s][0] = 1.0;
    t->p[s][1] = (y - 3.0) / 2.0;
    t->p[s][2] = (y2 - 10.0 * y + 15.0) / 8.0;
    t->p[s][3] = (y3 - 21.0 * y2 + 105.0 * y - 105.0) / 48.0;
    t->p[s][4] = (y4 - 36.0 * y3 + 378.0 * y2 - 1260.0 * y + 945.0) / 384.0;
    t->w[s] = w[s];
    for (int k = 0; k < 5; ++k) t->wp[s][k] = w[s] * t->p[s][k];
  }

  // Coefficients (in eta) of <W~/rho, c_x^4> and <W~/rho, c_x^2 c_y^2>, summed over the 81
  // directions, then the numerators of A and B over theta^2 = theta0^2 (1 + eta)^2.
  double mxx[5] = {0, 0, 0, 0, 0}, mxy[5] = {0, 0, 0, 0, 0};
  for (int i = 0; i < kQ; ++i) {
    const double cx = 0.5 * kDirs[i].hx, cy = 0.5 * kDirs[i].hy;
    const int s = kDirs[i].shell;
    for (int k = 0; k < 5; ++k) {
      mxx[k] += t->wp[s][k] * cx * cx * cx * cx;
      mxy[k] += t->wp[s][k] * cx * cx * cy * cy;
    }
  }
  const double th2[5] = {t0 * t0, 2.0 * t0 * t0, t0 * t0, 0.0, 0.0};
  for (int k = 0; k < 5; ++k) {
    t->nb[k] = mxy[k] - th2[k];
    t->na[k] = mxx[k] - 3.0 * mxy[k];
  }
  t->theta0 = t0;

  for (int s = 0; s < kShells; ++s) {
    t->wf[s] = static_cast<float>(t->w[s]);
    for (int k = 0; k < 5; ++k) {
      t->wpf[s][k] = static_cast<float>(t->wp[s][k]);
      t->pf[s][k] = static_cast<float>(t->p[s][k]);
    }
  }
  for (int k = 0; k < 5; ++k) {
    t->naf[k] = static_cast<float>(t->na[k]);
    t->nbf[k] = static_cast<float>(t->nb[k]);
  }
  t->theta0f = static_cast<float>(t0);
  t->theta0x3_dw[0] = static_cast<float>(3.0 * t0);
  t->theta0x3_dw[1] = static_cast<float>(3.0 * t0 - static_cast<double>(t->theta0x3_dw[0]));
  // k_s: the largest |h_a| over the shell's members (every nonzero component has it)
  int kmax[kShells] = {};
  for (int i = 1; i < kQ; ++i) {
    const int a[3] = {kDirs[i].hx, kDirs[i].hy, kDirs[i].hz};
    for (int c = 0; c < 3; ++c) kmax[kDirs[i].shell] = std::max(kmax[kDirs[i].shell], std::abs(a[c]));
  }
  auto split = [](double v, float* out) {
    out[0] = static_cast<float>(v);
    out[1] = static_cast<float>(v - static_cast<double>(out[0]));
  };
  for (int s = 0; s < kShells; ++s) {
    t->wc2f[s] = static_cast<float>(w[s] * kShellC2[s]);
    t->whkf[s] = static_cast<float>(w[s] * 0.5 * kmax[s]);
    split(w[s], t->w_dw[s]);
    split(w[s] * kShellC2[s], t->wc2_dw[s]);
    split(w[s] * 0.5 * kmax[s], t->whk_dw[s]);
  }
  for (int i = 0; i < kQ; ++i) t->wdir[i] = w[kDirs[i].shell];
  for (int i = 0; i < kQ; ++i) {
    t->opp[i] = i == 0 ? 0 : (i % 2 == 1 ? i + 1 : i - 1);
    const Dir& d = kDirs[i];
    for (int s = 0; s < 2; ++s) {
      // the site that pulls f_i from (s, n) is the source of -c_i at (s, n)
      t->push_d[s][i][0] = static_cast<signed char>(pull_disp(-d.hx, s));
      t->push_d[s][i][1] = static_cast<signed char>(pull_disp(-d.hy, s));
      t->push_d[s][i][2] = static_cast<signed char>(pull_disp(-d.hz, s));
      t->push_d[s][i][3] = static_cast<signed char>(d.hx % 2 != 0 ? 1 - s : s);
    }
  }
}

void fill_slab_bases(StepParams* p, size_t elem, int kind) {
  const char* src = static_cast<const char*>(p->src);
  char* dst = static_cast<char*>(p->dst);
  const long long e = static_cast<long long>(elem);
  p->z0 = 0;
  p->z1 = p->g.nz;
  for (int sub = 0; sub < 2; ++sub)
    for (int i = 0; i < kQ; ++i) {
      const int other = (rd3q81::kDirs[i].hx % 2 != 0) ? 1 - sub : sub;  // sublattice across link i
      const int opp = i == 0 ? 0 : (i % 2 == 1 ? i + 1 : i - 1);
      int ls = other, li = i, ss = sub, si = i;  // load sublattice / slot, store sublattice / slot
      if (kind == kStepAANeighbour) {
        li = opp;    // the neighbour left f_i in its slot of -c_i
        ss = other;  // and f_i goes to the neighbour that pulls it, slot i
      } else if (kind == kStepAAOwn) {
        ls = sub;    // own site, slot i (pushed there by the neighbour step)
        si = opp;    // own site, slot of -c_i
      }
      p->src_slab[sub][i] = src + (ls * p->g.sub_stride + li * p->g.dir_stride) * e;
      p->dst_slab[sub][i] = dst + (ss * p->g.sub_stride + si * p->g.dir_stride) * e;
    }
}

}  // namespace lbm
