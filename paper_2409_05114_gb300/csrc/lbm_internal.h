// Internal declarations shared by the kernels and the C-ABI layer of liblbm_rd3q81.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <string>

#include "lbm.h"
#include "rd3q81.h"

namespace lbm {

using rd3q81::kPairs;
using rd3q81::kQ;
using rd3q81::kShells;

// Lattice constants derived on the host in FP64 from Table "tab:weights" and App. B, passed
// to every kernel by value (they live in the kernel-parameter constant bank).
//
//   W~_s(theta) / rho      = sum_k wp[s][k] eta^k          (App. B, Eq. (zeroveleqseries))
//   W~_s(theta) / (rho w_s) = sum_k p[s][k] eta^k
//   A = (sum_k na[k] eta^k) / theta^2,  B = (sum_k nb[k] eta^k) / theta^2,  R-bar = A/5 + B
//
// where the cubic-symmetric R-bar tensor of App. B is written as
//   R-bar_{k a z e} = A delta_{kaze} + B Delta_{kaze}
// (delta_{kaze} = 1 iff all four indices agree, Delta = the isotropic 4th-order tensor), so
//   B = <W~/rho, c_x^2 c_y^2>/theta^2 - 1,   A = <W~/rho, c_x^4>/theta^2 - 3 - 3B,
// and R-bar = <W~/rho, c^4>/(15 theta^2) - 1 = A/5 + B because <c^4> = 3<c_x^4> + 6<c_x^2 c_y^2>.
struct LatticeTables {
  double w[kShells];
  double wp[kShells][5];
  double p[kShells][5];
  double na[5], nb[5];
  double theta0;
  float wf[kShells];
  float wpf[kShells][5];
  float pf[kShells][5];
  float naf[5], nbf[5];
  float theta0f;
  float theta0x3_dw[2];  // 3 theta0 as a double word hi + lo (moment read-back of offset storage)
  float wc2f[kShells];   // w_s c_s^2 (moment sums of offset storage)
  float whkf[kShells];   // w_s k_s / 2, k_s the nonzero |h_a| of shell s (momentum sums)
  // the same three and w_s as double words hi + lo (FP64-quality moment sums of offset storage)
  float w_dw[kShells][2], wc2_dw[kShells][2], whk_dw[kShells][2];
  double wdir[kQ];  // w_i per direction (decoding offset storage in the auxiliary kernels)
  // In-place (AA) streaming: opp[i] = index of -c_i; the site that pulls f_i from site n of
  // sublattice s is n - push_d[s][i][0..2] on sublattice push_d[s][i][3].
  int opp[kQ];
  signed char push_d[2][kQ][4];
};

// Where the stored state keeps population i of site (s, n):
//   kLayoutPlain    (ping-pong)                           at (s, n), slot i;
//   kLayoutAAOwn    (AA, after init or an own-site step)  at (s, n), slot opp[i];
//   kLayoutAAPushed (AA, after a neighbour step)          at the site that pulls it, slot i.
enum StateLayout { kLayoutPlain = 0, kLayoutAAOwn = 1, kLayoutAAPushed = 2 };
// Kinds of step: ping-pong; AA from the own layout (pulls from the neighbours' opp slots and
// pushes into their slots: leaves kLayoutAAPushed); AA from the pushed layout (reads and
// writes its own site: leaves kLayoutAAOwn).
enum StepKind { kStepPingPong = 0, kStepAANeighbour = 1, kStepAAOwn = 2 };

// Builds the tables (host, FP64).  Defined in lattice_tables.cu.
void build_lattice_tables(LatticeTables* t);

// Geometry of one case's population buffers.  A buffer holds both sublattices; each
// sublattice holds 81 direction slabs; a slab is nz planes of ny rows of `pitch` elements,
// the interior x range being [xoff, xoff + nx).  Non-periodic x faces keep kReach ghost
// layers on each side of the interior (xoff >= 4); periodic axes have none and wrap.
struct Geometry {
  int nx, ny, nz;
  int pitch;             // elements per row
  int xoff;              // element index of interior x = 0 within a row
  int x_periodic;        // 1: x wraps; 0: ghost layers at both x faces
  long long plane;       // pitch * ny
  long long dir_stride;  // elements between direction slabs (>= plane * nz, padded)
  long long sub_stride;  // elements between the P and R halves (= 81 * dir_stride)
};

struct StepParams {
  const void* src;
  void* dst;
  Geometry g;
  double omega;          // alpha * beta = 2 / (2 tau + 1)
  unsigned int* flag;    // set to nonzero when a site sees rho <= 0, theta <= 0 or non-finite
  LatticeTables tab;
  // Base addresses, per target sublattice and direction, of the slab a pull reads from
  // (the other sublattice for half links) and of the slab the update writes to.  Filled by
  // fill_slab_bases(); they spare the kernel the 64-bit slab arithmetic of every access.
  const void* src_slab[2][kQ];
  void* dst_slab[2][kQ];
  // The update covers the z planes [z0, z1) of both sublattices (fill_slab_bases sets the
  // whole grid, 0 and nz; a narrower range lets a step run slab by slab).
  int z0, z1;
};

// Fills p.src_slab / p.dst_slab from p.src, p.dst, p.g and the element size, for a step of
// the given kind (StepKind; the AA kinds use p.src == p.dst).
void fill_slab_bases(StepParams* p, size_t elem, int kind = kStepPingPong);

// Validates cfg and derives its buffer geometry (api.cu); LBM_OK or LBM_EINVAL with *why.
lbm_status plan_geometry(const lbm_config* cfg, Geometry* g, std::string* why);

// Storage codecs.  FP64 / FP32 store f_i itself.  FP16 / BF16 store the offset
// d_i = f_i / w_i - 1 (f_i = w_i (1 + d_i)); the collide then works on d directly.  store_evict_first
// stores with the evict-first cache hint (st.global.cs; the in-place AA steps).
template <class S>
struct Codec;
template <>
struct Codec<double> {
  using Real = double;
  static constexpr bool kOffset = false;
  static __device__ __forceinline__ double load(const double* p) { return *p; }
  static __device__ __forceinline__ void store(double* p, double v) { *p = v; }
  static __device__ __forceinline__ void store_evict_first(double* p, double v) { __stcs(p, v); }
};
template <>
struct Codec<float> {
  using Real = float;
  static constexpr bool kOffset = false;
  static __device__ __forceinline__ float load(const float* p) { return *p; }
  static __device__ __forceinline__ void store(float* p, float v) { *p = v; }
  static __device__ __forceinline__ void store_evict_first(float* p, float v) { __stcs(p, v); }
};
template <>
struct Codec<__half> {
  using Real = float;
  static constexpr bool kOffset = true;
  static __device__ __forceinline__ float load(const __half* p) { return __half2float(*p); }
  static __device__ __forceinline__ void store(__half* p, float v) { *p = __float2half_rn(v); }
  static __device__ __forceinline__ void store_evict_first(__half* p, float v) { __stcs(p, __float2half_rn(v)); }
};
template <>
struct Codec<__nv_bfloat16> {
  using Real = float;
  static constexpr bool kOffset = true;
  static __device__ __forceinline__ float load(const __nv_bfloat16* p) { return __bfloat162float(*p); }
  static __device__ __forceinline__ void store(__nv_bfloat16* p, float v) { *p = __float2bfloat16_rn(v); }
  static __device__ __forceinline__ void store_evict_first(__nv_bfloat16* p, float v) {
    __stcs(p, __float2bfloat16_rn(v));
  }
};

// Storage kinds (values match lbm_storage in include/lbm.h).
enum StorageKind { kF64 = 0, kF32 = 1, kF16Off = 2, kBF16Off = 3 };
// Equilibrium + collision variants of the fused kernel.
enum Equilibrium { kEqSeries = 0, kEqEntropic = 1, kEqEntropicAlpha = 2, kEqSeriesExactW = 3 };
RD3Q81_HD constexpr bool eq_is_series(int eq) { return eq == kEqSeries || eq == kEqSeriesExactW; }
inline size_t storage_bytes(int s) { return s == kF64 ? 8 : s == kF32 ? 4 : 2; }

// ---- launchers (each defined in the translation unit of its storage type) --------------
// Fused pull-stream + moments + equilibrium + BGK over every interior site of both
// sublattices.  fp64_moments selects FP64 moment sums and temperature recovery.
// eq: kEqSeries (App. B equilibrium, BGK), kEqSeriesExactW (the same with the exact
// temperature weights of Eq. (zeroveleq)), kEqEntropic (exact entropic equilibrium of Sec. III,
// BGK) or kEqEntropicAlpha (exact entropic equilibrium, entropic alpha of Eq. (delH)).
// kind: StepKind (AA kinds in the sc_aa_*.cu units).
cudaError_t launch_stream_collide(int storage, int fp64_moments, int eq, int kind, const StepParams& p, cudaStream_t s);
cudaError_t launch_sc_f64(int fp64_moments, int eq, const StepParams& p, cudaStream_t s);
cudaError_t launch_sc_f32(int fp64_moments, int eq, const StepParams& p, cudaStream_t s);
cudaError_t launch_sc_f16(int fp64_moments, int eq, const StepParams& p, cudaStream_t s);
cudaError_t launch_sc_bf16(int fp64_moments, int eq, const StepParams& p, cudaStream_t s);
cudaError_t launch_sc_aa_f64(int fp64_moments, int eq, int kind, const StepParams& p, cudaStream_t s);
cudaError_t launch_sc_aa_f32(int fp64_moments, int eq, int kind, const StepParams& p, cudaStream_t s);
cudaError_t launch_sc_aa_f16(int fp64_moments, int eq, int kind, const StepParams& p, cudaStream_t s);
cudaError_t launch_sc_aa_bf16(int fp64_moments, int eq, int kind, const StepParams& p, cudaStream_t s);

// Auxiliary kernels (aux_kernels.cu).  `layout` (StateLayout) says where the stored state
// keeps each population; own_slots = 1 writes the initial state in the AA own layout.
cudaError_t launch_init(int storage, int eq, const Geometry& g, const LatticeTables& tab, void* buf,
                        const double* rho, const double* u, const double* theta,
                        long long first_site, long long count, long long u_stride, cudaStream_t s,
                        unsigned int* flag, int own_slots = 0);
struct Feq81 {
  double v[kQ];
};
cudaError_t launch_fill_inflow(int storage, const Geometry& g, const LatticeTables& tab, void* buf,
                               int face, const Feq81& feq, cudaStream_t s);
// Zero-gradient ghost layers of one x face, for the z planes [z0, z1) (z1 < 0: through nz).
cudaError_t launch_fill_zero_gradient(int storage, const Geometry& g, void* buf, int face, cudaStream_t s,
                                      int z0 = 0, int z1 = -1);
// Bounce-back wall on one x face for the z planes [z0, z1) (z1 < 0: through nz).  mode 0: ghost
// fill before a ping-pong step; 1: ghost fill in the AA own layout before a neighbour step; 2: after
// that neighbour step, what the wall returns into the fluid sites' slots.
cudaError_t launch_bounce_back(int storage, const Geometry& g, const LatticeTables& tab, void* buf, int face,
                               int mode, cudaStream_t s, int z0 = 0, int z1 = -1);
// AA: after a neighbour step, what the ghost sites of one x face push into the interior.
cudaError_t launch_aa_ghost_push(int storage, const Geometry& g, const LatticeTables& tab, void* buf, int face,
                                 int zero_grad, const Feq81& feq, cudaStream_t s);
cudaError_t launch_moments(int storage, const Geometry& g, const LatticeTables& tab, const void* buf,
                           double* rho, double* u, double* theta, long long first_site,
                           long long count, long long u_stride, cudaStream_t s, int layout = kLayoutPlain);
cudaError_t launch_get_populations(int storage, const Geometry& g, const LatticeTables& tab,
                                   const void* buf, double* f, long long first, long long count,
                                   cudaStream_t s, int layout = kLayoutPlain);
cudaError_t launch_set_populations(int storage, const Geometry& g, const LatticeTables& tab, void* buf,
                                   const double* f, long long first, long long count, cudaStream_t s,
                                   int layout = kLayoutPlain);
cudaError_t launch_totals(int storage, const Geometry& g, const LatticeTables& tab, const void* buf,
                          double* partials, int nblocks, double* out5, cudaStream_t s, int layout = kLayoutPlain);

// Mean kinetic energy and enstrophy (Sec. IV C) from FP64 fields rho[sites], u[3][sites] (sites
// ordered sub, z, y, x); partials holds 2 * diagnostics_blocks(sites) doubles; out2 (device) gets
// {KE, eps}.  Two launches (diagnostics.cu).
long long diagnostics_blocks(long long sites);
cudaError_t launch_diagnostics(const Geometry& g, const double* rho, const double* u, long long sites,
                               double* partials, double* out2, cudaStream_t s);
int totals_blocks(const Geometry& g);
cudaError_t launch_probe(int storage, const Geometry& g, const LatticeTables& tab, const void* buf,
                         const long long* sites, long long count, double* f, cudaStream_t s,
                         int layout = kLayoutPlain);

// The App. B equilibrium of one state in FP64 (host and device) is equilibrium_f64() in
// device_common.cuh; init and the inflow faces use it.
}  // namespace lbm
