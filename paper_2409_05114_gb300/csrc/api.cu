// C-ABI of liblbm_rd3q81 (declared and documented in include/lbm.h): context lifetime,
// validation, device memory, chunked host transfers and the step loop.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <string>
#include <vector>

#include "lbm.h"
#include "device_common.cuh"

namespace {

constexpr uint32_t kMagic = 0x52443831u;  // "RD81"
constexpr long long kChunkSites = 1LL << 22;  // sites per host-transfer chunk
constexpr int kGraphSteps = 8;                // steps per replayed CUDA graph (even)
// Pinned host fields move through staging slots, one z slab of both sublattices at a time:
// a slab holds about kSlabSites sites per sublattice (whole planes), and kRing slots per
// direction let the copy engines run ahead of (host to device) or behind (device to host)
// the kernels.
constexpr long long kSlabSites = 1LL << 20;
constexpr int kRing = 3;
constexpr int kSlabRows = 10;  // rho (2 sublattices), u (3 components x 2), theta (2)

thread_local std::string g_create_error = "no error";

long long round_up(long long a, long long b) { return (a + b - 1) / b * b; }

// Restores the caller's current device on scope exit.
struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) == cudaSuccess && prev != dev) cudaSetDevice(dev);
    else prev = -1;
  }
  ~DeviceGuard() {
    if (prev >= 0) cudaSetDevice(prev);
  }
};

}  // namespace

namespace lbm {

lbm_status plan_geometry(const lbm_config* cfg, Geometry* g, std::string* why) {
  if (!cfg) return *why = "config is NULL", LBM_EINVAL;
  if (cfg->velset != LBM_RD3Q81) return *why = "velset must be LBM_RD3Q81", LBM_EINVAL;
  if (cfg->nx < 1 || cfg->ny < 1 || cfg->nz < 1) return *why = "nx, ny, nz must be >= 1", LBM_EINVAL;
  if (!(std::isfinite(cfg->tau) && cfg->tau >= 0.0)) return *why = "tau must be finite and >= 0", LBM_EINVAL;
  if (cfg->storage < LBM_F64 || cfg->storage > LBM_BF16_OFFSET) return *why = "unknown storage", LBM_EINVAL;
  if (cfg->fp64_moments != 0 && cfg->fp64_moments != 1) return *why = "fp64_moments must be 0 or 1", LBM_EINVAL;
  if (cfg->equilibrium != LBM_EQ_SERIES && cfg->equilibrium != LBM_EQ_ENTROPIC &&
      cfg->equilibrium != LBM_EQ_SERIES_EXACT_W)
    return *why = "equilibrium must be LBM_EQ_SERIES, LBM_EQ_ENTROPIC or LBM_EQ_SERIES_EXACT_W", LBM_EINVAL;
  if (cfg->equilibrium != LBM_EQ_SERIES && cfg->fp64_moments)
    return *why = "fp64_moments is available with the series equilibrium (LBM_EQ_SERIES) only", LBM_EINVAL;
  if (cfg->streaming != LBM_STREAM_PINGPONG && cfg->streaming != LBM_STREAM_AA)
    return *why = "streaming must be LBM_STREAM_PINGPONG or LBM_STREAM_AA", LBM_EINVAL;
  if (cfg->collision != LBM_COLLISION_BGK && cfg->collision != LBM_COLLISION_ENTROPIC)
    return *why = "collision must be LBM_COLLISION_BGK or LBM_COLLISION_ENTROPIC", LBM_EINVAL;
  if (cfg->collision == LBM_COLLISION_ENTROPIC && cfg->equilibrium != LBM_EQ_ENTROPIC)
    return *why = "the entropic alpha is defined with the exact entropic equilibrium (equilibrium = LBM_EQ_ENTROPIC)",
           LBM_EINVAL;
  for (int f = 0; f < 6; ++f) {
    const lbm_bc& b = cfg->face[f];
    if (b.kind < LBM_BC_PERIODIC || b.kind > LBM_BC_BOUNCE_BACK) return *why = "unknown boundary kind", LBM_EINVAL;
    if (f >= 2 && b.kind != LBM_BC_PERIODIC)
      return *why = "only the x faces may be non-periodic in this version", LBM_EINVAL;
    if (b.kind == LBM_BC_EQ_INFLOW &&
        !(std::isfinite(b.rho) && b.rho > 0 && std::isfinite(b.theta) && b.theta > 0 &&
          std::isfinite(b.ux) && std::isfinite(b.uy) && std::isfinite(b.uz)))
      return *why = "inflow state needs finite u, rho > 0, theta > 0", LBM_EINVAL;
  }
  const bool xp0 = cfg->face[0].kind == LBM_BC_PERIODIC, xp1 = cfg->face[1].kind == LBM_BC_PERIODIC;
  if (xp0 != xp1) return *why = "a periodic x face must be paired with a periodic x face", LBM_EINVAL;
  const long long n = static_cast<long long>(cfg->nx) * cfg->ny * cfg->nz;
  if (n >= (1LL << 31)) return *why = "nx*ny*nz must be < 2^31", LBM_EINVAL;

  const long long elem = static_cast<long long>(storage_bytes(cfg->storage));
  g->nx = cfg->nx;
  g->ny = cfg->ny;
  g->nz = cfg->nz;
  g->x_periodic = xp0 ? 1 : 0;
  if (xp0) {
    g->xoff = 0;
    g->pitch = cfg->nx;
  } else {
    // Ghost layers; the interior row starts on a 128-byte boundary.
    const long long align = 128 / elem;
    g->xoff = static_cast<int>(align);
    const long long pitch = round_up(align + cfg->nx + rd3q81::kReach, align);
    if (pitch >= (1LL << 31)) return *why = "row too long", LBM_EINVAL;
    g->pitch = static_cast<int>(pitch);
  }
  g->plane = static_cast<long long>(g->pitch) * cfg->ny;
  const long long slab = g->plane * cfg->nz;
  if (slab >= (1LL << 31)) return *why = "one direction slab must hold < 2^31 elements", LBM_EINVAL;
  g->dir_stride = round_up(slab, 64);
  g->sub_stride = kQ * g->dir_stride;
  return LBM_OK;
}

}  // namespace lbm

struct lbm_ctx {
  uint32_t magic = kMagic;
  lbm_config cfg{};
  lbm::Geometry g{};
  lbm::LatticeTables tab{};
  int storage = 0;
  size_t elem = 0;
  long long sites = 0;  // 2 * nx * ny * nz
  void* buf[2] = {nullptr, nullptr};  // AA streaming uses buf[0] only
  int cur = 0;                        // ping-pong: the buffer holding the state
  bool aa = false;
  int layout = lbm::kLayoutPlain;     // StateLayout of the stored state
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  int device = 0;
  unsigned int* d_flag = nullptr;
  double* d_scratch = nullptr;
  long long chunk = 0;
  double* d_partials = nullptr;
  double* d_totals = nullptr;
  int totals_nb = 0;
  double omega = 0.0;
  bool initialized = false;
  bool zero_grad[2] = {false, false};
  bool inflow[2] = {false, false};
  bool bounce[2] = {false, false};
  lbm::Feq81 feq_in[2]{};
  lbm::Feq81 feq_in_own[2]{};  // feq_in with direction i in the slot of -c_i (AA own layout)
  long long launches = 0;
  // Staged host transfers: copy streams, a stream for the initialisation of arriving slabs
  // (it overlaps the steps and moments of earlier ones), slot events, kRing input then kRing
  // output slots.
  cudaStream_t xfer_in = nullptr, xfer_out = nullptr, init_stream = nullptr;
  cudaEvent_t in_ready[kRing] = {}, in_free[kRing] = {}, out_ready[kRing] = {}, out_free[kRing] = {};
  cudaEvent_t mark = nullptr;
  double* d_stage = nullptr;
  int slab_planes = 0;
  long long slab_m = 0;  // sites per sublattice in a full slab (the row pitch of a slot)
  cudaGraphExec_t graph = nullptr;  // kGraphSteps steps starting from buffer 0 (AA: the own layout)
  long long graph_launches = 0;     // kernel launches in one replay
  long long direct_steps = 0;       // steps issued by plain launches (the first ones load the kernels)
  std::string err = "no error";
};

namespace {

lbm_status fail(lbm_ctx* ctx, lbm_status st, const std::string& msg) {
  if (ctx) ctx->err = msg;
  else g_create_error = msg;
  return st;
}

#define LBM_CK(ctx, call)                                                                       \
  do {                                                                                         \
    cudaError_t e_ = (call);                                                                   \
    if (e_ != cudaSuccess)                                                                     \
      return fail(ctx, LBM_ECUDA, std::string(#call) + " failed: " + cudaGetErrorString(e_));  \
  } while (0)

bool valid(const lbm_ctx* ctx) { return ctx != nullptr && ctx->magic == kMagic; }

size_t buffer_bytes(const lbm::Geometry& g, int storage) {
  return static_cast<size_t>(2 * g.sub_stride) * lbm::storage_bytes(storage);
}

long long chunk_sites(long long sites) { return sites < kChunkSites ? sites : kChunkSites; }

// Scratch doubles: 5 fields per chunk site, and room for at least 256 probed sites.
long long scratch_doubles(long long sites) {
  const long long a = 5 * chunk_sites(sites), b = 256 * (1 + lbm::kQ);
  return a > b ? a : b;
}
size_t scratch_bytes(long long sites) { return static_cast<size_t>(scratch_doubles(sites)) * sizeof(double); }

// z planes per staged slab, and the staging bytes (2 kRing slots of kSlabRows rows).
int slab_planes(int nx, int ny, int nz) {
  const long long nxy = static_cast<long long>(nx) * ny;
  const long long z = kSlabSites / nxy;
  return static_cast<int>(z < 1 ? 1 : z > nz ? nz : z);
}
size_t stage_bytes(int nx, int ny, int nz) {
  const long long m = static_cast<long long>(slab_planes(nx, ny, nz)) * nx * ny;
  return static_cast<size_t>(2 * kRing * kSlabRows * m) * sizeof(double);
}

size_t aux_bytes(const lbm::Geometry& g) {
  return static_cast<size_t>(lbm::totals_blocks(g)) * 5 * sizeof(double) + 8 * sizeof(double) + 256;
}

// Device-side address of host memory p if it is page-locked and mapped into the device's
// address space (cudaHostAlloc'd or cudaHostRegister'ed, as pinned torch tensors are): kernels
// then read and write it directly over the host link, with no staging copies.  nullptr
// otherwise (pageable memory goes through the chunked copies).
void* mapped_host(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return a.type == cudaMemoryTypeHost ? a.devicePointer : nullptr;
}

lbm_status fill_inflow_faces(lbm_ctx* ctx) {
  if (ctx->aa) return LBM_OK;  // AA refills the inflow ghosts before every neighbour step
  for (int face = 0; face < 2; ++face) {
    if (!ctx->inflow[face]) continue;
    for (int b = 0; b < 2; ++b) {
      LBM_CK(ctx, lbm::launch_fill_inflow(ctx->storage, ctx->g, ctx->tab, ctx->buf[b], face,
                                          ctx->feq_in[face], ctx->stream));
      ++ctx->launches;
    }
  }
  return LBM_OK;
}

lbm_status check_flag(lbm_ctx* ctx) {
  unsigned int flag = 0;
  LBM_CK(ctx, cudaMemcpyAsync(&flag, ctx->d_flag, sizeof(flag), cudaMemcpyDeviceToHost, ctx->stream));
  LBM_CK(ctx, cudaStreamSynchronize(ctx->stream));
  if (flag) return fail(ctx, LBM_EUNSTABLE, "a site saw rho <= 0, theta <= 0 or a non-finite value");
  return LBM_OK;
}

}  // namespace

extern "C" {

lbm_status lbm_footprint(const lbm_config* cfg, size_t* bytes) {
  lbm::Geometry g;
  std::string why;
  if (!bytes) return fail(nullptr, LBM_EINVAL, "bytes is NULL");
  if (lbm::plan_geometry(cfg, &g, &why) != LBM_OK) return fail(nullptr, LBM_EINVAL, why);
  const long long sites = 2LL * cfg->nx * cfg->ny * cfg->nz;
  *bytes = (cfg->streaming == LBM_STREAM_AA ? 1 : 2) * buffer_bytes(g, cfg->storage) + scratch_bytes(sites) +
           aux_bytes(g) + stage_bytes(cfg->nx, cfg->ny, cfg->nz);
  return LBM_OK;
}

lbm_status lbm_create(const lbm_config* cfg, lbm_ctx** out) {
  if (!out) return fail(nullptr, LBM_EINVAL, "out is NULL");
  *out = nullptr;
  lbm::Geometry g;
  std::string why;
  if (lbm::plan_geometry(cfg, &g, &why) != LBM_OK) return fail(nullptr, LBM_EINVAL, why);

  lbm_ctx* ctx = new (std::nothrow) lbm_ctx();
  if (!ctx) return fail(nullptr, LBM_ENOMEM, "host allocation failed");
  ctx->cfg = *cfg;
  ctx->g = g;
  ctx->storage = cfg->storage;
  ctx->elem = lbm::storage_bytes(cfg->storage);
  ctx->sites = 2LL * cfg->nx * cfg->ny * cfg->nz;
  ctx->chunk = chunk_sites(ctx->sites);
  ctx->omega = 2.0 / (2.0 * cfg->tau + 1.0);
  lbm::build_lattice_tables(&ctx->tab);
  for (int face = 0; face < 2; ++face) {
    const lbm_bc& b = cfg->face[face];
    ctx->zero_grad[face] = b.kind == LBM_BC_ZERO_GRADIENT;
    ctx->inflow[face] = b.kind == LBM_BC_EQ_INFLOW;
    ctx->bounce[face] = b.kind == LBM_BC_BOUNCE_BACK;
    if (ctx->inflow[face]) {
      if (cfg->equilibrium == LBM_EQ_ENTROPIC)
        lbm::entropic_all<double>(b.rho, b.ux, b.uy, b.uz, b.theta, ctx->tab, ctx->feq_in[face].v);
      else if (cfg->equilibrium == LBM_EQ_SERIES_EXACT_W)
        lbm::equilibrium_all<double, false, true>(b.rho, b.ux, b.uy, b.uz, b.theta, ctx->tab, ctx->feq_in[face].v);
      else
        lbm::equilibrium_f64(b.rho, b.ux, b.uy, b.uz, b.theta, ctx->tab, ctx->feq_in[face].v);
    }
  }

  auto bail = [&](lbm_status st, const std::string& msg) {
    lbm_destroy(ctx);
    return fail(nullptr, st, msg);
  };
  cudaError_t e = cudaGetDevice(&ctx->device);
  if (e != cudaSuccess) return bail(LBM_ECUDA, std::string("cudaGetDevice failed: ") + cudaGetErrorString(e));
  if (cfg->cuda_stream) {
    ctx->stream = static_cast<cudaStream_t>(cfg->cuda_stream);
  } else {
    e = cudaStreamCreate(&ctx->stream);
    if (e != cudaSuccess) return bail(LBM_ECUDA, std::string("cudaStreamCreate failed: ") + cudaGetErrorString(e));
    ctx->own_stream = true;
  }
  const size_t bb = buffer_bytes(g, ctx->storage);
  ctx->aa = cfg->streaming == LBM_STREAM_AA;
  for (int face = 0; face < 2; ++face)
    for (int i = 0; i < lbm::kQ; ++i) ctx->feq_in_own[face].v[i] = ctx->feq_in[face].v[i == 0 ? 0 : (i % 2 ? i + 1 : i - 1)];
  for (int b = 0; b < (ctx->aa ? 1 : 2); ++b) {
    e = cudaMalloc(&ctx->buf[b], bb);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return bail(LBM_ENOMEM, "cudaMalloc of a population buffer (" + std::to_string(bb) + " bytes) failed: " +
                                  cudaGetErrorString(e));
    }
  }
  ctx->totals_nb = lbm::totals_blocks(g);
  e = cudaMalloc(&ctx->d_scratch, scratch_bytes(ctx->sites));
  if (e == cudaSuccess) e = cudaMalloc(&ctx->d_partials, ctx->totals_nb * 5 * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&ctx->d_totals, 8 * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&ctx->d_flag, 256);
  if (e == cudaSuccess) e = cudaMemsetAsync(ctx->d_flag, 0, 256, ctx->stream);
  ctx->slab_planes = slab_planes(cfg->nx, cfg->ny, cfg->nz);
  ctx->slab_m = static_cast<long long>(ctx->slab_planes) * cfg->nx * cfg->ny;
  if (e == cudaSuccess) e = cudaMalloc(&ctx->d_stage, stage_bytes(cfg->nx, cfg->ny, cfg->nz));
  if (e != cudaSuccess) {
    cudaGetLastError();
    return bail(LBM_ENOMEM, std::string("device allocation failed: ") + cudaGetErrorString(e));
  }
  e = cudaStreamCreateWithFlags(&ctx->xfer_in, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&ctx->xfer_out, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&ctx->init_stream, cudaStreamNonBlocking);
  for (int k = 0; k < kRing && e == cudaSuccess; ++k) {
    e = cudaEventCreateWithFlags(&ctx->in_ready[k], cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ctx->in_free[k], cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ctx->out_ready[k], cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ctx->out_free[k], cudaEventDisableTiming);
  }
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ctx->mark, cudaEventDisableTiming);
  if (e != cudaSuccess) return bail(LBM_ECUDA, std::string("stream/event creation failed: ") + cudaGetErrorString(e));
  *out = ctx;
  return LBM_OK;
}

lbm_status lbm_init(lbm_ctx* ctx, const double* rho, const double* u, const double* theta, int on_device) {
  if (!valid(ctx)) return LBM_EINVAL;
  if (!rho || !u || !theta) return fail(ctx, LBM_EINVAL, "NULL field pointer");
  DeviceGuard dg(ctx->device);
  const long long S = ctx->sites;
  ctx->cur = 0;
  ctx->layout = ctx->aa ? lbm::kLayoutAAOwn : lbm::kLayoutPlain;
  LBM_CK(ctx, cudaMemsetAsync(ctx->d_flag, 0, sizeof(unsigned int), ctx->stream));
  void* hr = on_device ? nullptr : mapped_host(rho);
  void* hu = on_device ? nullptr : mapped_host(u);
  void* ht = on_device ? nullptr : mapped_host(theta);
  if (on_device || (hr && hu && ht)) {
    // device fields, or pinned host fields read in place by the kernel
    LBM_CK(ctx, lbm::launch_init(ctx->storage, ctx->cfg.equilibrium, ctx->g, ctx->tab, ctx->buf[0],
                                 on_device ? rho : static_cast<const double*>(hr),
                                 on_device ? u : static_cast<const double*>(hu),
                                 on_device ? theta : static_cast<const double*>(ht), 0, S, S, ctx->stream, ctx->d_flag,
                                 ctx->aa ? 1 : 0));
    ++ctx->launches;
  } else {
    double* sr = ctx->d_scratch;
    double* su = sr + ctx->chunk;
    double* st = su + 3 * ctx->chunk;
    for (long long first = 0; first < S; first += ctx->chunk) {
      const long long cnt = S - first < ctx->chunk ? S - first : ctx->chunk;
      const size_t nb = static_cast<size_t>(cnt) * sizeof(double);
      LBM_CK(ctx, cudaMemcpyAsync(sr, rho + first, nb, cudaMemcpyHostToDevice, ctx->stream));
      for (int a = 0; a < 3; ++a)
        LBM_CK(ctx, cudaMemcpyAsync(su + a * cnt, u + a * S + first, nb, cudaMemcpyHostToDevice, ctx->stream));
      LBM_CK(ctx, cudaMemcpyAsync(st, theta + first, nb, cudaMemcpyHostToDevice, ctx->stream));
      LBM_CK(ctx, lbm::launch_init(ctx->storage, ctx->cfg.equilibrium, ctx->g, ctx->tab, ctx->buf[0], sr, su, st,
                                   first, cnt, cnt, ctx->stream, ctx->d_flag, ctx->aa ? 1 : 0));
      ++ctx->launches;
    }
  }
  lbm_status st = fill_inflow_faces(ctx);
  if (st != LBM_OK) return st;
  if (!on_device) LBM_CK(ctx, cudaStreamSynchronize(ctx->stream));
  ctx->initialized = true;
  return LBM_OK;
}

namespace {

int step_mode(const lbm_ctx* ctx) {
  return ctx->cfg.equilibrium == LBM_EQ_ENTROPIC
             ? (ctx->cfg.collision == LBM_COLLISION_ENTROPIC ? lbm::kEqEntropicAlpha : lbm::kEqEntropic)
         : ctx->cfg.equilibrium == LBM_EQ_SERIES_EXACT_W ? lbm::kEqSeriesExactW
                                                          : lbm::kEqSeries;
}

// The step that follows a stored state: ping-pong, or by AA layout (own -> neighbour step,
// pushed -> own-site step).
int step_kind(const lbm_ctx* ctx, int layout) {
  return !ctx->aa ? lbm::kStepPingPong : layout == lbm::kLayoutAAPushed ? lbm::kStepAAOwn : lbm::kStepAANeighbour;
}

enum FillKinds { kFillZeroGrad = 1, kFillInflow = 2, kFillWalls = 4, kFillAll = 7 };

// Boundary work before a step of `kind` from buffer `cur`, for the z planes [z0, z1) (z1 < 0:
// all): zero-gradient and bounce-back ghosts of the source (ping-pong) or of the own layout (AA
// neighbour step, which also refills the inflow ghosts it overwrites).  Ping-pong inflow ghosts
// are constant, written at init; an own-site step reads no ghost.
cudaError_t pre_step_fills(lbm_ctx* ctx, int cur, int kind, int kinds, cudaStream_t s, long long* launches,
                           int z0 = 0, int z1 = -1) {
  if (kind == lbm::kStepAAOwn) return cudaSuccess;
  void* b = ctx->buf[kind == lbm::kStepPingPong ? cur : 0];
  cudaError_t e = cudaSuccess;
  for (int face = 0; face < 2 && e == cudaSuccess; ++face) {
    if (ctx->zero_grad[face] && (kinds & kFillZeroGrad))
      e = lbm::launch_fill_zero_gradient(ctx->storage, ctx->g, b, face, s, z0, z1);
    else if (ctx->inflow[face] && kind == lbm::kStepAANeighbour && (kinds & kFillInflow))
      e = lbm::launch_fill_inflow(ctx->storage, ctx->g, ctx->tab, b, face, ctx->feq_in_own[face], s);
    else if (ctx->bounce[face] && (kinds & kFillWalls))
      e = lbm::launch_bounce_back(ctx->storage, ctx->g, ctx->tab, b, face, kind == lbm::kStepPingPong ? 0 : 1, s, z0, z1);
    else
      continue;
    ++*launches;
  }
  return e;
}

// The fused kernel of a step of `kind` from buffer `cur` over the z planes [z0, z1) (z1 < 0: all).
cudaError_t launch_step_kernel(lbm_ctx* ctx, int cur, int kind, cudaStream_t s, long long* launches, int z0 = 0,
                               int z1 = -1) {
  lbm::StepParams p;
  p.g = ctx->g;
  p.omega = ctx->omega;
  p.flag = ctx->d_flag;
  p.tab = ctx->tab;
  p.src = ctx->buf[ctx->aa ? 0 : cur];
  p.dst = ctx->buf[ctx->aa ? 0 : cur ^ 1];
  lbm::fill_slab_bases(&p, ctx->elem, kind);
  if (z1 >= 0) {
    p.z0 = z0;
    p.z1 = z1;
  }
  ++*launches;
  return lbm::launch_stream_collide(ctx->storage, ctx->cfg.fp64_moments,
                                    step_mode(ctx), kind, p, s);
}

// After an AA neighbour step (interior sites only): what each x face returns into the fluid
// sites' slots -- the ghosts' pushes (zero gradient, inflow) or the wall's reflections.
cudaError_t post_step_returns(lbm_ctx* ctx, int kind, cudaStream_t s, long long* launches) {
  if (kind != lbm::kStepAANeighbour) return cudaSuccess;
  cudaError_t e = cudaSuccess;
  for (int face = 0; face < 2 && e == cudaSuccess; ++face) {
    if (ctx->bounce[face])
      e = lbm::launch_bounce_back(ctx->storage, ctx->g, ctx->tab, ctx->buf[0], face, 2, s);
    else if (ctx->zero_grad[face] || ctx->inflow[face])
      e = lbm::launch_aa_ghost_push(ctx->storage, ctx->g, ctx->tab, ctx->buf[0], face, ctx->zero_grad[face] ? 1 : 0,
                                    ctx->feq_in[face], s);
    else
      continue;
    ++*launches;
  }
  return e;
}

// Issues one step on stream s and adds its launches to *launches.  Ping-pong: ghost fills,
// then the fused kernel from buffer `cur` into the other.  AA (buffer 0, in place): from the
// own layout, ghost fills in that layout, the neighbour step, then what the faces return into
// the interior (leaves the pushed layout); from the pushed layout, the own-site step.
cudaError_t issue_step(lbm_ctx* ctx, int cur, int layout, cudaStream_t s, long long* launches) {
  static_assert(kGraphSteps % 2 == 0, "a captured run must return to its starting state");
  const int kind = step_kind(ctx, layout);
  cudaError_t e = pre_step_fills(ctx, cur, kind, kFillAll, s, launches);
  if (e == cudaSuccess) e = launch_step_kernel(ctx, cur, kind, s, launches);
  if (e == cudaSuccess) e = post_step_returns(ctx, kind, s, launches);
  return e;
}

// The state after one step: ping-pong flips the buffer; AA flips the layout.
void advance(lbm_ctx* ctx) {
  if (ctx->aa)
    ctx->layout = ctx->layout == lbm::kLayoutAAOwn ? lbm::kLayoutAAPushed : lbm::kLayoutAAOwn;
  else
    ctx->cur ^= 1;
}

// True when the state is where a captured run starts: buffer 0 (ping-pong) or the AA own layout.
bool at_graph_start(const lbm_ctx* ctx) { return ctx->aa ? ctx->layout == lbm::kLayoutAAOwn : ctx->cur == 0; }

// Captures kGraphSteps steps starting from buffer 0 / the AA own layout (an even number of
// steps returns there).
cudaError_t build_graph(lbm_ctx* ctx) {
  cudaStream_t cap;
  cudaError_t e = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking);
  if (e != cudaSuccess) return e;
  cudaGraph_t g = nullptr;
  e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
  ctx->graph_launches = 0;
  for (int k = 0; e == cudaSuccess && k < kGraphSteps; ++k)
    e = issue_step(ctx, k & 1, (k & 1) ? lbm::kLayoutAAPushed : lbm::kLayoutAAOwn, cap, &ctx->graph_launches);
  cudaError_t e2 = cudaStreamEndCapture(cap, &g);
  if (e == cudaSuccess) e = e2;
  if (e == cudaSuccess) e = cudaGraphInstantiate(&ctx->graph, g, 0);
  if (g) cudaGraphDestroy(g);
  cudaStreamDestroy(cap);
  if (e != cudaSuccess) {
    ctx->graph = nullptr;
    cudaGetLastError();
  }
  return e;
}

// n steps on the context's stream (lbm_step after its checks).
lbm_status run_steps(lbm_ctx* ctx, long long n) {
  // Runs of kGraphSteps steps are replayed from one captured graph (launch overhead matters
  // for small grids), unless the caller is capturing the context's stream itself.
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  LBM_CK(ctx, cudaStreamIsCapturing(ctx->stream, &cs));
  const bool graphs = cs == cudaStreamCaptureStatusNone && n >= kGraphSteps + 2;
  long long k = 0;
  if (graphs) {
    // plain steps first: until two have run (kernels loaded before any capture) and until
    // the state is back in buffer 0, where the graph starts
    while (ctx->direct_steps < 2 || !at_graph_start(ctx)) {
      LBM_CK(ctx, issue_step(ctx, ctx->cur, ctx->layout, ctx->stream, &ctx->launches));
      ++ctx->direct_steps;
      advance(ctx);
      ++k;
    }
    if (!ctx->graph && n - k >= kGraphSteps) LBM_CK(ctx, build_graph(ctx));
    for (; n - k >= kGraphSteps; k += kGraphSteps) {
      LBM_CK(ctx, cudaGraphLaunch(ctx->graph, ctx->stream));
      ctx->launches += ctx->graph_launches;
    }
  }
  for (; k < n; ++k) {
    LBM_CK(ctx, issue_step(ctx, ctx->cur, ctx->layout, ctx->stream, &ctx->launches));
    ++ctx->direct_steps;
    advance(ctx);
  }
  return LBM_OK;
}


// ---- staged host transfers --------------------------------------------------------------
// A slab is the z planes [z0, z1) of both sublattices.  In a staging slot its fields are
// kSlabRows rows of slab_m doubles: rows 0-1 rho, 2-7 u (row 2a + s: component a on
// sublattice s), 8-9 theta.  In the field layout the same rows start s n, (2a + s) n and s n
// elements into the field (n = nx ny nz), plus z0 nx ny: one 2-D copy per field.
struct Slab {
  int z0, z1;
  long long m;  // sites per sublattice
};

int slab_count(const lbm_ctx* ctx) { return (ctx->cfg.nz + ctx->slab_planes - 1) / ctx->slab_planes; }

Slab slab_at(const lbm_ctx* ctx, int k) {
  const int z0 = k * ctx->slab_planes;
  const int z1 = z0 + ctx->slab_planes < ctx->cfg.nz ? z0 + ctx->slab_planes : ctx->cfg.nz;
  return {z0, z1, static_cast<long long>(z1 - z0) * ctx->cfg.nx * ctx->cfg.ny};
}

// Slot q % kRing of the input (out = 0) or output (out = 1) ring.
double* stage_slot(const lbm_ctx* ctx, int out, long long q) {
  return ctx->d_stage + ((out ? kRing : 0) + q % kRing) * kSlabRows * ctx->slab_m;
}

cudaError_t copy_slab(const lbm_ctx* ctx, const Slab& sl, double* slot, double* const host[3], bool to_device,
                      cudaStream_t s) {
  const long long nxy = static_cast<long long>(ctx->cfg.nx) * ctx->cfg.ny;
  const size_t width = static_cast<size_t>(sl.m) * sizeof(double);
  const size_t hp = static_cast<size_t>(nxy * ctx->cfg.nz) * sizeof(double);
  const size_t dp = static_cast<size_t>(ctx->slab_m) * sizeof(double);
  const int row0[3] = {0, 2, 8}, rows[3] = {2, 6, 2};
  cudaError_t e = cudaSuccess;
  for (int f = 0; f < 3 && e == cudaSuccess; ++f) {
    double* d = slot + row0[f] * ctx->slab_m;
    double* h = host[f] + sl.z0 * nxy;
    e = to_device ? cudaMemcpy2DAsync(d, dp, h, hp, width, rows[f], cudaMemcpyHostToDevice, s)
                  : cudaMemcpy2DAsync(h, hp, d, dp, width, rows[f], cudaMemcpyDeviceToHost, s);
  }
  return e;
}

// Host to device copy of slab k's fields into input slot k, once lbm::launch_init is done with
// the slot's previous slab.
cudaError_t stage_in(lbm_ctx* ctx, int k, double* const host[3]) {
  const int r = k % kRing;
  cudaError_t e = cudaStreamWaitEvent(ctx->xfer_in, ctx->in_free[r], 0);
  if (e == cudaSuccess) e = copy_slab(ctx, slab_at(ctx, k), stage_slot(ctx, 0, k), host, true, ctx->xfer_in);
  if (e == cudaSuccess) e = cudaEventRecord(ctx->in_ready[r], ctx->xfer_in);
  return e;
}

// Equilibrium initialisation of slab k from its input slot (buffer 0), and the zero-gradient
// ghosts of its planes when a step follows, on the init stream; in_free[k % kRing] marks its end.
cudaError_t init_slab(lbm_ctx* ctx, int k, bool fill_ghosts) {
  const int r = k % kRing;
  const Slab sl = slab_at(ctx, k);
  const long long n = ctx->sites / 2, M = ctx->slab_m, nxy = static_cast<long long>(ctx->cfg.nx) * ctx->cfg.ny;
  double* slot = stage_slot(ctx, 0, k);
  cudaStream_t s = ctx->init_stream;
  cudaError_t e = cudaStreamWaitEvent(s, ctx->in_ready[r], 0);
  for (int sub = 0; sub < 2 && e == cudaSuccess; ++sub) {
    e = lbm::launch_init(ctx->storage, ctx->cfg.equilibrium, ctx->g, ctx->tab, ctx->buf[0], slot + sub * M,
                         slot + (2 + sub) * M, slot + (8 + sub) * M, sub * n + sl.z0 * nxy, sl.m, 2 * M, s,
                         ctx->d_flag, ctx->aa ? 1 : 0);
    ++ctx->launches;
  }
  for (int face = 0; face < 2 && e == cudaSuccess && fill_ghosts; ++face) {
    if (!ctx->zero_grad[face]) continue;
    e = lbm::launch_fill_zero_gradient(ctx->storage, ctx->g, ctx->buf[0], face, s, sl.z0, sl.z1);
    ++ctx->launches;
  }
  if (e == cudaSuccess) e = cudaEventRecord(ctx->in_free[r], s);
  return e;
}

// Moments of slab k of `buf` into output slot q (once that slot's previous copy has left),
// then its device to host copy on the output copy stream.
cudaError_t moments_out(lbm_ctx* ctx, int k, long long q, const void* buf, int layout, double* const host[3]) {
  const int r = q % kRing;
  const Slab sl = slab_at(ctx, k);
  const long long n = ctx->sites / 2, M = ctx->slab_m, nxy = static_cast<long long>(ctx->cfg.nx) * ctx->cfg.ny;
  double* slot = stage_slot(ctx, 1, q);
  cudaError_t e = cudaStreamWaitEvent(ctx->stream, ctx->out_free[r], 0);
  for (int sub = 0; sub < 2 && e == cudaSuccess; ++sub) {
    e = lbm::launch_moments(ctx->storage, ctx->g, ctx->tab, buf, slot + sub * M, slot + (2 + sub) * M,
                            slot + (8 + sub) * M, sub * n + sl.z0 * nxy, sl.m, 2 * M, ctx->stream, layout);
    ++ctx->launches;
  }
  if (e == cudaSuccess) e = cudaEventRecord(ctx->out_ready[r], ctx->stream);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(ctx->xfer_out, ctx->out_ready[r], 0);
  if (e == cudaSuccess) e = copy_slab(ctx, sl, slot, host, false, ctx->xfer_out);
  if (e == cudaSuccess) e = cudaEventRecord(ctx->out_free[r], ctx->xfer_out);
  return e;
}

// The copy and init streams start after the work already queued on the context's stream ...
cudaError_t fork_copies(lbm_ctx* ctx) {
  cudaError_t e = cudaEventRecord(ctx->mark, ctx->stream);
  for (cudaStream_t xs : {ctx->xfer_in, ctx->xfer_out, ctx->init_stream})
    if (e == cudaSuccess) e = cudaStreamWaitEvent(xs, ctx->mark, 0);
  return e;
}

// ... and the context's stream continues after their last copy or kernel.
cudaError_t join_copies(lbm_ctx* ctx) {
  cudaError_t e = cudaSuccess;
  for (cudaStream_t xs : {ctx->init_stream, ctx->xfer_in, ctx->xfer_out}) {
    if (e == cudaSuccess) e = cudaEventRecord(ctx->mark, xs);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(ctx->stream, ctx->mark, 0);
  }
  return e;
}

// lbm_advance_fields for pinned host fields.  Slab by slab: the input copy engine fills input
// slots, init runs on each slab as it lands (on its own stream), and the output copy engine drains
// each slab's moments as soon as they are computed, so both directions of the host link and the
// kernels overlap.  n == 0: moments follow init; n == 1: the step of a slab follows the init of
// every slab within the pull reach of its planes; n >= 2: init for all slabs, n - 1 whole-grid
// steps, then the last step slab by slab with its moments.  AA streaming: the neighbour step of
// a slab reads and writes only slots of sites within its reach, each slot by one site, so slab
// steps may run in any order once those sites are initialised; the moments of the pushed layout
// read only what the slab's own sites pushed; what the x faces return into the fluid (for the
// next step) follows all slab steps.
lbm_status advance_staged(lbm_ctx* ctx, double* const in[3], long long n, double* const out[3]) {
  const int N = slab_count(ctx);
  ctx->cur = 0;
  ctx->layout = ctx->aa ? lbm::kLayoutAAOwn : lbm::kLayoutPlain;
  ctx->initialized = false;
  LBM_CK(ctx, cudaMemsetAsync(ctx->d_flag, 0, sizeof(unsigned int), ctx->stream));
  lbm_status st = fill_inflow_faces(ctx);  // ping-pong: constant inflow ghosts of both buffers
  if (st != LBM_OK) return st;
  const int kind1 = step_kind(ctx, ctx->layout);  // the first step's kind
  if (n == 1) LBM_CK(ctx, pre_step_fills(ctx, 0, kind1, kFillInflow, ctx->stream, &ctx->launches));
  LBM_CK(ctx, fork_copies(ctx));
  for (int k = 0; k < N && k < kRing; ++k) LBM_CK(ctx, stage_in(ctx, k, in));
  // n == 1: need[k] = the last slab, in init order, holding a plane within kReach of slab k.  A
  // bounce-back wall's ghosts on slab k's planes read fluid sites within that reach (they run once
  // need[k] is initialised), and slab k's step reads the ghosts of every slab within its reach:
  // with walls a step waits for step_need[k] = max(need[k'] : k' within reach of k).
  std::vector<int> need(N, 0), step_need(N, 0), order(N), fill_order(N);
  auto slabs_within_reach = [&](int k, auto&& fn) {
    const Slab sl = slab_at(ctx, k);
    for (int z = sl.z0 - rd3q81::kReach; z < sl.z1 + rd3q81::kReach; ++z)
      fn((((z % ctx->cfg.nz) + ctx->cfg.nz) % ctx->cfg.nz) / ctx->slab_planes);
  };
  for (int k = 0; k < N; ++k) slabs_within_reach(k, [&](int k2) { need[k] = std::max(need[k], k2); });
  const bool walls = ctx->bounce[0] || ctx->bounce[1];
  for (int k = 0; k < N; ++k) {
    order[k] = fill_order[k] = k;
    step_need[k] = need[k];
    if (walls) slabs_within_reach(k, [&](int k2) { step_need[k] = std::max(step_need[k], need[k2]); });
  }
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return step_need[a] < step_need[b]; });
  std::stable_sort(fill_order.begin(), fill_order.end(), [&](int a, int b) { return need[a] < need[b]; });
  size_t next = 0, next_fill = 0;
  long long q = 0;
  // where the moments of the state after a step of `kind` are read
  auto after = [&](int kind) {
    return kind == lbm::kStepPingPong ? lbm::kLayoutPlain
                                      : kind == lbm::kStepAANeighbour ? lbm::kLayoutAAPushed : lbm::kLayoutAAOwn;
  };
  void* const out_buf = ctx->buf[ctx->aa ? 0 : 1];  // holds the state after one step from buffer 0
  for (int j = 0; j < N; ++j) {
    LBM_CK(ctx, init_slab(ctx, j, n == 1));
    if (j + kRing < N) LBM_CK(ctx, stage_in(ctx, j + kRing, in));
    // what follows needs init up to slab j (and no further): wait for in_free[j % kRing]
    if (n == 0) {
      LBM_CK(ctx, cudaStreamWaitEvent(ctx->stream, ctx->in_free[j % kRing], 0));
      LBM_CK(ctx, moments_out(ctx, j, q++, ctx->buf[0], ctx->layout, out));
    } else if (n == 1 && ((next < order.size() && step_need[order[next]] <= j) ||
                          (walls && next_fill < fill_order.size() && need[fill_order[next_fill]] <= j))) {
      LBM_CK(ctx, cudaStreamWaitEvent(ctx->stream, ctx->in_free[j % kRing], 0));
      for (; walls && next_fill < fill_order.size() && need[fill_order[next_fill]] <= j; ++next_fill) {
        const Slab sl = slab_at(ctx, fill_order[next_fill]);
        LBM_CK(ctx, pre_step_fills(ctx, 0, kind1, kFillWalls, ctx->stream, &ctx->launches, sl.z0, sl.z1));
      }
      for (; next < order.size() && step_need[order[next]] <= j; ++next) {
        const Slab sl = slab_at(ctx, order[next]);
        LBM_CK(ctx, launch_step_kernel(ctx, 0, kind1, ctx->stream, &ctx->launches, sl.z0, sl.z1));
        LBM_CK(ctx, moments_out(ctx, order[next], q++, out_buf, after(kind1), out));
      }
    }
  }
  ctx->initialized = true;
  if (n == 1) LBM_CK(ctx, post_step_returns(ctx, kind1, ctx->stream, &ctx->launches));
  if (n >= 2) {
    LBM_CK(ctx, cudaEventRecord(ctx->mark, ctx->init_stream));
    LBM_CK(ctx, cudaStreamWaitEvent(ctx->stream, ctx->mark, 0));
    st = run_steps(ctx, n - 1);
    if (st != LBM_OK) return st;
    const int kind = step_kind(ctx, ctx->layout);
    LBM_CK(ctx, pre_step_fills(ctx, ctx->cur, kind, kFillAll, ctx->stream, &ctx->launches));
    void* const last_buf = ctx->buf[ctx->aa ? 0 : ctx->cur ^ 1];
    for (int k = 0; k < N; ++k) {
      const Slab sl = slab_at(ctx, k);
      LBM_CK(ctx, launch_step_kernel(ctx, ctx->cur, kind, ctx->stream, &ctx->launches, sl.z0, sl.z1));
      LBM_CK(ctx, moments_out(ctx, k, q++, last_buf, after(kind), out));
    }
    LBM_CK(ctx, post_step_returns(ctx, kind, ctx->stream, &ctx->launches));
  }
  if (n >= 1) advance(ctx);
  LBM_CK(ctx, join_copies(ctx));
  return check_flag(ctx);
}

}  // namespace

lbm_status lbm_step(lbm_ctx* ctx, long long n) {
  if (!valid(ctx)) return LBM_EINVAL;
  if (n < 0) return fail(ctx, LBM_EINVAL, "n must be >= 0");
  if (!ctx->initialized) return fail(ctx, LBM_EINVAL, "lbm_init or lbm_set_populations was never called");
  DeviceGuard dg(ctx->device);
  return run_steps(ctx, n);
}

lbm_status lbm_advance_fields(lbm_ctx* ctx, const double* rho, const double* u, const double* theta, long long n,
                              double* rho_out, double* u_out, double* theta_out, int on_device) {
  if (!valid(ctx)) return LBM_EINVAL;
  if (!rho || !u || !theta || !rho_out || !u_out || !theta_out) return fail(ctx, LBM_EINVAL, "NULL field pointer");
  if (n < 0) return fail(ctx, LBM_EINVAL, "n must be >= 0");
  DeviceGuard dg(ctx->device);
  bool pinned = !on_device;
  for (const void* f : {static_cast<const void*>(rho), static_cast<const void*>(u), static_cast<const void*>(theta),
                        static_cast<const void*>(rho_out), static_cast<const void*>(u_out),
                        static_cast<const void*>(theta_out)})
    if (pinned && !mapped_host(f)) pinned = false;
  if (pinned) {
    double* const in[3] = {const_cast<double*>(rho), const_cast<double*>(u), const_cast<double*>(theta)};
    double* const out[3] = {rho_out, u_out, theta_out};
    return advance_staged(ctx, in, n, out);
  }
  lbm_status st = lbm_init(ctx, rho, u, theta, on_device);
  if (st == LBM_OK) st = run_steps(ctx, n);
  if (st == LBM_OK) st = lbm_moments(ctx, rho_out, u_out, theta_out, on_device);
  return st;
}

lbm_status lbm_moments(lbm_ctx* ctx, double* rho, double* u, double* theta, int on_device) {
  if (!valid(ctx)) return LBM_EINVAL;
  if (!rho || !u || !theta) return fail(ctx, LBM_EINVAL, "NULL field pointer");
  if (!ctx->initialized) return fail(ctx, LBM_EINVAL, "lbm_init or lbm_set_populations was never called");
  DeviceGuard dg(ctx->device);
  const long long S = ctx->sites;
  const void* b = ctx->buf[ctx->cur];
  const bool pinned = !on_device && mapped_host(rho) && mapped_host(u) && mapped_host(theta);
  if (on_device) {
    LBM_CK(ctx, lbm::launch_moments(ctx->storage, ctx->g, ctx->tab, b, rho, u, theta, 0, S, S, ctx->stream,
                                    ctx->layout));
    ++ctx->launches;
  } else if (pinned) {
    // slab by slab through the output ring: the copy engine drains one slab while the next
    // one's moments are computed
    double* const out[3] = {rho, u, theta};
    for (int k = 0; k < slab_count(ctx); ++k) LBM_CK(ctx, moments_out(ctx, k, k, b, ctx->layout, out));
    LBM_CK(ctx, join_copies(ctx));
  } else {
    double* sr = ctx->d_scratch;
    double* su = sr + ctx->chunk;
    double* st = su + 3 * ctx->chunk;
    for (long long first = 0; first < S; first += ctx->chunk) {
      const long long cnt = S - first < ctx->chunk ? S - first : ctx->chunk;
      const size_t nb = static_cast<size_t>(cnt) * sizeof(double);
      LBM_CK(ctx, lbm::launch_moments(ctx->storage, ctx->g, ctx->tab, b, sr, su, st, first, cnt, cnt, ctx->stream,
                                      ctx->layout));
      ++ctx->launches;
      LBM_CK(ctx, cudaMemcpyAsync(rho + first, sr, nb, cudaMemcpyDeviceToHost, ctx->stream));
      for (int a = 0; a < 3; ++a)
        LBM_CK(ctx, cudaMemcpyAsync(u + a * S + first, su + a * cnt, nb, cudaMemcpyDeviceToHost, ctx->stream));
      LBM_CK(ctx, cudaMemcpyAsync(theta + first, st, nb, cudaMemcpyDeviceToHost, ctx->stream));
    }
  }
  return check_flag(ctx);
}

lbm_status lbm_totals(lbm_ctx* ctx, double* out5) {
  if (!valid(ctx)) return LBM_EINVAL;
  if (!out5) return fail(ctx, LBM_EINVAL, "out5 is NULL");
  if (!ctx->initialized) return fail(ctx, LBM_EINVAL, "lbm_init or lbm_set_populations was never called");
  DeviceGuard dg(ctx->device);
  LBM_CK(ctx, lbm::launch_totals(ctx->storage, ctx->g, ctx->tab, ctx->buf[ctx->cur], ctx->d_partials,
                                 ctx->totals_nb, ctx->d_totals, ctx->stream, ctx->layout));
  ctx->launches += 2;
  LBM_CK(ctx, cudaMemcpyAsync(out5, ctx->d_totals, 5 * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
  LBM_CK(ctx, cudaStreamSynchronize(ctx->stream));
  return LBM_OK;
}

lbm_status lbm_diagnostics(lbm_ctx* ctx, double* out2) {
  if (!valid(ctx)) return LBM_EINVAL;
  if (!out2) return fail(ctx, LBM_EINVAL, "out2 is NULL");
  if (!ctx->initialized) return fail(ctx, LBM_EINVAL, "lbm_init or lbm_set_populations was never called");
  if (!ctx->g.x_periodic && ctx->cfg.nx < 3)
    return fail(ctx, LBM_EINVAL, "the one-sided x differences of a non-periodic grid need nx >= 3");
  DeviceGuard dg(ctx->device);
  const long long S = ctx->sites;
  const long long nb = lbm::diagnostics_blocks(S);
  const size_t bytes = static_cast<size_t>(5 * S + 2 * nb + 2) * sizeof(double);
  void* scratch = nullptr;
  if (cudaMallocAsync(&scratch, bytes, ctx->stream) != cudaSuccess) {
    cudaGetLastError();
    return fail(ctx, LBM_ENOMEM, "no device memory for the diagnostics fields (40 bytes per site)");
  }
  double* rho = static_cast<double*>(scratch);
  double* u = rho + S;
  double* theta = u + 3 * S;
  double* partials = theta + S;
  double* dout = partials + 2 * nb;
  cudaError_t e = lbm::launch_moments(ctx->storage, ctx->g, ctx->tab, ctx->buf[ctx->cur], rho, u, theta, 0, S, S,
                                      ctx->stream, ctx->layout);
  if (e == cudaSuccess) e = lbm::launch_diagnostics(ctx->g, rho, u, S, partials, dout, ctx->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(out2, dout, 2 * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream);
  ctx->launches += 3;
  cudaFreeAsync(scratch, ctx->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
  if (e != cudaSuccess) return fail(ctx, LBM_ECUDA, std::string("lbm_diagnostics: ") + cudaGetErrorString(e));
  return LBM_OK;
}

lbm_status lbm_get_populations(lbm_ctx* ctx, double* f, int on_device) {
  if (!valid(ctx)) return LBM_EINVAL;
  if (!f) return fail(ctx, LBM_EINVAL, "f is NULL");
  if (!ctx->initialized) return fail(ctx, LBM_EINVAL, "lbm_init or lbm_set_populations was never called");
  DeviceGuard dg(ctx->device);
  const long long total = ctx->sites * lbm::kQ;
  const void* b = ctx->buf[ctx->cur];
  if (on_device) {
    LBM_CK(ctx, lbm::launch_get_populations(ctx->storage, ctx->g, ctx->tab, b, f, 0, total, ctx->stream, ctx->layout));
    ++ctx->launches;
  } else {
    const long long ck = 5 * ctx->chunk;
    for (long long first = 0; first < total; first += ck) {
      const long long cnt = total - first < ck ? total - first : ck;
      LBM_CK(ctx, lbm::launch_get_populations(ctx->storage, ctx->g, ctx->tab, b, ctx->d_scratch, first, cnt,
                                              ctx->stream, ctx->layout));
      ++ctx->launches;
      LBM_CK(ctx, cudaMemcpyAsync(f + first, ctx->d_scratch, static_cast<size_t>(cnt) * sizeof(double),
                                  cudaMemcpyDeviceToHost, ctx->stream));
    }
  }
  LBM_CK(ctx, cudaStreamSynchronize(ctx->stream));
  return LBM_OK;
}

lbm_status lbm_set_populations(lbm_ctx* ctx, const double* f, int on_device) {
  if (!valid(ctx)) return LBM_EINVAL;
  if (!f) return fail(ctx, LBM_EINVAL, "f is NULL");
  DeviceGuard dg(ctx->device);
  const long long total = ctx->sites * lbm::kQ;
  ctx->cur = 0;
  ctx->layout = ctx->aa ? lbm::kLayoutAAOwn : lbm::kLayoutPlain;
  if (on_device) {
    LBM_CK(ctx, lbm::launch_set_populations(ctx->storage, ctx->g, ctx->tab, ctx->buf[0], f, 0, total, ctx->stream,
                                            ctx->layout));
    ++ctx->launches;
  } else {
    const long long ck = 5 * ctx->chunk;
    for (long long first = 0; first < total; first += ck) {
      const long long cnt = total - first < ck ? total - first : ck;
      LBM_CK(ctx, cudaMemcpyAsync(ctx->d_scratch, f + first, static_cast<size_t>(cnt) * sizeof(double),
                                  cudaMemcpyHostToDevice, ctx->stream));
      LBM_CK(ctx, lbm::launch_set_populations(ctx->storage, ctx->g, ctx->tab, ctx->buf[0], ctx->d_scratch, first,
                                              cnt, ctx->stream, ctx->layout));
      ++ctx->launches;
    }
  }
  lbm_status st = fill_inflow_faces(ctx);
  if (st != LBM_OK) return st;
  LBM_CK(ctx, cudaMemsetAsync(ctx->d_flag, 0, sizeof(unsigned int), ctx->stream));
  LBM_CK(ctx, cudaStreamSynchronize(ctx->stream));
  ctx->initialized = true;
  return LBM_OK;
}

lbm_status lbm_probe(lbm_ctx* ctx, const long long* sites, long long count, double* f) {
  if (!valid(ctx)) return LBM_EINVAL;
  if (count < 0 || (count > 0 && (!sites || !f))) return fail(ctx, LBM_EINVAL, "bad probe arguments");
  if (!ctx->initialized) return fail(ctx, LBM_EINVAL, "lbm_init or lbm_set_populations was never called");
  for (long long k = 0; k < count; ++k)
    if (sites[k] < 0 || sites[k] >= ctx->sites) return fail(ctx, LBM_EINVAL, "probe site index out of range");
  DeviceGuard dg(ctx->device);
  // Scratch holds 5 * chunk doubles: site indices (as 64-bit integers) and then the values.
  const long long per = scratch_doubles(ctx->sites) / (1 + lbm::kQ);
  long long* d_sites = reinterpret_cast<long long*>(ctx->d_scratch);
  double* d_vals = ctx->d_scratch + per;
  for (long long first = 0; first < count; first += per) {
    const long long cnt = count - first < per ? count - first : per;
    LBM_CK(ctx, cudaMemcpyAsync(d_sites, sites + first, cnt * sizeof(long long), cudaMemcpyHostToDevice,
                                ctx->stream));
    LBM_CK(ctx, lbm::launch_probe(ctx->storage, ctx->g, ctx->tab, ctx->buf[ctx->cur], d_sites, cnt, d_vals,
                                  ctx->stream, ctx->layout));
    ++ctx->launches;
    LBM_CK(ctx, cudaMemcpyAsync(f + first * lbm::kQ, d_vals, cnt * lbm::kQ * sizeof(double),
                                cudaMemcpyDeviceToHost, ctx->stream));
    LBM_CK(ctx, cudaStreamSynchronize(ctx->stream));
  }
  return LBM_OK;
}

lbm_status lbm_sync(lbm_ctx* ctx) {
  if (!valid(ctx)) return LBM_EINVAL;
  DeviceGuard dg(ctx->device);
  return check_flag(ctx);
}

lbm_status lbm_launch_count(const lbm_ctx* ctx, long long* count) {
  if (!valid(ctx) || !count) return LBM_EINVAL;
  *count = ctx->launches;
  return LBM_OK;
}

lbm_status lbm_destroy(lbm_ctx* ctx) {
  if (!valid(ctx)) return LBM_EINVAL;
  {
    DeviceGuard dg(ctx->device);
    for (cudaStream_t xs : {ctx->stream, ctx->xfer_in, ctx->xfer_out, ctx->init_stream})
      if (xs) cudaStreamSynchronize(xs);
    for (int b = 0; b < 2; ++b)
      if (ctx->buf[b]) cudaFree(ctx->buf[b]);
    if (ctx->d_scratch) cudaFree(ctx->d_scratch);
    if (ctx->d_partials) cudaFree(ctx->d_partials);
    if (ctx->d_totals) cudaFree(ctx->d_totals);
    if (ctx->d_flag) cudaFree(ctx->d_flag);
    if (ctx->graph) cudaGraphExecDestroy(ctx->graph);
    if (ctx->d_stage) cudaFree(ctx->d_stage);
    for (cudaStream_t xs : {ctx->xfer_in, ctx->xfer_out, ctx->init_stream})
      if (xs) cudaStreamDestroy(xs);
    for (int k = 0; k < kRing; ++k)
      for (cudaEvent_t ev : {ctx->in_ready[k], ctx->in_free[k], ctx->out_ready[k], ctx->out_free[k]})
        if (ev) cudaEventDestroy(ev);
    if (ctx->mark) cudaEventDestroy(ctx->mark);
    if (ctx->own_stream && ctx->stream) cudaStreamDestroy(ctx->stream);
  }
  ctx->magic = 0;
  delete ctx;
  return LBM_OK;
}

const char* lbm_last_error(const lbm_ctx* ctx) {
  if (ctx == nullptr) return g_create_error.c_str();
  if (!valid(ctx)) return "invalid context";
  return ctx->err.c_str();
}

int lbm_velocities(int* h, double* w) {
  lbm::LatticeTables t;
  lbm::build_lattice_tables(&t);
  for (int i = 0; i < lbm::kQ; ++i) {
    if (h) {
      h[3 * i + 0] = rd3q81::kDirs[i].hx;
      h[3 * i + 1] = rd3q81::kDirs[i].hy;
      h[3 * i + 2] = rd3q81::kDirs[i].hz;
    }
    if (w) w[i] = t.wdir[i];
  }
  return lbm::kQ;
}

}  // extern "C"
