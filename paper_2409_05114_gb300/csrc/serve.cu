// Continuous-batching server: many independent RD3Q81 cases resident on one GPU, advanced
// together by one persistent fused kernel per time step and per kind of case (storage type and
// equilibrium: the App. B series, or the exact entropic equilibrium of Sec. III, both with BGK).
//
// Each admitted case owns two population buffers (ping-pong) and a slot in a device case
// table.  A step of the whole batch is (a) one batched zero-gradient ghost fill (only if a
// resident case has such a face) and (b) one persistent kernel whose blocks walk a packed
// index of 128-site tiles over all cases: the tile's case is found by binary search over the
// cases' first-tile offsets, and the site is updated by the same device function as the
// single-case kernel's (site_update_table, with the case's slab bases from a table).  Sites are independent, so a case's result is bitwise
// the same served alone and in any mix.  K steps form one "tick", captured once per (membership, K) as a CUDA graph and
// replayed.  A scheduler thread admits queued requests by HBM footprint on a separate
// stream while the current tick runs, and retires finished or unstable cases after it.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "lbm.h"
#include "stream_collide.cuh"

namespace lbm {
namespace {

constexpr int kMaxServerCases = 1024;
constexpr int kTickSteps = 16;            // longest tick (steps between scheduler decisions)
// Admission is first fit in submission order over the oldest kAdmitLookahead waiting requests;
// a request passed over kMaxBypass times holds back every later one until it is admitted.
constexpr int kAdmitLookahead = 16;
constexpr int kMaxBypass = 8;

struct CaseDesc {
  Geometry g;
  void* buf[2];
  double omega;
  unsigned int* flag;
  int storage;         // kF32, kF16Off or kBF16Off
  int eq;              // kEqSeries or kEqEntropic
  int parity;          // buffer holding the state at the start of the tick
  int tiles_sub;       // ceil(nx*ny*nz / kScBlock)
  int zg_face[2];      // zero-gradient at -x / +x
  long long tile0;     // first packed tile of this case within its storage group's P half
  long long row0;      // first packed ghost row (zero-gradient faces)
  long long rows_face; // rows per zero-gradient face: 2 * 81 * nz * ny
};

__device__ __forceinline__ int find_case(const long long* first, int ncases, long long idx) {
  int lo = 0, hi = ncases - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (first[mid] <= idx) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// Slab base addresses of one resident case for one parity of its buffers (source buf[par],
// destination buf[par ^ 1]), per target sublattice and direction: the table fill_slab_bases
// writes for a single-case step.
struct CaseSlabs {
  const void* src[2][kQ];
  void* dst[2][kQ];
};

// Step k of the current tick, sublattice SUB, for the resident cases of one group (storage type S,
// equilibrium kEq): one kernel per group and sublattice, so each holds one site update.  A kernel
// with several (the three storage types once, then both sublattices) overflowed the instruction
// cache: with the entropic update, 6.7 "no instruction" stalls per issue against 1.0 for the
// single-case kernel, whose blocks each run one sublattice.  Grid: persistent (SMs x resident
// blocks); block b handles tiles b, b + gridDim.x, ... of the group's packed tiles (`half` of them
// per sublattice).  No block waits on another.  When a block's tile belongs to another
// (case, parity) than its last one, the block copies that case's 81 source and 81 destination
// slab bases into shared memory; the site update then reads them there, as the single-case
// kernel reads its kernel parameters.
template <class S, int kEq, int SUB>
__global__ void __launch_bounds__(kScBlock, 4) served_step_kernel(const CaseDesc* __restrict__ cases,
                                                               const CaseSlabs* __restrict__ slabs, int ncases,
                                                               long long half, int k, const LatticeTables tab) {
  __shared__ long long s_first[kMaxServerCases];
  __shared__ const void* s_src[kQ];
  __shared__ void* s_dst[kQ];
  for (int c = threadIdx.x; c < ncases; c += blockDim.x) s_first[c] = cases[c].tile0;
  __syncthreads();
  int have = -1;  // (case, parity) whose slab bases are in shared memory
  for (long long tile = blockIdx.x; tile < half; tile += gridDim.x) {
    const int c = find_case(s_first, ncases, tile);
    const CaseDesc& cd = cases[c];
    const int par = (cd.parity + k) & 1;
    const int key = 2 * c + par;
    if (key != have) {  // the same for every thread of the block
      __syncthreads();
      const CaseSlabs& tb = slabs[key];
      for (int i = threadIdx.x; i < kQ; i += blockDim.x) {
        s_src[i] = tb.src[SUB][i];
        s_dst[i] = tb.dst[SUB][i];
      }
      __syncthreads();
      have = key;
    }
    const long long t = (tile - cd.tile0) * kScBlock + threadIdx.x;
    const long long n = static_cast<long long>(cd.g.nx) * cd.g.ny * cd.g.nz;
    if (t >= n) continue;
    site_update_table<S, false, SUB, kEq, kStepPingPong>(cd.g, cd.omega, cd.flag, tab, SharedSlabs{s_src, s_dst},
                                                         static_cast<int>(t));
  }
}

// Resident cases grouped by kind (storage type, equilibrium): the case table lists the groups
// in this order; each group's tiles are numbered from 0 for its own kernel.
constexpr int kGroups = 6;
constexpr int kGroupStorage[kGroups] = {kF32, kF16Off, kBF16Off, kF32, kF16Off, kBF16Off};
constexpr int kGroupEq[kGroups] = {kEqSeries, kEqSeries, kEqSeries, kEqEntropic, kEqEntropic, kEqEntropic};
struct TickPlan {
  int first[kGroups] = {};      // first case of the group in the table
  int count[kGroups] = {};
  long long tiles[kGroups] = {};  // tiles of the group per sublattice
};

// Both sublattices of one step of a group: the P kernel, then the R kernel.
template <class S, int kEq>
void launch_served(const CaseDesc* d, const CaseSlabs* sl, int count, long long tiles, int k, const LatticeTables& tab,
                   int grid, cudaStream_t s) {
  served_step_kernel<S, kEq, 0><<<grid, kScBlock, 0, s>>>(d, sl, count, tiles, k, tab);
  served_step_kernel<S, kEq, 1><<<grid, kScBlock, 0, s>>>(d, sl, count, tiles, k, tab);
}

void launch_group(int gi, const CaseDesc* d, const CaseSlabs* sl, int count, long long tiles, int k,
                  const LatticeTables& tab, int grid, cudaStream_t s) {
  switch (gi) {
    case 0: launch_served<float, kEqSeries>(d, sl, count, tiles, k, tab, grid, s); break;
    case 1: launch_served<__half, kEqSeries>(d, sl, count, tiles, k, tab, grid, s); break;
    case 2: launch_served<__nv_bfloat16, kEqSeries>(d, sl, count, tiles, k, tab, grid, s); break;
    case 3: launch_served<float, kEqEntropic>(d, sl, count, tiles, k, tab, grid, s); break;
    case 4: launch_served<__half, kEqEntropic>(d, sl, count, tiles, k, tab, grid, s); break;
    default: launch_served<__nv_bfloat16, kEqEntropic>(d, sl, count, tiles, k, tab, grid, s);
  }
}

template <class T>
__device__ __forceinline__ void copy_edge(T* buf, const CaseDesc& cd, long long row, int face) {
  const Geometry& g = cd.g;
  if (face == 0) {
    const T v = buf[row + g.xoff];
    for (int l = 1; l <= rd3q81::kReach; ++l) buf[row + g.xoff - l] = v;
  } else {
    const T v = buf[row + g.xoff + g.nx - 1];
    for (int l = 0; l < rd3q81::kReach; ++l) buf[row + g.xoff + g.nx + l] = v;
  }
}

// Zero-gradient ghost fill of step k for all resident cases: thread per (case, face, sub,
// i, z, y) row; raw copies of the stored values (no decode needed).
__global__ void served_zero_gradient_kernel(const CaseDesc* __restrict__ cases, int ncases, long long total_rows,
                                            int k) {
  __shared__ long long s_first[kMaxServerCases];
  for (int c = threadIdx.x; c < ncases; c += blockDim.x) s_first[c] = cases[c].row0;
  __syncthreads();
  for (long long r = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x; r < total_rows;
       r += static_cast<long long>(gridDim.x) * blockDim.x) {
    const int c = find_case(s_first, ncases, r);
    const CaseDesc& cd = cases[c];
    long long local = r - cd.row0;
    int which = static_cast<int>(local / cd.rows_face);  // index among this case's zg faces
    local -= which * cd.rows_face;
    const int face = (cd.zg_face[0] && which == 0) ? 0 : 1;
    const Geometry& g = cd.g;
    const int y = static_cast<int>(local % g.ny);
    const long long q = local / g.ny;
    const int z = static_cast<int>(q % g.nz);
    const long long si = q / g.nz;
    const long long row = (si / kQ) * g.sub_stride + (si % kQ) * g.dir_stride + z * g.plane +
                          static_cast<long long>(y) * g.pitch;
    void* b = cd.buf[(cd.parity + k) & 1];
    if (cd.storage == kF32)
      copy_edge(static_cast<uint32_t*>(b), cd, row, face);
    else
      copy_edge(static_cast<uint16_t*>(b), cd, row, face);
  }
}

using Clock = std::chrono::steady_clock;

// Pinned, device-mapped host memory (a request's fields), freed with its owner.  The kernels read
// and write it in place over the host link: no staging copy, nothing for the scheduler to wait on.
struct HostFields {
  double* p = nullptr;
  HostFields() = default;
  HostFields(const HostFields&) = delete;
  HostFields& operator=(const HostFields&) = delete;
  ~HostFields() {
    if (p) cudaFreeHost(p);
  }
  bool alloc(long long n) {
    void* q = nullptr;
    if (cudaHostAlloc(&q, static_cast<size_t>(n) * sizeof(double), cudaHostAllocMapped | cudaHostAllocPortable) !=
        cudaSuccess) {
      cudaGetLastError();
      return false;
    }
    p = static_cast<double*>(q);
    return true;
  }
};

struct Request {
  long long ticket = 0;
  lbm_config cfg{};
  long long nsteps = 0;
  long long sites = 0;
  size_t footprint = 0;
  HostFields in;   // rho | u (3 * sites) | theta
  HostFields out;  // same layout, written at retirement
  Clock::time_point t_submit, t_done;
  lbm_status status = LBM_EBUSY;
  bool done = false;
  int bypassed = 0;         // later requests admitted before this one
};

// A case whose fields are being read back (on the retire stream) and whose memory is being freed.
struct Retiring {
  std::shared_ptr<Request> req;
  int slot = -1;
  lbm_status status = LBM_OK;
  cudaEvent_t done = nullptr;
};

struct Resident {
  std::shared_ptr<Request> req;
  Geometry g{};
  void* buf[2] = {nullptr, nullptr};
  int slot = -1;
  int parity = 0;
  long long steps_left = 0;
  double omega = 0.0;
  bool zg[2] = {false, false};
  cudaEvent_t ready = nullptr;  // admission finished (on the admission stream)
};

}  // namespace
}  // namespace lbm

struct lbm_server {
  using Request = lbm::Request;
  using Resident = lbm::Resident;
  using Retiring = lbm::Retiring;

  size_t budget = 0;
  int max_cases = 0;
  int device = 0;
  lbm::LatticeTables tab{};
  cudaStream_t compute = nullptr, admit = nullptr, retire = nullptr;
  cudaEvent_t tick_done = nullptr;
  lbm::CaseDesc* d_cases = nullptr;
  lbm::CaseDesc* h_cases = nullptr;  // pinned staging
  lbm::CaseSlabs* d_slabs = nullptr;  // per table position and parity (2 per case)
  lbm::CaseSlabs* h_slabs = nullptr;  // pinned staging
  long long slabs_version = -1;       // membership version the device table was written for
  unsigned int* d_flags = nullptr;
  unsigned int* h_flags = nullptr;   // pinned
  int grid_blocks = 0;

  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<std::shared_ptr<Request>> queue;          // submitted, not admitted
  std::unordered_map<long long, std::shared_ptr<Request>> requests;
  std::vector<Resident> active, joining;
  std::vector<Retiring> retiring;
  std::vector<int> free_slots;
  size_t resident_bytes = 0;
  long long next_ticket = 1;
  bool stop = false;
  lbm_status fatal = LBM_OK;
  std::string err = "no error";
  lbm_server_stats stats{};
  lbm::Clock::time_point busy_since;

  // graphs per (version, K)
  long long version = 0;
  std::map<std::pair<long long, int>, cudaGraphExec_t> graphs;
  std::thread worker;
};

namespace lbm {
namespace {

thread_local std::string g_server_error = "no error";

lbm_status set_fatal(lbm_server* s, const std::string& msg) {
  std::lock_guard<std::mutex> lk(s->mu);
  s->fatal = LBM_ECUDA;
  s->err = msg;
  s->cv_done.notify_all();
  return LBM_ECUDA;
}

#define SRV_CK(s, call)                                                                         \
  do {                                                                                         \
    cudaError_t e_ = (call);                                                                   \
    if (e_ != cudaSuccess) return set_fatal(s, std::string(#call) + " failed: " + cudaGetErrorString(e_)); \
  } while (0)

// Starts the admission of request r into a free slot (asynchronous, on the admission stream).
lbm_status start_admission(lbm_server* s, const std::shared_ptr<Request>& r, int slot) {
  Resident res;
  res.req = r;
  res.slot = slot;
  res.steps_left = r->nsteps;
  res.omega = 2.0 / (2.0 * r->cfg.tau + 1.0);
  std::string why;
  plan_geometry(&r->cfg, &res.g, &why);
  res.zg[0] = r->cfg.face[0].kind == LBM_BC_ZERO_GRADIENT;
  res.zg[1] = r->cfg.face[1].kind == LBM_BC_ZERO_GRADIENT;
  const size_t bb = static_cast<size_t>(2 * res.g.sub_stride) * storage_bytes(r->cfg.storage);
  for (int b = 0; b < 2; ++b) SRV_CK(s, cudaMallocAsync(&res.buf[b], bb, s->admit));
  SRV_CK(s, cudaMemsetAsync(s->d_flags + slot, 0, sizeof(unsigned int), s->admit));
  // the init kernel reads the request's pinned fields in place
  const long long S = r->sites;
  double* din = nullptr;
  SRV_CK(s, cudaHostGetDevicePointer(reinterpret_cast<void**>(&din), r->in.p, 0));
  SRV_CK(s, launch_init(r->cfg.storage, r->cfg.equilibrium, res.g, s->tab, res.buf[0], din, din + S, din + 4 * S, 0, S,
                        S, s->admit, s->d_flags + slot));
  long long launches = 1;  // published under the lock below, with the stats' readers
  for (int face = 0; face < 2; ++face) {
    const lbm_bc& b = r->cfg.face[face];
    if (b.kind != LBM_BC_EQ_INFLOW) continue;
    Feq81 feq;
    if (r->cfg.equilibrium == LBM_EQ_ENTROPIC)
      entropic_all<double>(b.rho, b.ux, b.uy, b.uz, b.theta, s->tab, feq.v);
    else
      equilibrium_f64(b.rho, b.ux, b.uy, b.uz, b.theta, s->tab, feq.v);
    for (int k = 0; k < 2; ++k) {
      SRV_CK(s, launch_fill_inflow(r->cfg.storage, res.g, s->tab, res.buf[k], face, feq, s->admit));
      ++launches;
    }
  }
  SRV_CK(s, cudaEventCreateWithFlags(&res.ready, cudaEventDisableTiming));
  SRV_CK(s, cudaEventRecord(res.ready, s->admit));
  s->joining.push_back(res);
  std::lock_guard<std::mutex> lk(s->mu);
  s->stats.kernel_launches += launches;
  return LBM_OK;
}

lbm_status finish_retirements(lbm_server* s);

// Admits queued requests while a slot is free: the first of the oldest kAdmitLookahead that fits
// the remaining budget, so that one large request at the head does not leave the budget idle;
// a request passed over kMaxBypass times is admitted before any later one.
lbm_status admit_some(lbm_server* s) {
  const lbm_status fr = finish_retirements(s);
  if (fr != LBM_OK) return fr;
  for (;;) {
    std::shared_ptr<Request> r;
    int slot = -1;
    {
      std::lock_guard<std::mutex> lk(s->mu);
      if (s->queue.empty() || s->free_slots.empty()) return LBM_OK;
      const int look = static_cast<int>(std::min<size_t>(s->queue.size(), kAdmitLookahead));
      int pick = -1;
      for (int q = 0; q < look; ++q) {
        if (s->resident_bytes + s->queue[q]->footprint <= s->budget) {
          pick = q;
          break;
        }
        if (s->queue[q]->bypassed >= kMaxBypass) break;
      }
      if (pick < 0) return LBM_OK;
      for (int q = 0; q < pick; ++q) ++s->queue[q]->bypassed;
      r = s->queue[pick];
      s->queue.erase(s->queue.begin() + pick);
      slot = s->free_slots.back();
      s->free_slots.pop_back();
      s->resident_bytes += r->footprint;
      s->stats.peak_resident_bytes = std::max(s->stats.peak_resident_bytes, s->resident_bytes);
      ++s->stats.admitted;
    }
    lbm_status st = start_admission(s, r, slot);
    if (st != LBM_OK) return st;
  }
}

cudaGraphExec_t tick_graph(lbm_server* s, int ncases, const TickPlan& plan, long long total_rows, int K) {
  auto key = std::make_pair(s->version, K);
  auto it = s->graphs.find(key);
  if (it != s->graphs.end()) return it->second;
  cudaStream_t cap;
  if (cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking) != cudaSuccess) return nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  bool ok = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
  for (int k = 0; ok && k < K; ++k) {
    if (total_rows > 0) {
      const int zb = static_cast<int>(std::min<long long>((total_rows + 255) / 256, 4096));
      served_zero_gradient_kernel<<<zb, 256, 0, cap>>>(s->d_cases, ncases, total_rows, k);
    }
    for (int gi = 0; gi < kGroups; ++gi) {
      if (plan.count[gi] == 0) continue;
      const int grid = static_cast<int>(std::min<long long>(s->grid_blocks, plan.tiles[gi]));
      launch_group(gi, s->d_cases + plan.first[gi], s->d_slabs + 2 * plan.first[gi], plan.count[gi], plan.tiles[gi], k,
                   s->tab, grid, cap);
    }
  }
  if (ok) ok = cudaStreamEndCapture(cap, &graph) == cudaSuccess;
  if (ok) ok = cudaGraphInstantiate(&exec, graph, 0) == cudaSuccess;
  if (graph) cudaGraphDestroy(graph);
  cudaStreamDestroy(cap);
  if (!ok) {
    cudaGetLastError();
    return nullptr;
  }
  s->graphs[key] = exec;
  return exec;
}

void drop_graphs(lbm_server* s) {
  for (auto& kv : s->graphs) cudaGraphExecDestroy(kv.second);
  s->graphs.clear();
}

// Starts a case's retirement on the retire stream, after the tick that finished it: the moments
// kernel writes its fields into the request's pinned output in place, then its buffers are freed.
// The scheduler goes on with the next tick; finish_retirements completes the request.
lbm_status begin_retire(lbm_server* s, Resident& res, lbm_status status) {
  Request& r = *res.req;
  const long long S = r.sites;
  double* dout = nullptr;
  SRV_CK(s, cudaHostGetDevicePointer(reinterpret_cast<void**>(&dout), r.out.p, 0));
  SRV_CK(s, cudaStreamWaitEvent(s->retire, s->tick_done, 0));
  SRV_CK(s, launch_moments(r.cfg.storage, res.g, s->tab, res.buf[res.parity], dout, dout + S, dout + 4 * S, 0, S, S,
                           s->retire));
  for (int b = 0; b < 2; ++b) SRV_CK(s, cudaFreeAsync(res.buf[b], s->retire));
  Retiring rt;
  rt.req = res.req;
  rt.slot = res.slot;
  rt.status = status;
  SRV_CK(s, cudaEventCreateWithFlags(&rt.done, cudaEventDisableTiming));
  SRV_CK(s, cudaEventRecord(rt.done, s->retire));
  if (res.ready) cudaEventDestroy(res.ready);
  s->retiring.push_back(rt);
  std::lock_guard<std::mutex> lk(s->mu);
  ++s->stats.kernel_launches;
  return LBM_OK;
}

// Completes the retirements whose read-back has finished: the request is done, its footprint and
// slot return to the pool.
lbm_status finish_retirements(lbm_server* s) {
  for (size_t k = 0; k < s->retiring.size();) {
    Retiring& rt = s->retiring[k];
    const cudaError_t e = cudaEventQuery(rt.done);
    if (e == cudaErrorNotReady) {
      ++k;
      continue;
    }
    if (e != cudaSuccess) return set_fatal(s, std::string("retirement failed: ") + cudaGetErrorString(e));
    cudaEventDestroy(rt.done);
    // the scheduler drops its reference before the request shows as done, so that the client's
    // poll releases the pinned fields on its own thread
    std::lock_guard<std::mutex> lk(s->mu);
    Request& r = *rt.req;
    r.t_done = Clock::now();
    r.status = rt.status;
    s->resident_bytes -= r.footprint;
    s->free_slots.push_back(rt.slot);
    ++s->stats.completed;
    if (rt.status == LBM_EUNSTABLE) ++s->stats.unstable;
    else s->stats.site_updates += r.sites * r.nsteps;
    r.done = true;
    s->retiring[k] = std::move(s->retiring.back());
    s->retiring.pop_back();
    s->cv_done.notify_all();
    s->cv_work.notify_all();
  }
  return LBM_OK;
}

lbm_status run_tick(lbm_server* s) {
  // join cases whose admission finished
  if (!s->joining.empty()) {
    for (auto& j : s->joining) {
      SRV_CK(s, cudaStreamWaitEvent(s->compute, j.ready, 0));
      s->active.push_back(j);
    }
    s->joining.clear();
    ++s->version;
    drop_graphs(s);
  }
  if (s->active.empty()) return LBM_OK;
  const int ncases = static_cast<int>(s->active.size());
  long long total_rows = 0, min_left = s->active[0].steps_left;
  TickPlan plan;
  std::vector<int> order;  // active cases grouped by kind
  for (int gi = 0; gi < kGroups; ++gi) {
    plan.first[gi] = static_cast<int>(order.size());
    for (int c = 0; c < ncases; ++c) {
      const lbm_config& cf = s->active[c].req->cfg;
      if (cf.storage == kGroupStorage[gi] && cf.equilibrium == kGroupEq[gi]) order.push_back(c);
    }
    plan.count[gi] = static_cast<int>(order.size()) - plan.first[gi];
  }
  if (static_cast<int>(order.size()) != ncases) return set_fatal(s, "a resident case has an unserved kind");
  for (int c = 0; c < ncases; ++c) {
    Resident& a = s->active[order[c]];
    CaseDesc& d = s->h_cases[c];
    int gi = 0;
    while (gi + 1 < kGroups && c >= plan.first[gi + 1]) ++gi;
    d.g = a.g;
    d.buf[0] = a.buf[0];
    d.buf[1] = a.buf[1];
    d.omega = a.omega;
    d.flag = s->d_flags + a.slot;
    d.storage = a.req->cfg.storage;
    d.eq = a.req->cfg.equilibrium;
    d.parity = a.parity;
    const long long n = static_cast<long long>(a.g.nx) * a.g.ny * a.g.nz;
    d.tiles_sub = static_cast<int>((n + kScBlock - 1) / kScBlock);
    d.tile0 = plan.tiles[gi];
    plan.tiles[gi] += d.tiles_sub;
    d.zg_face[0] = a.zg[0];
    d.zg_face[1] = a.zg[1];
    d.rows_face = 2LL * kQ * a.g.nz * a.g.ny;
    d.row0 = total_rows;
    total_rows += (a.zg[0] + a.zg[1]) * d.rows_face;
    min_left = std::min(min_left, a.steps_left);
  }
  const int K = static_cast<int>(std::min<long long>(kTickSteps, min_left));
  SRV_CK(s, cudaMemcpyAsync(s->d_cases, s->h_cases, sizeof(CaseDesc) * ncases, cudaMemcpyHostToDevice, s->compute));
  if (s->slabs_version != s->version) {
    // table positions change only with membership; parity selects the table's half
    for (int c = 0; c < ncases; ++c) {
      const Resident& a = s->active[order[c]];
      for (int par = 0; par < 2; ++par) {
        StepParams sp{};
        sp.src = a.buf[par];
        sp.dst = a.buf[par ^ 1];
        sp.g = a.g;
        fill_slab_bases(&sp, storage_bytes(a.req->cfg.storage));
        CaseSlabs& t = s->h_slabs[2 * c + par];
        std::memcpy(t.src, sp.src_slab, sizeof(t.src));
        std::memcpy(t.dst, sp.dst_slab, sizeof(t.dst));
      }
    }
    SRV_CK(s, cudaMemcpyAsync(s->d_slabs, s->h_slabs, sizeof(CaseSlabs) * 2 * ncases, cudaMemcpyHostToDevice,
                              s->compute));
    s->slabs_version = s->version;
  }
  cudaGraphExec_t g = tick_graph(s, ncases, plan, total_rows, K);
  if (!g) return set_fatal(s, "CUDA graph capture of a serving tick failed");
  SRV_CK(s, cudaGraphLaunch(g, s->compute));
  SRV_CK(s, cudaEventRecord(s->tick_done, s->compute));
  int groups = 0;
  for (int gi = 0; gi < kGroups; ++gi) groups += plan.count[gi] > 0;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    ++s->stats.graph_launches;
    s->stats.kernel_launches += static_cast<long long>(K) * ((total_rows > 0 ? 1 : 0) + 2 * groups);
    ++s->stats.ticks;
  }
  SRV_CK(s, cudaMemcpyAsync(s->h_flags, s->d_flags, sizeof(unsigned int) * s->max_cases, cudaMemcpyDeviceToHost,
                            s->compute));
  // overlap: admit newly arrived requests while the tick runs
  lbm_status st = admit_some(s);
  if (st != LBM_OK) return st;
  SRV_CK(s, cudaStreamSynchronize(s->compute));
  std::vector<Resident> keep;
  for (auto& a : s->active) {
    a.steps_left -= K;
    a.parity ^= (K & 1);
    const bool unstable = s->h_flags[a.slot] != 0;
    if (a.steps_left == 0 || unstable) {
      st = begin_retire(s, a, unstable ? LBM_EUNSTABLE : LBM_OK);
      if (st != LBM_OK) return st;
    } else {
      keep.push_back(a);
    }
  }
  if (keep.size() != s->active.size()) {
    ++s->version;
    drop_graphs(s);
  }
  s->active.swap(keep);
  return LBM_OK;
}

void worker_main(lbm_server* s) {
  cudaSetDevice(s->device);
  while (true) {
    {
      std::unique_lock<std::mutex> lk(s->mu);
      if (s->stop || s->fatal != LBM_OK) break;
      if (s->active.empty() && s->joining.empty() && s->queue.empty())
        s->cv_work.wait_for(lk, std::chrono::milliseconds(s->retiring.empty() ? 20 : 1));
      if (s->stop) break;
    }
    if (admit_some(s) != LBM_OK) break;
    if (s->active.empty() && s->joining.empty()) continue;  // (admit_some also finished retirements)
    const auto t0 = Clock::now();
    size_t held = 0;
    bool backlog = false;  // requests waiting for admission when the tick starts
    {
      std::lock_guard<std::mutex> lk(s->mu);
      held = s->resident_bytes;
      backlog = !s->queue.empty();
    }
    if (run_tick(s) != LBM_OK) break;
    const auto t1 = Clock::now();
    std::lock_guard<std::mutex> lk(s->mu);
    const double dt = std::chrono::duration<double>(t1 - t0).count();
    s->stats.busy_seconds += dt;
    const double bytes = static_cast<double>(std::max(held, s->resident_bytes));
    s->stats.resident_byte_seconds += dt * bytes;
    if (backlog) {
      s->stats.backlog_seconds += dt;
      s->stats.backlog_byte_seconds += dt * bytes;
    }
    s->stats.resident_cases = static_cast<int>(s->active.size());
  }
}

}  // namespace
}  // namespace lbm

extern "C" {

lbm_status lbm_server_create(size_t hbm_budget_bytes, int max_cases, lbm_server** out) {
  using namespace lbm;
  if (!out) return LBM_EINVAL;
  *out = nullptr;
  if (hbm_budget_bytes == 0 || max_cases < 1 || max_cases > kMaxServerCases) {
    g_server_error = "need hbm_budget_bytes > 0 and 1 <= max_cases <= 1024";
    return LBM_EINVAL;
  }
  auto* s = new (std::nothrow) lbm_server();
  if (!s) return LBM_ENOMEM;
  s->budget = hbm_budget_bytes;
  s->max_cases = max_cases;
  build_lattice_tables(&s->tab);
  for (int i = max_cases - 1; i >= 0; --i) s->free_slots.push_back(i);
  auto bail = [&](const std::string& msg) {
    g_server_error = msg;
    lbm_server_destroy(s);
    return LBM_ECUDA;
  };
  if (cudaGetDevice(&s->device) != cudaSuccess) return bail("cudaGetDevice failed");
  if (cudaStreamCreateWithFlags(&s->compute, cudaStreamNonBlocking) != cudaSuccess ||
      cudaStreamCreateWithFlags(&s->admit, cudaStreamNonBlocking) != cudaSuccess ||
      cudaStreamCreateWithFlags(&s->retire, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&s->tick_done, cudaEventDisableTiming) != cudaSuccess)
    return bail("stream creation failed");
  if (cudaMalloc(&s->d_cases, sizeof(CaseDesc) * max_cases) != cudaSuccess ||
      cudaMallocHost(&s->h_cases, sizeof(CaseDesc) * max_cases) != cudaSuccess ||
      cudaMalloc(&s->d_slabs, sizeof(CaseSlabs) * 2 * max_cases) != cudaSuccess ||
      cudaMallocHost(&s->h_slabs, sizeof(CaseSlabs) * 2 * max_cases) != cudaSuccess ||
      cudaMalloc(&s->d_flags, sizeof(unsigned int) * max_cases) != cudaSuccess ||
      cudaMallocHost(&s->h_flags, sizeof(unsigned int) * max_cases) != cudaSuccess) {
    cudaGetLastError();
    return bail("device allocation failed");
  }
  cudaMemset(s->d_flags, 0, sizeof(unsigned int) * max_cases);
  int sms = 0, per_sm = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, s->device);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, served_step_kernel<float, kEqSeries, 0>, kScBlock, 0);
  s->grid_blocks = std::max(1, sms * std::max(1, per_sm));
  s->worker = std::thread(worker_main, s);
  *out = s;
  return LBM_OK;
}

lbm_status lbm_submit(lbm_server* s, const lbm_config* cfg, const double* rho, const double* u, const double* theta,
                      long long nsteps, long long* ticket) {
  using namespace lbm;
  if (!s || !cfg || !rho || !u || !theta || !ticket || nsteps < 1) return LBM_EINVAL;
  Geometry g;
  std::string why;
  if (plan_geometry(cfg, &g, &why) != LBM_OK) {
    std::lock_guard<std::mutex> lk(s->mu);
    s->err = why;
    return LBM_EINVAL;
  }
  if (cfg->face[0].kind == LBM_BC_BOUNCE_BACK || cfg->face[1].kind == LBM_BC_BOUNCE_BACK) {
    std::lock_guard<std::mutex> lk(s->mu);
    s->err = "served cases take periodic, zero-gradient or equilibrium-inflow faces";
    return LBM_EINVAL;
  }
  if (cfg->storage == LBM_F64 || cfg->fp64_moments ||
      (cfg->equilibrium != LBM_EQ_SERIES && cfg->equilibrium != LBM_EQ_ENTROPIC) ||
      cfg->collision != LBM_COLLISION_BGK || cfg->streaming != LBM_STREAM_PINGPONG) {
    std::lock_guard<std::mutex> lk(s->mu);
    s->err = "served cases use FP32, FP16 or BF16 storage with FP32 moments, the series or the exact entropic "
             "equilibrium, BGK collision and ping-pong streaming";
    return LBM_EINVAL;
  }
  auto r = std::make_shared<Request>();
  r->cfg = *cfg;
  r->nsteps = nsteps;
  r->sites = 2LL * cfg->nx * cfg->ny * cfg->nz;
  r->footprint = static_cast<size_t>(2 * 2 * g.sub_stride) * storage_bytes(cfg->storage);
  if (r->footprint > s->budget) {
    std::lock_guard<std::mutex> lk(s->mu);
    s->err = "case footprint exceeds the server's HBM budget";
    ++s->stats.rejected;
    return LBM_ENOMEM;
  }
  const long long S = r->sites;
  if (!r->in.alloc(5 * S) || !r->out.alloc(5 * S)) {
    std::lock_guard<std::mutex> lk(s->mu);
    s->err = "pinned host memory for the request's fields could not be allocated";
    return LBM_ENOMEM;
  }
  std::memcpy(r->in.p, rho, S * sizeof(double));
  std::memcpy(r->in.p + S, u, 3 * S * sizeof(double));
  std::memcpy(r->in.p + 4 * S, theta, S * sizeof(double));
  r->t_submit = Clock::now();
  {
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->fatal != LBM_OK) return s->fatal;
    r->ticket = s->next_ticket++;
    s->queue.push_back(r);
    s->requests[r->ticket] = r;
    ++s->stats.submitted;
  }
  s->cv_work.notify_all();
  *ticket = r->ticket;
  return LBM_OK;
}

lbm_status lbm_poll(lbm_server* s, long long ticket, double* rho, double* u, double* theta, double* latency_s) {
  using namespace lbm;
  if (!s) return LBM_EINVAL;
  std::shared_ptr<Request> r;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->requests.find(ticket);
    if (it == s->requests.end()) return LBM_ENOTFOUND;
    r = it->second;
    if (!r->done) return s->fatal != LBM_OK ? s->fatal : LBM_EBUSY;
    s->requests.erase(it);
  }
  const long long S = r->sites;
  if (rho) std::memcpy(rho, r->out.p, S * sizeof(double));
  if (u) std::memcpy(u, r->out.p + S, 3 * S * sizeof(double));
  if (theta) std::memcpy(theta, r->out.p + 4 * S, S * sizeof(double));
  if (latency_s) *latency_s = std::chrono::duration<double>(r->t_done - r->t_submit).count();
  return r->status;
}

lbm_status lbm_wait(lbm_server* s, long long ticket, double timeout_s) {
  using namespace lbm;
  if (!s || !(timeout_s >= 0)) return LBM_EINVAL;
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->requests.find(ticket);
  if (it == s->requests.end()) return LBM_ENOTFOUND;
  auto r = it->second;
  const bool ok = s->cv_done.wait_for(lk, std::chrono::duration<double>(timeout_s),
                                      [&] { return r->done || s->fatal != LBM_OK; });
  if (s->fatal != LBM_OK) return s->fatal;
  return ok ? LBM_OK : LBM_ETIMEOUT;
}

lbm_status lbm_server_get_stats(lbm_server* s, lbm_server_stats* out) {
  if (!s || !out) return LBM_EINVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  *out = s->stats;
  out->resident_bytes = s->resident_bytes;
  out->queued = static_cast<long long>(s->queue.size());
  return LBM_OK;
}

const char* lbm_server_last_error(const lbm_server* s) {
  if (!s) return lbm::g_server_error.c_str();
  // a copy taken under the lock: the scheduler thread may replace the message meanwhile
  thread_local std::string copy;
  {
    std::lock_guard<std::mutex> lk(const_cast<lbm_server*>(s)->mu);
    copy = s->err;
  }
  return copy.c_str();
}

lbm_status lbm_server_destroy(lbm_server* s) {
  using namespace lbm;
  if (!s) return LBM_EINVAL;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
  }
  s->cv_work.notify_all();
  if (s->worker.joinable()) s->worker.join();
  int prev = -1;
  cudaGetDevice(&prev);
  if (prev != s->device) cudaSetDevice(s->device);
  if (s->compute) cudaStreamSynchronize(s->compute);
  if (s->admit) cudaStreamSynchronize(s->admit);
  if (s->retire) cudaStreamSynchronize(s->retire);
  for (auto& rt : s->retiring)
    if (rt.done) cudaEventDestroy(rt.done);
  s->retiring.clear();
  for (auto* v : {&s->active, &s->joining})
    for (auto& a : *v) {
      for (int b = 0; b < 2; ++b)
        if (a.buf[b]) cudaFree(a.buf[b]);
      if (a.ready) cudaEventDestroy(a.ready);
    }
  drop_graphs(s);
  if (s->d_cases) cudaFree(s->d_cases);
  if (s->h_cases) cudaFreeHost(s->h_cases);
  if (s->d_slabs) cudaFree(s->d_slabs);
  if (s->h_slabs) cudaFreeHost(s->h_slabs);
  if (s->d_flags) cudaFree(s->d_flags);
  if (s->h_flags) cudaFreeHost(s->h_flags);
  if (s->tick_done) cudaEventDestroy(s->tick_done);
  if (s->compute) cudaStreamDestroy(s->compute);
  if (s->admit) cudaStreamDestroy(s->admit);
  if (s->retire) cudaStreamDestroy(s->retire);
  if (prev >= 0 && prev != s->device) cudaSetDevice(prev);
  delete s;
  return LBM_OK;
}

}  // extern "C"
