/*
 * liblbm_rd3q81 -- GB300 (sm_103a) implementation of the RD3Q81 lattice Boltzmann step.
 *
 * Paper: M. Atif, N. H. Maruthi, P. K. Kolluru, C. Thantanapally, S. Ansumali,
 * "Lattice Boltzmann Model for Transonic Flows", arXiv 2409.05114.
 *
 * One step (lbm_step) is, for every site x of the grid and every velocity c_i,
 *   f_i(x + c_i, t + 1) = f_i(x, t) + alpha beta [f~eq_i(rho, u, theta) - f_i(x, t)]
 * with alpha = 2 and beta = 1 / (2 tau + 1) (Sec. II, Eq. (discretelbm)); rho, rho u and
 * rho u^2 + 3 rho theta are the moments <f, 1>, <f, c>, <f, c^2> (Eq. (conslaws)); f~eq is
 * the series entropic equilibrium with temperature-dependent weights W~_i(theta) to eta^4,
 * f^(2), f^(3) and R-bar (App. B); the 81 velocities and weights are Table "tab:weights".
 *
 * Grid.  The physical lattice is body-centred cubic: a primary sublattice P (site index
 * n = (x, y, z), position n) and a replica sublattice R (same index range, position
 * n + (1/2, 1/2, 1/2)).  Half-integer velocities (BCC-1/2, 3/2, 5/2) move populations
 * between P and R (Sec. I, replica grid).  A grid nx*ny*nz therefore has 2*nx*ny*nz sites.
 *
 * Field layout (lbm_init, lbm_moments): site-major, all P sites then all R sites, each
 * block ordered z, y, x with x fastest: site k = sub*nx*ny*nz + (z*ny + y)*nx + x.
 * Scalars rho[k], theta[k] have 2*nx*ny*nz entries; velocity u is [3][2*nx*ny*nz]
 * (all u_x, then all u_y, then all u_z).
 * Population layout (lbm_get_populations / lbm_set_populations): dense FP64
 * f[sub][i][z][y][x], i in the library's direction order (lbm_velocities).
 *
 * Memory.  The context owns its device memory (two population buffers, ping-pong; one with
 * AA streaming).  The caller owns every field buffer it passes; the library copies in or out
 * and keeps no caller pointer after a call returns.  on_device = 1 means the pointers are
 * device pointers of the context's device (for example a torch tensor's data_ptr()), read or
 * written in order on the context's stream; on_device = 0 means host memory.  Host fields
 * that are page-locked (cudaHostAlloc / cudaHostRegister, e.g. pinned torch tensors; each
 * field one allocation) move without extra host copies: lbm_init reads them in place from its
 * kernel over the host link; lbm_moments and lbm_advance_fields move them with the copy
 * engines, one z slab at a time through a ring of device staging slots (part of the context's
 * footprint), overlapped with the kernels.  Pageable host memory goes through chunked copies.
 *
 * Errors.  Every call returns an lbm_status; no C++ exception crosses this interface.
 * A NULL or destroyed context gives LBM_EINVAL.  lbm_last_error() describes the last
 * failure.  LBM_EUNSTABLE is returned by the synchronising calls once any site has seen a
 * non-finite value, rho <= 0 or theta <= 0 (the series equilibrium has a limited range in
 * temperature deviation and Mach number; the populations are left as computed).
 *
 * Threads.  Calls on one context must not overlap; different contexts are independent.
 */
#ifndef LBM_RD3Q81_H
#define LBM_RD3Q81_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lbm_ctx lbm_ctx;

typedef enum {
  LBM_OK = 0,
  LBM_EINVAL = 1,    /* invalid argument or configuration */
  LBM_ENOMEM = 2,    /* device memory (or the server's HBM budget) exhausted */
  LBM_ECUDA = 3,     /* a CUDA call failed; see lbm_last_error */
  LBM_EUNSTABLE = 4, /* a site saw rho <= 0, theta <= 0 or a non-finite value */
  LBM_ETIMEOUT = 5,  /* a bounded wait ran out */
  LBM_EBUSY = 6,     /* result not ready yet (serving) */
  LBM_ENOTFOUND = 7  /* unknown ticket (serving) */
} lbm_status;

typedef enum { LBM_RD3Q81 = 1 } lbm_velset;

typedef enum {
  LBM_BC_PERIODIC = 0,      /* wrap-around; the opposite face must be periodic too */
  LBM_BC_ZERO_GRADIENT = 1, /* outflow: ghost sites copy the nearest interior site of the
                               same sublattice (all 81 populations) before every step */
  LBM_BC_EQ_INFLOW = 2,     /* ghost sites hold f~eq(rho, u, theta) of the face's state */
  LBM_BC_BOUNCE_BACK = 3    /* solid wall (the Sod tube's x ends, Sec. IV A): a population whose
                               link from a fluid site would end outside the fluid index range
                               0 <= x < nx comes back to that site one step later with the reversed
                               velocity, f_-i(x, t+1) = f*_i(x, t).  Keeps every population, so mass
                               and energy are conserved exactly.  Not available to served cases. */
} lbm_bc_kind;

typedef enum {
  LBM_F64 = 0,        /* populations stored as FP64, all arithmetic FP64 */
  LBM_F32 = 1,        /* stored as FP32, collide in FP32 */
  LBM_F16_OFFSET = 2, /* stored as FP16 offsets d_i = f_i / w_i - 1, collide in FP32 */
  LBM_BF16_OFFSET = 3 /* stored as BF16 offsets d_i = f_i / w_i - 1, collide in FP32 */
} lbm_storage;

typedef enum {
  LBM_EQ_SERIES = 0,  /* the series form of App. B (temperature weights to eta^4, f^(2), f^(3), R-bar) */
  LBM_EQ_ENTROPIC = 1, /* the exact entropic equilibrium of Sec. III: w_i rho exp(mu + zeta.c_i + gamma c_i^2)
                          minimising H = <f, log(f/w) - 1>, its multipliers found per site by Newton on
                          the paper's 5x5 moment system (positive populations; the Mach-2 regime) */
  LBM_EQ_SERIES_EXACT_W = 2 /* the series form of App. B with the exact temperature weights
                               W_i(theta) = w_i A G^(4 c_i^2) of Eq. (zeroveleq) (G per site by a 1-D
                               Newton on theta'(G) = F2 / (3 theta0 F0)) in place of the eta^4 series */
} lbm_equilibrium;

typedef enum {
  LBM_COLLISION_BGK = 0,     /* f += alpha beta (feq - f) with alpha = 2 (Eq. (discretelbm)) */
  LBM_COLLISION_ENTROPIC = 1 /* alpha per site: the nontrivial root of H[f + alpha (feq - f)] - H[f] = 0
                                (Eq. (delH), H = <f, log(f/w) - 1>), kept where every population stays
                                positive; needs LBM_EQ_ENTROPIC */
} lbm_collision;

typedef enum {
  LBM_STREAM_PINGPONG = 0, /* two population buffers: each step reads one and writes the other */
  LBM_STREAM_AA = 1        /* one buffer, updated in place by two alternating step kinds: one reads and writes
                              each site's own populations (into the slots of the opposite directions), the
                              next pulls from and pushes to the neighbours.  Half the memory of ping-pong;
                              the same arithmetic, so results agree with ping-pong to rounding (the step
                              kinds are separately compiled, and a multiply-add may contract differently) */
} lbm_streaming;

typedef struct {
  int kind;                          /* lbm_bc_kind */
  double rho, ux, uy, uz, theta;     /* state of an LBM_BC_EQ_INFLOW face; ignored otherwise */
} lbm_bc;

typedef struct {
  int nx, ny, nz;     /* sites per sublattice along x, y, z (each >= 1) */
  int velset;         /* LBM_RD3Q81 */
  double tau;         /* the paper's relaxation time: beta = 1 / (2 tau + 1), tau >= 0 */
  lbm_bc face[6];     /* -x, +x, -y, +y, -z, +z.  This version accepts non-periodic kinds
                         on the two x faces only; y and z must be periodic. */
  int storage;        /* lbm_storage */
  int fp64_moments;   /* 1: moment sums and temperature recovery to FP64 quality for FP32/FP16/
                         BF16 storage (no effect for LBM_F64), without FP64 arithmetic: FP32
                         storage by exact 64-bit integer sums of the values scaled by a power
                         of two, FP16/BF16 by cascaded double-word (float + float, ~2^-48
                         relative) sums of each shell's offsets, weighted by the shell's
                         weights held as double words; u and theta then in double-word
                         arithmetic; 0: FP32 */
  void* cuda_stream;  /* cudaStream_t the context issues its work on; NULL: the context
                         creates its own stream (which synchronises with the legacy
                         default stream) */
  int equilibrium;    /* lbm_equilibrium (init, inflow faces and every step).  fp64_moments = 1
                         is available with LBM_EQ_SERIES only; a site whose Newton iteration
                         breaks down raises the instability flag (LBM_EUNSTABLE) */
  int collision;      /* lbm_collision.  LBM_COLLISION_ENTROPIC needs equilibrium =
                         LBM_EQ_ENTROPIC.  A site with a population <= 0 (where H is not
                         defined) takes alpha = 2. */
  int streaming;      /* lbm_streaming */
} lbm_config;

/* Device bytes lbm_create would allocate for this configuration (both population buffers
 * and internal scratch).  Returns LBM_EINVAL for an invalid configuration. */
lbm_status lbm_footprint(const lbm_config* cfg, size_t* bytes);

/* Creates a context on the current CUDA device: validates cfg, allocates the population
 * buffers (two, or one with AA streaming).  On failure *out is NULL and lbm_last_error(NULL)
 * tells why. */
lbm_status lbm_create(const lbm_config* cfg, lbm_ctx** out);

/* Sets every site's populations to f~eq(rho, u, theta) (App. B).  Fields as described
 * above; they must be finite with rho > 0 and theta > 0 (not checked element-wise: a bad
 * value shows up as LBM_EUNSTABLE later).  Also writes the equilibrium-inflow ghost layers.
 * With on_device = 0 the call returns after the host data has been consumed. */
lbm_status lbm_init(lbm_ctx* ctx, const double* rho, const double* u, const double* theta, int on_device);

/* Advances n >= 0 time steps: per step, zero-gradient ghost fills (if any) then one fused
 * pull-stream-collide kernel over all sites.  Stream-ordered: returns once the work is
 * queued.  Returns LBM_EINVAL if lbm_init / lbm_set_populations was never called. */
lbm_status lbm_step(lbm_ctx* ctx, long long n);

/* lbm_init, lbm_step(n) and lbm_moments as one call: sets every site to f~eq of the fields
 * rho, u, theta, advances n >= 0 steps and writes the fields of the result to rho_out, u_out,
 * theta_out (layouts as lbm_init; the outputs may be the inputs).  The context keeps the state
 * afterwards, as after the three calls, and the fields are bitwise those of the three calls.
 * With page-locked host fields the work runs slab by slab in z (ping-pong or AA streaming): the
 * host-to-device copy of later slabs, the kernels, and the device-to-host copy of finished slabs
 * overlap (both directions of the host link at once when n <= 1; for n >= 2 the input overlaps
 * initialisation and the output overlaps the last step).  Device fields and pageable memory
 * run the three calls one after the other.  Synchronises; LBM_EUNSTABLE as lbm_moments;
 * LBM_EINVAL for NULL fields or n < 0. */
lbm_status lbm_advance_fields(lbm_ctx* ctx, const double* rho, const double* u, const double* theta, long long n,
                              double* rho_out, double* u_out, double* theta_out, int on_device);

/* rho, u, theta of the stored (post-collision) state (Eq. (conslaws)), returned in FP64;
 * layout as for lbm_init.  FP64 storage sums and divides in FP64.  FP32/FP16/BF16 storage sums
 * each velocity shell in FP32, then combines the shells, divides and forms theta in double-word
 * (float + float) arithmetic: relative error ~1e-14 beyond the FP32 shell sums, at FP32 speed
 * (this GPU runs FP64 at a small fraction of its FP32 rate).  Synchronises the stream; returns LBM_EUNSTABLE (after writing
 * the fields) if any step so far was flagged. */
lbm_status lbm_moments(lbm_ctx* ctx, double* rho, double* u, double* theta, int on_device);

/* Mean kinetic energy and mean enstrophy of the stored state (Sec. IV C, compressible
 * Taylor-Green vortex): out2[0] = KE = <rho u.u / 2>, out2[1] = eps = <rho w.w / 2>, w = curl u,
 * averages over all 2 nx ny nz sites (host memory, 2 doubles).  The paper gives no
 * discretisation of the curl: it is taken on each sublattice's own grid (unit spacing) by
 * second-order central differences; y and z wrap, x wraps when the x faces are periodic and
 * otherwise uses second-order one-sided differences at the end planes.  FP64 fields and
 * deterministic sums.  Allocates 40 bytes per site of device memory for the call (stream-
 * ordered, freed before it returns); synchronises.  LBM_EINVAL: NULL out2, context not
 * initialised, or non-periodic x with nx < 3; LBM_ENOMEM: no room for the fields. */
lbm_status lbm_diagnostics(lbm_ctx* ctx, double* out2);

/* Self-check, no counterpart in the paper: the largest relative difference between the FP32
 * log(1 + y) that the entropic-alpha solve uses and CUDA's log1pf over n points of a fixed sweep
 * of y in (-0.999, 100), written to *max_rel_err (host).  Runs on the current device and
 * synchronises.  LBM_EINVAL: n < 1 or NULL output; LBM_ENOMEM / LBM_ECUDA on device errors. */
lbm_status lbm_selftest_log1p(long long n, double* max_rel_err);

/* Global sums over all sites of rho, rho u_x, rho u_y, rho u_z and <f, c^2>, FP64,
 * bitwise reproducible for a given state (fixed reduction order).  out5: host double[5].
 * Synchronises. */
lbm_status lbm_totals(lbm_ctx* ctx, double* out5);

/* Copies the populations out as dense FP64 f[sub][i][z][y][x] (2*81*nx*ny*nz values),
 * decoding offset storage (f = w_i (1 + d_i)).  Synchronises. */
lbm_status lbm_get_populations(lbm_ctx* ctx, double* f, int on_device);

/* Sets the populations from dense FP64 f[sub][i][z][y][x] (encoding to the storage type).
 * Also writes the equilibrium-inflow ghost layers.  Synchronises. */
lbm_status lbm_set_populations(lbm_ctx* ctx, const double* f, int on_device);

/* Gathers the 81 populations (FP64, decoded, library direction order) of `count` sites:
 * f[k*81 + i] for site index sites[k] (0 <= sites[k] < 2*nx*ny*nz, field layout order).
 * Host arrays.  Out-of-range indices give LBM_EINVAL before any work.  Synchronises. */
lbm_status lbm_probe(lbm_ctx* ctx, const long long* sites, long long count, double* f);

/* Waits for the context's queued work; LBM_EUNSTABLE if any step so far was flagged. */
lbm_status lbm_sync(lbm_ctx* ctx);

/* Number of kernel launches the context has issued so far (host-side count; every step
 * issues 1 fused kernel plus 1 per zero-gradient face). */
lbm_status lbm_launch_count(const lbm_ctx* ctx, long long* count);

/* Frees the context and its device memory (after waiting for its queued work). */
lbm_status lbm_destroy(lbm_ctx* ctx);

/* Message of the last failure on ctx, or of the last failed lbm_create on this thread when
 * ctx is NULL.  Never NULL; valid until the next call on the same context / thread. */
const char* lbm_last_error(const lbm_ctx* ctx);

/* The library's velocity set: h[3*i + a] = 2 c_{i,a} (integers) and w[i] = w_i, for the
 * 81 directions in the library's order (rest first, then +v/-v pairs shell by shell as in
 * Table "tab:weights").  Either pointer may be NULL.  Returns 81. */
int lbm_velocities(int* h, double* w);

/* The global sums of lbm_totals (rho, rho u_x, rho u_y, rho u_z, <f, c^2>) for a caller that
 * cannot allocate device memory -- for example because its own memory pool already holds
 * the device's free memory, or because it must not call cudaMalloc/cudaFree, which can
 * synchronise the whole device.  The paper has no counterpart; this is plumbing.  It needs
 * no context and allocates nothing.  f: device pointer to dense populations
 * f[sub][i][z][y][x] in the storage type `storage` (lbm_storage; offset types hold
 * d = f/w - 1), i in the library's direction order; out5: device pointer to 5 doubles;
 * cuda_stream: the stream to run on (NULL: legacy default).  Asynchronous: returns after
 * queueing two kernels.  Its scratch is a fixed 160 KiB device array inside the library
 * (4096 partial sums of 8192 sites each), which every device that loads the library holds
 * until exit; grids with 2*nx*ny*nz > 33,554,432 sites are rejected with LBM_EINVAL.  The
 * first call on a device, with that device current, looks up the array's device address
 * (cudaGetSymbolAddress), so make it before any stream capture; the address is kept for the
 * life of the process, so a cudaDeviceReset by the application invalidates the entry point on
 * that device.  All calls share the array,
 * which keeps the last call's contents; calls that overlap on the GPU (different streams)
 * race on it.  Returns LBM_EINVAL for bad arguments, LBM_ECUDA if a launch fails. */
lbm_status lbm_totals_noalloc(const void* f, int storage, int nx, int ny, int nz, double* out5, void* cuda_stream);

/* ---- serving: continuous batching of independent cases on one GPU --------------------
 *
 * A server keeps many cases (each an lbm_config with its own grid, tau, faces and storage)
 * resident on the current device and advances all of them together: every time step is
 * one persistent fused kernel per kind of case present (storage type and equilibrium), over a
 * packed index of those cases'
 * sites (plus one batched zero-gradient fill if any resident case needs it), and runs of up
 * to 16 steps are replayed as CUDA graphs.  Requests are admitted in submission order whenever a slot is
 * free and the sum of resident case footprints (2 population buffers each) stays within
 * the HBM budget; when the oldest waiting request does not fit the free budget, the first of
 * the next 15 that fits goes ahead of it, but no request is passed over more than 8 times.
 * Admission (an initialisation kernel that reads the request's fields in place from pinned,
 * device-mapped host memory) runs on its own stream while the resident cases compute.  A case
 * leaves after its step count, or early when one of its sites becomes unstable; its fields are
 * then written back, again in place into pinned host memory, on a third stream while the
 * next steps run.  Its result is bitwise the same whether it is
 * served alone or in any mix (sites are independent and every case runs the same kernel),
 * and equals lbm_step's to rounding (the same arithmetic, compiled into another kernel).
 * A scheduler thread owned by the server does all GPU work; the calls are thread-safe. */
typedef struct lbm_server lbm_server;

typedef struct {
  long long submitted, admitted, completed, unstable, rejected, queued;
  long long site_updates;           /* sum of sites x steps over cases completed OK */
  long long ticks, kernel_launches, graph_launches;
  int resident_cases;
  size_t resident_bytes, peak_resident_bytes;
  double busy_seconds;              /* scheduler time spent running ticks */
  double resident_byte_seconds;     /* resident bytes integrated over that time (per tick, the larger of
                                       the counts before and after it): mean resident = this / busy */
  double backlog_seconds;           /* the part of busy_seconds in ticks that began with requests waiting */
  double backlog_byte_seconds;      /* resident bytes integrated over backlog_seconds */
} lbm_server_stats;

/* Creates a server on the current device.  hbm_budget_bytes bounds the resident cases'
 * population memory (the server adds about 5 KB of tables per case slot); 1 <= max_cases <= 1024. */
lbm_status lbm_server_create(size_t hbm_budget_bytes, int max_cases, lbm_server** out);

/* Queues one case: configuration (storage FP32, FP16 or BF16 offsets, fp64_moments = 0,
 * the series equilibrium of App. B or the exact entropic equilibrium of Sec. III, BGK collision,
 * ping-pong streaming, x faces periodic, zero-gradient or equilibrium inflow; cuda_stream is
 * ignored), initial fields in host memory (layout as lbm_init; copied into pinned host memory
 * of the request's own, 80 bytes per site with its result, before the call returns; released
 * when lbm_poll hands the result over, or by lbm_server_destroy) and
 * nsteps >= 1.  Returns a ticket.  LBM_ENOMEM if the case alone exceeds the budget or its
 * pinned memory cannot be allocated, LBM_EINVAL for an invalid configuration. */
lbm_status lbm_submit(lbm_server* srv, const lbm_config* cfg, const double* rho, const double* u,
                      const double* theta, long long nsteps, long long* ticket);

/* Non-blocking.  LBM_EBUSY while the case is queued or running; once it is done, copies
 * rho, u, theta (host arrays, layout as lbm_moments; any may be NULL) and the time from
 * submission to completion, returns the case's status (LBM_OK or LBM_EUNSTABLE) and
 * forgets the ticket (LBM_ENOTFOUND afterwards). */
lbm_status lbm_poll(lbm_server* srv, long long ticket, double* rho, double* u, double* theta,
                    double* latency_s);

/* Blocks until the case is done (LBM_OK, then lbm_poll for the result) or timeout_s
 * seconds passed (LBM_ETIMEOUT). */
lbm_status lbm_wait(lbm_server* srv, long long ticket, double timeout_s);

lbm_status lbm_server_get_stats(lbm_server* srv, lbm_server_stats* out);

/* Message of the server's last failure (or of the last failed lbm_server_create when srv
 * is NULL).  The string stays valid until the calling thread's next call of this function. */
const char* lbm_server_last_error(const lbm_server* srv);

/* Stops the scheduler (queued and running cases are dropped) and frees everything. */
lbm_status lbm_server_destroy(lbm_server* srv);

#ifdef __cplusplus
}
#endif

#endif /* LBM_RD3Q81_H */
