// lbm_totals_noalloc: the global conservation sums of lbm_totals for callers that cannot
// allocate device memory themselves or through the library -- for example an application
// whose memory pool already holds the device's free memory, or code that must not call
// cudaMalloc/cudaFree because those calls can synchronise the whole device.  It needs no
// context (lbm_create allocates) and allocates nothing: the caller passes the populations
// and the output, and the per-block partial sums live in a fixed-size array in this file.
#include <mutex>

#include "device_common.cuh"
#include "reduce.cuh"
#include "lbm.h"

namespace lbm {
namespace {

constexpr int kNaThreads = 256;
constexpr long long kNaSitesPerBlock = 8192;  // sites reduced by one block (32 per thread)
constexpr int kNaMaxBlocks = 4096;            // capacity of the static partial-sum array
constexpr int kNaMaxDevices = 64;

// Partial sums (rho, j_x, j_y, j_z, <f, c^2>) of every block: 4096 x 5 doubles = 160 KiB,
// held by every device that loads the library until the process exits.  Each call
// overwrites the slots of the blocks it launches before reading them, so nothing needs
// clearing; calls that overlap on the GPU (different streams) share it and race.
static __device__ __align__(256) double g_na_partials[kNaMaxBlocks * 5];

std::mutex g_na_mu;
double* g_na_ptr[kNaMaxDevices] = {};  // device address of g_na_partials, per device

template <class S>
__device__ __forceinline__ double na_decode(const S* p, double w) {
  if constexpr (Codec<S>::kOffset) return w * (1.0 + static_cast<double>(Codec<S>::load(p)));
  else return static_cast<double>(*p);
}

// Pass 1: block b sums sites [b * kNaSitesPerBlock, (b+1) * kNaSitesPerBlock) of the dense
// layout f[sub][i][z][y][x] (site index k = sub*n + t), in a fixed order, into partials[b].
template <class S>
__global__ void na_pass1(const S* __restrict__ f, long long n, LatticeTables tab, double* partials) {
  const long long sites = 2 * n;
  const long long first = static_cast<long long>(blockIdx.x) * kNaSitesPerBlock;
  const long long last = first + kNaSitesPerBlock < sites ? first + kNaSitesPerBlock : sites;
  double acc[5] = {0, 0, 0, 0, 0};
  for (long long k = first + threadIdx.x; k < last; k += kNaThreads) {
    const long long sub = k >= n ? 1 : 0;
    const S* base = f + sub * kQ * n + (k - sub * n);
    double r = 0, jx = 0, jy = 0, jz = 0, e = 0;
    static_for<kQ>([&](auto Ic) {
      constexpr int i = decltype(Ic)::value;
      constexpr rd3q81::Dir d = rd3q81::kDirs[i];
      constexpr double c2 = rd3q81::kShellC2[d.shell];
      const double v = na_decode(base + i * n, tab.w[d.shell]);
      r += v;
      jx += 0.5 * d.hx * v;
      jy += 0.5 * d.hy * v;
      jz += 0.5 * d.hz * v;
      e += c2 * v;
    });
    acc[0] += r;
    acc[1] += jx;
    acc[2] += jy;
    acc[3] += jz;
    acc[4] += e;
  }
  block_sum5_fixed<kNaThreads>(acc);
  if (threadIdx.x == 0)
    for (int q = 0; q < 5; ++q) partials[blockIdx.x * 5 + q] = acc[q];
}

// one warp
__global__ void na_pass2(const double* partials, int nblocks, double* out) {
  warp_total5_fixed(partials, nblocks, out);
}

// Address of the static array on the current device, looked up once per device (the first
// call on a device, with that device current).
lbm_status na_scratch(double** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return LBM_ECUDA;
  if (dev < 0 || dev >= kNaMaxDevices) return LBM_EINVAL;
  std::lock_guard<std::mutex> lk(g_na_mu);
  if (!g_na_ptr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_na_partials) != cudaSuccess) return LBM_ECUDA;
    g_na_ptr[dev] = static_cast<double*>(p);
  }
  *out = g_na_ptr[dev];
  return LBM_OK;
}

}  // namespace
}  // namespace lbm

extern "C" {

lbm_status lbm_totals_noalloc(const void* f, int storage, int nx, int ny, int nz, double* out5, void* cuda_stream) {
  using namespace lbm;
  if (!f || !out5) return LBM_EINVAL;
  if (storage < LBM_F64 || storage > LBM_BF16_OFFSET) return LBM_EINVAL;
  if (nx < 1 || ny < 1 || nz < 1) return LBM_EINVAL;
  const long long n = static_cast<long long>(nx) * ny * nz;
  const long long nblocks = (2 * n + kNaSitesPerBlock - 1) / kNaSitesPerBlock;
  if (nblocks > kNaMaxBlocks) return LBM_EINVAL;  // more partial sums than the static array holds
  double* partials = nullptr;
  lbm_status st = na_scratch(&partials);
  if (st != LBM_OK) return st;
  LatticeTables tab;
  build_lattice_tables(&tab);
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  const int nb = static_cast<int>(nblocks);
  switch (storage) {
    case LBM_F64: na_pass1<double><<<nb, kNaThreads, 0, s>>>(static_cast<const double*>(f), n, tab, partials); break;
    case LBM_F32: na_pass1<float><<<nb, kNaThreads, 0, s>>>(static_cast<const float*>(f), n, tab, partials); break;
    case LBM_F16_OFFSET:
      na_pass1<__half><<<nb, kNaThreads, 0, s>>>(static_cast<const __half*>(f), n, tab, partials);
      break;
    default:
      na_pass1<__nv_bfloat16><<<nb, kNaThreads, 0, s>>>(static_cast<const __nv_bfloat16*>(f), n, tab, partials);
      break;
  }
  if (cudaGetLastError() != cudaSuccess) return LBM_ECUDA;
  na_pass2<<<1, 32, 0, s>>>(partials, nb, out5);
  if (cudaGetLastError() != cudaSuccess) return LBM_ECUDA;
  return LBM_OK;
}

}  // extern "C"
