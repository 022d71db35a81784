// Self-check of the FP32 log(1 + y) that the entropic alpha solve uses (log1p_alpha in
// stream_collide.cuh) against CUDA's log1pf, on a fixed sweep of y over (-0.999, 100).
#include "stream_collide.cuh"

namespace lbm {
namespace {

constexpr int kSelfBlock = 256;

__global__ void log1p_check_kernel(long long n, float* worst) {
  __shared__ float sw[kSelfBlock];
  float w = 0.0f;
  for (long long k = static_cast<long long>(blockIdx.x) * kSelfBlock + threadIdx.x; k < n;
       k += static_cast<long long>(gridDim.x) * kSelfBlock) {
    // three ranges: (-0.999, -0.25), [-0.25, 0.25) densely, [0.25, 100) geometrically
    const double t = (k + 0.5) / static_cast<double>(n);
    double yd;
    if (t < 0.3) yd = -0.999 + (0.749) * (t / 0.3);
    else if (t < 0.7) yd = -0.25 + 0.5 * ((t - 0.3) / 0.4);
    else yd = 0.25 * pow(400.0, (t - 0.7) / 0.3);
    const float y = static_cast<float>(yd);
    const float ref = log1pf(y);
    const float got = log1p_alpha(y);
    const float err = fabsf(got - ref) / fmaxf(fabsf(ref), 1e-30f);
    w = fmaxf(w, err);
  }
  sw[threadIdx.x] = w;
  __syncthreads();
  for (int h = kSelfBlock / 2; h > 0; h >>= 1) {
    if (threadIdx.x < h) sw[threadIdx.x] = fmaxf(sw[threadIdx.x], sw[threadIdx.x + h]);
    __syncthreads();
  }
  if (threadIdx.x == 0) worst[blockIdx.x] = sw[0];
}

}  // namespace
}  // namespace lbm

extern "C" lbm_status lbm_selftest_log1p(long long n, double* max_rel_err) {
  if (n < 1 || !max_rel_err) return LBM_EINVAL;
  constexpr int kBlocks = 152;
  float* d = nullptr;
  if (cudaMalloc(&d, kBlocks * sizeof(float)) != cudaSuccess) return LBM_ENOMEM;
  lbm::log1p_check_kernel<<<kBlocks, lbm::kSelfBlock>>>(n, d);
  float h[kBlocks];
  cudaError_t e = cudaMemcpy(h, d, sizeof(h), cudaMemcpyDeviceToHost);
  cudaFree(d);
  if (e != cudaSuccess) return LBM_ECUDA;
  float w = 0.0f;
  for (float v : h) w = v > w ? v : w;
  *max_rel_err = w;
  return LBM_OK;
}
