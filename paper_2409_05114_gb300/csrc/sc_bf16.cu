// Fused stream-collide instantiations for __nv_bfloat16 storage (one translation unit per storage
// type so that they compile in parallel): series equilibrium with FP32 or FP64 moments, and
// the exact entropic equilibrium with BGK or entropic alpha.  The series equilibrium with FP32
// moments runs two sites per thread (stream_collide_pair.cuh) when nx is even.
#include "stream_collide.cuh"
#include "stream_collide_pair.cuh"

namespace lbm {

cudaError_t launch_sc_bf16(int fp64_moments, int eq, const StepParams& p, cudaStream_t s) {
  if (eq == kEqEntropic) return launch_sc<__nv_bfloat16, false, kEqEntropic>(p, s);
  if (eq == kEqEntropicAlpha) return launch_sc<__nv_bfloat16, false, kEqEntropicAlpha>(p, s);
  if (eq == kEqSeriesExactW) return launch_sc<__nv_bfloat16, false, kEqSeriesExactW>(p, s);
  if (pair_kernel_applies(fp64_moments, eq, p)) return launch_sc_pair<__nv_bfloat16>(p, s);
  return fp64_moments ? launch_sc<__nv_bfloat16, true>(p, s) : launch_sc<__nv_bfloat16, false>(p, s);
}

}  // namespace lbm
