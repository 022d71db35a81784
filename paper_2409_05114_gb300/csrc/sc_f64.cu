// Fused stream-collide instantiations for double storage (one translation unit per storage
// type so that they compile in parallel): series equilibrium with FP32 or FP64 moments, and
// the exact entropic equilibrium with BGK or entropic alpha.
#include "stream_collide.cuh"

namespace lbm {

cudaError_t launch_sc_f64(int fp64_moments, int eq, const StepParams& p, cudaStream_t s) {
  (void)fp64_moments;  // FP64 storage already sums its moments in FP64
  if (eq == kEqEntropic) return launch_sc<double, false, kEqEntropic>(p, s);
  if (eq == kEqEntropicAlpha) return launch_sc<double, false, kEqEntropicAlpha>(p, s);
  if (eq == kEqSeriesExactW) return launch_sc<double, false, kEqSeriesExactW>(p, s);
  return launch_sc<double, false, kEqSeries>(p, s);
}

}  // namespace lbm
