// Fused stream-collide instantiations for double storage (one translation unit per storage
// type so that they compile in parallel).
#include "stream_collide.cuh"

namespace lbm {

cudaError_t launch_sc_f64(int fp64_moments, const StepParams& p, cudaStream_t s) {
  (void)fp64_moments;  // FP64 storage already sums its moments in FP64
  return launch_sc<double, false>(p, s);
}

}  // namespace lbm
