// Fused stream-collide instantiations for float storage (one translation unit per storage
// type so that they compile in parallel).
#include "stream_collide.cuh"

namespace lbm {

cudaError_t launch_sc_f32(int fp64_moments, const StepParams& p, cudaStream_t s) {
  return fp64_moments ? launch_sc<float, true>(p, s) : launch_sc<float, false>(p, s);
}

}  // namespace lbm
