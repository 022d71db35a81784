// Fused stream-collide instantiations for __nv_bfloat16 storage (one translation unit per storage
// type so that they compile in parallel).
#include "stream_collide.cuh"

namespace lbm {

cudaError_t launch_sc_bf16(int fp64_moments, const StepParams& p, cudaStream_t s) {
  return fp64_moments ? launch_sc<__nv_bfloat16, true>(p, s) : launch_sc<__nv_bfloat16, false>(p, s);
}

}  // namespace lbm
