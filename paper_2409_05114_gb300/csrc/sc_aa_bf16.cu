// Fused stream-collide instantiations for __nv_bfloat16 storage with in-place (AA) streaming: both step
// kinds for every equilibrium and collision (own translation unit so that it compiles in
// parallel with the ping-pong one).
#include "stream_collide.cuh"

namespace lbm {

cudaError_t launch_sc_aa_bf16(int fp64_moments, int eq, int kind, const StepParams& p, cudaStream_t s) {
  return launch_sc_aa_all<__nv_bfloat16>(fp64_moments, eq, kind, p, s);
}

}  // namespace lbm
