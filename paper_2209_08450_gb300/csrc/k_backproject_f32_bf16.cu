// CUDA-core LineRec backprojector kernels for FP32 sinograms and BF16
// volumes (every configuration), instantiated in a unit of their own.
#include "k_backproject_impl.cuh"

namespace tcp {

KernPair bp_pick_f32_bf16(const tcp_bp_config& c, bool check) { return pick<float, __nv_bfloat16>(c, check); }

}  // namespace tcp
