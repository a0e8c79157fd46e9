// CUDA-core LineRec backprojector kernels for FP32 sinograms and FP16
// volumes (every configuration), instantiated in a unit of their own.
#include "k_backproject_impl.cuh"

namespace tcp {

KernPair bp_pick_f32_f16(const tcp_bp_config& c, bool check) { return pick<float, __half>(c, check); }

}  // namespace tcp
