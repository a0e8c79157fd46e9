// CUDA-core LineRec backprojector kernels for FP32 sinograms and FP32
// volumes (every configuration), instantiated in a unit of their own.
#include "k_backproject_impl.cuh"

namespace tcp {

KernPair bp_pick_f32_f32(const tcp_bp_config& c, bool check) { return pick<float, float>(c, check); }

}  // namespace tcp
