// CUDA-core LineRec backprojector kernels for BF16 sinograms (every
// configuration and volume dtype), instantiated in a unit of their own.
#include "k_backproject_impl.cuh"

namespace tcp {

KernPair bp_pick_bf16(int vdt, const tcp_bp_config& c, bool check) { return pick_vol<__nv_bfloat16>(vdt, c, check); }

}  // namespace tcp
