// LineRec backprojection on the CUDA cores: launchers (the kernels and
// their configurations are in k_backproject_impl.cuh, instantiated in
// k_backproject_f32_{f32,f16,bf16}.cu, k_backproject_f16.cu and
// k_backproject_bf16.cu, compiled in parallel).
#include <mutex>
#include <set>

#include "k_backproject_impl.cuh"

namespace tcp {
namespace {

// Opt every kernel of a pair in to its dynamic shared memory once.
tcp_status prepare(const KernPair& kp) {
  static std::mutex mu;
  static std::set<const void*> done;
  std::lock_guard<std::mutex> lk(mu);
  if (done.count(reinterpret_cast<const void*>(kp.direct))) return TCP_OK;
  TCP_CUDA_TRY(cudaFuncSetAttribute(kp.direct, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kp.smem));
  TCP_CUDA_TRY(cudaFuncSetAttribute(kp.persistent, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kp.smem));
  done.insert(reinterpret_cast<const void*>(kp.direct));
  return TCP_OK;
}

KernPair pick_all(int sdt, int vdt, const tcp_bp_config& c, bool check) {
  switch (sdt) {
    case TCP_F32:
      return vdt == TCP_F32 ? bp_pick_f32_f32(c, check)
             : vdt == TCP_F16 ? bp_pick_f32_f16(c, check)
             : vdt == TCP_BF16 ? bp_pick_f32_bf16(c, check)
             : KernPair{nullptr, nullptr, 0};
    case TCP_F16: return bp_pick_f16(vdt, c, check);
    case TCP_BF16: return bp_pick_bf16(vdt, c, check);
  }
  return {nullptr, nullptr, 0};
}

}  // namespace

}  // namespace tcp

extern "C" tcp_status tcp_tc_launch_shape(int64_t nz, int32_t sino_dtype, int32_t theta_stage, int32_t blocks_per_sm,
                                          tcp_tc_shape* shape) {
  using namespace tcp;
  if (!shape || nz < 1) return fail(TCP_ERR_ARG, "tc_launch_shape: null shape or nz < 1");
  if (sino_dtype != TCP_F16 && sino_dtype != TCP_BF16 && sino_dtype != TCP_F16X2)
    return fail(TCP_ERR_DTYPE, "tc_launch_shape: sinogram dtype must be F16, BF16 or F16X2");
  TcShape sh;
  if (!tc_shape(nz, sino_dtype == TCP_F16X2, theta_stage, blocks_per_sm, &sh))
    return fail(TCP_ERR_UNSUPPORTED, "tc_launch_shape: shared memory too small for the rings");
  shape->slices_per_block = sh.N;
  shape->angles_per_stage = sh.S;
  shape->blocks_per_sm = sh.blocks;
  shape->weight_stages = sh.na;
  shape->sinogram_stages = sh.nbb;
  shape->smem_bytes = (int64_t)sh.smem;
  return TCP_OK;
}

namespace tcp {

bool valid_bp_config(const tcp_bp_config& c) {
  if (c.kernel < 0 || c.kernel > 3) return false;
  // tensor cores: theta_stage 1 or 2 picks the stage size; the rest is ignored
  if (c.kernel == 1 || c.kernel == 3) return true;
  return bp_pick_f32_f32(c, false).direct != nullptr;
}

int bp_threads(const tcp_bp_config& c) { return 32 * (32 / c.rows_per_thread); }

tcp_status bp_persistent_grid(int sdt, int vdt, const tcp_bp_config& cfg, int* blocks) {
  KernPair kp = pick_all(sdt, vdt, cfg, checked_mode());
  if (!kp.persistent) return fail(TCP_ERR_UNSUPPORTED, "backproject: no persistent kernel for this dtype/config");
  tcp_status s = prepare(kp);
  if (s != TCP_OK) return s;
  int per_sm = 0, dev = 0, sms = 0;
  TCP_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kp.persistent, bp_threads(cfg), kp.smem));
  TCP_CUDA_TRY(cudaGetDevice(&dev));
  TCP_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  *blocks = std::max(1, per_sm) * sms;
  return TCP_OK;
}

tcp_status launch_backproject_persistent(const BpWork& w, int sdt, int vdt, const tcp_bp_config& cfg, int blocks,
                                         cudaStream_t st) {
  KernPair kp = pick_all(sdt, vdt, cfg, checked_mode());
  if (!kp.persistent) return fail(TCP_ERR_UNSUPPORTED, "backproject: no persistent kernel for this dtype/config");
  tcp_status s = prepare(kp);
  if (s != TCP_OK) return s;
  kp.persistent<<<blocks, bp_threads(cfg), kp.smem, st>>>(w);
  TCP_CUDA_TRY(cudaGetLastError());
  return TCP_OK;
}

tcp_bp_config default_bp_config(int64_t nz, int64_t, int64_t, int64_t, int sdt, int) {
  tcp_bp_config c{8, 16, 4, 0};
  if (nz <= 1) c = tcp_bp_config{1, 32, 4, 0};
  else if (nz <= 2) c = tcp_bp_config{2, 16, 4, 0};
  else if (nz <= 4) c = tcp_bp_config{4, 16, 4, 0};
  // FP32 sinograms: the slice-pair form (1.21x the one-column-per-lane form at
  // 2048^2 x 32 slices x 2048 angles)
  if (sdt == TCP_F32 && nz >= 3) c = tcp_bp_config{nz >= 5 ? 8 : 4, 16, 4, 2};
  // 16-bit sinograms with enough slices to fill the MMA's N dimension go to
  // the tensor cores (inputs whose strides do not suit TMA fall back), two
  // blocks per SM where the slice block allows it (at 2048^2 x 2048 angles:
  // 40.9 / 43.6 / 52.5 ms against 62.2 / 63.3 / 67.0 ms with one block, for
  // 32 / 64 / 128 slices; the weight builders bind there, and a second block
  // doubles them).
  if ((sdt == TCP_F16 || sdt == TCP_BF16) && nz >= 32) c.kernel = 3;
  if (sdt == TCP_F16X2) c.kernel = 1;  // split FP16 pairs exist only on the tensor cores
  return c;
}

tcp_status launch_backproject(const View3& sino, const TrigTable& trig, double center, const View3& vol,
                              const tcp_bp_config& cfg, cudaStream_t st, float scale) {
  if (sino.dtype == TCP_F16X2 || ((cfg.kernel == 1 || cfg.kernel == 3) && tc_eligible(sino))) {
    if (!tc_eligible(sino))
      return fail(TCP_ERR_ALIGN, "backproject: F16X2 sinograms need 16-byte aligned planes, slices and rows");
    if (sino.d0 == 0 || vol.d1 == 0) return TCP_OK;
    return launch_backproject_tc(sino, trig, center, vol, scale, cfg.theta_stage, cfg.kernel == 3 ? 2 : 1, st);
  }
  const KernPair kp = pick_all(sino.dtype, vol.dtype, cfg, checked_mode());
  Kern k = kp.direct;
  if (!k) return fail(TCP_ERR_UNSUPPORTED, "backproject: no kernel for this dtype/config");
  tcp_status ps = prepare(kp);
  if (ps != TCP_OK) return ps;
  if (sino.d0 == 0 || vol.d1 == 0) return TCP_OK;
  BpArgs a = make_bp_args(sino, trig, center, vol, scale);
  const int threads = bp_threads(cfg);
  dim3 grid((unsigned)(a.ntx * a.ntx), (unsigned)((a.nz + cfg.k_slices - 1) / cfg.k_slices));
  if (grid.y > 65535u) return fail(TCP_ERR_SHAPE, "backproject: too many slice blocks");
  k<<<grid, threads, kp.smem, st>>>(a);
  TCP_CUDA_TRY(cudaGetLastError());
  return TCP_OK;
}

BpArgs make_bp_args(const View3& sino, const TrigTable& trig, double center, const View3& vol, float scale) {
  BpArgs a;
  a.scale = scale;
  a.sino = sino.p;
  a.s_z = sino.s0;
  a.s_t = sino.s1;
  a.nz = (int)sino.d0;
  a.ntheta = (int)sino.d1;
  a.ndet = (int)sino.d2;
  a.vol = vol.p;
  a.v_z = vol.s0;
  a.v_y = vol.s1;
  a.n = (int)vol.d1;
  a.ntx = (a.n + kTile - 1) / kTile;
  a.trig = trig.dev;
  a.center = center;
  a.half_n = 0.5 * (double)a.n;
  a.err = device_error_word();
  return a;
}

}  // namespace tcp
