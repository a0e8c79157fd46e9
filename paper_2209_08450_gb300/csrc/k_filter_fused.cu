// tcp_normalize_filter: dark/flat normalisation, -log and the FBP filter in
// one pass over the raw frames (kernels in k_filter_impl.cuh).
#include "k_filter_impl.cuh"

namespace tcp {
// Fused: raw [ntheta][nz][nd] u16, means [1][nz][nd] (s1 = z stride) ->
// filtered sino [nz][ntheta][nd].
tcp_status launch_normalize_filter(const View3& raw, const View3& dark, const View3& flat, const View3& sino,
                                   const FilterTable& ft, int pad_mode, cudaStream_t st) {
  FiltArgs a;
  a.src = raw.p;
  a.s0 = raw.s0;
  a.s1 = raw.s1;
  a.dark = reinterpret_cast<const float*>(dark.p);
  a.flat = reinterpret_cast<const float*>(flat.p);
  a.dm = dark.s1;
  a.fm = flat.s1;
  a.dst = sino.p;
  a.t0 = sino.s0;
  a.t1 = sino.s1;
  a.d1 = (int)sino.d1;
  a.rows = sino.d0 * sino.d1;
  a.nd = (int)sino.d2;
  a.plane = sino.dtype == TCP_F16X2 ? sino.plane : 0;
  // 8-byte raw loads and 16-byte mean loads need aligned row starts
  a.vec4 = ((uintptr_t)raw.p % 8 == 0) && (raw.s0 % 4 == 0) && (raw.s1 % 4 == 0) && ((uintptr_t)dark.p % 16 == 0) &&
           ((uintptr_t)flat.p % 16 == 0) && (dark.s1 % 4 == 0) && (flat.s1 % 4 == 0);
  return run(pick_out<true, uint16_t>(sino.dtype), a, ft, pad_mode, st);
}

}  // namespace tcp
