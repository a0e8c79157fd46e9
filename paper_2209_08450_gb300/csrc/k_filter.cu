// tcp_filter: the FBP filter of every detector row in place (kernels in
// k_filter_impl.cuh; the fused normalise + filter launcher is in
// k_filter_fused.cu, compiled in parallel with this unit).
#include "k_filter_impl.cuh"

namespace tcp {

// In place: sino [d0][d1][nd] rows (d0*d1 rows).
tcp_status launch_filter(const View3& sino, const FilterTable& ft, int pad_mode, cudaStream_t st) {
  FiltArgs a;
  a.src = sino.p;
  a.s0 = sino.s0;
  a.s1 = sino.s1;
  a.dst = sino.p;
  a.t0 = sino.s0;
  a.t1 = sino.s1;
  a.dark = a.flat = nullptr;
  a.dm = a.fm = 0;
  a.vec4 = 0;
  a.plane = 0;
  a.d1 = (int)sino.d1;
  a.rows = sino.d0 * sino.d1;
  a.nd = (int)sino.d2;
  void (*k)(FiltArgs) = nullptr;
  switch (sino.dtype) {
    case TCP_F32: k = k_filter<false, float, float>; break;
    case TCP_F16: k = k_filter<false, __half, __half>; break;
    case TCP_BF16: k = k_filter<false, __nv_bfloat16, __nv_bfloat16>; break;
  }
  return run(k, a, ft, pad_mode, st);
}

}  // namespace tcp
