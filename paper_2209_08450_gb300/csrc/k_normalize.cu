// Dark/flat-field correction and negative logarithm (Sec. 2.2 of the
// TomocuPy paper), fused with the transposition from projection-major raw
// frames raw[theta][z][j] to sinograms sino[z][theta][j].
//
// The step is a pure stream: 2 bytes in, 2 or 4 bytes out per pixel, so it is
// bound by HBM bandwidth.  Each thread handles 8 consecutive detector pixels
// with one 16-byte uint16 load and 16/32-byte stores when the layout is
// aligned (the common case), one pixel otherwise.  The arithmetic is FP32 even
// for 16-bit output: raw counts up to 65535 do not fit FP16 (max 65504,
// Sec. 2.1).
#include "tcp_internal.cuh"

namespace tcp {
namespace {

__global__ void k_frame_mean(const uint16_t* f, int nf, int64_t f0, int64_t f1, int nz, int nd,
                             float* mean, int64_t m0) {
  const int64_t total = (int64_t)nz * nd;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int z = (int)(e / nd), j = (int)(e - (int64_t)z * nd);
    uint64_t acc = 0;
    for (int k = 0; k < nf; ++k) acc += __ldg(f + (int64_t)k * f0 + (int64_t)z * f1 + j);
    mean[(int64_t)z * m0 + j] = (float)((double)acc / (double)nf);
  }
}

struct NormArgs {
  const uint16_t* raw;
  int64_t r0, r1;  // raw strides: theta, z
  const float* dark;
  const float* flat;
  int64_t d0, f0;  // mean strides: z
  void* sino;
  int64_t s0, s1;  // sino strides: z, theta
  int ntheta, nz, nd;
  int jblocks;     // blocks per row
};

template <class TS, int VEC>
__global__ void __launch_bounds__(256) k_normalize(NormArgs a) {
  const int64_t rows = (int64_t)a.ntheta * a.nz;
  for (int64_t b = blockIdx.x; b < rows * a.jblocks; b += gridDim.x) {
    const int64_t row = b / a.jblocks;
    const int jb = (int)(b - row * a.jblocks);
    const int t = (int)(row / a.nz), z = (int)(row - (int64_t)t * a.nz);
    const int j = (jb * 256 + threadIdx.x) * VEC;
    if (j >= a.nd) continue;
    const uint16_t* rp = a.raw + (int64_t)t * a.r0 + (int64_t)z * a.r1 + j;
    const float* dp = a.dark + (int64_t)z * a.d0 + j;
    const float* fp = a.flat + (int64_t)z * a.f0 + j;
    TS* op = reinterpret_cast<TS*>(a.sino) + (int64_t)z * a.s0 + (int64_t)t * a.s1 + j;
    if constexpr (VEC == 8) {
      const uint4 rv = __ldcs(reinterpret_cast<const uint4*>(rp));
      const float4 d_lo = __ldg(reinterpret_cast<const float4*>(dp));
      const float4 d_hi = __ldg(reinterpret_cast<const float4*>(dp) + 1);
      const float4 f_lo = __ldg(reinterpret_cast<const float4*>(fp));
      const float4 f_hi = __ldg(reinterpret_cast<const float4*>(fp) + 1);
      const float d[8] = {d_lo.x, d_lo.y, d_lo.z, d_lo.w, d_hi.x, d_hi.y, d_hi.z, d_hi.w};
      const float f[8] = {f_lo.x, f_lo.y, f_lo.z, f_lo.w, f_hi.x, f_hi.y, f_hi.z, f_hi.w};
      const uint32_t w[4] = {rv.x, rv.y, rv.z, rv.w};
      float p[8];
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        const float raw = (float)((w[k >> 1] >> ((k & 1) * 16)) & 0xffffu);
        p[k] = neglog_ratio(raw, d[k], f[k]);
      }
      if constexpr (std::is_same<TS, float>::value) {
        __stcs(reinterpret_cast<float4*>(op), make_float4(p[0], p[1], p[2], p[3]));
        __stcs(reinterpret_cast<float4*>(op) + 1, make_float4(p[4], p[5], p[6], p[7]));
      } else {
        TS h[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) Store<TS>::put(&h[k], p[k]);
        __stcs(reinterpret_cast<uint4*>(op), *reinterpret_cast<const uint4*>(h));
      }
    } else {
      Store<TS>::put(op, neglog_ratio((float)__ldg(rp), __ldg(dp), __ldg(fp)));
    }
  }
}

template <class TS>
void (*pick(int vec))(NormArgs) {
  return vec == 8 ? k_normalize<TS, 8> : k_normalize<TS, 1>;
}

bool aligned(const void* p, int bytes) { return ((uintptr_t)p % bytes) == 0; }

}  // namespace

tcp_status launch_frame_mean(const View3& fr, const View3& mean, cudaStream_t st) {
  const int64_t total = fr.d1 * fr.d2;
  if (total == 0) return TCP_OK;
  const int blocks = (int)std::min<int64_t>((total + 255) / 256, 65536);
  k_frame_mean<<<blocks, 256, 0, st>>>(reinterpret_cast<const uint16_t*>(fr.p), (int)fr.d0, fr.s0, fr.s1,
                                       (int)fr.d1, (int)fr.d2, reinterpret_cast<float*>(mean.p), mean.s1);
  TCP_CUDA_TRY(cudaGetLastError());
  return TCP_OK;
}

// raw: [ntheta][nz][nd] u16; dark/flat: [1][nz][nd] f32 (s1 = z stride);
// sino: [nz][ntheta][nd].
tcp_status launch_normalize(const View3& raw, const View3& dark, const View3& flat, const View3& sino,
                            cudaStream_t st) {
  NormArgs a;
  a.raw = reinterpret_cast<const uint16_t*>(raw.p);
  a.r0 = raw.s0;
  a.r1 = raw.s1;
  a.dark = reinterpret_cast<const float*>(dark.p);
  a.flat = reinterpret_cast<const float*>(flat.p);
  a.d0 = dark.s1;
  a.f0 = flat.s1;
  a.sino = sino.p;
  a.s0 = sino.s0;
  a.s1 = sino.s1;
  a.ntheta = (int)raw.d0;
  a.nz = (int)raw.d1;
  a.nd = (int)raw.d2;
  if (a.ntheta == 0 || a.nz == 0 || a.nd == 0) return TCP_OK;
  const int ssz = sino.dtype == TCP_F32 ? 4 : 2;
  const bool vec = a.nd % 8 == 0 && a.r0 % 8 == 0 && a.r1 % 8 == 0 && a.d0 % 8 == 0 && a.f0 % 8 == 0 &&
                   a.s0 % 8 == 0 && a.s1 % 8 == 0 && aligned(raw.p, 16) && aligned(dark.p, 16) &&
                   aligned(flat.p, 16) && aligned(sino.p, 16) && ssz > 0;
  const int v = vec ? 8 : 1;
  a.jblocks = (a.nd + 256 * v - 1) / (256 * v);
  const int64_t work = (int64_t)a.ntheta * a.nz * a.jblocks;
  const int blocks = (int)std::min<int64_t>(work, 152 * 64);
  void (*k)(NormArgs) = nullptr;
  switch (sino.dtype) {
    case TCP_F32: k = pick<float>(v); break;
    case TCP_F16: k = pick<__half>(v); break;
    case TCP_BF16: k = pick<__nv_bfloat16>(v); break;
  }
  if (!k) return fail(TCP_ERR_DTYPE, "normalize: sinogram dtype must be F32, F16 or BF16");
  k<<<blocks, 256, 0, st>>>(a);
  TCP_CUDA_TRY(cudaGetLastError());
  return TCP_OK;
}

}  // namespace tcp
