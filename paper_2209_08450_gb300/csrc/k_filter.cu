// One-dimensional FBP filter of every detector row (Sec. 2.2 of the TomocuPy
// paper: Shepp-Logan / Parzen filtering in Fourier space, rows padded before
// the FFT).
//
// GB300 design: the whole padded row lives in shared memory; no padded copy
// ever touches HBM.  Two real rows travel as one complex row z = a + i b:
// because the filter response is Hermitian (F[N-k] = conj(F[k])), filtering z
// filters a and b independently, so one complex FFT pair serves two rows
// without a separation step.  The FFT is a Stockham auto-sort transform with
// radix-4 passes (one radix-2 pass when log2 N is odd), each thread holding up
// to four butterflies in registers between the shared-memory read and write
// phases.  Twiddles and the response are FP64-derived tables; the arithmetic
// is FP32.  The response folds in the window, the pi/N_theta FBP weight, the
// 1/N of the inverse transform and the phase that moves the rotation axis to
// ndet/2.
#include "tcp_internal.cuh"

namespace tcp {
namespace {

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(__fmaf_rn(a.x, b.x, -a.y * b.y), __fmaf_rn(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
// multiply by -i (forward) or +i (inverse)
template <bool INV> __device__ __forceinline__ float2 rot(float2 a) {
  return INV ? make_float2(-a.y, a.x) : make_float2(a.y, -a.x);
}

constexpr int kMaxB = 4;  // butterflies per thread per pass

template <bool INV>
__device__ void radix2_first(float2* x, int N, int nthreads) {
  // Ns = 1: no twiddles.
  const int nb = N / 2;
  float2 v[2 * kMaxB][2];
#pragma unroll
  for (int i = 0; i < 2 * kMaxB; ++i) {
    const int b = threadIdx.x + i * nthreads;
    if (b < nb) {
      v[i][0] = x[b];
      v[i][1] = x[b + nb];
    }
  }
  __syncthreads();
#pragma unroll
  for (int i = 0; i < 2 * kMaxB; ++i) {
    const int b = threadIdx.x + i * nthreads;
    if (b < nb) {
      x[2 * b] = cadd(v[i][0], v[i][1]);
      x[2 * b + 1] = csub(v[i][0], v[i][1]);
    }
  }
  __syncthreads();
}

template <bool INV>
__device__ void radix4_pass(float2* x, int N, int Ns, const float2* tw, int nthreads) {
  const int nb = N / 4;
  const int step = N / (4 * Ns);
  float2 v[kMaxB][4];
#pragma unroll
  for (int i = 0; i < kMaxB; ++i) {
    const int b = threadIdx.x + i * nthreads;
    if (b < nb) {
#pragma unroll
      for (int r = 0; r < 4; ++r) v[i][r] = x[b + r * nb];
    }
  }
  __syncthreads();
#pragma unroll
  for (int i = 0; i < kMaxB; ++i) {
    const int b = threadIdx.x + i * nthreads;
    if (b < nb) {
      const int k = b & (Ns - 1);
      if (Ns > 1) {
#pragma unroll
        for (int r = 1; r < 4; ++r) {
          float2 w = __ldg(tw + r * k * step);
          if (INV) w.y = -w.y;
          v[i][r] = cmul(v[i][r], w);
        }
      }
      const float2 s02 = cadd(v[i][0], v[i][2]), d02 = csub(v[i][0], v[i][2]);
      const float2 s13 = cadd(v[i][1], v[i][3]), d13 = rot<INV>(csub(v[i][1], v[i][3]));
      const int o = (b - k) * 4 + k;
      x[o] = cadd(s02, s13);
      x[o + Ns] = cadd(d02, d13);
      x[o + 2 * Ns] = csub(s02, s13);
      x[o + 3 * Ns] = csub(d02, d13);
    }
  }
  __syncthreads();
}

template <bool INV>
__device__ void fft(float2* x, int N, int log2N, const float2* tw, int nthreads) {
  int Ns = 1;
  if (log2N & 1) {
    radix2_first<INV>(x, N, nthreads);
    Ns = 2;
  }
  for (; Ns < N; Ns *= 4) radix4_pass<INV>(x, N, Ns, tw, nthreads);
}

struct FiltArgs {
  void* sino;
  int64_t s0, s1;  // strides of the [d0][d1] row grid
  int d1;          // rows per outer index
  int64_t rows;
  int nd, npad, log2n, left;
  int pad_zero;
  const float2* resp;
  const float2* tw;
};

template <class TS>
__global__ void k_filter(FiltArgs a) {
  extern __shared__ float2 buf[];
  const int nthreads = blockDim.x;
  TS* base = reinterpret_cast<TS*>(a.sino);
  const int64_t npairs = (a.rows + 1) / 2;
  for (int64_t p = blockIdx.x; p < npairs; p += gridDim.x) {
    const int64_t r0 = 2 * p, r1 = 2 * p + 1;
    const bool has1 = r1 < a.rows;
    TS* row0 = base + (r0 / a.d1) * a.s0 + (r0 % a.d1) * a.s1;
    TS* row1 = has1 ? base + (r1 / a.d1) * a.s0 + (r1 % a.d1) * a.s1 : row0;
    for (int m = threadIdx.x; m < a.npad; m += nthreads) {
      int j = m - a.left;
      float re = 0.f, im = 0.f;
      if (a.pad_zero) {
        if (j >= 0 && j < a.nd) {
          re = Store<TS>::load(row0 + j);
          im = has1 ? Store<TS>::load(row1 + j) : 0.f;
        }
      } else {
        j = min(max(j, 0), a.nd - 1);
        re = Store<TS>::load(row0 + j);
        im = has1 ? Store<TS>::load(row1 + j) : 0.f;
      }
      buf[m] = make_float2(re, im);
    }
    __syncthreads();
    fft<false>(buf, a.npad, a.log2n, a.tw, nthreads);
    const int half = a.npad / 2;
    for (int k = threadIdx.x; k < a.npad; k += nthreads) {
      float2 F = __ldg(a.resp + (k <= half ? k : a.npad - k));
      if (k > half) F.y = -F.y;
      buf[k] = cmul(buf[k], F);
    }
    __syncthreads();
    fft<true>(buf, a.npad, a.log2n, a.tw, nthreads);
    for (int j = threadIdx.x; j < a.nd; j += nthreads) {
      const float2 v = buf[a.left + j];
      Store<TS>::put(row0 + j, v.x);
      if (has1) Store<TS>::put(row1 + j, v.y);
    }
    __syncthreads();
  }
}

}  // namespace

// sino: [d0][d1][nd] rows (d0*d1 rows).
tcp_status launch_filter(const View3& sino, const FilterTable& ft, int pad_mode, cudaStream_t st) {
  FiltArgs a;
  a.sino = sino.p;
  a.s0 = sino.s0;
  a.s1 = sino.s1;
  a.d1 = (int)sino.d1;
  a.rows = sino.d0 * sino.d1;
  a.nd = (int)sino.d2;
  a.npad = ft.npad;
  a.log2n = 0;
  while ((1 << a.log2n) < a.npad) ++a.log2n;
  a.left = (a.npad - a.nd) / 2;
  a.pad_zero = pad_mode == TCP_PAD_ZERO;
  a.resp = ft.response;
  a.tw = ft.twiddle;
  if (a.rows == 0 || a.nd == 0) return TCP_OK;
  const int threads = std::max(32, std::min(512, a.npad / (4 * kMaxB)));
  const size_t smem = (size_t)a.npad * sizeof(float2);
  void (*k)(FiltArgs) = nullptr;
  switch (sino.dtype) {
    case TCP_F32: k = k_filter<float>; break;
    case TCP_F16: k = k_filter<__half>; break;
    case TCP_BF16: k = k_filter<__nv_bfloat16>; break;
  }
  if (!k) return fail(TCP_ERR_DTYPE, "filter: sinogram dtype must be F32, F16 or BF16");
  TCP_CUDA_TRY(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  const int64_t npairs = (a.rows + 1) / 2;
  const int blocks = (int)std::min<int64_t>(npairs, 152 * 32);
  k<<<blocks, threads, smem, st>>>(a);
  TCP_CUDA_TRY(cudaGetLastError());
  return TCP_OK;
}

}  // namespace tcp
