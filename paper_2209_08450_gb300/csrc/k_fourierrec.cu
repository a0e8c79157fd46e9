// FourierRec: backprojection through the Fourier-slice theorem with a
// transform on unequally spaced frequencies (Sec. 1, Sec. 2.2 and Sec. 3 of
// arXiv 2209.08450: frequency-domain interpolation with exponential
// functions, frequencies oversampled by 2, controllable accuracy).
//
// What is computed.  Each filtered row q[j] (j < ndet), extended by zeros to
// the period M = the next power of two >= 2 ndet, is replaced by its
// trigonometric interpolant (the Nyquist term split into two halves), and
//   vol[z][iy][ix] = scale * sum_theta q~_theta(x cos theta + y sin theta + center),
// x = ix - n/2, y = iy - n/2, n even.  With P[theta][k] =
// (w_k / M) e^{2 pi i k center / M} Q_theta[k] (Q the DFT of the padded row)
// that is sum_{theta,k} P e^{2 pi i nu.(x, y)} at the polar frequencies
// nu = (k / M)(cos theta, sin theta), evaluated in three kernels per batch of
// slice pairs (two slices ride as the real and imaginary parts of one complex
// row, since the map is real-linear):
//   k_frec_rows       one CTA per (angle, pair): FFT of the padded row,
//                     times the centre phase -> P[pair][theta][k + M/2];
//   k_frec_spread     one CTA per strip of cw columns of the L x L Cartesian
//                     frequency grid (L = next power of two >= 2n, so the
//                     oversampling is >= 2): every polar sample whose window
//                     reaches the strip is spread into shared memory with the
//                     separable "exponential of semicircle" window of width
//                     W (Barnett, Magland, af Klinteberg, SIAM J. Sci.
//                     Comput. 41, 2019); then the strip's columns are
//                     inverse-transformed and the n needed rows kept, divided
//                     by the window's Fourier transform in y -> H[pair][iy][gx];
//   k_frec_out        one CTA per (row, pair): inverse FFT of the row, the
//                     n needed columns divided by the window's transform in x,
//                     times scale, real part -> slice 2p, imaginary -> 2p+1.
// FFTs are in-place radix-4 (and one radix-2) decimation in frequency in
// shared memory; their outputs are read at digit-reversed positions.
#include <cmath>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "tcp_internal.cuh"

namespace tcp {
namespace {

constexpr int kMaxLg = 14;  // M, L <= 16384 (128 KB of complex FP32 in shared memory)
constexpr int kMaxTheta = 16384;
constexpr size_t kBatchBytes = size_t(1) << 30;  // P + H workspace per batch

__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }

// Position of output k of fft_dif of length 2^lg: radix-4 digits first, the
// radix-2 digit last (mixed-radix digit reversal).
__device__ __forceinline__ int dif_pos(int k, int lg) {
  int pos = 0, lgs = lg;
  for (; lgs >= 2; lgs -= 2) {
    pos += (k & 3) << (lgs - 2);
    k >>= 2;
  }
  if (lgs == 1) pos += k & 1;
  return pos;
}

// In-place decimation-in-frequency FFT of `count` sequences of length
// N = 2^lg stored back to back in shared memory.  tw[j] = e^{-2 pi i j / N};
// INV takes the conjugates (positive exponent, no 1/N).  The caller
// synchronises before; this returns synchronised.
template <bool INV>
__device__ void fft_dif(float2* a, int lg, int count, const float2* __restrict__ tw) {
  const int nthr = blockDim.x, tid = threadIdx.x;
  int lgs = lg, ts = 1;
  for (; lgs >= 2; lgs -= 2, ts <<= 2) {
    const int lgm = lgs - 2, m = 1 << lgm;
    const int per_seq = 1 << (lg - 2);
    const int nb = count * per_seq;
    for (int b = tid; b < nb; b += nthr) {
      const int seq = b >> (lg - 2), bb = b & (per_seq - 1);
      const int blk = bb >> lgm, j = bb & (m - 1);
      float2* p = a + (seq << lg) + (blk << lgs) + j;
      const float2 x0 = p[0], x1 = p[m], x2 = p[2 * m], x3 = p[3 * m];
      const float2 s02 = cadd(x0, x2), d02 = csub(x0, x2), s13 = cadd(x1, x3), d13 = csub(x1, x3);
      // omega_4 = -i (forward) or +i (inverse) times d13
      const float2 r13 = INV ? make_float2(-d13.y, d13.x) : make_float2(d13.y, -d13.x);
      float2 w1 = __ldg(tw + j * ts), w2 = __ldg(tw + 2 * j * ts), w3 = __ldg(tw + 3 * j * ts);
      if (INV) {
        w1.y = -w1.y;
        w2.y = -w2.y;
        w3.y = -w3.y;
      }
      p[0] = cadd(s02, s13);
      p[m] = cmul(cadd(d02, r13), w1);
      p[2 * m] = cmul(csub(s02, s13), w2);
      p[3 * m] = cmul(csub(d02, r13), w3);
    }
    __syncthreads();
  }
  if (lgs == 1) {
    const int nb = count << (lg - 1);
    for (int b = tid; b < nb; b += nthr) {
      float2* p = a + 2 * b;
      const float2 x0 = p[0], x1 = p[1];
      p[0] = cadd(x0, x1);
      p[1] = csub(x0, x1);
    }
    __syncthreads();
  }
}

// --------------------------------------------------------------- tables --

// Per-call geometry: (L/M) cos theta and (L/M) sin theta as FP32 hi + lo
// pairs (from the FP64 angle table), and the row phase factors
// (w_k / M) e^{2 pi i k center / M}, k = -M/2 .. M/2, made in FP64.
__global__ void k_frec_geom(const double2* __restrict__ trig, int nt, double ratio, float4* __restrict__ geom,
                            double center, int M, float2* __restrict__ phase) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < nt) {
    const double cx = trig[i].x * ratio, sy = trig[i].y * ratio;
    const float chi = (float)cx, shi = (float)sy;
    geom[i] = make_float4(chi, (float)(cx - (double)chi), shi, (float)(sy - (double)shi));
  }
  if (i <= M) {
    const double k = (double)(i - M / 2);
    const double w = (i == 0 || i == M) ? 0.5 : 1.0;
    const double a = fmod(k * center, (double)M);  // phase turns * M, reduced
    double sn, cs;
    sincospi(2.0 * a / (double)M, &sn, &cs);
    phase[i] = make_float2((float)(w * cs / M), (float)(w * sn / M));
  }
}

// ------------------------------------------------------------- kernel 1 --

template <class TS>
__global__ void __launch_bounds__(256) k_frec_rows(const TS* __restrict__ sino, int64_t s0, int64_t s1, int nz,
                                                   int nd, int z0, int lgM, const float2* __restrict__ twM,
                                                   const float2* __restrict__ phase, float2* __restrict__ P,
                                                   int64_t p_pair, int ms) {
  extern __shared__ float2 frec_buf[];
  const int t = blockIdx.x, pb = blockIdx.y;
  const int M = 1 << lgM;
  const int z1 = z0 + 2 * pb, z2 = z1 + 1;
  const TS* r1 = sino + (int64_t)z1 * s0 + (int64_t)t * s1;
  const TS* r2 = sino + (int64_t)z2 * s0 + (int64_t)t * s1;
  const bool two = z2 < nz;
  for (int j = threadIdx.x; j < M; j += blockDim.x) {
    float a = 0.f, b = 0.f;
    if (j < nd) {
      a = Store<TS>::load(r1 + j);
      if (two) b = Store<TS>::load(r2 + j);
    }
    frec_buf[j] = make_float2(a, b);
  }
  __syncthreads();
  fft_dif<false>(frec_buf, lgM, 1, twM);
  float2* out = P + (int64_t)pb * p_pair + (int64_t)t * ms;
  for (int i = threadIdx.x; i <= M; i += blockDim.x)
    out[i] = cmul(frec_buf[dif_pos((i - M / 2) & (M - 1), lgM)], __ldg(phase + i));
}

// ------------------------------------------------------------- kernel 2 --

// Conservative k range of the samples of one angle whose window can reach
// grid columns [lo, hi]: k * c in (lo - W/2, hi + W/2), widened by one on each
// side (the exact column test is made per node), clipped to [-M/2, M/2].
__device__ __forceinline__ void k_range(float c, float A, float B, int M, int* klo, int* khi) {
  const float lim = (float)M;
  if (fabsf(c) < 1e-30f) {
    if (A < 0.f && B > 0.f) {
      *klo = -M / 2;
      *khi = M / 2;
    } else {
      *klo = 1;
      *khi = 0;
    }
    return;
  }
  float qa = A / c, qb = B / c;
  if (qa > qb) {
    const float tmp = qa;
    qa = qb;
    qb = tmp;
  }
  qa = fminf(fmaxf(qa, -lim), lim);
  qb = fminf(fmaxf(qb, -lim), lim);
  *klo = max((int)floorf(qa) - 1, -M / 2);
  *khi = min((int)ceilf(qb) + 1, M / 2);
}

// k * (hi + lo) as an integer part and a fraction accurate to ~1e-7.
__device__ __forceinline__ void split_pos(float fk, float hi, float lo, int* gi, float* fr) {
  const float ph = fk * hi;
  const float pe = fmaf(fk, hi, -ph) + fk * lo;
  float fl = floorf(ph);
  float f = (ph - fl) + pe;
  if (f < 0.f) {
    f += 1.f;
    fl -= 1.f;
  } else if (f >= 1.f) {
    f -= 1.f;
    fl += 1.f;
  }
  *gi = (int)fl;
  *fr = f;
}

template <int W>
__device__ __forceinline__ float es_weight(float d, float beta) {
  const float s = d * (2.f / (float)W);
  const float z2 = s * s;
  return z2 < 1.f ? expf(beta * (sqrtf(1.f - z2) - 1.f)) : 0.f;
}

// Exclusive scan of v[0..n) in place, v[n] = total; all threads take part.
__device__ void block_scan(int* v, int n) {
  __shared__ int warp_tot[32];
  const int nthr = blockDim.x, tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const int per = (n + nthr - 1) / nthr;
  const int b = min(n, tid * per), e = min(n, b + per);
  int sum = 0;
  for (int i = b; i < e; ++i) sum += v[i];
  int inc = sum;
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += y;
  }
  if (lane == 31) warp_tot[wid] = inc;
  __syncthreads();
  if (wid == 0) {
    const int nw = nthr >> 5;
    int x = lane < nw ? warp_tot[lane] : 0;
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (lane < nw) warp_tot[lane] = x;  // inclusive over warps
  }
  __syncthreads();
  int run = inc - sum + (wid > 0 ? warp_tot[wid - 1] : 0);
  for (int i = b; i < e; ++i) {
    const int c = v[i];
    v[i] = run;
    run += c;
  }
  if (tid == nthr - 1) v[n] = run;
  __syncthreads();
}

template <int W>
__global__ void __launch_bounds__(512) k_frec_spread(const float2* __restrict__ P, int64_t p_pair, int ms,
                                                     const float4* __restrict__ geom, int nt, int M, int lgL,
                                                     int cw, int n, const float2* __restrict__ twL,
                                                     const float* __restrict__ dec, float beta,
                                                     float2* __restrict__ H, int64_t h_pair) {
  extern __shared__ float4 frec_smem4[];
  const int L = 1 << lgL;
  float2* strip = reinterpret_cast<float2*>(frec_smem4);  // [cw][L]
  int* off = reinterpret_cast<int*>(strip + cw * L);      // [nt + 1]
  const int gx0 = blockIdx.x * cw, pb = blockIdx.y;
  const float2* Pp = P + (int64_t)pb * p_pair;
  for (int i = threadIdx.x; i < cw * L; i += blockDim.x) strip[i] = make_float2(0.f, 0.f);
  __syncthreads();
  // The strip's columns as signed frequencies: image 0 is [gx0, gx0 + cw),
  // image -1 the same columns minus L (nodes lie in (-L/2 - W/2, L/2 + W/2)).
  for (int img = 0; img >= -1; --img) {
    const int lo = gx0 + img * L, hi = lo + cw - 1;
    if (2 * hi <= -L - W || 2 * lo >= L + W) continue;  // uniform over the CTA
    const float A = (float)lo - 0.5f * W, B = (float)hi + 0.5f * W;
    for (int t = threadIdx.x; t < nt; t += blockDim.x) {
      int klo, khi;
      k_range(__ldg(&geom[t].x), A, B, M, &klo, &khi);
      off[t] = max(0, khi - klo + 1);
    }
    __syncthreads();
    block_scan(off, nt);
    const int total = off[nt];
    const int per = (total + (int)blockDim.x - 1) / (int)blockDim.x;
    const int i0 = min(total, (int)threadIdx.x * per), i1 = min(total, i0 + per);
    if (i0 < i1) {
      int a = 0, b = nt;  // largest t with off[t] <= i0
      while (b - a > 1) {
        const int mid = (a + b) >> 1;
        if (off[mid] <= i0) a = mid; else b = mid;
      }
      int t = a;
      int klo, khi;
      float4 g = __ldg(geom + t);
      k_range(g.x, A, B, M, &klo, &khi);
      int k = klo + (i0 - off[t]);
      for (int it = i0; it < i1; ++it, ++k) {
        while (it >= off[t + 1]) {
          ++t;
          g = __ldg(geom + t);
          k_range(g.x, A, B, M, &klo, &khi);
          k = klo;
        }
        const float2 v = __ldg(Pp + (int64_t)t * ms + k + M / 2);
        const float fk = (float)k;
        int gix, giy;
        float frx, fry;
        split_pos(fk, g.x, g.y, &gix, &frx);
        split_pos(fk, g.z, g.w, &giy, &fry);
        const float bx = frx - 0.5f * W, by = fry - 0.5f * W;
        const float fbx = floorf(bx), fby = floorf(by);
        const float tx = bx - fbx, ty = by - fby;
        const int g0x = gix + (int)fbx + 1, g0y = giy + (int)fby + 1;
        float wy[W];
#pragma unroll
        for (int r = 0; r < W; ++r) wy[r] = es_weight<W>(ty + (0.5f * W - 1.f - r), beta);
#pragma unroll
        for (int i = 0; i < W; ++i) {
          const int c = g0x + i - lo;
          if (c < 0 || c >= cw) continue;
          const float2 vx = cscale(v, es_weight<W>(tx + (0.5f * W - 1.f - i), beta));
          float2* col = strip + c * L;
#pragma unroll
          for (int r = 0; r < W; ++r) {
            float2* q = col + ((g0y + r) & (L - 1));
            atomicAdd(&q->x, vx.x * wy[r]);
            atomicAdd(&q->y, vx.y * wy[r]);
          }
        }
      }
    }
    __syncthreads();
  }
  fft_dif<true>(strip, lgL, cw, twL);
  float2* Hp = H + (int64_t)pb * h_pair;
  for (int i = threadIdx.x; i < n * cw; i += blockDim.x) {
    const int iy = i / cw, c = i - iy * cw;
    const float2 v = strip[c * L + dif_pos((iy - n / 2) & (L - 1), lgL)];
    Hp[(int64_t)iy * L + gx0 + c] = cscale(v, __ldg(dec + iy));
  }
}

// ------------------------------------------------------------- kernel 3 --

template <class TV>
__global__ void __launch_bounds__(256) k_frec_out(const float2* __restrict__ H, int64_t h_pair, int lgL, int n,
                                                  const float2* __restrict__ twL, const float* __restrict__ dec,
                                                  float scale, TV* __restrict__ vol, int64_t v0, int64_t v1,
                                                  int nz, int z0) {
  extern __shared__ float2 frec_buf[];
  const int iy = blockIdx.x, pb = blockIdx.y;
  const int L = 1 << lgL;
  const float2* row = H + (int64_t)pb * h_pair + (int64_t)iy * L;
  for (int j = threadIdx.x; j < L; j += blockDim.x) frec_buf[j] = __ldg(row + j);
  __syncthreads();
  fft_dif<true>(frec_buf, lgL, 1, twL);
  const int z1 = z0 + 2 * pb, z2 = z1 + 1;
  TV* o1 = vol + (int64_t)z1 * v0 + (int64_t)iy * v1;
  TV* o2 = vol + (int64_t)z2 * v0 + (int64_t)iy * v1;
  const bool two = z2 < nz;
  for (int ix = threadIdx.x; ix < n; ix += blockDim.x) {
    const float2 v = frec_buf[dif_pos((ix - n / 2) & (L - 1), lgL)];
    const float d = __ldg(dec + ix) * scale;
    Store<TV>::put(o1 + ix, v.x * d);
    if (two) Store<TV>::put(o2 + ix, v.y * d);
  }
}

// --------------------------------------------------------- host tables --

struct HostTables {
  std::map<std::pair<int, int>, float2*> tw;                 // (dev, N) -> e^{-2 pi i j / N}
  std::map<std::tuple<int, int, int, int>, float*> dec;      // (dev, n, L, W) -> 1 / Phi(x / L)
};
std::mutex g_frec_mu;
HostTables g_frec;

int ilog2(int64_t v) {
  int l = 0;
  while ((int64_t(1) << l) < v) ++l;
  return l;
}

double es_beta(int W) { return 0.98 * M_PI * W * (1.0 - 1.0 / (2.0 * 2.0)); }

// Phi(xi) = 2 int_0^{W/2} phi(u) cos(2 pi u xi) du with u = (W/2) sin(a):
// 2 (W/2) int_0^{pi/2} e^{beta (cos a - 1)} cos(pi W xi sin a) cos a da,
// composite Simpson on 1024 intervals (the integrand is smooth in a).
double es_fourier(double xi, int W) {
  const double beta = es_beta(W), half = 0.5 * W;
  const int N = 1024;
  const double h = (M_PI / 2) / N;
  double s = 0.0;
  for (int i = 0; i <= N; ++i) {
    const double a = i * h;
    const double f = std::exp(beta * (std::cos(a) - 1.0)) * std::cos(2.0 * M_PI * half * std::sin(a) * xi) * std::cos(a);
    s += f * ((i == 0 || i == N) ? 1.0 : (i & 1) ? 4.0 : 2.0);
  }
  return 2.0 * half * s * h / 3.0;
}

tcp_status get_twiddles(int dev, int N, const float2** out) {
  std::lock_guard<std::mutex> lk(g_frec_mu);
  auto it = g_frec.tw.find({dev, N});
  if (it != g_frec.tw.end()) {
    *out = it->second;
    return TCP_OK;
  }
  std::vector<float2> h((size_t)N);
  for (int j = 0; j < N; ++j) {
    const double a = -2.0 * M_PI * (double)j / (double)N;
    h[(size_t)j] = make_float2((float)std::cos(a), (float)std::sin(a));
  }
  float2* d = nullptr;
  TCP_CUDA_TRY(cudaMalloc(&d, h.size() * sizeof(float2)));
  const cudaError_t e = cudaMemcpy(d, h.data(), h.size() * sizeof(float2), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    cudaFree(d);
    return cuda_fail(e, "upload FourierRec twiddles");
  }
  g_frec.tw[{dev, N}] = d;
  *out = d;
  return TCP_OK;
}

tcp_status get_deconv(int dev, int n, int L, int W, const float** out) {
  std::lock_guard<std::mutex> lk(g_frec_mu);
  const auto key = std::make_tuple(dev, n, L, W);
  auto it = g_frec.dec.find(key);
  if (it != g_frec.dec.end()) {
    *out = it->second;
    return TCP_OK;
  }
  std::vector<float> h((size_t)n);
  for (int i = 0; i < n; ++i) h[(size_t)i] = (float)(1.0 / es_fourier((double)(i - n / 2) / (double)L, W));
  float* d = nullptr;
  TCP_CUDA_TRY(cudaMalloc(&d, h.size() * sizeof(float)));
  const cudaError_t e = cudaMemcpy(d, h.data(), h.size() * sizeof(float), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    cudaFree(d);
    return cuda_fail(e, "upload FourierRec deconvolution table");
  }
  g_frec.dec[key] = d;
  *out = d;
  return TCP_OK;
}

template <class TS>
void launch_rows(const View3& sv, int z0, int nb, int lgM, const float2* twM, const float2* phase, float2* P,
                 int64_t p_pair, int ms, cudaStream_t st) {
  const size_t sm = sizeof(float2) << lgM;
  cudaFuncSetAttribute(k_frec_rows<TS>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  k_frec_rows<TS><<<dim3((unsigned)sv.d1, (unsigned)nb), 256, sm, st>>>(
      (const TS*)sv.p, sv.s0, sv.s1, (int)sv.d0, (int)sv.d2, z0, lgM, twM, phase, P, p_pair, ms);
}

template <int W>
void launch_spread(const float2* P, int64_t p_pair, int ms, const float4* geom, int nt, int M, int lgL, int cw, int n,
                   const float2* twL, const float* dec, float2* H, int64_t h_pair, int nb, cudaStream_t st) {
  const int L = 1 << lgL;
  const size_t sm = sizeof(float2) * (size_t)cw * L + sizeof(int) * (size_t)(nt + 1);
  cudaFuncSetAttribute(k_frec_spread<W>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  k_frec_spread<W><<<dim3((unsigned)(L / cw), (unsigned)nb), 512, sm, st>>>(P, p_pair, ms, geom, nt, M, lgL, cw, n, twL,
                                                                          dec, (float)es_beta(W), H, h_pair);
}

template <class TV>
void launch_out(const float2* H, int64_t h_pair, int lgL, int n, const float2* twL, const float* dec, float scale,
                const View3& vv, int z0, int nb, cudaStream_t st) {
  const size_t sm = sizeof(float2) << lgL;
  cudaFuncSetAttribute(k_frec_out<TV>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  k_frec_out<TV><<<dim3((unsigned)n, (unsigned)nb), 256, sm, st>>>(H, h_pair, lgL, n, twL, dec, scale, (TV*)vv.p,
                                                                   vv.s0, vv.s1, (int)vv.d0, z0);
}

}  // namespace

int fourierrec_default_width(int vol_dtype, int64_t n) {
  int64_t L = 1;
  while (L < 2 * n) L *= 2;
  return (int)std::max<int64_t>(2, std::min<int64_t>(L, vol_dtype == TCP_F32 ? 7 : 5));
}

tcp_status fourierrec_check(int64_t nt, int64_t nd, int64_t n, int width) {
  if (n % 2) return fail(TCP_ERR_SHAPE, "fourierrec: n must be even");
  int64_t M = 1, L = 1;
  while (M < 2 * nd) M *= 2;
  while (L < 2 * n) L *= 2;
  if (M > (int64_t(1) << kMaxLg)) return fail(TCP_ERR_SHAPE, "fourierrec: ndet must be <= 8192");
  if (L > (int64_t(1) << kMaxLg)) return fail(TCP_ERR_SHAPE, "fourierrec: n must be <= 8192");
  if (nt > kMaxTheta) return fail(TCP_ERR_SHAPE, "fourierrec: ntheta must be <= 16384");
  if (width < 2 || width > 16) return fail(TCP_ERR_ARG, "fourierrec: width must be in [2, 16]");
  if (width > L) return fail(TCP_ERR_ARG, "fourierrec: width must not exceed the grid size (2n rounded up)");
  return TCP_OK;
}

tcp_status launch_fourierrec(const View3& sv, const TrigTable& trig, double center, const View3& vv, float scale,
                             int width, cudaStream_t st) {
  const int nz = (int)sv.d0, nt = (int)sv.d1, nd = (int)sv.d2, n = (int)vv.d1;
  tcp_status s;
  if ((s = fourierrec_check(nt, nd, n, width)) != TCP_OK) return s;
  const int lgM = std::max(1, ilog2(2 * (int64_t)nd)), lgL = std::max(1, ilog2(2 * (int64_t)n));
  const int M = 1 << lgM, L = 1 << lgL;
  const int ms = M + 1;
  const int cw = std::max(1, std::min(std::min(4, L), (1 << kMaxLg) / L));
  int dev = 0;
  TCP_CUDA_TRY(cudaGetDevice(&dev));
  const float2 *twM = nullptr, *twL = nullptr;
  const float* dec = nullptr;
  if ((s = get_twiddles(dev, M, &twM)) != TCP_OK) return s;
  if ((s = get_twiddles(dev, L, &twL)) != TCP_OK) return s;
  if ((s = get_deconv(dev, n, L, width, &dec)) != TCP_OK) return s;

  const int npairs = (nz + 1) / 2;
  const int64_t p_pair = (int64_t)nt * ms, h_pair = (int64_t)n * L;
  const size_t per_pair = sizeof(float2) * (size_t)(p_pair + h_pair);
  const int nb = (int)std::max<int64_t>(1, std::min<int64_t>(npairs, (int64_t)(kBatchBytes / per_pair)));

  struct Ws {
    cudaStream_t st;
    std::vector<void*> p;
    ~Ws() {
      for (void* q : p) cudaFreeAsync(q, st);
    }
    tcp_status alloc(void** q, size_t bytes) {
      const cudaError_t e = cudaMallocAsync(q, bytes ? bytes : 16, st);
      if (e != cudaSuccess) return cuda_fail(e, "cudaMallocAsync");
      p.push_back(*q);
      return TCP_OK;
    }
  } ws{st, {}};
  void *geom = nullptr, *phase = nullptr, *P = nullptr, *H = nullptr;
  if ((s = ws.alloc(&geom, sizeof(float4) * (size_t)nt)) != TCP_OK) return s;
  if ((s = ws.alloc(&phase, sizeof(float2) * (size_t)ms)) != TCP_OK) return s;
  if ((s = ws.alloc(&P, sizeof(float2) * (size_t)p_pair * nb)) != TCP_OK) return s;
  if ((s = ws.alloc(&H, sizeof(float2) * (size_t)h_pair * nb)) != TCP_OK) return s;
  {
    const int cnt = std::max(nt, ms);
    k_frec_geom<<<(cnt + 255) / 256, 256, 0, st>>>(trig.dev, nt, (double)L / (double)M, (float4*)geom, center, M,
                                                     (float2*)phase);
    TCP_CUDA_TRY(cudaGetLastError());
  }
  for (int p0 = 0; p0 < npairs; p0 += nb) {
    const int b = std::min(nb, npairs - p0), z0 = 2 * p0;
    switch (sv.dtype) {
      case TCP_F32: launch_rows<float>(sv, z0, b, lgM, twM, (const float2*)phase, (float2*)P, p_pair, ms, st); break;
      case TCP_F16: launch_rows<__half>(sv, z0, b, lgM, twM, (const float2*)phase, (float2*)P, p_pair, ms, st); break;
      case TCP_BF16:
        launch_rows<__nv_bfloat16>(sv, z0, b, lgM, twM, (const float2*)phase, (float2*)P, p_pair, ms, st);
        break;
      default: return fail(TCP_ERR_DTYPE, "fourierrec: sino must be F32, F16 or BF16");
    }
    TCP_CUDA_TRY(cudaGetLastError());
#define TCP_FREC_W(w)                                                                                         \
  case w:                                                                                                     \
    launch_spread<w>((const float2*)P, p_pair, ms, (const float4*)geom, nt, M, lgL, cw, n, twL, dec, (float2*)H, \
                     h_pair, b, st);                                                                          \
    break;
    switch (width) {
      TCP_FREC_W(2) TCP_FREC_W(3) TCP_FREC_W(4) TCP_FREC_W(5) TCP_FREC_W(6) TCP_FREC_W(7) TCP_FREC_W(8)
      TCP_FREC_W(9) TCP_FREC_W(10) TCP_FREC_W(11) TCP_FREC_W(12) TCP_FREC_W(13) TCP_FREC_W(14) TCP_FREC_W(15)
      TCP_FREC_W(16)
      default: return fail(TCP_ERR_ARG, "fourierrec: width must be in [2, 16]");
    }
#undef TCP_FREC_W
    TCP_CUDA_TRY(cudaGetLastError());
    View3 ov = vv;
    switch (vv.dtype) {
      case TCP_F32: launch_out<float>((const float2*)H, h_pair, lgL, n, twL, dec, scale, ov, z0, b, st); break;
      case TCP_F16: launch_out<__half>((const float2*)H, h_pair, lgL, n, twL, dec, scale, ov, z0, b, st); break;
      case TCP_BF16:
        launch_out<__nv_bfloat16>((const float2*)H, h_pair, lgL, n, twL, dec, scale, ov, z0, b, st);
        break;
      default: return fail(TCP_ERR_DTYPE, "fourierrec: vol must be F32, F16 or BF16");
    }
    TCP_CUDA_TRY(cudaGetLastError());
  }
  return TCP_OK;
}

}  // namespace tcp
