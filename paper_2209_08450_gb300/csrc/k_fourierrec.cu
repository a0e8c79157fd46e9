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
// nu = (k / M)(cos theta, sin theta), evaluated in four kernels per batch of
// slice pairs (two slices ride as the real and imaginary parts of one complex
// row, since the map is real-linear):
//   k_frec_rows       one CTA per (angle, pair): FFT of the padded row,
//                     times the centre phase -> P[pair][theta][k + M/2];
//   k_frec_gather     the L x L Cartesian frequency grid (L = next power of
//                     two >= 2n, at least 16: oversampling >= 2), one 4 x 4 node
//                     block per thread: every polar sample whose window
//                     reaches the block is added with the separable
//                     "exponential of semicircle" window of width W (Barnett,
//                     Magland, af Klinteberg, SIAM J. Sci. Comput. 41, 2019),
//                     visiting only the angles whose line passes near the
//                     block (angles folded to [0, pi) and sorted on the host);
//                     no atomics -> G[pair][gx][gy];
//   k_frec_cols       strips of grid columns: inverse FFTs, the n needed rows
//                     kept, divided by the window's Fourier transform in y
//                     -> H[pair][iy][gx];
//   k_frec_out        one CTA per (row, pair): inverse FFT of the row, the
//                     n needed columns divided by the window's transform in x,
//                     times scale, real part -> slice 2p, imaginary -> 2p+1.
// FFTs are in-place radix-4 (and one radix-2) decimation in frequency in
// shared memory (XOR-swizzled layout); their outputs are read at
// digit-reversed positions.
#include <cmath>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "tcp_internal.cuh"

namespace tcp {
namespace {

constexpr int kMaxLg = 14;  // M, L <= 16384 (128 KB of complex FP32 in shared memory)
constexpr int kMaxTheta = 1 << 24;  // angle indices and counts stay far inside int
constexpr size_t kBatchBytes = size_t(3) << 29;  // P + G + H workspace per batch (1.5 GiB)

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

// Shared-memory index of logical element g of an FFT buffer: the low four
// bits are XORed with bits 4..7 (rotated), a bijection within every aligned
// block of 16 elements.  It spreads the radix-4 stages with butterfly stride 4
// and 1 (and the output gathers) over all banks; stages with stride >= 16 see
// a permutation of 16 consecutive elements, as before.  Every access to an
// FFT buffer goes through it.
__device__ __forceinline__ int swz(int g) {
  const int h = g >> 4;
  return g ^ (((h & 3) << 2) | ((h >> 2) & 3));
}

// In-place decimation-in-frequency FFT of `count` sequences of length
// N = 2^lg stored back to back in shared memory (swizzled, swz).
// tw[j] = e^{-2 pi i j / N}; INV takes the conjugates (positive exponent, no
// 1/N); w^2 and w^3 of a butterfly are formed from w.  The caller
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
      const int e0 = (seq << lg) + (blk << lgs) + j;
      const int i0 = swz(e0), i1 = swz(e0 + m), i2 = swz(e0 + 2 * m), i3 = swz(e0 + 3 * m);
      const float2 x0 = a[i0], x1 = a[i1], x2 = a[i2], x3 = a[i3];
      const float2 s02 = cadd(x0, x2), d02 = csub(x0, x2), s13 = cadd(x1, x3), d13 = csub(x1, x3);
      // omega_4 = -i (forward) or +i (inverse) times d13
      const float2 r13 = INV ? make_float2(-d13.y, d13.x) : make_float2(d13.y, -d13.x);
      float2 w1 = __ldg(tw + j * ts);
      if (INV) w1.y = -w1.y;
      const float2 w2 = cmul(w1, w1), w3 = cmul(w2, w1);
      a[i0] = cadd(s02, s13);
      a[i1] = cmul(cadd(d02, r13), w1);
      a[i2] = cmul(csub(s02, s13), w2);
      a[i3] = cmul(csub(d02, r13), w3);
    }
    __syncthreads();
  }
  if (lgs == 1) {
    const int nb = count << (lg - 1);
    for (int b = tid; b < nb; b += nthr) {
      const int i0 = swz(2 * b), i1 = swz(2 * b + 1);
      const float2 x0 = a[i0], x1 = a[i1];
      a[i0] = cadd(x0, x1);
      a[i1] = csub(x0, x1);
    }
    __syncthreads();
  }
}

// --------------------------------------------------------------- tables --

// Per-call geometry in sorted-angle order: for sorted position u, meta[u] =
// (original angle t, sign s) with theta' = theta_t - pi (1 - s)/2 in [0, pi);
// geomS[u] = (L/M) s (cos theta_t, sin theta_t) as FP32 hi + lo pairs (from
// the FP64 angle table).  Also the row phase factors
// (w_k / M) e^{2 pi i k center / M}, k = -M/2 .. M/2, made in FP64.
__global__ void k_frec_geom(const double2* __restrict__ trig, const int2* __restrict__ meta, int nt, double ratio,
                            float4* __restrict__ geomS, double center, int M, float2* __restrict__ phase) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < nt) {
    const int2 m = meta[i];
    const double cx = trig[m.x].x * ratio * m.y, sy = trig[m.x].y * ratio * m.y;
    const float chi = (float)cx, shi = (float)sy;
    geomS[i] = make_float4(chi, (float)(cx - (double)chi), shi, (float)(sy - (double)shi));
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
    frec_buf[swz(j)] = make_float2(a, b);
  }
  __syncthreads();
  fft_dif<false>(frec_buf, lgM, 1, twM);
  float2* out = P + (int64_t)pb * p_pair + (int64_t)t * ms;
  for (int i = threadIdx.x; i <= M; i += blockDim.x)
    out[i] = cmul(frec_buf[swz(dif_pos((i - M / 2) & (M - 1), lgM))], __ldg(phase + i));
}

// ------------------------------------------------------------- kernel 2 --

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

// Window weight at distance d (grid points): exp(beta (sqrt(1 - (2d/W)^2) - 1))
// inside |d| < W/2, else 0, as 2^(bl2 (sqrt(z) - 1)) with bl2 = beta log2(e).
// The approximate square root and base-2 exponential (~2^-22 relative each)
// keep the weight within ~2e-6 relative, inside the window's own error at the
// default widths.
__device__ __forceinline__ float es_weight(float d, float bl2, float two_over_w) {
  const float s = d * two_over_w;
  const float z = fmaf(-s, s, 1.f);
  float q, w;
  asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(q) : "f"(z));
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(w) : "f"(fmaf(bl2, q, -bl2)));
  return z > 0.f ? w : 0.f;  // z <= 0: outside the window (sqrt of a negative is NaN, discarded)
}

// Intersect [klo, khi] with the integers k for which k * c lies in (A, B),
// up to a margin of 2e-3 in k: the quotients carry a relative error of a few
// 1e-7 (|k| <= 8192), and a sample that close to the window's edge has weight
// below 2e-7 (e^-beta scale), far inside the window's own error.
__device__ __forceinline__ void clip_k(float c, float A, float B, float lim, int* klo, int* khi) {
  if (fabsf(c) < 1e-30f) {
    if (!(A < 0.f && B > 0.f)) *khi = *klo - 1;
    return;
  }
  float qa = __fdividef(A, c), qb = __fdividef(B, c);
  if (qa > qb) {
    const float t = qa;
    qa = qb;
    qb = t;
  }
  *klo = max(*klo, (int)ceilf(fmaxf(qa, -lim) - 2e-3f));
  *khi = min(*khi, (int)floorf(fminf(qb, lim) + 2e-3f));
}

// Sorted-angle index range [u0, u1) of the angles theta' in [lo, hi] (thS
// ascending in [0, pi)).
__device__ __forceinline__ void angle_range(const float* __restrict__ thS, int nt, float lo, float hi, int* u0,
                                            int* u1) {
  int a = 0, b = nt;  // first index with thS >= lo
  while (a < b) {
    const int m = (a + b) >> 1;
    if (__ldg(thS + m) < lo) a = m + 1; else b = m;
  }
  *u0 = a;
  b = nt;  // first index with thS > hi
  while (a < b) {
    const int m = (a + b) >> 1;
    if (__ldg(thS + m) <= hi) a = m + 1; else b = m;
  }
  *u1 = a;
}

// Candidate angles for the nodes [bx0, bx0 + CW) x [by0, by0 + R): lines
// through the origin at angle theta' reach a window of a node only if they
// pass within hd + W/sqrt(2) of the block centre (hd: half diagonal).  Up to
// two sorted-index ranges (the angle interval may wrap at pi).
template <int R, int CW>
__device__ __forceinline__ int block_angles(int W, int bx0, int by0, const float* __restrict__ thS, int nt, int2* rng) {
  const float xc = bx0 + 0.5f * (CW - 1), yc = by0 + 0.5f * (R - 1);
  const float rho = sqrtf(xc * xc + yc * yc);
  const float reach = 0.5f * sqrtf((float)((CW - 1) * (CW - 1) + (R - 1) * (R - 1))) + 0.7072f * W + 0.5f;
  if (reach >= rho) {
    rng[0] = make_int2(0, nt);
    return 1;
  }
  const float kPi = 3.14159265358979f;
  const float alpha = asinf(reach / rho) + 1e-4f;
  float phi = atan2f(yc, xc);
  if (phi < 0.f) phi += kPi;
  if (phi >= kPi) phi -= kPi;
  const float lo = phi - alpha, hi = phi + alpha;
  int u0, u1;
  if (lo < 0.f) {
    angle_range(thS, nt, 0.f, hi, &u0, &u1);
    rng[0] = make_int2(u0, u1);
    angle_range(thS, nt, lo + kPi, kPi, &u0, &u1);
    rng[1] = make_int2(u0, u1);
    return 2;
  }
  if (hi >= kPi) {
    angle_range(thS, nt, lo, kPi, &u0, &u1);
    rng[0] = make_int2(u0, u1);
    angle_range(thS, nt, 0.f, hi - kPi, &u0, &u1);
    rng[1] = make_int2(u0, u1);
    return 2;
  }
  angle_range(thS, nt, lo, hi, &u0, &u1);
  rng[0] = make_int2(u0, u1);
  return 1;
}

// Adds to acc[r][c] the window-weighted samples of sorted angle u that reach
// node (bx0 + c, by0 + r).
template <int R, int CW>
__device__ __forceinline__ void gather_angle(int W, int u, int bx0, int by0, const float2* __restrict__ Pp, int ms,
                                             int M, const float4* __restrict__ geomS, const int2* __restrict__ meta,
                                             float bl2, float2 (&acc)[R][CW]) {
  const float tw = 2.f / (float)W;
  const float4 g = __ldg(geomS + u);
  int klo = -M / 2, khi = M / 2;
  const float lim = (float)M;
  clip_k(g.x, bx0 - 0.5f * W, bx0 + (CW - 1) + 0.5f * W, lim, &klo, &khi);
  clip_k(g.z, by0 - 0.5f * W, by0 + (R - 1) + 0.5f * W, lim, &klo, &khi);
  if (klo > khi) return;
  const int2 m = __ldg(meta + u);  // original angle, sign of k
  const float2* row = Pp + (int64_t)m.x * ms + M / 2;
  // positions k * (hi + lo) as integer part + fraction: exact split at klo,
  // then steps by the exact integer/fraction split of the increment (the
  // fraction's rounding is <= 2^-24 per step)
  const float fk0 = (float)klo;
  int gix, giy;
  float frx, fry;
  split_pos(fk0, g.x, g.y, &gix, &frx);
  split_pos(fk0, g.z, g.w, &giy, &fry);
  const float flx = floorf(g.x), fly = floorf(g.z);
  const int sxi = (int)flx, syi = (int)fly;
  const float sxf = (g.x - flx) + g.y, syf = (g.z - fly) + g.w;
  for (int k = klo; k <= khi; ++k) {
    const float dx = (float)(gix - bx0) + frx, dy = (float)(giy - by0) + fry;
    float wy[R];
#pragma unroll
    for (int r = 0; r < R; ++r) wy[r] = es_weight(dy - (float)r, bl2, tw);
    const float2 v = __ldg(row + m.y * k);
#pragma unroll
    for (int c = 0; c < CW; ++c) {
      const float wx = es_weight(dx - (float)c, bl2, tw);
      const float2 vx = make_float2(v.x * wx, v.y * wx);
#pragma unroll
      for (int r = 0; r < R; ++r) {
        acc[r][c].x = fmaf(vx.x, wy[r], acc[r][c].x);
        acc[r][c].y = fmaf(vx.y, wy[r], acc[r][c].y);
      }
    }
    frx += sxf;
    gix += sxi;
    if (frx >= 1.f) {
      frx -= 1.f;
      ++gix;
    } else if (frx < 0.f) {
      frx += 1.f;
      --gix;
    }
    fry += syf;
    giy += syi;
    if (fry >= 1.f) {
      fry -= 1.f;
      ++giy;
    } else if (fry < 0.f) {
      fry += 1.f;
      --giy;
    }
  }
}

// Gather: thread t owns a block of R x CW grid nodes (CW columns, R rows) in
// a 64 x 64-node tile per CTA (warps: 8 x 4 blocks), with signed node
// coordinates and their images shifted by -L (samples lie in [-L/2, L/2]),
// and adds every sample whose window reaches the block -- no atomics, no
// shared memory.  Warps with a block within kCoopRadius of the zero
// frequency (where every angle contributes) are "near": their nodes come
// from the near-node sparse table when the geometry has one (skip_near);
// without it they take their blocks one at a time and share each block's
// angles among the lanes, reducing with shuffles.
// Output: the grid G[pair][gx][gy] (column-major), written from registers.
// The radius was measured at 2048^2 x 64 slices, window 7: 64, 96, 128, 192,
// 256, 384, 512 gave 24.8, 24.6, 24.4, 24.6, 24.9, 25.9, 27.2 ms per call
// (the table's 0.21 GB at 128).
constexpr float kCoopRadius = 128.f;
constexpr int kTile = 64;  // nodes per CTA tile side

// Lane `lane` of warp `wid` in the CTA of tile `tile` owns the R x CW node
// block at (gx0, gy0); `own` tells whether it lies inside the L x L grid, and
// the return value whether that block, or its image shifted by -L in x or y,
// lies within kCoopRadius of the zero frequency.  A warp is "near" when any of
// its lanes is; the gather, the near-node table build and its application
// all decide it with this function.
template <int R, int CW>
__device__ __forceinline__ bool lane_block_near(int2 tile, int wid, int lane, int L, int W, int* gx0, int* gy0,
                                                bool* own) {
  constexpr int kWarpCols = 8 * CW, kWarpRows = 4 * R;
  constexpr int kWarpsX = kTile / kWarpCols;
  const int tx0 = tile.x * kTile + (wid % kWarpsX) * kWarpCols;
  const int ty0 = tile.y * kTile + (wid / kWarpsX) * kWarpRows;
  *gx0 = tx0 + (lane & 7) * CW;
  *gy0 = ty0 + (lane >> 3) * R;
  *own = *gx0 < L && *gy0 < L;
  bool near = false;
  if (*own) {
    for (int mx = 0; mx >= -1; --mx)
      for (int my = 0; my >= -1; --my) {
        const int bx0 = *gx0 + mx * L, by0 = *gy0 + my * L;
        if ((2 * (bx0 + CW - 1) <= -L - W || 2 * bx0 >= L + W) || (2 * (by0 + R - 1) <= -L - W || 2 * by0 >= L + W))
          continue;
        const float xc = bx0 + 0.5f * (CW - 1), yc = by0 + 0.5f * (R - 1);
        near |= xc * xc + yc * yc < kCoopRadius * kCoopRadius;
      }
  }
  return near;
}

// CTAs run in the order of `order`: tiles sorted by their distance from the
// zero frequency (nearest first), every slice pair of a tile in a row.  Near
// the origin every angle contributes and a tile takes many times the work of
// an outer one; started last, those tiles left most SMs idle at the end of
// the launch.
template <int R, int CW>
__global__ void __launch_bounds__(256) k_frec_gather(int W, const float2* __restrict__ P, int64_t p_pair, int ms,
                                                     const float4* __restrict__ geomS, const int2* __restrict__ meta,
                                                     const float* __restrict__ thS, int nt, int M, int lgL, float bl2,
                                                     float2* __restrict__ G, int64_t g_pair,
                                                     const int2* __restrict__ order, int nb, int skip_near) {
  const int L = 1 << lgL;
  const int rank = (int)(blockIdx.x / (unsigned)nb);
  const int pb = (int)(blockIdx.x - (unsigned)rank * (unsigned)nb);
  const int2 tile = __ldg(order + rank);
  const float2* Pp = P + (int64_t)pb * p_pair;
  float2* Gp = G + (int64_t)pb * g_pair;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  // warp tile: 8 blocks across (8 CW columns), 4 blocks down (4 R rows)
  constexpr int kWarpCols = 8 * CW, kWarpRows = 4 * R;
  constexpr int kWarpsX = kTile / kWarpCols;
  const int tx0 = tile.x * kTile + (wid % kWarpsX) * kWarpCols;
  const int ty0 = tile.y * kTile + (wid / kWarpsX) * kWarpRows;
  int gx0, gy0;
  bool own;
  const bool near = lane_block_near<R, CW>(tile, wid, lane, L, W, &gx0, &gy0, &own);
  auto reachable = [&](int b0, int ext) { return !(2 * (b0 + ext - 1) <= -L - W || 2 * b0 >= L + W); };
  const bool warp_near = __any_sync(0xffffffffu, near);
  if (warp_near && skip_near) return;  // the near-node table covers this warp's nodes
  float2 acc[R][CW];
  if (!warp_near) {
    if (!own) return;
#pragma unroll
    for (int r = 0; r < R; ++r)
#pragma unroll
      for (int c = 0; c < CW; ++c) acc[r][c] = make_float2(0.f, 0.f);
    for (int mx = 0; mx >= -1; --mx)
      for (int my = 0; my >= -1; --my) {
        const int bx0 = gx0 + mx * L, by0 = gy0 + my * L;
        if (!reachable(bx0, CW) || !reachable(by0, R)) continue;
        int2 rng[2];
        const int nr = block_angles<R, CW>(W, bx0, by0, thS, nt, rng);
        for (int q = 0; q < nr; ++q)
          for (int u = rng[q].x; u < rng[q].y; ++u)
            gather_angle<R, CW>(W, u, bx0, by0, Pp, ms, M, geomS, meta, bl2, acc);
      }
#pragma unroll
    for (int c = 0; c < CW; ++c)
#pragma unroll
      for (int r = 0; r < R; ++r) Gp[(int64_t)(gx0 + c) * L + gy0 + r] = acc[r][c];
    return;
  }
  // cooperative: the warp's 32 blocks one at a time, angles split over lanes
  for (int bi = 0; bi < 32; ++bi) {
    const int bx = tx0 + (bi & 7) * CW, by = ty0 + (bi >> 3) * R;
    if (bx >= L || by >= L) continue;  // uniform over the warp
#pragma unroll
    for (int r = 0; r < R; ++r)
#pragma unroll
      for (int c = 0; c < CW; ++c) acc[r][c] = make_float2(0.f, 0.f);
    for (int mx = 0; mx >= -1; --mx)
      for (int my = 0; my >= -1; --my) {
        const int bx0 = bx + mx * L, by0 = by + my * L;
        if (!reachable(bx0, CW) || !reachable(by0, R)) continue;
        int2 rng[2];
        const int nr = block_angles<R, CW>(W, bx0, by0, thS, nt, rng);
        for (int q = 0; q < nr; ++q)
          for (int u = rng[q].x + lane; u < rng[q].y; u += 32)
            gather_angle<R, CW>(W, u, bx0, by0, Pp, ms, M, geomS, meta, bl2, acc);
      }
#pragma unroll
    for (int r = 0; r < R; ++r)
#pragma unroll
      for (int c = 0; c < CW; ++c) {
        float x = acc[r][c].x, y = acc[r][c].y;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
          x += __shfl_xor_sync(0xffffffffu, x, o);
          y += __shfl_xor_sync(0xffffffffu, y, o);
        }
        if (lane == (r * CW + c) % 32) Gp[(int64_t)(bx + c) * L + by + r] = make_float2(x, y);
      }
  }
}

// ---------------------------------------------- near-node sparse table --
//
// The nodes of near warps (within ~kCoopRadius of the zero frequency, where
// every angle contributes) cost the gather far more per node than any other,
// and their window weights do not depend on the data: they are listed once
// per geometry as a
// sparse table, row = node (16 rows per lane block, 8 warps x 32 lanes per
// tile, tiles in gather order), entries (P offset within a slice pair,
// weight wx * wy), in the gather's visiting order (images, sorted angles, k).
// Applying the table to a batch reads each entry once for up to 8 slice pairs.

// Calls f(P offset, weight) for every sample of sorted angle u whose window
// reaches node (bx0, by0) with a non-zero weight, k ascending: the gather's
// positions and weights for a one-node block.
template <class F>
__device__ __forceinline__ void node_angle(int W, int u, int bx0, int by0, int ms, int M,
                                           const float4* __restrict__ geomS, const int2* __restrict__ meta,
                                           float bl2, F&& f) {
  const float tw = 2.f / (float)W;
  const float4 g = __ldg(geomS + u);
  int klo = -M / 2, khi = M / 2;
  const float lim = (float)M;
  clip_k(g.x, bx0 - 0.5f * W, bx0 + 0.5f * W, lim, &klo, &khi);
  clip_k(g.z, by0 - 0.5f * W, by0 + 0.5f * W, lim, &klo, &khi);
  if (klo > khi) return;
  const int2 m = __ldg(meta + u);
  const int row = m.x * ms + M / 2;
  const float fk0 = (float)klo;
  int gix, giy;
  float frx, fry;
  split_pos(fk0, g.x, g.y, &gix, &frx);
  split_pos(fk0, g.z, g.w, &giy, &fry);
  const float flx = floorf(g.x), fly = floorf(g.z);
  const int sxi = (int)flx, syi = (int)fly;
  const float sxf = (g.x - flx) + g.y, syf = (g.z - fly) + g.w;
  for (int k = klo; k <= khi; ++k) {
    const float dx = (float)(gix - bx0) + frx, dy = (float)(giy - by0) + fry;
    const float w = es_weight(dx, bl2, tw) * es_weight(dy, bl2, tw);
    if (w != 0.f) f(row + m.y * k, w);
    frx += sxf;
    gix += sxi;
    if (frx >= 1.f) {
      frx -= 1.f;
      ++gix;
    } else if (frx < 0.f) {
      frx += 1.f;
      --gix;
    }
    fry += syf;
    giy += syi;
    if (fry >= 1.f) {
      fry -= 1.f;
      ++giy;
    } else if (fry < 0.f) {
      fry += 1.f;
      --giy;
    }
  }
}

// Count (FILL = false: counts[row]) or write (FILL: ent[off[row] ..]) the
// entries of every node of the near warps of tiles order[0 .. gridDim.x).
template <int R, int CW, bool FILL>
__global__ void __launch_bounds__(256) k_frec_near_build(int W, const float4* __restrict__ geomS,
                                                         const int2* __restrict__ meta, const float* __restrict__ thS,
                                                         int nt, int M, int lgL, float bl2,
                                                         const int2* __restrict__ order, int* __restrict__ counts,
                                                         const int64_t* __restrict__ off, int2* __restrict__ ent) {
  const int L = 1 << lgL, ms = M + 1;
  const int rank = blockIdx.x;
  const int2 tile = __ldg(order + rank);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  int gx0, gy0;
  bool own;
  const bool near = lane_block_near<R, CW>(tile, wid, lane, L, W, &gx0, &gy0, &own);
  if (!__any_sync(0xffffffffu, near) || !own) return;
  const int64_t rowb = ((int64_t)(rank * 8 + wid) * 32 + lane) * (R * CW);
  for (int r = 0; r < R; ++r)
    for (int c = 0; c < CW; ++c) {
      const int64_t row = rowb + r * CW + c;
      int cnt = 0;
      int64_t pos = FILL ? off[row] : 0;
      for (int mx = 0; mx >= -1; --mx)
        for (int my = 0; my >= -1; --my) {
          const int bx = gx0 + c + mx * L, by = gy0 + r + my * L;
          if ((2 * bx <= -L - W || 2 * bx >= L + W) || (2 * by <= -L - W || 2 * by >= L + W)) continue;
          int2 rng[2];
          const int nr = block_angles<1, 1>(W, bx, by, thS, nt, rng);
          for (int q = 0; q < nr; ++q)
            for (int u = rng[q].x; u < rng[q].y; ++u)
              node_angle(W, u, bx, by, ms, M, geomS, meta, bl2, [&](int o, float w) {
                if (FILL) ent[pos++] = make_int2(o, __float_as_int(w));
                else ++cnt;
              });
        }
      if (!FILL) counts[row] = cnt;
    }
}

// G[pair][node] = sum of weight x P[pair][offset] over the node's entries,
// for the nodes of near warps and slice pairs 0 .. nb - 1, at most kPairs at
// a time.  One warp per row, the lanes splitting the row's entries, then a
// shuffle reduction; rows with more than kHeavyRow entries (the nodes next to
// the zero frequency, where every angle contributes) are left to
// k_frec_near_heavy, one CTA each.
constexpr int kNearPairs = 8;
constexpr int kHeavyRow = 4096;

// Node coordinates of table row `row` (16 rows per lane block, 32 lane blocks
// per warp, 8 warps per tile in gather order).
__device__ __forceinline__ void near_row_node(int64_t row, const int2* __restrict__ order, int* gx, int* gy, int* rank,
                                              int* w, int* l) {
  const int64_t blk = row >> 4;
  const int rc = (int)(row & 15);
  *rank = (int)(blk >> 8);
  *w = (int)((blk >> 5) & 7);
  *l = (int)(blk & 31);
  const int2 tile = __ldg(order + *rank);
  *gx = tile.x * kTile + (*w % 2) * 32 + (*l & 7) * 4 + (rc & 3);
  *gy = tile.y * kTile + (*w / 2) * 16 + (*l >> 3) * 4 + (rc >> 2);
}

// nearw[rank * 8 + warp] = 1 for the near warps of tiles order[0 .. gridDim.x).
template <int R, int CW>
__global__ void __launch_bounds__(256) k_frec_near_flags(int W, int lgL, const int2* __restrict__ order,
                                                         unsigned char* __restrict__ nearw) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  int gx0, gy0;
  bool own;
  const bool near = lane_block_near<R, CW>(__ldg(order + blockIdx.x), wid, lane, 1 << lgL, W, &gx0, &gy0, &own);
  const bool any = __any_sync(0xffffffffu, near);
  if (lane == 0) nearw[blockIdx.x * 8 + wid] = any ? 1 : 0;
}

__device__ __forceinline__ void near_accumulate(const float2* __restrict__ Pp, int64_t p_pair, int np, int2 en,
                                                float2 (&acc)[kNearPairs]) {
  const float w = __int_as_float(en.y);
#pragma unroll
  for (int p = 0; p < kNearPairs; ++p)
    if (p < np) {
      const float2 v = __ldg(Pp + p * p_pair + en.x);
      acc[p].x = fmaf(w, v.x, acc[p].x);
      acc[p].y = fmaf(w, v.y, acc[p].y);
    }
}

__global__ void __launch_bounds__(256) k_frec_near_apply(const float2* __restrict__ P, int64_t p_pair, int nb,
                                                         const int64_t* __restrict__ off,
                                                         const int2* __restrict__ ent,
                                                         const unsigned char* __restrict__ nearw, int lgL,
                                                         int64_t rows, const int2* __restrict__ order,
                                                         float2* __restrict__ G, int64_t g_pair) {
  const int L = 1 << lgL;
  const int lane = threadIdx.x & 31;
  const int64_t row = (int64_t)blockIdx.x * 8 + (threadIdx.x >> 5);
  if (row >= rows || !__ldg(nearw + (row >> 9))) return;  // 512 rows per gather warp
  int gx, gy, rank, w, l;
  near_row_node(row, order, &gx, &gy, &rank, &w, &l);
  if (gx - (int)(row & 3) >= L || gy - (int)((row >> 2) & 3) >= L) return;  // block outside the grid
  const int64_t e0 = __ldg(off + row), e1 = __ldg(off + row + 1);
  if (e1 - e0 > kHeavyRow) return;
  for (int p0 = 0; p0 < nb; p0 += kNearPairs) {
    const int np = min(kNearPairs, nb - p0);
    float2 acc[kNearPairs];
#pragma unroll
    for (int p = 0; p < kNearPairs; ++p) acc[p] = make_float2(0.f, 0.f);
    const float2* Pp = P + (int64_t)p0 * p_pair;
    int64_t e = e0 + lane;
    for (; e + 32 < e1; e += 64) {  // two entries in flight per lane
      const int2 a = __ldg(ent + e), b = __ldg(ent + e + 32);
      near_accumulate(Pp, p_pair, np, a, acc);
      near_accumulate(Pp, p_pair, np, b, acc);
    }
    if (e < e1) near_accumulate(Pp, p_pair, np, __ldg(ent + e), acc);
#pragma unroll
    for (int p = 0; p < kNearPairs; ++p) {
      if (p >= np) break;  // uniform over the warp
      float x = acc[p].x, y = acc[p].y;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        x += __shfl_xor_sync(0xffffffffu, x, o);
        y += __shfl_xor_sync(0xffffffffu, y, o);
      }
      if (lane == p) G[(int64_t)(p0 + p) * g_pair + (int64_t)gx * L + gy] = make_float2(x, y);
    }
  }
}

// The heavy rows, one CTA (256 threads) each: the threads split the entries,
// warp shuffles then shared memory reduce them in a fixed order.
__global__ void __launch_bounds__(256) k_frec_near_heavy(const float2* __restrict__ P, int64_t p_pair, int nb,
                                                         const int64_t* __restrict__ off,
                                                         const int2* __restrict__ ent,
                                                         const int64_t* __restrict__ heavy, int lgL,
                                                         const int2* __restrict__ order, float2* __restrict__ G,
                                                         int64_t g_pair) {
  __shared__ float2 red[8][kNearPairs];
  const int L = 1 << lgL;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int64_t row = __ldg(heavy + blockIdx.x);
  int gx, gy, rank, w, l;
  near_row_node(row, order, &gx, &gy, &rank, &w, &l);
  const int64_t e0 = __ldg(off + row), e1 = __ldg(off + row + 1);
  for (int p0 = 0; p0 < nb; p0 += kNearPairs) {
    const int np = min(kNearPairs, nb - p0);
    float2 acc[kNearPairs];
#pragma unroll
    for (int p = 0; p < kNearPairs; ++p) acc[p] = make_float2(0.f, 0.f);
    const float2* Pp = P + (int64_t)p0 * p_pair;
    int64_t e = e0 + threadIdx.x;
    for (; e + 256 < e1; e += 512) {
      const int2 a = __ldg(ent + e), b = __ldg(ent + e + 256);
      near_accumulate(Pp, p_pair, np, a, acc);
      near_accumulate(Pp, p_pair, np, b, acc);
    }
    if (e < e1) near_accumulate(Pp, p_pair, np, __ldg(ent + e), acc);
#pragma unroll
    for (int p = 0; p < kNearPairs; ++p) {
      float x = acc[p].x, y = acc[p].y;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        x += __shfl_xor_sync(0xffffffffu, x, o);
        y += __shfl_xor_sync(0xffffffffu, y, o);
      }
      if (lane == 0) red[wid][p] = make_float2(x, y);
    }
    __syncthreads();
    if (threadIdx.x < np) {
      float2 t = red[0][threadIdx.x];
      for (int q = 1; q < 8; ++q) t = make_float2(t.x + red[q][threadIdx.x].x, t.y + red[q][threadIdx.x].y);
      G[(int64_t)(p0 + threadIdx.x) * g_pair + (int64_t)gx * L + gy] = t;
    }
    __syncthreads();
  }
}

// Column pass: one CTA per strip of CW grid columns (contiguous in G): the
// columns' inverse FFTs in shared memory, then rows y in [-n/2, n/2) are
// kept, times 1/Phi(y/L) -> H[pair][iy][gx].
__global__ void __launch_bounds__(1024) k_frec_cols(const float2* __restrict__ G, int64_t g_pair, int lgL, int cw,
                                                    int n, const float2* __restrict__ twL,
                                                    const float* __restrict__ dec, float2* __restrict__ H,
                                                    int64_t h_pair) {
  extern __shared__ float4 frec_smem4[];
  const int L = 1 << lgL;
  float2* strip = reinterpret_cast<float2*>(frec_smem4);  // [cw][L]
  const int gx0 = blockIdx.x * cw, pb = blockIdx.y;
  const float2* src = G + (int64_t)pb * g_pair + (int64_t)gx0 * L;
  for (int i = threadIdx.x; i < cw * L; i += blockDim.x) strip[swz(i)] = __ldg(src + i);
  __syncthreads();
  fft_dif<true>(strip, lgL, cw, twL);
  float2* Hp = H + (int64_t)pb * h_pair;
  for (int i = threadIdx.x; i < n * cw; i += blockDim.x) {
    const int iy = i / cw, c = i - iy * cw;
    const float2 v = strip[swz(c * L + dif_pos((iy - n / 2) & (L - 1), lgL))];
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
  for (int j = threadIdx.x; j < L; j += blockDim.x) frec_buf[swz(j)] = __ldg(row + j);
  __syncthreads();
  fft_dif<true>(frec_buf, lgL, 1, twL);
  const int z1 = z0 + 2 * pb, z2 = z1 + 1;
  TV* o1 = vol + (int64_t)z1 * v0 + (int64_t)iy * v1;
  TV* o2 = vol + (int64_t)z2 * v0 + (int64_t)iy * v1;
  const bool two = z2 < nz;
  for (int ix = threadIdx.x; ix < n; ix += blockDim.x) {
    const float2 v = frec_buf[swz(dif_pos((ix - n / 2) & (L - 1), lgL))];
    const float d = __ldg(dec + ix) * scale;
    Store<TV>::put(o1 + ix, v.x * d);
    if (two) Store<TV>::put(o2 + ix, v.y * d);
  }
}

// --------------------------------------------------------- host tables --

struct SortedAngles {
  std::vector<double> theta;
  uint64_t hash = 0;      // of the angle array's bytes
  uint64_t used = 0;      // last-use stamp (least recently used goes first)
  int2* meta = nullptr;   // (original index, sign of k) per sorted position
  float* thS = nullptr;   // theta' in [0, pi), ascending
};
// Angle sets kept per device; beyond this the least recently used set is freed.
constexpr size_t kAngleCacheCap = 64;
uint64_t g_frec_stamp = 0;

uint64_t bytes_hash(const void* p, size_t n) {  // FNV-1a
  const unsigned char* b = reinterpret_cast<const unsigned char*>(p);
  uint64_t h = 1469598103934665603ull;
  for (size_t i = 0; i < n; ++i) h = (h ^ b[i]) * 1099511628211ull;
  return h;
}
struct NearEntry;  // near-node table of one geometry (defined with its builder)
struct HostTables {
  std::map<std::pair<int, int>, float2*> tw;                 // (dev, N) -> e^{-2 pi i j / N}
  std::map<std::tuple<int, int, int, int>, float*> dec;      // (dev, n, L, W) -> 1 / Phi(x / L)
  std::map<int, std::vector<SortedAngles>> ang;              // dev -> angle arrays seen
  std::map<std::pair<int, int>, int2*> order;                // (dev, L) -> gather tile order
  std::vector<NearEntry*> nearT;                             // near-node tables (least recently used freed)
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

// Angles folded to theta' = theta mod pi in [0, pi) (k changes sign when
// theta mod 2 pi >= pi: the same line through the origin), sorted ascending:
// per sorted position the original index and the sign of k, and theta'.
void sort_angles(const double* theta, int nt, std::vector<int2>* meta, std::vector<float>* ths) {
  std::vector<std::pair<double, int2>> v((size_t)nt);
  for (int t = 0; t < nt; ++t) {
    double a = std::fmod(theta[t], 2.0 * M_PI);
    if (a < 0.0) a += 2.0 * M_PI;
    int sg = 1;
    if (a >= M_PI) {
      a -= M_PI;
      sg = -1;
    }
    if (a >= M_PI) a = 0.0;  // rounding at the top of the range
    v[(size_t)t] = {a, make_int2(t, sg)};
  }
  std::stable_sort(v.begin(), v.end(), [](const std::pair<double, int2>& x, const std::pair<double, int2>& y) {
    return x.first < y.first;
  });
  meta->resize((size_t)std::max(nt, 1));
  ths->resize((size_t)std::max(nt, 1));
  for (int u = 0; u < nt; ++u) {
    (*meta)[(size_t)u] = v[(size_t)u].second;
    (*ths)[(size_t)u] = (float)v[(size_t)u].first;
  }
}

// Cached per device and angle set.
tcp_status get_sorted_angles(int dev, const double* theta, int nt, const int2** meta, const float** thS) {
  std::lock_guard<std::mutex> lk(g_frec_mu);
  auto& lst = g_frec.ang[dev];
  const uint64_t h = bytes_hash(theta, sizeof(double) * (size_t)nt);
  for (auto& e : lst)
    if (e.hash == h && (int)e.theta.size() == nt && std::equal(e.theta.begin(), e.theta.end(), theta)) {
      e.used = ++g_frec_stamp;
      *meta = e.meta;
      *thS = e.thS;
      return TCP_OK;
    }
  if (lst.size() >= kAngleCacheCap) {
    // cudaFree waits for the device, so no queued kernel still reads the set
    auto lru = std::min_element(lst.begin(), lst.end(),
                                [](const SortedAngles& a, const SortedAngles& b) { return a.used < b.used; });
    cudaFree(lru->meta);
    cudaFree(lru->thS);
    lst.erase(lru);
  }
  std::vector<int2> hm;
  std::vector<float> ht;
  sort_angles(theta, nt, &hm, &ht);
  SortedAngles e;
  e.theta.assign(theta, theta + nt);
  e.hash = h;
  e.used = ++g_frec_stamp;
  TCP_CUDA_TRY(cudaMalloc(&e.meta, sizeof(int2) * (size_t)std::max(nt, 1)));
  cudaError_t err = cudaMalloc(&e.thS, sizeof(float) * (size_t)std::max(nt, 1));
  if (err != cudaSuccess) {
    cudaFree(e.meta);
    return cuda_fail(err, "cudaMalloc");
  }
  err = cudaMemcpy(e.meta, hm.data(), sizeof(int2) * (size_t)nt, cudaMemcpyHostToDevice);
  if (err == cudaSuccess) err = cudaMemcpy(e.thS, ht.data(), sizeof(float) * (size_t)nt, cudaMemcpyHostToDevice);
  if (err != cudaSuccess) {
    cudaFree(e.meta);
    cudaFree(e.thS);
    return cuda_fail(err, "upload FourierRec angle table");
  }
  lst.push_back(e);
  *meta = e.meta;
  *thS = e.thS;
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

template <int R, int CW>
void launch_gather(int W, const float2* P, int64_t p_pair, int ms, const float4* geomS, const int2* meta,
                   const float* thS, int nt, int M, int lgL, float2* G, int64_t g_pair, int nb, const int2* order,
                   const FrecTables& tb, cudaStream_t st) {
  const int L = 1 << lgL;
  const unsigned tiles = (unsigned)((L + kTile - 1) / kTile);
  const int skip = tb.t_near > 0 ? 1 : 0;
  k_frec_gather<R, CW><<<dim3(tiles * tiles * (unsigned)nb), 256, 0, st>>>(
      W, P, p_pair, ms, geomS, meta, thS, nt, M, lgL, (float)(es_beta(W) / M_LN2), G, g_pair, order, nb, skip);
  if (skip) {
    const int64_t rows = (int64_t)tb.t_near * 4096;
    k_frec_near_apply<<<dim3((unsigned)((rows + 7) / 8)), 256, 0, st>>>(P, p_pair, nb, tb.near_off, tb.near_ent,
                                                                         tb.near_warps, lgL, rows, order, G, g_pair);
    if (tb.n_heavy > 0)
      k_frec_near_heavy<<<dim3((unsigned)tb.n_heavy), 256, 0, st>>>(P, p_pair, nb, tb.near_off, tb.near_ent,
                                                                     tb.near_heavy, lgL, order, G, g_pair);
  }
}

std::vector<int2> gather_tile_order(int L);

// Near-node table of one geometry: tiles order[0 .. t_near) (every tile with
// a near warp: their centres lie within kCoopRadius + 64 of the zero
// frequency), 4096 rows each.  Sample positions as k_frec_geom makes them
// (FP64 cos/sin times L/M, split into FP32 hi + lo).  Returns t_near = 0
// without a table when the device memory for it is not available.
struct NearTable {
  int t_near = 0;
  int64_t* off = nullptr;
  int2* ent = nullptr;
  int64_t n_heavy = 0;
  int64_t* heavy = nullptr;  // rows above kHeavyRow entries
  unsigned char* warps = nullptr;  // near flag per gather warp of the t_near tiles
  size_t bytes = 0;
};
tcp_status build_near_table(const double* theta, int nt, int lgM, int lgL, int W, const std::vector<int2>& hmeta,
                            const int2* d_meta, const float* d_thS, const int2* d_order,
                            const std::vector<int2>& horder, NearTable* out) {
  const int M = 1 << lgM, L = 1 << lgL;
  *out = NearTable();
  int t_near = 0;
  for (const int2& t : horder) {
    const double cx = t.x * kTile + 0.5 * kTile, cy = t.y * kTile + 0.5 * kTile;
    const double dx = std::min(cx, L - cx), dy = std::min(cy, L - cy);
    if (std::sqrt(dx * dx + dy * dy) >= (double)kCoopRadius + 64.0) break;
    ++t_near;
  }
  // entries hold the P offset of a sample as an int: the spectra of one slice
  // pair must stay below 2^31 samples
  if (t_near == 0 || nt == 0 || (int64_t)nt * (M + 1) >= (int64_t(1) << 31)) return TCP_OK;
  std::vector<float4> hg((size_t)nt);
  const double ratio = (double)L / (double)M;
  for (int u = 0; u < nt; ++u) {
    const int2 m = hmeta[(size_t)u];
    const double cx = std::cos(theta[m.x]) * ratio * m.y, sy = std::sin(theta[m.x]) * ratio * m.y;
    const float chi = (float)cx, shi = (float)sy;
    hg[(size_t)u] = make_float4(chi, (float)(cx - (double)chi), shi, (float)(sy - (double)shi));
  }
  const int64_t rows = (int64_t)t_near * 4096;
  float4* dg = nullptr;
  int* dc = nullptr;
  int64_t* doff = nullptr;
  int2* dent = nullptr;
  int64_t* dheavy = nullptr;
  unsigned char* dwarps = nullptr;
  auto release = [&]() {
    cudaFree(dg);
    cudaFree(dc);
    cudaFree(doff);
    cudaFree(dent);
    cudaFree(dheavy);
    cudaFree(dwarps);
  };
  if (cudaMalloc(&dg, sizeof(float4) * (size_t)nt) != cudaSuccess ||
      cudaMalloc(&dc, sizeof(int) * (size_t)rows) != cudaSuccess ||
      cudaMalloc(&doff, sizeof(int64_t) * (size_t)(rows + 1)) != cudaSuccess) {
    release();
    cudaGetLastError();  // an allocation failure is not sticky; the gather keeps these nodes
    return TCP_OK;
  }
  cudaError_t e = cudaMemcpy(dg, hg.data(), sizeof(float4) * (size_t)nt, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemset(dc, 0, sizeof(int) * (size_t)rows);
  const float bl2 = (float)(es_beta(W) / M_LN2);
  if (e == cudaSuccess) {
    k_frec_near_build<4, 4, false><<<dim3((unsigned)t_near), 256>>>(W, dg, d_meta, d_thS, nt, M, lgL, bl2, d_order,
                                                                    dc, nullptr, nullptr);
    e = cudaGetLastError();
  }
  std::vector<int> hc((size_t)rows);
  if (e == cudaSuccess) e = cudaMemcpy(hc.data(), dc, sizeof(int) * (size_t)rows, cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) {
    release();
    return cuda_fail(e, "FourierRec near-node table (count)");
  }
  std::vector<int64_t> ho((size_t)rows + 1), hh;
  ho[0] = 0;
  for (int64_t i = 0; i < rows; ++i) {
    ho[(size_t)i + 1] = ho[(size_t)i] + hc[(size_t)i];
    if (hc[(size_t)i] > kHeavyRow) hh.push_back(i);
  }
  const int64_t total = ho[(size_t)rows];
  if (total > (int64_t(1) << 29)) {  // above 4 GB the gather keeps these nodes
    release();
    return TCP_OK;
  }
  if (cudaMalloc(&dent, sizeof(int2) * (size_t)std::max<int64_t>(total, 1)) != cudaSuccess ||
      cudaMalloc(&dheavy, sizeof(int64_t) * std::max<size_t>(hh.size(), 1)) != cudaSuccess ||
      cudaMalloc(&dwarps, (size_t)t_near * 8) != cudaSuccess) {
    release();
    cudaGetLastError();
    return TCP_OK;
  }
  e = cudaMemcpy(doff, ho.data(), sizeof(int64_t) * (size_t)(rows + 1), cudaMemcpyHostToDevice);
  if (e == cudaSuccess && !hh.empty())
    e = cudaMemcpy(dheavy, hh.data(), sizeof(int64_t) * hh.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) {
    k_frec_near_build<4, 4, true><<<dim3((unsigned)t_near), 256>>>(W, dg, d_meta, d_thS, nt, M, lgL, bl2, d_order,
                                                                   nullptr, doff, dent);
    k_frec_near_flags<4, 4><<<dim3((unsigned)t_near), 256>>>(W, lgL, d_order, dwarps);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  cudaFree(dg);
  cudaFree(dc);
  if (e != cudaSuccess) {
    cudaFree(doff);
    cudaFree(dent);
    cudaFree(dheavy);
    cudaFree(dwarps);
    return cuda_fail(e, "FourierRec near-node table (fill)");
  }
  out->t_near = t_near;
  out->off = doff;
  out->ent = dent;
  out->n_heavy = (int64_t)hh.size();
  out->heavy = dheavy;
  out->warps = dwarps;
  out->bytes = sizeof(int64_t) * (size_t)(rows + 1) + sizeof(int2) * (size_t)std::max<int64_t>(total, 1) +
               sizeof(int64_t) * std::max<size_t>(hh.size(), 1);
  return TCP_OK;
}

// Cached near-node tables: a few geometries (each up to ~1 GB at 2048^2),
// the least recently used freed beyond the cap.
struct NearEntry {
  int dev = 0, M = 0, L = 0, W = 0;
  std::vector<double> theta;
  uint64_t hash = 0, used = 0;
  NearTable t;
};
constexpr size_t kNearCacheCap = 4;

tcp_status get_near_table(int dev, const double* theta, int nt, int lgM, int lgL, int W, const int2* d_meta,
                          const float* d_thS, const int2* d_order, NearTable* out) {
  std::lock_guard<std::mutex> lk(g_frec_mu);
  const uint64_t h = bytes_hash(theta, sizeof(double) * (size_t)nt);
  for (NearEntry* e : g_frec.nearT)
    if (e->dev == dev && e->M == (1 << lgM) && e->L == (1 << lgL) && e->W == W && e->hash == h &&
        (int)e->theta.size() == nt && std::equal(e->theta.begin(), e->theta.end(), theta)) {
      e->used = ++g_frec_stamp;
      *out = e->t;
      return TCP_OK;
    }
  if (g_frec.nearT.size() >= kNearCacheCap) {
    auto lru = std::min_element(g_frec.nearT.begin(), g_frec.nearT.end(),
                                [](const NearEntry* a, const NearEntry* b) { return a->used < b->used; });
    cudaFree((*lru)->t.off);  // cudaFree waits for the device: no queued kernel still reads it
    cudaFree((*lru)->t.ent);
    cudaFree((*lru)->t.heavy);
    cudaFree((*lru)->t.warps);
    delete *lru;
    g_frec.nearT.erase(lru);
  }
  std::vector<int2> hm;
  std::vector<float> ht;
  sort_angles(theta, nt, &hm, &ht);
  NearTable t;
  tcp_status s = build_near_table(theta, nt, lgM, lgL, W, hm, d_meta, d_thS, d_order, gather_tile_order(1 << lgL), &t);
  if (s != TCP_OK) return s;
  NearEntry* e = new NearEntry;
  e->dev = dev;
  e->M = 1 << lgM;
  e->L = 1 << lgL;
  e->W = W;
  e->theta.assign(theta, theta + nt);
  e->hash = h;
  e->used = ++g_frec_stamp;
  e->t = t;
  g_frec.nearT.push_back(e);
  *out = t;
  return TCP_OK;
}

// Gather tiles of an L x L grid, nearest to the zero frequency (node 0 and
// its image at L) first.
std::vector<int2> gather_tile_order(int L) {
  const int tiles = (L + kTile - 1) / kTile;
  std::vector<std::pair<double, int2>> v;
  v.reserve((size_t)tiles * tiles);
  for (int ty = 0; ty < tiles; ++ty)
    for (int tx = 0; tx < tiles; ++tx) {
      const double cx = tx * kTile + 0.5 * kTile, cy = ty * kTile + 0.5 * kTile;
      const double dx = std::min(cx, L - cx), dy = std::min(cy, L - cy);
      v.push_back({dx * dx + dy * dy, make_int2(tx, ty)});
    }
  std::stable_sort(v.begin(), v.end(), [](const std::pair<double, int2>& a, const std::pair<double, int2>& b) {
    return a.first < b.first;
  });
  std::vector<int2> out(v.size());
  for (size_t i = 0; i < v.size(); ++i) out[i] = v[i].second;
  return out;
}

void launch_cols(const float2* G, int64_t g_pair, int lgL, int n, const float2* twL, const float* dec, float2* H,
                 int64_t h_pair, int nb, cudaStream_t st) {
  const int L = 1 << lgL;
  // two columns (64 KB at L = 4096) per CTA: several CTAs per SM overlap one
  // another's stage barriers
  const int cw = std::max(1, std::min(std::min(2, L), (1 << (kMaxLg - 1)) / L));
  const size_t sm = sizeof(float2) * (size_t)cw * L;
  cudaFuncSetAttribute(k_frec_cols, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  k_frec_cols<<<dim3((unsigned)(L / cw), (unsigned)nb), 512, sm, st>>>(G, g_pair, lgL, cw, n, twL, dec, H, h_pair);
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

void fourierrec_cache_clear() {
  std::lock_guard<std::mutex> lk(g_frec_mu);
  for (auto& kv : g_frec.tw) cudaFree(kv.second);
  g_frec.tw.clear();
  for (auto& kv : g_frec.dec) cudaFree(kv.second);
  g_frec.dec.clear();
  for (auto& kv : g_frec.order) cudaFree(kv.second);
  g_frec.order.clear();
  for (auto& kv : g_frec.ang)
    for (auto& e : kv.second) {
      cudaFree(e.meta);
      cudaFree(e.thS);
    }
  g_frec.ang.clear();
  for (NearEntry* e : g_frec.nearT) {
    cudaFree(e->t.off);
    cudaFree(e->t.ent);
    cudaFree(e->t.heavy);
    cudaFree(e->t.warps);
    delete e;
  }
  g_frec.nearT.clear();
}

// Cartesian grid side: the next power of two >= 2n, at least 16 (oversampling
// >= 2, and every window width 2..16 fits).
int64_t fourierrec_grid(int64_t n) {
  int64_t L = 16;
  while (L < 2 * n) L *= 2;
  return L;
}

int fourierrec_default_width(int vol_dtype, int64_t n) {
  return (int)std::min<int64_t>(fourierrec_grid(n), vol_dtype == TCP_F32 ? 7 : 5);
}

tcp_status fourierrec_check(int64_t nt, int64_t nd, int64_t n, int width) {
  if (n % 2) return fail(TCP_ERR_SHAPE, "fourierrec: n must be even");
  int64_t M = 1;
  while (M < 2 * nd) M *= 2;
  const int64_t L = fourierrec_grid(n);
  if (M > (int64_t(1) << kMaxLg)) return fail(TCP_ERR_SHAPE, "fourierrec: ndet must be <= 8192");
  if (L > (int64_t(1) << kMaxLg)) return fail(TCP_ERR_SHAPE, "fourierrec: n must be <= 8192");
  if (nt > kMaxTheta) return fail(TCP_ERR_SHAPE, "fourierrec: ntheta must be <= 2^24");
  if (width < 2 || width > 16) return fail(TCP_ERR_ARG, "fourierrec: width must be in [2, 16]");
  if (width > L) return fail(TCP_ERR_ARG, "fourierrec: width must not exceed the grid size (2n rounded up)");
  return TCP_OK;
}

// Slice pairs per batch and workspace bytes of one FourierRec call on nz
// slices (the batch is capped at about 1.5 GiB of P + H + G).
size_t fourierrec_workspace_bytes(int64_t nt, int64_t nd, int64_t n, int64_t nz, int* nb_out) {
  const int lgM = std::max(1, ilog2(2 * nd)), lgL = ilog2(fourierrec_grid(n));
  const int64_t ms = (int64_t(1) << lgM) + 1, L = int64_t(1) << lgL;
  const int64_t npairs = std::max<int64_t>(1, (nz + 1) / 2);
  const int64_t p_pair = nt * ms, h_pair = n * L, g_pair = L * L;
  const size_t per_pair = sizeof(float2) * (size_t)(p_pair + h_pair + g_pair);
  const int nb = (int)std::max<int64_t>(1, std::min<int64_t>(npairs, (int64_t)(kBatchBytes / per_pair)));
  if (nb_out) *nb_out = nb;
  auto up = [](size_t b) { return (b + 255) / 256 * 256; };
  return up(sizeof(float4) * (size_t)std::max<int64_t>(nt, 1)) + up(sizeof(float2) * (size_t)ms) +
         up(sizeof(float2) * (size_t)p_pair * nb) + up(sizeof(float2) * (size_t)h_pair * nb) +
         up(sizeof(float2) * (size_t)g_pair * nb);
}

// Carve the workspace of fourierrec_workspace_bytes out of `base`.
FrecWorkspace fourierrec_workspace(void* base, int64_t nt, int64_t nd, int64_t n, int64_t nz) {
  FrecWorkspace w;
  const int lgM = std::max(1, ilog2(2 * nd)), lgL = ilog2(fourierrec_grid(n));
  const int64_t ms = (int64_t(1) << lgM) + 1, L = int64_t(1) << lgL;
  fourierrec_workspace_bytes(nt, nd, n, nz, &w.nb);
  auto up = [](size_t b) { return (b + 255) / 256 * 256; };
  char* p = (char*)base;
  w.geom = p;
  p += up(sizeof(float4) * (size_t)std::max<int64_t>(nt, 1));
  w.phase = p;
  p += up(sizeof(float2) * (size_t)ms);
  w.P = p;
  p += up(sizeof(float2) * (size_t)(nt * ms) * w.nb);
  w.H = p;
  p += up(sizeof(float2) * (size_t)(n * L) * w.nb);
  w.G = p;
  return w;
}

// Cached tables (built on first use of a size, width or angle set).
tcp_status fourierrec_tables_cached(const double* theta, int64_t nt, int64_t nd, int64_t n, int width,
                                    FrecTables* t) {
  const int lgM = std::max(1, ilog2(2 * nd)), lgL = ilog2(fourierrec_grid(n));
  int dev = 0;
  TCP_CUDA_TRY(cudaGetDevice(&dev));
  tcp_status s;
  if ((s = get_twiddles(dev, 1 << lgM, &t->twM)) != TCP_OK) return s;
  if ((s = get_twiddles(dev, 1 << lgL, &t->twL)) != TCP_OK) return s;
  if ((s = get_deconv(dev, (int)n, 1 << lgL, width, &t->dec)) != TCP_OK) return s;
  {
    std::lock_guard<std::mutex> lk(g_frec_mu);
    auto it = g_frec.order.find({dev, 1 << lgL});
    if (it == g_frec.order.end()) {
      const std::vector<int2> h = gather_tile_order(1 << lgL);
      int2* d = nullptr;
      TCP_CUDA_TRY(cudaMalloc(&d, h.size() * sizeof(int2)));
      const cudaError_t e = cudaMemcpy(d, h.data(), h.size() * sizeof(int2), cudaMemcpyHostToDevice);
      if (e != cudaSuccess) {
        cudaFree(d);
        return cuda_fail(e, "upload FourierRec tile order");
      }
      it = g_frec.order.emplace(std::make_pair(dev, 1 << lgL), d).first;
    }
    t->order = it->second;
  }
  if ((s = get_sorted_angles(dev, theta, (int)nt, &t->meta, &t->thS)) != TCP_OK) return s;
  NearTable nt_;
  if ((s = get_near_table(dev, theta, (int)nt, lgM, lgL, width, t->meta, t->thS, t->order, &nt_)) != TCP_OK) return s;
  t->t_near = nt_.t_near;
  t->near_off = nt_.off;
  t->near_ent = nt_.ent;
  t->n_heavy = nt_.n_heavy;
  t->near_heavy = nt_.heavy;
  t->near_warps = nt_.warps;
  return TCP_OK;
}

// Tables owned by the caller (a plan): cudaMalloc and synchronous upload, the
// allocations appended to `owned`.
tcp_status fourierrec_tables_owned(const double* theta, int64_t nt, int64_t nd, int64_t n, int width,
                                   std::vector<void*>* owned, FrecTables* t) {
  const int lgM = std::max(1, ilog2(2 * nd)), lgL = ilog2(fourierrec_grid(n));
  auto upload = [&](const void* h, size_t bytes, const void** out) -> tcp_status {
    void* d = nullptr;
    TCP_CUDA_TRY(cudaMalloc(&d, bytes ? bytes : 16));
    owned->push_back(d);
    if (bytes) TCP_CUDA_TRY(cudaMemcpy(d, h, bytes, cudaMemcpyHostToDevice));
    *out = d;
    return TCP_OK;
  };
  auto twiddles = [](int N) {
    std::vector<float2> h((size_t)N);
    for (int j = 0; j < N; ++j) {
      const double a = -2.0 * M_PI * (double)j / (double)N;
      h[(size_t)j] = make_float2((float)std::cos(a), (float)std::sin(a));
    }
    return h;
  };
  tcp_status s;
  const std::vector<float2> hM = twiddles(1 << lgM), hL = twiddles(1 << lgL);
  if ((s = upload(hM.data(), hM.size() * sizeof(float2), (const void**)&t->twM)) != TCP_OK) return s;
  if ((s = upload(hL.data(), hL.size() * sizeof(float2), (const void**)&t->twL)) != TCP_OK) return s;
  std::vector<float> hd((size_t)n);
  for (int64_t i = 0; i < n; ++i) hd[(size_t)i] = (float)(1.0 / es_fourier((double)(i - n / 2) / (double)(1 << lgL), width));
  if ((s = upload(hd.data(), hd.size() * sizeof(float), (const void**)&t->dec)) != TCP_OK) return s;
  std::vector<int2> hm;
  std::vector<float> ht;
  sort_angles(theta, (int)nt, &hm, &ht);
  if ((s = upload(hm.data(), hm.size() * sizeof(int2), (const void**)&t->meta)) != TCP_OK) return s;
  const std::vector<int2> ho = gather_tile_order(1 << lgL);
  if ((s = upload(ho.data(), ho.size() * sizeof(int2), (const void**)&t->order)) != TCP_OK) return s;
  if ((s = upload(ht.data(), ht.size() * sizeof(float), (const void**)&t->thS)) != TCP_OK) return s;
  NearTable nt_;
  if ((s = build_near_table(theta, (int)nt, lgM, lgL, width, hm, t->meta, t->thS, t->order, ho, &nt_)) != TCP_OK)
    return s;
  if (nt_.t_near > 0) {
    owned->push_back(nt_.off);
    owned->push_back(nt_.ent);
    owned->push_back(nt_.heavy);
    owned->push_back(nt_.warps);
  }
  t->t_near = nt_.t_near;
  t->near_off = nt_.off;
  t->near_ent = nt_.ent;
  t->n_heavy = nt_.n_heavy;
  t->near_heavy = nt_.heavy;
  t->near_warps = nt_.warps;
  return TCP_OK;
}

tcp_status launch_fourierrec_ws(const View3& sv, const FrecTables& tb, const FrecWorkspace& w, const TrigTable& trig,
                                double center, const View3& vv, float scale, int width, cudaStream_t st) {
  const int nz = (int)sv.d0, nt = (int)sv.d1, nd = (int)sv.d2, n = (int)vv.d1;
  tcp_status s;
  if ((s = fourierrec_check(nt, nd, n, width)) != TCP_OK) return s;
  const int lgM = std::max(1, ilog2(2 * (int64_t)nd)), lgL = ilog2(fourierrec_grid(n));
  const int M = 1 << lgM, L = 1 << lgL;
  const int ms = M + 1;
  const int npairs = (nz + 1) / 2;
  const int64_t p_pair = (int64_t)nt * ms, h_pair = (int64_t)n * L, g_pair = (int64_t)L * L;
  const int nb = std::max(1, std::min(npairs, w.nb));
  {
    const int cnt = std::max(nt, ms);
    k_frec_geom<<<(cnt + 255) / 256, 256, 0, st>>>(trig.dev, tb.meta, nt, (double)L / (double)M, (float4*)w.geom,
                                                     center, M, (float2*)w.phase);
    TCP_CUDA_TRY(cudaGetLastError());
  }
  for (int p0 = 0; p0 < npairs; p0 += nb) {
    const int b = std::min(nb, npairs - p0), z0 = 2 * p0;
    switch (sv.dtype) {
      case TCP_F32:
        launch_rows<float>(sv, z0, b, lgM, tb.twM, (const float2*)w.phase, (float2*)w.P, p_pair, ms, st);
        break;
      case TCP_F16:
        launch_rows<__half>(sv, z0, b, lgM, tb.twM, (const float2*)w.phase, (float2*)w.P, p_pair, ms, st);
        break;
      case TCP_BF16:
        launch_rows<__nv_bfloat16>(sv, z0, b, lgM, tb.twM, (const float2*)w.phase, (float2*)w.P, p_pair, ms, st);
        break;
      default: return fail(TCP_ERR_DTYPE, "fourierrec: sino must be F32, F16 or BF16");
    }
    TCP_CUDA_TRY(cudaGetLastError());
    launch_gather<4, 4>(width, (const float2*)w.P, p_pair, ms, (const float4*)w.geom, tb.meta, tb.thS, nt, M, lgL,
                        (float2*)w.G, g_pair, b, tb.order, tb, st);
    TCP_CUDA_TRY(cudaGetLastError());
    launch_cols((const float2*)w.G, g_pair, lgL, n, tb.twL, tb.dec, (float2*)w.H, h_pair, b, st);
    TCP_CUDA_TRY(cudaGetLastError());
    View3 ov = vv;
    switch (vv.dtype) {
      case TCP_F32: launch_out<float>((const float2*)w.H, h_pair, lgL, n, tb.twL, tb.dec, scale, ov, z0, b, st); break;
      case TCP_F16: launch_out<__half>((const float2*)w.H, h_pair, lgL, n, tb.twL, tb.dec, scale, ov, z0, b, st); break;
      case TCP_BF16:
        launch_out<__nv_bfloat16>((const float2*)w.H, h_pair, lgL, n, tb.twL, tb.dec, scale, ov, z0, b, st);
        break;
      default: return fail(TCP_ERR_DTYPE, "fourierrec: vol must be F32, F16 or BF16");
    }
    TCP_CUDA_TRY(cudaGetLastError());
  }
  return TCP_OK;
}

tcp_status launch_fourierrec(const View3& sv, const double* theta, const TrigTable& trig, double center,
                             const View3& vv, float scale, int width, cudaStream_t st) {
  const int64_t nz = sv.d0, nt = sv.d1, nd = sv.d2, n = vv.d1;
  tcp_status s;
  if ((s = fourierrec_check(nt, nd, n, width)) != TCP_OK) return s;
  FrecTables tb;
  if ((s = fourierrec_tables_cached(theta, nt, nd, n, width, &tb)) != TCP_OK) return s;
  const size_t bytes = fourierrec_workspace_bytes(nt, nd, n, nz, nullptr);
  void* base = nullptr;
  TCP_CUDA_TRY(cudaMallocAsync(&base, bytes, st));
  s = launch_fourierrec_ws(sv, tb, fourierrec_workspace(base, nt, nd, n, nz), trig, center, vv, scale, width, st);
  const cudaError_t e = cudaFreeAsync(base, st);
  if (s == TCP_OK && e != cudaSuccess) return cuda_fail(e, "cudaFreeAsync");
  return s;
}

}  // namespace tcp
