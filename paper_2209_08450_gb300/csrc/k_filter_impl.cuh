#pragma once
// Shared by k_filter.cu (tcp_filter) and k_filter_fused.cu
// (tcp_normalize_filter): the two launchers compile in separate units.
// One-dimensional FBP filter of every detector row (Sec. 2.2 of the TomocuPy
// paper: Shepp-Logan / Parzen filtering in Fourier space, rows padded before
// the FFT), optionally fused with the dark/flat normalisation and -log.
//
// GB300 design: the whole padded row lives in shared memory; no padded copy
// ever touches HBM.  Two real rows travel as one complex row z = a + i b:
// because the filter response is Hermitian (F[N-k] = conj(F[k])), filtering z
// filters a and b independently, so one complex FFT pair serves two rows
// without a separation step.  The FFT is a Stockham auto-sort transform
// between two shared-memory buffers, one barrier per pass: radix-16 register
// butterflies, then one pass of 8, 4 or 2 for the rest of the power of two,
// then radix 3 or 5 for padded lengths 3 * 2^k or 5 * 2^k.  The forward last pass, the
// response and the inverse first pass run in registers (the inverse takes the
// radices in reverse order), and the inverse last pass writes the output
// rows.  Twiddles (a two-level table in shared memory) and the response are
// FP64-derived; the arithmetic is FP32.  The response folds in the window, the
// pi/N_theta FBP weight (or a caller's storage weight), the 1/N of the inverse
// transform and the phase that moves the rotation axis to ndet/2.
//
// Fused mode reads uint16 projections and computes -ln((raw-dark)/(flat-dark))
// in FP32 while filling shared memory, so an FP16/BF16 sinogram is rounded
// once, after filtering.  Rounding the unfiltered sinogram to 16 bits would
// lose accuracy: the ramp removes its large low-frequency content and keeps
// the rounding noise (the large-minus-small hazard of Sec. 2.1).
#include <map>
#include <type_traits>
#include <mutex>
#include <tuple>

#include "tcp_internal.cuh"

namespace tcp {
namespace {

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(__fmaf_rn(a.x, b.x, -a.y * b.y), __fmaf_rn(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
// multiply by -i (forward transform) or +i (inverse)
template <bool INV> __device__ __forceinline__ float2 rot(float2 a) {
  return INV ? make_float2(-a.y, a.x) : make_float2(a.y, -a.x);
}

// ------------------------------------------------------------ small DFTs --
// In-register DFTs of 2, 4, 8 and 16 points, forward (W = e^{-2 pi i/R}) or
// inverse.  Radix 16 is 4 x 4 Cooley-Tukey: four 4-point DFTs over the
// stride-4 subsequences, twiddles W16^{kq}, four 4-point DFTs across them.

template <bool INV>
__device__ __forceinline__ void dft2(float2& a, float2& b) {
  const float2 t = a;
  a = cadd(t, b);
  b = csub(t, b);
}

template <bool INV>
__device__ __forceinline__ void dft4(float2& v0, float2& v1, float2& v2, float2& v3) {
  const float2 s02 = cadd(v0, v2), d02 = csub(v0, v2);
  const float2 s13 = cadd(v1, v3), d13 = rot<INV>(csub(v1, v3));
  v0 = cadd(s02, s13);
  v2 = csub(s02, s13);
  v1 = cadd(d02, d13);
  v3 = csub(d02, d13);
}

// multiply by W_R^e for a compile-time-known small angle (table of exact
// constants for R = 8 and 16).
template <bool INV>
__device__ __forceinline__ float2 tw_const(float2 a, int e, int R) {
  // e * (16 / R) indexes W16^m, m = 0..15
  const int m = (e * (16 / R)) & 15;
  constexpr float C1 = 0.92387953251128674f, S1 = 0.38268343236508978f, H = 0.70710678118654752f;
  const float cs[16] = {1.f, C1, H, S1, 0.f, -S1, -H, -C1, -1.f, -C1, -H, -S1, 0.f, S1, H, C1};
  const float sn[16] = {0.f, S1, H, C1, 1.f, C1, H, S1, 0.f, -S1, -H, -C1, -1.f, -C1, -H, -S1};
  // W16^m = cos(2 pi m/16) - i sin(2 pi m/16) (forward)
  const float c = cs[m], s = INV ? sn[m] : -sn[m];
  return make_float2(a.x * c - a.y * s, a.x * s + a.y * c);
}

// 3-point DFT: X_q = sum_r v_r W3^(r q), W3 = exp(-+2 pi i/3) = -1/2 -+ i sqrt(3)/2.
template <bool INV>
__device__ __forceinline__ void dft3(float2& v0, float2& v1, float2& v2) {
  constexpr float S3 = 0.86602540378443865f;  // sqrt(3)/2
  const float2 s = cadd(v1, v2), d = csub(v1, v2);
  const float2 m = make_float2(v0.x - 0.5f * s.x, v0.y - 0.5f * s.y);
  // (-+ i sqrt(3)/2) (v1 - v2)
  const float2 r = INV ? make_float2(-S3 * d.y, S3 * d.x) : make_float2(S3 * d.y, -S3 * d.x);
  v0 = cadd(v0, s);
  v1 = cadd(m, r);
  v2 = csub(m, r);
}

// 5-point DFT: with t1 = v1 + v4, t2 = v2 + v3, t3 = v1 - v4, t4 = v2 - v3,
// X0 = v0 + t1 + t2, X1,4 = v0 + c1 t1 + c2 t2 -+ i (s1 t3 + s2 t4),
// X2,3 = v0 + c2 t1 + c1 t2 -+ i (s2 t3 - s1 t4) (forward; the inverse flips
// the sign of i), c_m = cos(2 pi m / 5), s_m = sin(2 pi m / 5).
template <bool INV>
__device__ __forceinline__ void dft5(float2& v0, float2& v1, float2& v2, float2& v3, float2& v4) {
  constexpr float c1 = 0.309016994374947424f, c2 = -0.809016994374947424f;
  constexpr float s1 = 0.951056516295153572f, s2 = 0.587785252292473129f;
  const float2 t1 = cadd(v1, v4), t2 = cadd(v2, v3), t3 = csub(v1, v4), t4 = csub(v2, v3);
  const float2 b1 = make_float2(v0.x + c1 * t1.x + c2 * t2.x, v0.y + c1 * t1.y + c2 * t2.y);
  const float2 b2 = make_float2(v0.x + c2 * t1.x + c1 * t2.x, v0.y + c2 * t1.y + c1 * t2.y);
  const float2 d1 = rot<INV>(make_float2(s1 * t3.x + s2 * t4.x, s1 * t3.y + s2 * t4.y));  // -+ i (s1 t3 + s2 t4)
  const float2 d2 = rot<INV>(make_float2(s2 * t3.x - s1 * t4.x, s2 * t3.y - s1 * t4.y));
  v0 = cadd(v0, cadd(t1, t2));
  v1 = cadd(b1, d1);
  v4 = csub(b1, d1);
  v2 = cadd(b2, d2);
  v3 = csub(b2, d2);
}

template <int R, bool INV>
__device__ __forceinline__ void dft(float2 (&v)[R]) {
  if constexpr (R == 5) {
    dft5<INV>(v[0], v[1], v[2], v[3], v[4]);
  } else if constexpr (R == 3) {
    dft3<INV>(v[0], v[1], v[2]);
  } else if constexpr (R == 2) {
    dft2<INV>(v[0], v[1]);
  } else if constexpr (R == 4) {
    dft4<INV>(v[0], v[1], v[2], v[3]);
  } else if constexpr (R == 8) {
    // 2 x 4: two 4-point DFTs on even/odd, twiddle W8^q, 2-point across
#pragma unroll
    for (int k = 0; k < 2; ++k) dft4<INV>(v[k], v[k + 2], v[k + 4], v[k + 6]);
    // now v[k + 2q] holds Y_k[q]
    float2 o[8];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      float2 a = v[2 * q], b = tw_const<INV>(v[1 + 2 * q], q, 8);
      dft2<INV>(a, b);
      o[q] = a;
      o[q + 4] = b;
    }
#pragma unroll
    for (int i = 0; i < 8; ++i) v[i] = o[i];
  } else {
    static_assert(R == 16, "radix");
#pragma unroll
    for (int k = 0; k < 4; ++k) dft4<INV>(v[k], v[k + 4], v[k + 8], v[k + 12]);
    // v[k + 4q] = Y_k[q]; twiddle by W16^{kq}
#pragma unroll
    for (int k = 1; k < 4; ++k)
#pragma unroll
      for (int q = 1; q < 4; ++q) v[k + 4 * q] = tw_const<INV>(v[k + 4 * q], k * q, 16);
    float2 o[16];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      float2 a = v[4 * q], b = v[4 * q + 1], c = v[4 * q + 2], d = v[4 * q + 3];
      dft4<INV>(a, b, c, d);
      o[q] = a;
      o[q + 4] = b;
      o[q + 8] = c;
      o[q + 12] = d;
    }
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = o[i];
  }
}

// Shared-memory index of element i: one pad slot per 16 elements, so that the
// stride-16 stores of the first radix-16 pass fall in distinct banks.
__device__ __forceinline__ int pi16(int i) { return i + (i >> 4); }

// W^m (forward sign) from the two-level table in shared memory: entry m % 64
// times entry 64 + m / 64, both rounded from FP64 (about 1.5 ulp).
__device__ __forceinline__ float2 tw2(const float2* tw, int m) { return cmul(tw[m & 63], tw[64 + (m >> 6)]); }

// Stockham pass of radix R: in -> out, sub-transform size Ns, by the gs
// threads of one group (group-local index gt).  The R - 1 twiddles W^(r k
// step) of a butterfly: for R = 16 the powers r = 1, 2, 4, 8 come from the
// table and the others are products of at most three of them; for smaller R
// every power comes from the table.
template <int R, bool INV, bool P2 = true>
__device__ __forceinline__ void stockham_pass(const float2* in, float2* out, int N, int Ns, const float2* tw,
                                              int gt, int gs) {
  const int nb = N / R;
  const int step = N / (R * Ns);
  for (int b = gt; b < nb; b += gs) {
    float2 v[R];
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = in[pi16(b + r * nb)];
    const int k = P2 ? (b & (Ns - 1)) : b % Ns;  // P2: Ns is a power of two (else 3 * 2^i or 5 * 2^i)
    if (Ns > 1) {
      float2 w[R];
      const int m1 = k * step;
      if constexpr (R == 16) {
        w[1] = tw2(tw, m1);
        w[2] = tw2(tw, 2 * m1);
        w[4] = tw2(tw, 4 * m1);
        w[8] = tw2(tw, 8 * m1);
        w[3] = cmul(w[1], w[2]);
        w[5] = cmul(w[1], w[4]);
        w[6] = cmul(w[2], w[4]);
        w[7] = cmul(w[3], w[4]);
#pragma unroll
        for (int r = 9; r < 16; ++r) w[r] = cmul(w[r - 8], w[8]);
      } else {
#pragma unroll
        for (int r = 1; r < R; ++r) w[r] = tw2(tw, r * m1);
      }
#pragma unroll
      for (int r = 1; r < R; ++r) {
        if (INV) w[r].y = -w[r].y;
        v[r] = cmul(v[r], w[r]);
      }
    }
    dft<R, INV>(v);
    const int o = (b - k) * R + k;
#pragma unroll
    for (int r = 0; r < R; ++r) out[pi16(o + r * Ns)] = v[r];
  }
}

// Store one filtered sample.  With `plane` != 0 (TCP_F16X2, TOut = __half) the
// value is split: hi = fp16(v) at p[j], lo = fp16(v - hi) at p[j + plane].
template <class TOut>
__device__ __forceinline__ void put_sample(TOut* p, int j, float v, int64_t plane) {
  if constexpr (std::is_same<TOut, __half>::value) {
    if (plane) {
      const __half hi = __float2half_rn(v);
      p[j] = hi;
      p[j + plane] = __float2half_rn(v - __half2float(hi));
      return;
    }
  }
  Store<TOut>::put(p + j, v);
}

// Response factor for frequency index k (Hermitian: F[N - k] = conj F[k]).
__device__ __forceinline__ float2 response_at(const float2* resp, int k, int N) {
  const int half = N >> 1;
  float2 F = __ldg(resp + (k <= half ? k : N - k));
  if (k > half) F.y = -F.y;
  return F;
}

// The forward transform's last pass (radix R, Ns = N / R), the response and
// the inverse transform's first pass (radix R, Ns = 1) in registers: the
// forward butterfly b produces X[b + r N/R], which are exactly the inputs of
// inverse butterfly b, so the spectrum never returns to shared memory.
template <int R>
__device__ __forceinline__ void fused_turn(const float2* in, float2* out, int N, const float2* tw, const float2* resp,
                                           int gt, int gs) {
  const int nb = N / R;
  for (int b = gt; b < nb; b += gs) {
    float2 v[R];
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = in[pi16(b + r * nb)];
    if (nb > 1) {  // forward twiddles W^(r b), step 1
#pragma unroll
      for (int r = 1; r < R; ++r) v[r] = cmul(v[r], tw2(tw, r * b));
    }
    dft<R, false>(v);
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = cmul(v[r], response_at(resp, b + r * nb, N));
    dft<R, true>(v);
#pragma unroll
    for (int r = 0; r < R; ++r) out[pi16(b * R + r)] = v[r];
  }
}

// The inverse transform's last pass (radix 16, Ns = N / 16) with the result
// stored straight to the two output rows: butterfly b yields y[b + r N/16].
template <class TOut>
__device__ __forceinline__ void last_to_rows(const float2* in, int N, const float2* tw, int gt, int gs, int left,
                                             int nd, TOut* o0, TOut* o1, bool has1, int64_t plane) {
  constexpr int R = 16;
  const int nb = N / R;
  for (int b = gt; b < nb; b += gs) {
    float2 v[R];
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = in[pi16(b + r * nb)];
    float2 w[R];
    w[1] = tw2(tw, b);
    w[2] = tw2(tw, 2 * b);
    w[4] = tw2(tw, 4 * b);
    w[8] = tw2(tw, 8 * b);
    w[3] = cmul(w[1], w[2]);
    w[5] = cmul(w[1], w[4]);
    w[6] = cmul(w[2], w[4]);
    w[7] = cmul(w[3], w[4]);
#pragma unroll
    for (int r = 9; r < 16; ++r) w[r] = cmul(w[r - 8], w[8]);
#pragma unroll
    for (int r = 1; r < R; ++r) {
      w[r].y = -w[r].y;
      v[r] = cmul(v[r], w[r]);
    }
    dft<R, true>(v);
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int j = b + r * nb - left;
      if (j >= 0 && j < nd) {
        put_sample<TOut>(o0, j, v[r].x, plane);
        if (has1) put_sample<TOut>(o1, j, v[r].y, plane);
      }
    }
  }
}

// Transforms of N <= 16: one butterfly holds the whole row.
template <int R, class TOut>
__device__ __forceinline__ void single_pass(const float2* in, const float2* resp, int gt, int left, int nd, TOut* o0,
                                            TOut* o1, bool has1, int64_t plane) {
  if (gt != 0) return;
  float2 v[R];
#pragma unroll
  for (int r = 0; r < R; ++r) v[r] = in[pi16(r)];
  dft<R, false>(v);
#pragma unroll
  for (int r = 0; r < R; ++r) v[r] = cmul(v[r], response_at(resp, r, R));
  dft<R, true>(v);
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const int j = r - left;
    if (j >= 0 && j < nd) {
      put_sample<TOut>(o0, j, v[r].x, plane);
      if (has1) put_sample<TOut>(o1, j, v[r].y, plane);
    }
  }
}

// One Stockham pass of runtime radix r (2, 3, 4, 8 or 16).
template <bool INV>
__device__ __forceinline__ void pass_r(int r, const float2* in, float2* out, int N, int Ns, const float2* tw, int gt,
                                       int gs) {
  if ((Ns & (Ns - 1)) == 0) {
    switch (r) {
      case 16: stockham_pass<16, INV>(in, out, N, Ns, tw, gt, gs); break;
      case 8: stockham_pass<8, INV>(in, out, N, Ns, tw, gt, gs); break;
      case 4: stockham_pass<4, INV>(in, out, N, Ns, tw, gt, gs); break;
      case 3: stockham_pass<3, INV>(in, out, N, Ns, tw, gt, gs); break;
      case 5: stockham_pass<5, INV>(in, out, N, Ns, tw, gt, gs); break;
      default: stockham_pass<2, INV>(in, out, N, Ns, tw, gt, gs); break;
    }
  } else {  // after the inverse radix-3 or radix-5 pass: Ns = 3 * 2^i or 5 * 2^i
    switch (r) {
      case 16: stockham_pass<16, INV, false>(in, out, N, Ns, tw, gt, gs); break;
      case 8: stockham_pass<8, INV, false>(in, out, N, Ns, tw, gt, gs); break;
      case 4: stockham_pass<4, INV, false>(in, out, N, Ns, tw, gt, gs); break;
      default: stockham_pass<2, INV, false>(in, out, N, Ns, tw, gt, gs); break;
    }
  }
}

// Filter the row pair held in `a` (padded to N = prod rad[i]): forward
// transform with the radices rad[0..nrad) (16, ..., 16, then 2/4/8, then 3),
// the inverse with the same radices reversed so that its first pass meets the
// forward last pass in registers, and its last pass (radix 16) writes the rows.
// nrad == 1: N <= 16, one butterfly.  Every thread of the block takes part in
// the barriers; groups without a row pair (active == false) skip the
// arithmetic.  On return the shared buffers may be reused after a barrier.
template <class TOut>
__device__ void filter_pair(float2* a, float2* b, int N, const int* rad, int nrad, const float2* tw, const float2* resp,
                            int gt, int gs, bool active, int left, int nd, TOut* o0, TOut* o1, bool has1,
                            int64_t plane) {
  if (nrad == 1) {
    if (active) {
      if (N == 16) single_pass<16>(a, resp, gt, left, nd, o0, o1, has1, plane);
      else if (N == 8) single_pass<8>(a, resp, gt, left, nd, o0, o1, has1, plane);
      else if (N == 4) single_pass<4>(a, resp, gt, left, nd, o0, o1, has1, plane);
      else single_pass<2>(a, resp, gt, left, nd, o0, o1, has1, plane);
    }
    return;
  }
  int r8[8];  // the radices in registers (compile-time indices below)
#pragma unroll
  for (int i = 0; i < 8; ++i) r8[i] = i < nrad ? rad[i] : 1;
  int Ns = 1;
#pragma unroll
  for (int i = 0; i < 7; ++i) {
    if (i + 1 < nrad) {
      if (active) pass_r<false>(r8[i], a, b, N, Ns, tw, gt, gs);
      __syncthreads();
      float2* t = a;
      a = b;
      b = t;
      Ns *= r8[i];
    }
  }
  int rl = 1;
#pragma unroll
  for (int i = 0; i < 8; ++i)
    if (i == nrad - 1) rl = r8[i];
  if (active) {
    if (rl == 16) fused_turn<16>(a, b, N, tw, resp, gt, gs);
    else if (rl == 8) fused_turn<8>(a, b, N, tw, resp, gt, gs);
    else if (rl == 4) fused_turn<4>(a, b, N, tw, resp, gt, gs);
    else if (rl == 3) fused_turn<3>(a, b, N, tw, resp, gt, gs);
    else if (rl == 5) fused_turn<5>(a, b, N, tw, resp, gt, gs);
    else fused_turn<2>(a, b, N, tw, resp, gt, gs);
  }
  __syncthreads();
  {
    float2* t = a;
    a = b;
    b = t;
  }
  Ns = rl;
#pragma unroll
  for (int i = 6; i >= 1; --i) {
    if (i <= nrad - 2) {
      if (active) pass_r<true>(r8[i], a, b, N, Ns, tw, gt, gs);
      __syncthreads();
      float2* t = a;
      a = b;
      b = t;
      Ns *= r8[i];
    }
  }
  if (active) last_to_rows<TOut>(a, N, tw, gt, gs, left, nd, o0, o1, has1, plane);
}

// filter_pair for a power-of-two padded length N >= 256 known at compile
// time (radices 16, ..., 16 and a last 2, 4 or 8), with GS threads per row
// pair: the same passes in the same order as filter_pair (bit-identical
// results), but with N, every sub-transform size and the trip counts as
// constants, so that the shared-memory index arithmetic folds into address
// offsets.  The common padded lengths take this path.
template <int N>
__host__ __device__ constexpr int ct_log2() {
  int l = 0;
  while ((1 << l) < N) ++l;
  return l;
}
template <int N>
__host__ __device__ constexpr int ct_group() {  // threads per row pair, as the launch computes it
  return N / 16 < 32 ? 32 : (N / 16 > 256 ? 256 : N / 16);
}
template <int N, class TOut>
__device__ void filter_pair_ct(float2* a, float2* b, const float2* tw, const float2* resp, int gt, bool active,
                               int left, int nd, TOut* o0, TOut* o1, bool has1, int64_t plane) {
  constexpr int L2 = ct_log2<N>();
  static_assert((1 << L2) == N && L2 >= 8, "power-of-two padded length >= 256");
  constexpr int P16 = L2 / 4, Q = 1 << (L2 % 4);
  constexpr int NRAD = P16 + (Q > 1 ? 1 : 0);
  constexpr int RL = Q > 1 ? Q : 16;  // the last forward radix (met by the inverse first pass)
  constexpr int GS = ct_group<N>();
  int Ns = 1;
#pragma unroll
  for (int i = 0; i < NRAD - 1; ++i) {
    if (active) stockham_pass<16, false>(a, b, N, Ns, tw, gt, GS);
    __syncthreads();
    float2* t = a;
    a = b;
    b = t;
    Ns *= 16;
  }
  if (active) fused_turn<RL>(a, b, N, tw, resp, gt, GS);
  __syncthreads();
  {
    float2* t = a;
    a = b;
    b = t;
  }
  Ns = RL;
#pragma unroll
  for (int i = NRAD - 2; i >= 1; --i) {
    if (active) stockham_pass<16, true>(a, b, N, Ns, tw, gt, GS);
    __syncthreads();
    float2* t = a;
    a = b;
    b = t;
    Ns *= 16;
  }
  if (active) last_to_rows<TOut>(a, N, tw, gt, GS, left, nd, o0, o1, has1, plane);
}

struct FiltArgs {
  // source rows: filtered sinogram [d0][d1][nd] (in place) or raw projections
  const void* src;
  int64_t s0, s1;   // source strides (sino: z, theta; raw: theta, z)
  const float* dark;
  const float* flat;
  int64_t dm, fm;   // z strides of the means
  void* dst;        // sinogram [d0][d1][nd]
  int64_t t0, t1;   // destination strides (z, theta)
  int d1;           // rows per z (= ntheta)
  int64_t rows;
  int nd, npad, log2n, left;
  int gs;           // threads per row pair
  int pad_zero;
  int vec4;         // raw rows and means allow 4-sample vector loads
  int nrad;         // FFT radices, forward order (see filter_pair)
  int rad[8];
  int64_t plane;    // TCP_F16X2 output: elements from the hi to the lo plane (else 0)
  const float2* resp;
  const float2* tw;  // two-level twiddle table (global; copied to shared memory)
};

template <bool RAW, class TIn>
__device__ __forceinline__ float load_sample(const FiltArgs& a, int64_t z, int64_t t, int j) {
  if constexpr (RAW) {
    const uint16_t v = __ldg(reinterpret_cast<const uint16_t*>(a.src) + t * a.s0 + z * a.s1 + j);
    return neglog_ratio((float)v, __ldg(a.dark + z * a.dm + j), __ldg(a.flat + z * a.fm + j));
  } else {
    return Store<TIn>::load(reinterpret_cast<const TIn*>(a.src) + z * a.s0 + t * a.s1 + j);
  }
}

// A block of 256 threads works on G = 256/gs row pairs at once, gs threads
// per pair (gs = npad/16 clamped to [32, 256]): small transforms still fill the
// block and share its barriers.
template <bool RAW, class TIn, class TOut>
__global__ void __launch_bounds__(256, 3) k_filter(FiltArgs a) {
  extern __shared__ float2 smem[];
  const int gs = a.gs;
  const int G = blockDim.x / gs;
  const int g = threadIdx.x / gs, gt = threadIdx.x - g * gs;
  const int plen = a.npad + a.npad / 16;  // padded buffer length
  // [two-level twiddle table][G x (bufA, bufB)]
  const int ntw = 64 + (a.npad + 63) / 64;
  float2* tw = smem;
  for (int i = threadIdx.x; i < ntw; i += blockDim.x) tw[i] = __ldg(a.tw + i);
  float2* bufA = smem + ntw + (size_t)g * 2 * plen;
  float2* bufB = bufA + plen;
  const int64_t npairs = (a.rows + 1) / 2;
  for (int64_t p0 = (int64_t)blockIdx.x * G; p0 < npairs; p0 += (int64_t)gridDim.x * G) {
    const int64_t p = p0 + g;
    const bool active = p < npairs;
    const int64_t r0 = 2 * p, r1 = 2 * p + 1;
    const bool has1 = active && r1 < a.rows;
    const int64_t z0 = r0 / a.d1, t0 = r0 - z0 * a.d1;
    const int64_t z1 = has1 ? r1 / a.d1 : z0, t1 = has1 ? r1 - z1 * a.d1 : t0;
    if (active) {
      if constexpr (RAW) {
        // uint16 projections: 4 samples per load where the rows allow it;
        // the two rows of a pair share one slice (and its dark/flat means)
        // unless the pair straddles two slices
        const uint16_t* ra = reinterpret_cast<const uint16_t*>(a.src) + t0 * a.s0 + z0 * a.s1;
        const uint16_t* rb = reinterpret_cast<const uint16_t*>(a.src) + t1 * a.s0 + z1 * a.s1;
        const float* d0 = a.dark + z0 * a.dm;
        const float* f0 = a.flat + z0 * a.fm;
        const float* d1 = a.dark + z1 * a.dm;
        const float* f1 = a.flat + z1 * a.fm;
        const bool vec = a.vec4;
        const int nd4 = vec ? a.nd / 4 : 0;
#pragma unroll 2
        for (int q = gt; q < nd4; q += gs) {
          const uint2 ua = __ldg(reinterpret_cast<const uint2*>(ra) + q);
          const uint2 ub = has1 ? __ldg(reinterpret_cast<const uint2*>(rb) + q) : make_uint2(0, 0);
          const float4 da = __ldg(reinterpret_cast<const float4*>(d0) + q);
          const float4 fa = __ldg(reinterpret_cast<const float4*>(f0) + q);
          float4 db = da, fb = fa;
          if (has1 && z1 != z0) {
            db = __ldg(reinterpret_cast<const float4*>(d1) + q);
            fb = __ldg(reinterpret_cast<const float4*>(f1) + q);
          }
          const float va[4] = {(float)(ua.x & 0xffff), (float)(ua.x >> 16), (float)(ua.y & 0xffff), (float)(ua.y >> 16)};
          const float vb[4] = {(float)(ub.x & 0xffff), (float)(ub.x >> 16), (float)(ub.y & 0xffff), (float)(ub.y >> 16)};
          const float dA[4] = {da.x, da.y, da.z, da.w}, fA[4] = {fa.x, fa.y, fa.z, fa.w};
          const float dB[4] = {db.x, db.y, db.z, db.w}, fB[4] = {fb.x, fb.y, fb.z, fb.w};
#pragma unroll
          for (int e = 0; e < 4; ++e)
            bufA[pi16(a.left + 4 * q + e)] =
                make_float2(neglog_ratio(va[e], dA[e], fA[e]), has1 ? neglog_ratio(vb[e], dB[e], fB[e]) : 0.f);
        }
        for (int j = 4 * nd4 + gt; j < a.nd; j += gs) {
          const float re = neglog_ratio((float)__ldg(ra + j), __ldg(d0 + j), __ldg(f0 + j));
          const float im = has1 ? neglog_ratio((float)__ldg(rb + j), __ldg(d1 + j), __ldg(f1 + j)) : 0.f;
          bufA[pi16(a.left + j)] = make_float2(re, im);
        }
      } else {
        // real samples (unrolled so that several loads are in flight)
#pragma unroll 4
        for (int j = gt; j < a.nd; j += gs) {
          const float re = load_sample<RAW, TIn>(a, z0, t0, j);
          const float im = has1 ? load_sample<RAW, TIn>(a, z1, t1, j) : 0.f;
          bufA[pi16(a.left + j)] = make_float2(re, im);
        }
      }
      // padding: zeros or the edge samples (each thread evaluates the edges once)
      float2 lo = make_float2(0.f, 0.f), hi = lo;
      const int npadded = a.npad - a.nd;
      if (!a.pad_zero && gt < npadded) {
        lo = make_float2(load_sample<RAW, TIn>(a, z0, t0, 0), has1 ? load_sample<RAW, TIn>(a, z1, t1, 0) : 0.f);
        hi = make_float2(load_sample<RAW, TIn>(a, z0, t0, a.nd - 1),
                         has1 ? load_sample<RAW, TIn>(a, z1, t1, a.nd - 1) : 0.f);
      }
      for (int m = gt; m < npadded; m += gs) {
        if (m < a.left) bufA[pi16(m)] = lo;
        else bufA[pi16(a.nd + m)] = hi;
      }
    }
    __syncthreads();
    TOut* o0 = reinterpret_cast<TOut*>(a.dst) + z0 * a.t0 + t0 * a.t1;
    TOut* o1 = reinterpret_cast<TOut*>(a.dst) + z1 * a.t0 + t1 * a.t1;
    switch (a.npad) {
      case 1024: filter_pair_ct<1024, TOut>(bufA, bufB, tw, a.resp, gt, active, a.left, a.nd, o0, o1, has1, a.plane); break;
      case 2048: filter_pair_ct<2048, TOut>(bufA, bufB, tw, a.resp, gt, active, a.left, a.nd, o0, o1, has1, a.plane); break;
      case 4096: filter_pair_ct<4096, TOut>(bufA, bufB, tw, a.resp, gt, active, a.left, a.nd, o0, o1, has1, a.plane); break;
      case 8192: filter_pair_ct<8192, TOut>(bufA, bufB, tw, a.resp, gt, active, a.left, a.nd, o0, o1, has1, a.plane); break;
      default:
        filter_pair<TOut>(bufA, bufB, a.npad, a.rad, a.nrad, tw, a.resp, gt, gs, active, a.left, a.nd, o0, o1, has1,
                          a.plane);
    }
    __syncthreads();
  }
}

template <bool RAW, class TIn>
void (*pick_out(int dt))(FiltArgs) {
  switch (dt) {
    case TCP_F32: return k_filter<RAW, TIn, float>;
    case TCP_F16: return k_filter<RAW, TIn, __half>;
    case TCP_BF16: return k_filter<RAW, TIn, __nv_bfloat16>;
    case TCP_F16X2: return k_filter<RAW, TIn, __half>;
  }
  return nullptr;
}

tcp_status run(void (*k)(FiltArgs), FiltArgs& a, const FilterTable& ft, int pad_mode, cudaStream_t st) {
  a.npad = ft.npad;
  a.log2n = 0;
  // radices: N = 16^p 2^q (times 3 or 5), forward order 16, .., 16, 2^q, 3 or 5
  {
    const bool three = a.npad % 3 == 0, five = a.npad % 5 == 0;
    const int odd = three ? 3 : (five ? 5 : 1);
    int m = a.npad / odd, l2 = 0;
    while ((1 << l2) < m) ++l2;
    a.log2n = l2;
    a.nrad = 0;
    if (odd == 1 && l2 <= 4) {
      a.rad[a.nrad++] = a.npad;  // one butterfly
    } else {
      const int q = l2 % 4;
      for (int i = 0; i < l2 / 4; ++i) a.rad[a.nrad++] = 16;
      if (q) a.rad[a.nrad++] = 1 << q;
      if (odd > 1) a.rad[a.nrad++] = odd;
    }
    if (a.nrad > 8 || (a.nrad > 1 && a.rad[0] != 16))
      return fail(TCP_ERR_UNSUPPORTED, "filter: padded length " + std::to_string(a.npad) + " not supported");
  }
  a.left = (a.npad - a.nd) / 2;
  a.pad_zero = (pad_mode & TCP_PAD_ZERO) != 0;
  a.resp = ft.response;
  a.tw = ft.twiddle;
  if (a.rows == 0 || a.nd == 0) return TCP_OK;
  if (!k) return fail(TCP_ERR_DTYPE, "filter: sinogram dtype must be F32, F16 or BF16");
  // threads per row pair: a power of two (so that groups tile the block),
  // about one radix-16 butterfly each
  a.gs = 32;
  while (a.gs < 256 && 2 * a.gs <= a.npad / 16) a.gs *= 2;
  const int threads = 256;
  const size_t smem = ((size_t)(threads / a.gs) * 2 * (size_t)(a.npad + a.npad / 16) + 64 + (a.npad + 63) / 64) *
                      sizeof(float2);
  const int64_t npairs = (a.rows + 1) / 2;
  int dev = 0;
  TCP_CUDA_TRY(cudaGetDevice(&dev));
  // Kernel attributes and occupancy are looked up once per (device, kernel,
  // padded length), so that later launches, including ones under CUDA-graph
  // capture, only enqueue work.
  static std::mutex mu;
  static std::map<std::tuple<int, void*, int>, int> grid_cache;
  int cap = 0;
  {
    std::lock_guard<std::mutex> lk(mu);
    auto key = std::make_tuple(dev, reinterpret_cast<void*>(k), a.npad);
    auto it = grid_cache.find(key);
    if (it == grid_cache.end()) {
      TCP_CUDA_TRY(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)((2 * (8192 + 512) + 64 + 128) * sizeof(float2))));
      int per_sm = 1, sms = 0;
      TCP_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, threads, smem));
      TCP_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
      it = grid_cache.emplace(key, std::max(1, per_sm) * sms * 8).first;
    }
    cap = it->second;
  }
  const int G = threads / a.gs;
  const int blocks = (int)std::min<int64_t>((npairs + G - 1) / G, cap);
  k<<<blocks, threads, smem, st>>>(a);
  TCP_CUDA_TRY(cudaGetLastError());
  return TCP_OK;
}

}  // namespace
}  // namespace tcp
