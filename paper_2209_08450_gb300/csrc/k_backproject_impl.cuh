#pragma once
// Kernels and configuration dispatch of the CUDA-core LineRec backprojector,
// shared by k_backproject.cu (launchers) and the per-sinogram-dtype units
// k_backproject_f32.cu, k_backproject_f16.cu and k_backproject_bf16.cu, which
// instantiate the kernels in parallel.
// LineRec backprojection (Sec. 2.2, Sec. 3 of the TomocuPy paper): direct
// discretisation of the backprojection line integral with linear
// interpolation,
//   vol[z][iy][ix] = sum_theta q_{z,theta}(s),  s = x cos + y sin + center.
//
// GB300 design.  The work is a gather with two non-zeros per (voxel, angle),
// not a dense contraction, so it runs on the FP32 pipes and is bound by the
// shared-memory pipe (one 128-byte wavefront per warp-wide sample fetch).
//   * A thread block owns one aligned 32x32 voxel tile and K slices.
//   * Angles are processed in stages of T.  For each staged angle the block
//     copies, for each of its K slices, the window of WIN = 48 detector
//     samples that the tile's rays can touch into shared memory (zero outside
//     the detector).  32 * sqrt(2) < 46, so 48 samples always cover the tile.
//   * Each thread owns R voxels (one column lane, R rows) times K slices of
//     FP32 accumulators in registers.  The ray coordinate, floor and weights
//     are computed once per (voxel, angle) and reused for all K slices.
//   * FP32 sinograms: two 4-byte shared loads per interpolation.
//     FP16/BF16 sinograms: the window is stored as pairs (q[i], q[i+1]) so one
//     4-byte load fetches both neighbours, and PTX mixed-precision
//     fma.rn.f32.f16 / .bf16 accumulates the 16-bit samples in FP32 with
//     16-bit weights (Sec. 2.1: 16-bit storage, wider accumulation).
//   * Lanes of a warp are adjacent voxels in x, so their window indices are
//     consecutive or equal: every shared load is one conflict-free wavefront.
#include <mutex>
#include <set>

#include "tcp_internal.cuh"

namespace tcp {

using Kern = void (*)(BpArgs);
using PKern = void (*)(BpWork);

struct KernPair {
  Kern direct;
  PKern persistent;
  size_t smem;  // dynamic shared memory per block
};

// The configurations instantiated for FP32 (one unit per volume dtype), FP16
// and BF16 sinograms; {nullptr, ...} for a configuration that is not.
KernPair bp_pick_f32_f32(const tcp_bp_config& c, bool check);  // FP32 sinograms, by volume dtype
KernPair bp_pick_f32_f16(const tcp_bp_config& c, bool check);
KernPair bp_pick_f32_bf16(const tcp_bp_config& c, bool check);
KernPair bp_pick_f16(int vdt, const tcp_bp_config& c, bool check);
KernPair bp_pick_bf16(int vdt, const tcp_bp_config& c, bool check);

namespace {

constexpr int kWin = 48;

struct Geo {
  int base;  // i0 - window start
  float f0, c, s;
};

// Shared-memory element of the staged window.
template <class TS> struct Win;
template <> struct Win<__half> { using type = uint32_t; };         // (q[i], q[i+1]) as f16x2
template <> struct Win<__nv_bfloat16> { using type = uint32_t; };  // (q[i], q[i+1]) as bf16x2

template <class TS> struct Interp;

__device__ __forceinline__ uint16_t ld_u16(const void* row, int j, int ndet) {
  return (j >= 0 && j < ndet) ? __ldg(reinterpret_cast<const unsigned short*>(row) + j) : (uint16_t)0;
}

template <> struct Interp<__half> {
  static __device__ __forceinline__ uint32_t stage(const __half* row, int j, int ndet) {
    return (uint32_t)ld_u16(row, j, ndet) | ((uint32_t)ld_u16(row, j + 1, ndet) << 16);
  }
  struct W { uint16_t w0, w1; };
  static __device__ __forceinline__ W weights(float w) {
    return {__half_as_ushort(__float2half_rn(1.f - w)), __half_as_ushort(__float2half_rn(w))};
  }
  static __device__ __forceinline__ void acc(float& a, const uint32_t* p, int off, const W& w) {
    const uint32_t v = p[off];
    const uint16_t lo = (uint16_t)(v & 0xffffu), hi = (uint16_t)(v >> 16);
    asm("fma.rn.f32.f16 %0, %1, %2, %0;" : "+f"(a) : "h"(w.w0), "h"(lo));
    asm("fma.rn.f32.f16 %0, %1, %2, %0;" : "+f"(a) : "h"(w.w1), "h"(hi));
  }
};

template <> struct Interp<__nv_bfloat16> {
  static __device__ __forceinline__ uint32_t stage(const __nv_bfloat16* row, int j, int ndet) {
    return (uint32_t)ld_u16(row, j, ndet) | ((uint32_t)ld_u16(row, j + 1, ndet) << 16);
  }
  struct W { uint16_t w0, w1; };
  static __device__ __forceinline__ W weights(float w) {
    return {__bfloat16_as_ushort(__float2bfloat16_rn(1.f - w)),
            __bfloat16_as_ushort(__float2bfloat16_rn(w))};
  }
  static __device__ __forceinline__ void acc(float& a, const uint32_t* p, int off, const W& w) {
    const uint32_t v = p[off];
    const uint16_t lo = (uint16_t)(v & 0xffffu), hi = (uint16_t)(v >> 16);
    asm("fma.rn.f32.bf16 %0, %1, %2, %0;" : "+f"(a) : "h"(w.w0), "h"(lo));
    asm("fma.rn.f32.bf16 %0, %1, %2, %0;" : "+f"(a) : "h"(w.w1), "h"(hi));
  }
};

// ------------------------------------------------------- shared layouts --
//
// FP32 sinograms: two stage buffers win[2][T][K][WIN] (floats), filled with
//   4-byte cp.async (zero-filled outside the detector) one stage ahead of the
//   compute, so the global-load latency overlaps the interpolation loop.
// 16-bit sinograms, K >= 2: win[T][WIN][K] with the K slices of one detector
//   sample adjacent (K * 2 bytes), so that one vector load fetches sample i of
//   every slice and a second one sample i + 1; two slices are accumulated per
//   packed fma.rn.f32x2.
// 16-bit sinograms, K == 1: win[T][K][WIN] of (q[i], q[i+1]) pairs.

template <class TS, int K, int T>
struct BpLayout {
  static constexpr bool kF32 = std::is_same<TS, float>::value;
  static constexpr bool kInter = !kF32 && K >= 2;
  static constexpr int kStages = kF32 ? 2 : 1;
  // Geometry ring: FP32 writes the geometry of stage s+1 before the barrier
  // that ends stage s-1, so it needs three slots (s-1, s, s+1).
  static constexpr int kGeoSlots = kF32 ? 3 : 1;
  static constexpr int kWinWords = kInter ? T * kWin * K / 2 : T * K * kWin;  // 4-byte words per stage
  static constexpr size_t kGeoBytes = sizeof(Geo) * T * kGeoSlots;
  static constexpr size_t kWstBytes = sizeof(int) * T * kGeoSlots;
  static constexpr size_t kBytes = kGeoBytes + kWstBytes + 4ull * kWinWords * kStages;
};

__device__ __forceinline__ void cp_async4(void* smem, const void* gmem, bool valid) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(sa), "l"(gmem), "r"(valid ? 4 : 0)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

// Geometry of angle t0 + t for the tile: window start and in-tile constants.
__device__ __forceinline__ void tile_geometry(const BpArgs& a, int gx, int gy, int th, Geo* geo, int* wst) {
  const TileOrigin o = tile_origin(gx, gy, a.half_n, a.center, a.trig[th]);
  // Lowest reachable index over the tile, one sample of rounding margin.
  const float lo = o.f0 + fminf(0.f, 31.f * o.c) + fminf(0.f, 31.f * o.s);
  const int ws = o.i0 + (int)floorf(lo) - 1;
  *geo = Geo{o.i0 - ws, o.f0, o.c, o.s};
  *wst = ws;
}

template <bool CHECK>
__device__ __forceinline__ int window_index(const BpArgs& a, const Geo& g, float fdx, float fdy, float* w) {
  const float s = rel_coord(g.f0, g.c, g.s, fdx, fdy);
  const float fl = floorf(s);
  *w = s - fl;
  int idx = (int)fl + g.base;
  if (CHECK) {
    if (idx < 0 || idx > kWin - 2) {
      atomicOr(a.err, kErrBpWindow);
      idx = 0;
    }
  }
  return idx;
}

template <class TV, int K, int R>
__device__ __forceinline__ void store_tile(const BpArgs& a, int gx, int gy, int z0, const float (&acc)[R][K]) {
  constexpr int NW = 32 / R;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  TV* vol = reinterpret_cast<TV*>(a.vol);
  const int ix = gx * kTile + lane;
  if (ix >= a.n) return;
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const int iy = gy * kTile + warp + NW * r;
    if (iy >= a.n) continue;
#pragma unroll
    for (int k = 0; k < K; ++k) {
      const int z = z0 + k;
      if (z < a.nz) Store<TV>::put(vol + (int64_t)z * a.v_z + (int64_t)iy * a.v_y + ix, acc[r][k] * a.scale);
    }
  }
}

// --- FP32: double-buffered cp.async staging -------------------------------
template <class TV, int K, int T, int R, bool CHECK>
__device__ __forceinline__ void bp_tile_f32(const BpArgs& a, int gx, int gy, int z0, unsigned char* smem) {
  using L = BpLayout<float, K, T>;
  constexpr int NW = 32 / R, NT = 32 * NW;
  Geo* geo = reinterpret_cast<Geo*>(smem);
  int* wst = reinterpret_cast<int*>(smem + L::kGeoBytes);
  float* win = reinterpret_cast<float*>(smem + L::kGeoBytes + L::kWstBytes);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const float* sino = reinterpret_cast<const float*>(a.sino);
  const int nstages = (a.ntheta + T - 1) / T;

  float acc[R][K];
#pragma unroll
  for (int r = 0; r < R; ++r)
#pragma unroll
    for (int k = 0; k < K; ++k) acc[r][k] = 0.f;

  auto issue = [&](int s) {  // copy the windows of stage s into buffer s & 1
    const int b = s & 1, t0 = s * T, nt = min(T, a.ntheta - t0);
    float* wb = win + b * (T * K * kWin);
    const int* ws = wst + (s % 3) * T;
    for (int e = threadIdx.x; e < nt * K * kWin; e += NT) {
      const int t = e / (K * kWin);
      const int rem = e - t * (K * kWin);
      const int k = rem / kWin;
      const int i = rem - k * kWin;
      const int z = z0 + k, j = ws[t] + i;
      const bool ok = z < a.nz && j >= 0 && j < a.ndet;
      const float* src = ok ? sino + (int64_t)z * a.s_z + (int64_t)(t0 + t) * a.s_t + j : sino;
      cp_async4(wb + e, src, ok);
    }
    cp_async_commit();
  };

  if (threadIdx.x < min(T, a.ntheta)) tile_geometry(a, gx, gy, threadIdx.x, geo + threadIdx.x, wst + threadIdx.x);
  __syncthreads();
  issue(0);
  for (int s = 0; s < nstages; ++s) {
    const int b = s & 1;
    if (s + 1 < nstages) {
      // slot (s+1)%3 was last read by stage s-2, which every thread finished
      // before the previous iteration's barriers
      const int t1 = (s + 1) * T;
      const int gn = (s + 1) % 3;
      if ((int)threadIdx.x < min(T, a.ntheta - t1))
        tile_geometry(a, gx, gy, t1 + threadIdx.x, geo + gn * T + threadIdx.x, wst + gn * T + threadIdx.x);
    }
    __syncthreads();  // next geometry ready; window buffer (s+1)&1 no longer read
    if (s + 1 < nstages) {
      issue(s + 1);
      cp_async_wait<1>();
    } else {
      cp_async_wait<0>();
    }
    __syncthreads();  // stage s landed for every thread
    const int nt = min(T, a.ntheta - s * T);
    const float* wbase = win + b * (T * K * kWin);
    for (int t = 0; t < nt; ++t) {
      const Geo g = geo[(s % 3) * T + t];
      const float* wb = wbase + t * (K * kWin);
#pragma unroll
      for (int r = 0; r < R; ++r) {
        float w;
        const int idx = window_index<CHECK>(a, g, (float)lane, (float)(warp + NW * r), &w);
        const float w0 = 1.f - w;
#pragma unroll
        for (int k = 0; k < K; ++k) {
          acc[r][k] = __fmaf_rn(w0, wb[k * kWin + idx], acc[r][k]);
          acc[r][k] = __fmaf_rn(w, wb[k * kWin + idx + 1], acc[r][k]);
        }
      }
    }
  }
  __syncthreads();
  store_tile<TV, K, R>(a, gx, gy, z0, acc);
}

// --- FP32, 4 x 4 voxel blocks with register reuse of samples ---------------
//
// rows_per_thread == 16: 64 threads per 32 x 32 tile, each owning a 4 x 4 block
// of voxels times K slices.  Per angle the thread walks each of its 4 lines
// along the axis on which the ray coordinate changes least (|slope| <= 0.7072,
// in the direction in which it grows): the floor index then either stays or
// rises by one from voxel to voxel (the canonical coordinate is monotone in
// the walk, its FP32 rounding included), so the sample pair of the previous
// voxel is reused and one new sample per slice is read from shared memory,
// 5 loads per line instead of 8: 1.25 shared loads per interpolation instead
// of 2, which was the bound of the one-voxel-per-lane form.
template <int K, bool ALONG_X, bool FWD, bool CHECK>
__device__ __forceinline__ void rr_walk(const BpArgs& a, const Geo& g, const float* wb, float fx0, float fy0,
                                        float (&acc)[4][4][K]) {
#pragma unroll
  for (int line = 0; line < 4; ++line) {
    float va[K], vb[K];
    int prev = 0;
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      const int step = FWD ? v : 3 - v;
      const int col = ALONG_X ? step : line, row = ALONG_X ? line : step;
      float w;
      const int idx = window_index<CHECK>(a, g, fx0 + (float)col, fy0 + (float)row, &w);
      const float w0 = 1.f - w;
      if (v == 0) {
#pragma unroll
        for (int k = 0; k < K; ++k) {
          va[k] = wb[k * kWin + idx];
          vb[k] = wb[k * kWin + idx + 1];
        }
      } else {
        if (CHECK && idx != prev && idx != prev + 1) atomicOr(a.err, kErrBpWindow);
        const bool moved = idx != prev;
#pragma unroll
        for (int k = 0; k < K; ++k) {
          const float nb = wb[k * kWin + idx + 1];
          va[k] = moved ? vb[k] : va[k];
          vb[k] = nb;
        }
      }
      prev = idx;
#pragma unroll
      for (int k = 0; k < K; ++k) {
        acc[row][col][k] = __fmaf_rn(w0, va[k], acc[row][col][k]);
        acc[row][col][k] = __fmaf_rn(w, vb[k], acc[row][col][k]);
      }
    }
  }
}

template <class TV, int K>
__device__ __forceinline__ void store_tile_rr(const BpArgs& a, int gx, int gy, int z0, const float (&acc)[4][4][K]) {
  const int bx = threadIdx.x & 7, by = threadIdx.x >> 3;
  TV* vol = reinterpret_cast<TV*>(a.vol);
#pragma unroll
  for (int row = 0; row < 4; ++row) {
    const int iy = gy * kTile + 4 * by + row;
    if (iy >= a.n) continue;
#pragma unroll
    for (int col = 0; col < 4; ++col) {
      const int ix = gx * kTile + 4 * bx + col;
      if (ix >= a.n) continue;
#pragma unroll
      for (int k = 0; k < K; ++k)
        if (z0 + k < a.nz)
          Store<TV>::put(vol + (int64_t)(z0 + k) * a.v_z + (int64_t)iy * a.v_y + ix, acc[row][col][k] * a.scale);
    }
  }
}

template <class TV, int K, int T, bool CHECK>
__device__ __forceinline__ void bp_tile_f32_rr(const BpArgs& a, int gx, int gy, int z0, unsigned char* smem) {
  using L = BpLayout<float, K, T>;
  constexpr int NT = 64;
  Geo* geo = reinterpret_cast<Geo*>(smem);
  int* wst = reinterpret_cast<int*>(smem + L::kGeoBytes);
  float* win = reinterpret_cast<float*>(smem + L::kGeoBytes + L::kWstBytes);
  const float* sino = reinterpret_cast<const float*>(a.sino);
  const int nstages = (a.ntheta + T - 1) / T;
  const float fx0 = (float)(4 * (threadIdx.x & 7)), fy0 = (float)(4 * (threadIdx.x >> 3));

  float acc[4][4][K];
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int c = 0; c < 4; ++c)
#pragma unroll
      for (int k = 0; k < K; ++k) acc[r][c][k] = 0.f;

  auto issue = [&](int s) {  // copy the windows of stage s into buffer s & 1
    const int b = s & 1, t0 = s * T, nt = min(T, a.ntheta - t0);
    float* wb = win + b * (T * K * kWin);
    const int* ws = wst + (s % 3) * T;
    for (int e = threadIdx.x; e < nt * K * kWin; e += NT) {
      const int t = e / (K * kWin);
      const int rem = e - t * (K * kWin);
      const int k = rem / kWin;
      const int i = rem - k * kWin;
      const int z = z0 + k, j = ws[t] + i;
      const bool ok = z < a.nz && j >= 0 && j < a.ndet;
      const float* src = ok ? sino + (int64_t)z * a.s_z + (int64_t)(t0 + t) * a.s_t + j : sino;
      cp_async4(wb + e, src, ok);
    }
    cp_async_commit();
  };

  for (int t = threadIdx.x; t < min(T, a.ntheta); t += NT) tile_geometry(a, gx, gy, t, geo + t, wst + t);
  __syncthreads();
  issue(0);
  for (int s = 0; s < nstages; ++s) {
    const int b = s & 1;
    if (s + 1 < nstages) {
      const int t1 = (s + 1) * T;
      const int gn = (s + 1) % 3;
      for (int t = threadIdx.x; t < min(T, a.ntheta - t1); t += NT)
        tile_geometry(a, gx, gy, t1 + t, geo + gn * T + t, wst + gn * T + t);
    }
    __syncthreads();  // next geometry ready; window buffer (s+1)&1 no longer read
    if (s + 1 < nstages) {
      issue(s + 1);
      cp_async_wait<1>();
    } else {
      cp_async_wait<0>();
    }
    __syncthreads();  // stage s landed for every thread
    const int nt = min(T, a.ntheta - s * T);
    const float* wbase = win + b * (T * K * kWin);
    for (int t = 0; t < nt; ++t) {
      const Geo g = geo[(s % 3) * T + t];
      const float* wb = wbase + t * (K * kWin);
      // the branch is uniform over the block (one angle)
      if (fabsf(g.c) <= fabsf(g.s)) {
        if (g.c >= 0.f) rr_walk<K, true, true, CHECK>(a, g, wb, fx0, fy0, acc);
        else rr_walk<K, true, false, CHECK>(a, g, wb, fx0, fy0, acc);
      } else {
        if (g.s >= 0.f) rr_walk<K, false, true, CHECK>(a, g, wb, fx0, fy0, acc);
        else rr_walk<K, false, false, CHECK>(a, g, wb, fx0, fy0, acc);
      }
    }
  }
  __syncthreads();
  store_tile_rr<TV, K>(a, gx, gy, z0, acc);
}

// --- 16-bit, K >= 2: slice-interleaved window, packed FP32x2 FMAs ---------
template <class TS> __device__ __forceinline__ float2 unpack2(uint32_t v);
template <> __device__ __forceinline__ float2 unpack2<__half>(uint32_t v) {
  return __half22float2(*reinterpret_cast<const __half2*>(&v));
}
template <> __device__ __forceinline__ float2 unpack2<__nv_bfloat16>(uint32_t v) {
  return make_float2(__uint_as_float(v << 16), __uint_as_float(v & 0xffff0000u));
}

__device__ __forceinline__ unsigned long long pack2(float x, float y) {
  unsigned long long r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(x), "f"(y));
  return r;
}
__device__ __forceinline__ void ffma2(unsigned long long& acc, unsigned long long w, unsigned long long x) {
  asm("fma.rn.f32x2 %0, %1, %2, %0;" : "+l"(acc) : "l"(w), "l"(x));
}

template <int K>
__device__ __forceinline__ void load_words(const uint32_t* p, uint32_t (&v)[K / 2]) {
  if constexpr (K == 2) {
    v[0] = p[0];
  } else if constexpr (K == 4) {
    const uint2 q = *reinterpret_cast<const uint2*>(p);
    v[0] = q.x;
    v[1] = q.y;
  } else {
#pragma unroll
    for (int c = 0; c < K / 8; ++c) {
      const uint4 q = *reinterpret_cast<const uint4*>(p + 4 * c);
      v[4 * c] = q.x;
      v[4 * c + 1] = q.y;
      v[4 * c + 2] = q.z;
      v[4 * c + 3] = q.w;
    }
  }
}

template <class TS, class TV, int K, int T, int R, bool CHECK>
__device__ __forceinline__ void bp_tile_16i(const BpArgs& a, int gx, int gy, int z0, unsigned char* smem) {
  using L = BpLayout<TS, K, T>;
  constexpr int NW = 32 / R, NT = 32 * NW, KW = K / 2;  // words per detector sample
  Geo* geo = reinterpret_cast<Geo*>(smem);
  int* wst = reinterpret_cast<int*>(smem + L::kGeoBytes);
  uint32_t* win = reinterpret_cast<uint32_t*>(smem + L::kGeoBytes + L::kWstBytes);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const unsigned short* sino = reinterpret_cast<const unsigned short*>(a.sino);

  unsigned long long acc[R][KW];
#pragma unroll
  for (int r = 0; r < R; ++r)
#pragma unroll
    for (int c = 0; c < KW; ++c) acc[r][c] = 0ull;

  for (int t0 = 0; t0 < a.ntheta; t0 += T) {
    const int nt = min(T, a.ntheta - t0);
    if ((int)threadIdx.x < nt) tile_geometry(a, gx, gy, t0 + threadIdx.x, geo + threadIdx.x, wst + threadIdx.x);
    __syncthreads();
    // word e = ((t * WIN) + i) * KW + kp holds slices (2kp, 2kp + 1) of sample
    // i: consecutive threads write consecutive words (no bank conflicts).
    for (int e = threadIdx.x; e < nt * kWin * KW; e += NT) {
      const int t = e / (kWin * KW);
      const int rem = e - t * (kWin * KW);
      const int i = rem / KW;
      const int kp = rem - i * KW;
      const int z = z0 + 2 * kp, j = wst[t] + i;
      uint32_t v = 0;
      if (j >= 0 && j < a.ndet) {
        const int64_t off = (int64_t)(t0 + t) * a.s_t + j;
        const uint32_t lo = z < a.nz ? __ldg(sino + (int64_t)z * a.s_z + off) : 0u;
        const uint32_t hi = z + 1 < a.nz ? __ldg(sino + (int64_t)(z + 1) * a.s_z + off) : 0u;
        v = lo | (hi << 16);
      }
      win[e] = v;
    }
    __syncthreads();
    for (int t = 0; t < nt; ++t) {
      const Geo g = geo[t];
      const uint32_t* wb = win + t * (kWin * KW);
#pragma unroll
      for (int r = 0; r < R; ++r) {
        float w;
        const int idx = window_index<CHECK>(a, g, (float)lane, (float)(warp + NW * r), &w);
        uint32_t q0[KW], q1[KW];
        load_words<K>(wb + idx * KW, q0);
        load_words<K>(wb + (idx + 1) * KW, q1);
        const unsigned long long w0 = pack2(1.f - w, 1.f - w), w1 = pack2(w, w);
#pragma unroll
        for (int c = 0; c < KW; ++c) {
          const float2 x0 = unpack2<TS>(q0[c]), x1 = unpack2<TS>(q1[c]);
          ffma2(acc[r][c], w0, pack2(x0.x, x0.y));
          ffma2(acc[r][c], w1, pack2(x1.x, x1.y));
        }
      }
    }
    __syncthreads();
  }
  float out[R][K];
#pragma unroll
  for (int r = 0; r < R; ++r)
#pragma unroll
    for (int c = 0; c < KW; ++c) {
      float x, y;
      asm("mov.b64 {%0, %1}, %2;" : "=f"(x), "=f"(y) : "l"(acc[r][c]));
      out[r][2 * c] = x;
      out[r][2 * c + 1] = y;
    }
  store_tile<TV, K, R>(a, gx, gy, z0, out);
}

// --- FP32, slice pairs: packed FP32x2 FMAs, sample reuse along the column ----
//
// kernel == 2 (FP32 sinograms, K even): the window holds slice pairs
// win[t][p][i] = (q[z0 + 2p][i], q[z0 + 2p + 1][i]), so one 8-byte shared load
// fetches sample i of two slices and one fma.rn.f32x2 accumulates both.  A
// thread owns R consecutive rows of one voxel column; for angles with
// |sin| <= 0.99 it walks them in the direction in which the ray coordinate
// grows, where the canonical FP32 coordinate is monotone and rises by less than
// one sample per row, so the floor index steps by 0 or +1 and the previous
// voxel's sample pair is reused: one new 8-byte load per slice pair and voxel
// after the first.  Other angles load both samples.  Lanes are consecutive
// voxels of a row, so the loads of a warp are contiguous (no bank conflicts).
// The result equals the other CUDA-core forms to FP32 rounding (same weights;
// the same per-slice summation order).
template <int K, int R, bool UP, bool REUSE, bool CHECK>
__device__ __forceinline__ void pairs_column(const BpArgs& a, const Geo& g, const unsigned long long* wb, int lane,
                                             int y0, unsigned long long (&acc)[R][K / 2]) {
  constexpr int KP = K / 2;
  unsigned long long va[KP], vb[KP];
  int prev = 0;
#pragma unroll
  for (int v = 0; v < R; ++v) {
    const int r = UP ? v : R - 1 - v;
    float w;
    const int idx = window_index<CHECK>(a, g, (float)lane, (float)(y0 + r), &w);
    const unsigned long long w0 = pack2(1.f - w, 1.f - w), w1 = pack2(w, w);
    if (!REUSE || v == 0) {
#pragma unroll
      for (int p = 0; p < KP; ++p) {
        va[p] = wb[p * kWin + idx];
        vb[p] = wb[p * kWin + idx + 1];
      }
    } else {
      if (CHECK && idx != prev && idx != prev + 1) atomicOr(a.err, kErrBpWindow);
      const bool moved = idx != prev;
#pragma unroll
      for (int p = 0; p < KP; ++p) {
        const unsigned long long nb = wb[p * kWin + idx + 1];
        va[p] = moved ? vb[p] : va[p];
        vb[p] = nb;
      }
    }
    prev = idx;
#pragma unroll
    for (int p = 0; p < KP; ++p) {
      ffma2(acc[r][p], w0, va[p]);
      ffma2(acc[r][p], w1, vb[p]);
    }
  }
}

template <class TV, int K, int T, int R, bool CHECK>
__device__ __forceinline__ void bp_tile_f32_pairs(const BpArgs& a, int gx, int gy, int z0, unsigned char* smem) {
  static_assert(K % 2 == 0, "slice pairs");
  using L = BpLayout<float, K, T>;
  constexpr int NW = 32 / R, NT = 32 * NW, KP = K / 2;
  Geo* geo = reinterpret_cast<Geo*>(smem);
  int* wst = reinterpret_cast<int*>(smem + L::kGeoBytes);
  float* win = reinterpret_cast<float*>(smem + L::kGeoBytes + L::kWstBytes);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int y0 = warp * R;  // this thread's rows y0 .. y0 + R - 1 of the tile
  const float* sino = reinterpret_cast<const float*>(a.sino);
  const int nstages = (a.ntheta + T - 1) / T;

  unsigned long long acc[R][KP];
#pragma unroll
  for (int r = 0; r < R; ++r)
#pragma unroll
    for (int p = 0; p < KP; ++p) acc[r][p] = 0ull;

  auto issue = [&](int s) {  // stage s into buffer s & 1: float index ((t KP + p) WIN + i) 2 + h
    const int b = s & 1, t0 = s * T, nt = min(T, a.ntheta - t0);
    float* wb = win + b * (T * K * kWin);
    const int* ws = wst + (s % 3) * T;
    // one row (t, p) of 2 WIN floats per warp step: lane copies floats
    // lane, lane + 32, lane + 64 (sample i = f / 2 of slice 2p + f % 2)
    for (int row = warp; row < nt * KP; row += NW) {
      const int t = row / KP, pp = row - t * KP;
      const int64_t rbase = (int64_t)(t0 + t) * a.s_t;
      float* dst = wb + row * (2 * kWin);
#pragma unroll
      for (int c = 0; c < (2 * kWin) / 32; ++c) {
        const int f = lane + 32 * c;
        const int h = f & 1, i = f >> 1;
        const int z = z0 + 2 * pp + h, j = ws[t] + i;
        const bool ok = z < a.nz && j >= 0 && j < a.ndet;
        const float* src = ok ? sino + (int64_t)z * a.s_z + rbase + j : sino;
        cp_async4(dst + f, src, ok);
      }
    }
    cp_async_commit();
  };

  if (threadIdx.x < min(T, a.ntheta)) tile_geometry(a, gx, gy, threadIdx.x, geo + threadIdx.x, wst + threadIdx.x);
  __syncthreads();
  issue(0);
  for (int s = 0; s < nstages; ++s) {
    const int b = s & 1;
    if (s + 1 < nstages) {
      const int t1 = (s + 1) * T;
      const int gn = (s + 1) % 3;
      if ((int)threadIdx.x < min(T, a.ntheta - t1))
        tile_geometry(a, gx, gy, t1 + threadIdx.x, geo + gn * T + threadIdx.x, wst + gn * T + threadIdx.x);
    }
    __syncthreads();  // next geometry ready; window buffer (s+1)&1 no longer read
    if (s + 1 < nstages) {
      issue(s + 1);
      cp_async_wait<1>();
    } else {
      cp_async_wait<0>();
    }
    __syncthreads();  // stage s landed for every thread
    const int nt = min(T, a.ntheta - s * T);
    const unsigned long long* wbase = reinterpret_cast<const unsigned long long*>(win + b * (T * K * kWin));
    for (int t = 0; t < nt; ++t) {
      const Geo g = geo[(s % 3) * T + t];
      const unsigned long long* wb = wbase + t * (KP * kWin);
      if (fabsf(g.s) <= 0.99f) {  // uniform over the block (one angle)
        if (g.s >= 0.f) pairs_column<K, R, true, true, CHECK>(a, g, wb, lane, y0, acc);
        else pairs_column<K, R, false, true, CHECK>(a, g, wb, lane, y0, acc);
      } else {
        pairs_column<K, R, true, false, CHECK>(a, g, wb, lane, y0, acc);
      }
    }
  }
  __syncthreads();
  TV* vol = reinterpret_cast<TV*>(a.vol);
  const int ix = gx * kTile + lane;
  if (ix < a.n) {
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int iy = gy * kTile + y0 + r;
      if (iy >= a.n) continue;
#pragma unroll
      for (int p = 0; p < KP; ++p) {
        float lo, hi;
        asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(acc[r][p]));
        if (z0 + 2 * p < a.nz) Store<TV>::put(vol + (int64_t)(z0 + 2 * p) * a.v_z + (int64_t)iy * a.v_y + ix, lo * a.scale);
        if (z0 + 2 * p + 1 < a.nz)
          Store<TV>::put(vol + (int64_t)(z0 + 2 * p + 1) * a.v_z + (int64_t)iy * a.v_y + ix, hi * a.scale);
      }
    }
  }
}

// --- 16-bit, K == 1: (q[i], q[i+1]) pairs, mixed-precision FMAs -----------
template <class TS, class TV, int K, int T, int R, bool CHECK>
__device__ __forceinline__ void bp_tile_pairs(const BpArgs& a, int gx, int gy, int z0, unsigned char* smem) {
  using L = BpLayout<TS, K, T>;
  using I = Interp<TS>;
  constexpr int NW = 32 / R, NT = 32 * NW;
  Geo* geo = reinterpret_cast<Geo*>(smem);
  int* wst = reinterpret_cast<int*>(smem + L::kGeoBytes);
  uint32_t* win = reinterpret_cast<uint32_t*>(smem + L::kGeoBytes + L::kWstBytes);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const TS* sino = reinterpret_cast<const TS*>(a.sino);
  float acc[R][K];
#pragma unroll
  for (int r = 0; r < R; ++r)
#pragma unroll
    for (int k = 0; k < K; ++k) acc[r][k] = 0.f;
  for (int t0 = 0; t0 < a.ntheta; t0 += T) {
    const int nt = min(T, a.ntheta - t0);
    if ((int)threadIdx.x < nt) tile_geometry(a, gx, gy, t0 + threadIdx.x, geo + threadIdx.x, wst + threadIdx.x);
    __syncthreads();
    for (int e = threadIdx.x; e < nt * K * kWin; e += NT) {
      const int t = e / (K * kWin);
      const int rem = e - t * (K * kWin);
      const int k = rem / kWin;
      const int i = rem - k * kWin;
      const int z = z0 + k;
      uint32_t v = 0;
      if (z < a.nz) v = I::stage(sino + (int64_t)z * a.s_z + (int64_t)(t0 + t) * a.s_t, wst[t] + i, a.ndet);
      win[e] = v;
    }
    __syncthreads();
    for (int t = 0; t < nt; ++t) {
      const Geo g = geo[t];
      const uint32_t* wb = win + t * (K * kWin);
#pragma unroll
      for (int r = 0; r < R; ++r) {
        float w;
        const int idx = window_index<CHECK>(a, g, (float)lane, (float)(warp + NW * r), &w);
        const typename I::W wt = I::weights(w);
#pragma unroll
        for (int k = 0; k < K; ++k) I::acc(acc[r][k], wb, k * kWin + idx, wt);
      }
    }
    __syncthreads();
  }
  store_tile<TV, K, R>(a, gx, gy, z0, acc);
}

// One work unit: the aligned 32x32 voxel tile (gx, gy) times slices
// [z0, z0 + K), summed over every angle.  Ends with a block barrier, so the
// shared buffers may be reused by the next unit.
// V: 0 the forms above by dtype and R (R == 16: 4 x 4 blocks), 2 the FP32
// slice-pair form.
template <class TS, class TV, int K, int T, int R, bool CHECK, int V>
__device__ __forceinline__ void bp_tile(const BpArgs& a, int gx, int gy, int z0, unsigned char* smem) {
  using L = BpLayout<TS, K, T>;
  if constexpr (L::kF32 && V == 2) bp_tile_f32_pairs<TV, K, T, R, CHECK>(a, gx, gy, z0, smem);
  else if constexpr (L::kF32 && R == 16) bp_tile_f32_rr<TV, K, T, CHECK>(a, gx, gy, z0, smem);
  else if constexpr (L::kF32) bp_tile_f32<TV, K, T, R, CHECK>(a, gx, gy, z0, smem);
  else if constexpr (L::kInter) bp_tile_16i<TS, TV, K, T, R, CHECK>(a, gx, gy, z0, smem);
  else bp_tile_pairs<TS, TV, K, T, R, CHECK>(a, gx, gy, z0, smem);
  __syncthreads();
}

extern __shared__ __align__(16) unsigned char bp_smem[];

template <class TS, class TV, int K, int T, int R, bool CHECK, int V>
__global__ void __launch_bounds__(32 * (32 / R)) k_backproject(BpArgs a) {
  bp_tile<TS, TV, K, T, R, CHECK, V>(a, blockIdx.x % a.ntx, blockIdx.x / a.ntx, blockIdx.y * K, bp_smem);
}

// Persistent form for batches of datasets with uneven widths and angle
// counts: a grid sized to the resident capacity pulls work units from one
// atomic counter.  Unit u belongs to the item with prefix[i] <= u <
// prefix[i+1]; inside an item, units run over 32x32 tiles fastest, then slice
// blocks.  No block ever waits on another (the counter is the only shared
// state), so every launch completes regardless of scheduling.
template <class TS, class TV, int K, int T, int R, bool CHECK, int V>
__global__ void __launch_bounds__(32 * (32 / R)) k_backproject_persistent(BpWork w) {
  __shared__ long long s_unit;
  __shared__ int s_item;
  __shared__ BpArgs s_args;
  const long long total = w.prefix[w.nitems];
  for (;;) {
    if (threadIdx.x == 0) {
      const long long u = (long long)atomicAdd(w.counter, 1ull);
      int it = 0;
      if (u < total)
        while (u >= w.prefix[it + 1]) ++it;
      s_unit = u;
      s_item = it;
    }
    __syncthreads();
    const long long u = s_unit;
    if (u >= total) break;
    const int it = s_item;
    if (threadIdx.x == 0) s_args = w.items[it];
    __syncthreads();
    const long long local = u - w.prefix[it];
    const long long tiles = (long long)s_args.ntx * s_args.ntx;
    const int zb = (int)(local / tiles);
    const int tile = (int)(local - (long long)zb * tiles);
    bp_tile<TS, TV, K, T, R, CHECK, V>(s_args, tile % s_args.ntx, tile / s_args.ntx, zb * K, bp_smem);
  }
}

template <class TS, class TV, int K, int T, int R, int V = 0>
KernPair pick_check(bool check) {
  const size_t sm = BpLayout<TS, K, T>::kBytes;
  if (check)
    return {k_backproject<TS, TV, K, T, R, true, V>, k_backproject_persistent<TS, TV, K, T, R, true, V>, sm};
  return {k_backproject<TS, TV, K, T, R, false, V>, k_backproject_persistent<TS, TV, K, T, R, false, V>, sm};
}

// Instantiated configurations (k_slices, theta_stage, rows_per_thread).
template <class TS, class TV>
KernPair pick(const tcp_bp_config& c, bool check) {
  if (c.kernel == 2) {  // FP32 slice pairs
    if constexpr (std::is_same<TS, float>::value) {
#define TCP_BP_CASE2(K, T, R) \
  if (c.k_slices == K && c.theta_stage == T && c.rows_per_thread == R) return pick_check<TS, TV, K, T, R, 2>(check);
      TCP_BP_CASE2(8, 16, 4)
      TCP_BP_CASE2(16, 8, 4)
      TCP_BP_CASE2(4, 16, 4)
      TCP_BP_CASE2(8, 16, 8)
#undef TCP_BP_CASE2
    }
    return {nullptr, nullptr, 0};
  }
#define TCP_BP_CASE(K, T, R) \
  if (c.k_slices == K && c.theta_stage == T && c.rows_per_thread == R) return pick_check<TS, TV, K, T, R>(check);
  TCP_BP_CASE(8, 16, 4)
  TCP_BP_CASE(4, 32, 4)
  TCP_BP_CASE(4, 16, 4)
  TCP_BP_CASE(16, 8, 2)
  TCP_BP_CASE(8, 16, 2)
  TCP_BP_CASE(2, 16, 4)
  TCP_BP_CASE(1, 32, 4)
  if constexpr (std::is_same<TS, float>::value) {  // 4 x 4 voxel blocks: FP32 sinograms only
    TCP_BP_CASE(4, 16, 16)
    TCP_BP_CASE(2, 16, 16)
    TCP_BP_CASE(4, 32, 16)
    TCP_BP_CASE(8, 16, 16)
  }
#undef TCP_BP_CASE
  return {nullptr, nullptr, 0};
}

template <class TS>
KernPair pick_vol(int vdt, const tcp_bp_config& c, bool check) {
  switch (vdt) {
    case TCP_F32: return pick<TS, float>(c, check);
    case TCP_F16: return pick<TS, __half>(c, check);
    case TCP_BF16: return pick<TS, __nv_bfloat16>(c, check);
  }
  return {nullptr, nullptr, 0};
}

}  // namespace
}  // namespace tcp
