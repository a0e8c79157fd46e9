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
#include "tcp_internal.cuh"

namespace tcp {
namespace {

constexpr int kWin = 48;

struct Geo {
  int base;  // i0 - window start
  float f0, c, s;
};

// Shared-memory element of the staged window.
template <class TS> struct Win;
template <> struct Win<float> { using type = float; };
template <> struct Win<__half> { using type = uint32_t; };         // (q[i], q[i+1]) as f16x2
template <> struct Win<__nv_bfloat16> { using type = uint32_t; };  // (q[i], q[i+1]) as bf16x2

template <class TS> struct Interp;

template <> struct Interp<float> {
  static __device__ __forceinline__ float stage(const float* row, int j, int ndet) {
    return (j >= 0 && j < ndet) ? __ldg(row + j) : 0.f;
  }
  struct W { float w0, w1; };
  static __device__ __forceinline__ W weights(float w) { return {1.f - w, w}; }
  static __device__ __forceinline__ void acc(float& a, const float* p, int off, const W& w) {
    a = __fmaf_rn(w.w0, p[off], a);
    a = __fmaf_rn(w.w1, p[off + 1], a);
  }
};

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

template <class TS, int K, int T>
struct BpSmem {
  Geo geo[T];
  int wst[T];
  typename Win<TS>::type win[T * K * kWin];
};

// One work unit: the aligned 32x32 voxel tile (gx, gy) times slices
// [z0, z0 + K), summed over every angle.  Ends with a block barrier, so the
// shared buffers may be reused by the next unit.
template <class TS, class TV, int K, int T, int R, bool CHECK>
__device__ __forceinline__ void bp_tile(const BpArgs& a, int gx, int gy, int z0, BpSmem<TS, K, T>& sm) {
  using WT = typename Win<TS>::type;
  using I = Interp<TS>;
  constexpr int NW = 32 / R;  // warps per block (rows per pass)
  constexpr int NT = 32 * NW;
  Geo* geo = sm.geo;
  int* wst = sm.wst;
  WT* win = sm.win;

  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const TS* sino = reinterpret_cast<const TS*>(a.sino);

  float acc[R][K];
#pragma unroll
  for (int r = 0; r < R; ++r)
#pragma unroll
    for (int k = 0; k < K; ++k) acc[r][k] = 0.f;

  const float fdx = (float)lane;

  for (int t0 = 0; t0 < a.ntheta; t0 += T) {
    const int nt = min(T, a.ntheta - t0);
    if (threadIdx.x < nt) {
      const TileOrigin o = tile_origin(gx, gy, a.half_n, a.center, a.trig[t0 + threadIdx.x]);
      // Lowest reachable index over the tile, one sample of rounding margin.
      const float lo = o.f0 + fminf(0.f, 31.f * o.c) + fminf(0.f, 31.f * o.s);
      const int ws = o.i0 + (int)floorf(lo) - 1;
      geo[threadIdx.x] = Geo{o.i0 - ws, o.f0, o.c, o.s};
      wst[threadIdx.x] = ws;
    }
    __syncthreads();
    // Stage the windows: element e = (t, k, i), i fastest -> coalesced rows.
    for (int e = threadIdx.x; e < nt * K * kWin; e += NT) {
      const int t = e / (K * kWin);
      const int rem = e - t * (K * kWin);
      const int k = rem / kWin;
      const int i = rem - k * kWin;
      const int z = z0 + k;
      WT v = WT(0);
      if (z < a.nz) {
        const TS* row = sino + (int64_t)z * a.s_z + (int64_t)(t0 + t) * a.s_t;
        v = I::stage(row, wst[t] + i, a.ndet);
      }
      win[e] = v;
    }
    __syncthreads();

    for (int t = 0; t < nt; ++t) {
      const Geo g = geo[t];
      const WT* wb = win + t * (K * kWin);
#pragma unroll
      for (int r = 0; r < R; ++r) {
        const float s = rel_coord(g.f0, g.c, g.s, fdx, (float)(warp + NW * r));
        const float fl = floorf(s);
        const typename I::W w = I::weights(s - fl);
        int idx = (int)fl + g.base;
        if (CHECK) {
          if (idx < 0 || idx > kWin - 2) {
            atomicOr(a.err, kErrBpWindow);
            idx = 0;
          }
        }
#pragma unroll
        for (int k = 0; k < K; ++k) I::acc(acc[r][k], wb, k * kWin + idx, w);
      }
    }
    __syncthreads();
  }

  TV* vol = reinterpret_cast<TV*>(a.vol);
  const int ix = gx * kTile + lane;
  if (ix < a.n) {
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
}

template <class TS, class TV, int K, int T, int R, bool CHECK>
__global__ void __launch_bounds__(32 * (32 / R)) k_backproject(BpArgs a) {
  __shared__ BpSmem<TS, K, T> sm;
  bp_tile<TS, TV, K, T, R, CHECK>(a, blockIdx.x % a.ntx, blockIdx.x / a.ntx, blockIdx.y * K, sm);
}

// Persistent form for batches of datasets with uneven widths and angle
// counts: a grid sized to the resident capacity pulls work units from one
// atomic counter.  Unit u belongs to the item with prefix[i] <= u <
// prefix[i+1]; inside an item, units run over 32x32 tiles fastest, then slice
// blocks.  No block ever waits on another (the counter is the only shared
// state), so every launch completes regardless of scheduling.
template <class TS, class TV, int K, int T, int R, bool CHECK>
__global__ void __launch_bounds__(32 * (32 / R)) k_backproject_persistent(BpWork w) {
  __shared__ BpSmem<TS, K, T> sm;
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
    bp_tile<TS, TV, K, T, R, CHECK>(s_args, tile % s_args.ntx, tile / s_args.ntx, zb * K, sm);
  }
}

using Kern = void (*)(BpArgs);
using PKern = void (*)(BpWork);

struct KernPair {
  Kern direct;
  PKern persistent;
};

template <class TS, class TV, int K, int T, int R>
KernPair pick_check(bool check) {
  if (check) return {k_backproject<TS, TV, K, T, R, true>, k_backproject_persistent<TS, TV, K, T, R, true>};
  return {k_backproject<TS, TV, K, T, R, false>, k_backproject_persistent<TS, TV, K, T, R, false>};
}

// Instantiated configurations (k_slices, theta_stage, rows_per_thread).
template <class TS, class TV>
KernPair pick(const tcp_bp_config& c, bool check) {
#define TCP_BP_CASE(K, T, R) \
  if (c.k_slices == K && c.theta_stage == T && c.rows_per_thread == R) return pick_check<TS, TV, K, T, R>(check);
  TCP_BP_CASE(8, 16, 4)
  TCP_BP_CASE(4, 32, 4)
  TCP_BP_CASE(4, 16, 4)
  TCP_BP_CASE(16, 8, 2)
  TCP_BP_CASE(8, 16, 2)
  TCP_BP_CASE(2, 16, 4)
  TCP_BP_CASE(1, 32, 4)
#undef TCP_BP_CASE
  return {nullptr, nullptr};
}

template <class TS>
KernPair pick_vol(int vdt, const tcp_bp_config& c, bool check) {
  switch (vdt) {
    case TCP_F32: return pick<TS, float>(c, check);
    case TCP_F16: return pick<TS, __half>(c, check);
    case TCP_BF16: return pick<TS, __nv_bfloat16>(c, check);
  }
  return {nullptr, nullptr};
}

KernPair pick_all(int sdt, int vdt, const tcp_bp_config& c, bool check) {
  switch (sdt) {
    case TCP_F32: return pick_vol<float>(vdt, c, check);
    case TCP_F16: return pick_vol<__half>(vdt, c, check);
    case TCP_BF16: return pick_vol<__nv_bfloat16>(vdt, c, check);
  }
  return {nullptr, nullptr};
}

}  // namespace

bool valid_bp_config(const tcp_bp_config& c) {
  return pick<float, float>(c, false).direct != nullptr;
}

int bp_threads(const tcp_bp_config& c) { return 32 * (32 / c.rows_per_thread); }

tcp_status bp_persistent_grid(int sdt, int vdt, const tcp_bp_config& cfg, int* blocks) {
  KernPair kp = pick_all(sdt, vdt, cfg, checked_mode());
  if (!kp.persistent) return fail(TCP_ERR_UNSUPPORTED, "backproject: no persistent kernel for this dtype/config");
  int per_sm = 0, dev = 0, sms = 0;
  TCP_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kp.persistent, bp_threads(cfg), 0));
  TCP_CUDA_TRY(cudaGetDevice(&dev));
  TCP_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  *blocks = std::max(1, per_sm) * sms;
  return TCP_OK;
}

tcp_status launch_backproject_persistent(const BpWork& w, int sdt, int vdt, const tcp_bp_config& cfg, int blocks,
                                         cudaStream_t st) {
  KernPair kp = pick_all(sdt, vdt, cfg, checked_mode());
  if (!kp.persistent) return fail(TCP_ERR_UNSUPPORTED, "backproject: no persistent kernel for this dtype/config");
  kp.persistent<<<blocks, bp_threads(cfg), 0, st>>>(w);
  TCP_CUDA_TRY(cudaGetLastError());
  return TCP_OK;
}

tcp_bp_config default_bp_config(int64_t nz, int64_t, int64_t, int64_t, int sdt, int) {
  tcp_bp_config c{8, 16, 4, 0};
  if (nz <= 1) c = tcp_bp_config{1, 32, 4, 0};
  else if (nz <= 2) c = tcp_bp_config{2, 16, 4, 0};
  else if (nz <= 4) c = tcp_bp_config{4, 16, 4, 0};
  (void)sdt;
  return c;
}

tcp_status launch_backproject(const View3& sino, const TrigTable& trig, double center, const View3& vol,
                              const tcp_bp_config& cfg, cudaStream_t st, float scale) {
  Kern k = pick_all(sino.dtype, vol.dtype, cfg, checked_mode()).direct;
  if (!k) return fail(TCP_ERR_UNSUPPORTED, "backproject: no kernel for this dtype/config");
  if (sino.d0 == 0 || vol.d1 == 0) return TCP_OK;
  BpArgs a = make_bp_args(sino, trig, center, vol, scale);
  const int threads = bp_threads(cfg);
  dim3 grid((unsigned)(a.ntx * a.ntx), (unsigned)((a.nz + cfg.k_slices - 1) / cfg.k_slices));
  if (grid.y > 65535u) return fail(TCP_ERR_SHAPE, "backproject: too many slice blocks");
  k<<<grid, threads, 0, st>>>(a);
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
