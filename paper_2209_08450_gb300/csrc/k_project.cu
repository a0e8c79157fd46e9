// Radon projector, the adjoint of the LineRec backprojector (not in the
// paper; it makes backprojection differentiable and enables least-squares
// reconstruction):
//   sino[z][theta][j] = sum over voxels of vol * weight_j(s(voxel, theta)),
// where weight_j is the linear-interpolation weight that the backprojector
// gives detector pixel j at that voxel: (1 - w) if floor(s) == j, w if
// floor(s) + 1 == j, else 0.
//
// Gather form, one thread per (theta, j) and K slices: no atomics, a fixed
// summation order, deterministic.  The thread walks the major axis of the ray
// (y when |cos| >= |sin|, else x) and visits the <= 3 voxels per step whose
// ray coordinate can lie in [j - 1, j + 1).  Each candidate's coordinate is
// recomputed with the backprojector's canonical tile geometry, from a per-call
// table of FP64 tile origins built by the same function, so the two operators
// share bit-identical weights.
//
// Memory access: the lanes of a warp are consecutive detector bins j of one
// angle, so at each step they visit neighbouring voxels along the minor axis.
// For y-major angles that is along a row (coalesced); for x-major angles it
// would be down a column (one cache line per lane), so those angles read a
// transposed copy volT[z][ix][iy] made once per call by a tiled transpose.
// For FP32 volumes the slices are also interleaved in groups of 16
// (volI[g][a][q][b][4], slices 4q..4q+3 of voxel b adjacent; a row-major and a
// transposed copy), so that a hit reads its 16 slices with four 16-byte loads
// instead of sixteen 4-byte ones, while the lanes of a warp (neighbouring
// voxels b) still read neighbouring 16-byte words.
#include "tcp_internal.cuh"

namespace tcp {
namespace {

__global__ void k_origin_table(const double2* trig, int ntheta, int ntx, double half_n, double center,
                               int2* out) {
  const int64_t total = (int64_t)ntheta * ntx * ntx;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int t = (int)(e / ((int64_t)ntx * ntx));
    const int rem = (int)(e - (int64_t)t * ntx * ntx);
    const int gy = rem / ntx, gx = rem - gy * ntx;
    const TileOrigin o = tile_origin(gx, gy, half_n, center, trig[t]);
    out[e] = make_int2(o.i0, __float_as_int(o.f0));
  }
}

template <class TS> struct WRound {
  static __device__ __forceinline__ float r(float w) { return w; }
};
template <> struct WRound<__half> {
  static __device__ __forceinline__ float r(float w) { return __half2float(__float2half_rn(w)); }
};
template <> struct WRound<__nv_bfloat16> {
  static __device__ __forceinline__ float r(float w) { return __bfloat162float(__float2bfloat16_rn(w)); }
};

// volT[z][ix][iy] = vol[z][iy][ix], 32 x 32 tiles through shared memory.
template <class TV>
__global__ void k_transpose(const TV* vol, int64_t v_z, int64_t v_y, int n, TV* volT) {
  __shared__ TV t[32][33];
  const int z = blockIdx.z;
  const int x0 = blockIdx.x * 32, y0 = blockIdx.y * 32;
  const TV* src = vol + z * v_z;
  TV* dst = volT + (int64_t)z * n * n;
  for (int r = threadIdx.y; r < 32; r += 8) {
    const int y = y0 + r, x = x0 + threadIdx.x;
    if (y < n && x < n) t[r][threadIdx.x] = src[(int64_t)y * v_y + x];
  }
  __syncthreads();
  for (int r = threadIdx.y; r < 32; r += 8) {
    const int x = x0 + r, y = y0 + threadIdx.x;
    if (y < n && x < n) dst[(int64_t)x * n + y] = t[threadIdx.x][r];
  }
}

// dst[g][a][q][b][r] = src[16 g + 4 q + r][a][b] for slice groups g < G (FP32).
__global__ void k_interleave16(const float* src, int64_t s_z, int64_t s_row, int n, int G, float* dst) {
  const int64_t total = (int64_t)G * n * n;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int g = (int)(e / ((int64_t)n * n));
    const int64_t ab = e - (int64_t)g * n * n;
    const int a = (int)(ab / n), b = (int)(ab - (int64_t)a * n);
    const float* p = src + (int64_t)(16 * g) * s_z + (int64_t)a * s_row + b;
    float4* q = reinterpret_cast<float4*>(dst) + ((int64_t)g * n + a) * 4 * n + b;
#pragma unroll
    for (int c = 0; c < 4; ++c)
      q[(int64_t)c * n] = make_float4(__ldg(p + (int64_t)(4 * c) * s_z), __ldg(p + (int64_t)(4 * c + 1) * s_z),
                                      __ldg(p + (int64_t)(4 * c + 2) * s_z), __ldg(p + (int64_t)(4 * c + 3) * s_z));
  }
}

struct PjArgs {
  const void* vol;
  const float* volIy;  // FP32 volumes: [g][iy][ix][16] slice-interleaved copy
  const float* volIx;  // and [g][ix][iy][16]
  const void* volT;  // [z][ix][iy], row stride n, slice stride n * n
  int64_t v_z, v_y;
  int nz, n, ntx;
  void* sino;
  int64_t s_z, s_t;
  int ntheta, ndet;
  const double2* trig;
  const int2* orig;
  double center, half_n;
  int zbase;  // first slice of blockIdx.z == 0
};

// A block is 8 warps: 8 consecutive angles times the same 32 detector bins.
// Neighbouring angles visit nearly the same voxels at each step of the walk,
// so the block's warps share those rows through L1 instead of each streaming
// them from L2.
constexpr int kPjAngles = 8;
constexpr int kPjThreads = 32 * kPjAngles;

// FULL: all K slices of the block exist (no per-slice bound check).
template <class TV, class TS, int K, bool FULL>
__global__ void __launch_bounds__(kPjThreads) k_project(PjArgs a) {
  const int t = blockIdx.y * kPjAngles + (threadIdx.x >> 5);
  const int j = blockIdx.x * 32 + (threadIdx.x & 31);
  const int z0 = a.zbase + blockIdx.z * K;
  if (j >= a.ndet || t >= a.ntheta) return;
  const double2 cs = a.trig[t];
  const float c = __double2float_rn(cs.x), s = __double2float_rn(cs.y);
  const bool ymajor = fabs(cs.x) >= fabs(cs.y);
  const float inv = 1.0f / (ymajor ? c : s);
  const float hr = fabsf(inv) + 0.02f;
  const float hn = (float)a.half_n;
  const float jc = (float)((double)j - a.center);
  const int2* orig = a.orig + (int64_t)t * a.ntx * a.ntx;
  // x-major angles walk columns: read them as rows of the transposed copy
  const int64_t vy = ymajor ? a.v_y : a.n, vz = ymajor ? a.v_z : (int64_t)a.n * a.n;
  const TV* vol = reinterpret_cast<const TV*>(ymajor ? a.vol : a.volT) + (int64_t)z0 * vz;

  float acc[K];
#pragma unroll
  for (int k = 0; k < K; ++k) acc[k] = 0.f;

  for (int m = 0; m < a.n; ++m) {
    const float other = (float)m - hn;
    const float uc = (jc - other * (ymajor ? s : c)) * inv + hn;
    const int lo = max(0, (int)ceilf(uc - hr));
    const int hi = min(a.n - 1, (int)floorf(uc + hr));
    for (int u = lo; u <= hi; ++u) {
      const int ix = ymajor ? u : m, iy = ymajor ? m : u;
      const int2 o = __ldg(orig + (iy >> 5) * a.ntx + (ix >> 5));
      const float sr = rel_coord(__int_as_float(o.y), c, s, (float)(ix & 31), (float)(iy & 31));
      const float fl = floorf(sr);
      const float w = sr - fl;
      const int i = o.x + (int)fl;
      float wt = 0.f;
      if (i == j) wt = WRound<TS>::r(1.f - w);
      else if (i + 1 == j) wt = WRound<TS>::r(w);
      if (wt != 0.f) {
        const TV* p = vol + (int64_t)m * vy + u;  // (iy, ix) for y-major, (ix, iy) transposed otherwise
#pragma unroll
        for (int k = 0; k < K; ++k)
          if (FULL || z0 + k < a.nz) acc[k] = __fmaf_rn(wt, Store<TV>::load(p + (int64_t)k * vz), acc[k]);
      }
    }
  }
  TS* out = reinterpret_cast<TS*>(a.sino);
#pragma unroll
  for (int k = 0; k < K; ++k)
    if (z0 + k < a.nz) Store<TS>::put(out + (int64_t)(z0 + k) * a.s_z + (int64_t)t * a.s_t + j, acc[k]);
}

// FP32 volume, 16 slices per thread read from the slice-interleaved copies;
// otherwise the same walk, weights and summation order as k_project.
template <class TS>
__global__ void __launch_bounds__(kPjThreads) k_project_i16(PjArgs a) {
  const int t = blockIdx.y * kPjAngles + (threadIdx.x >> 5);
  const int j = blockIdx.x * 32 + (threadIdx.x & 31);
  const int g = blockIdx.z;
  const int z0 = 16 * g;
  if (j >= a.ndet || t >= a.ntheta) return;
  const double2 cs = a.trig[t];
  const float c = __double2float_rn(cs.x), s = __double2float_rn(cs.y);
  const bool ymajor = fabs(cs.x) >= fabs(cs.y);
  const float inv = 1.0f / (ymajor ? c : s);
  const float hr = fabsf(inv) + 0.02f;
  const float hn = (float)a.half_n;
  const float jc = (float)((double)j - a.center);
  const int2* orig = a.orig + (int64_t)t * a.ntx * a.ntx;
  const float* vol = (ymajor ? a.volIy : a.volIx) + (int64_t)g * a.n * a.n * 16;

  float acc[16];
#pragma unroll
  for (int k = 0; k < 16; ++k) acc[k] = 0.f;

  for (int m = 0; m < a.n; ++m) {
    const float other = (float)m - hn;
    const float uc = (jc - other * (ymajor ? s : c)) * inv + hn;
    const int lo = max(0, (int)ceilf(uc - hr));
    const int hi = min(a.n - 1, (int)floorf(uc + hr));
    for (int u = lo; u <= hi; ++u) {
      const int ix = ymajor ? u : m, iy = ymajor ? m : u;
      const int2 o = __ldg(orig + (iy >> 5) * a.ntx + (ix >> 5));
      const float sr = rel_coord(__int_as_float(o.y), c, s, (float)(ix & 31), (float)(iy & 31));
      const float fl = floorf(sr);
      const float w = sr - fl;
      const int i = o.x + (int)fl;
      float wt = 0.f;
      if (i == j) wt = WRound<TS>::r(1.f - w);
      else if (i + 1 == j) wt = WRound<TS>::r(w);
      if (wt != 0.f) {
        const float4* p = reinterpret_cast<const float4*>(vol) + (int64_t)m * 4 * a.n + u;
#pragma unroll
        for (int q4 = 0; q4 < 4; ++q4) {
          const float4 v = __ldg(p + (int64_t)q4 * a.n);
          acc[4 * q4] = __fmaf_rn(wt, v.x, acc[4 * q4]);
          acc[4 * q4 + 1] = __fmaf_rn(wt, v.y, acc[4 * q4 + 1]);
          acc[4 * q4 + 2] = __fmaf_rn(wt, v.z, acc[4 * q4 + 2]);
          acc[4 * q4 + 3] = __fmaf_rn(wt, v.w, acc[4 * q4 + 3]);
        }
      }
    }
  }
  TS* out = reinterpret_cast<TS*>(a.sino);
#pragma unroll
  for (int k = 0; k < 16; ++k) Store<TS>::put(out + (int64_t)(z0 + k) * a.s_z + (int64_t)t * a.s_t + j, acc[k]);
}

template <class TV, class TS>
void (*pick(int K, bool full))(PjArgs) {
  switch (K) {
    case 1: return full ? k_project<TV, TS, 1, true> : k_project<TV, TS, 1, false>;
    case 2: return full ? k_project<TV, TS, 2, true> : k_project<TV, TS, 2, false>;
    case 4: return full ? k_project<TV, TS, 4, true> : k_project<TV, TS, 4, false>;
    case 8: return full ? k_project<TV, TS, 8, true> : k_project<TV, TS, 8, false>;
    default: return full ? k_project<TV, TS, 16, true> : k_project<TV, TS, 16, false>;
  }
}

template <class TV>
void (*pick_s(int sdt, int K, bool full))(PjArgs) {
  switch (sdt) {
    case TCP_F32: return pick<TV, float>(K, full);
    case TCP_F16: return pick<TV, __half>(K, full);
    case TCP_BF16: return pick<TV, __nv_bfloat16>(K, full);
  }
  return nullptr;
}

}  // namespace

size_t project_origin_bytes(int64_t ntheta, int64_t n) {
  const int64_t ntx = (n + kTile - 1) / kTile;
  return (size_t)std::max<int64_t>(1, ntheta * ntx * ntx) * sizeof(int2);
}

size_t project_workspace_bytes(int64_t ntheta, int64_t n, int64_t nz, int vol_dtype) {
  const size_t ob = (project_origin_bytes(ntheta, n) + 255) / 256 * 256;
  const size_t tb = ((size_t)std::max<int64_t>(1, nz * n * n) * (vol_dtype == TCP_F32 ? 4 : 2) + 255) / 256 * 256;
  const size_t ib = vol_dtype == TCP_F32 ? (size_t)(nz / 16) * 16 * n * n * 4 : 0;  // two interleaved copies
  return ob + tb + 2 * ib;
}

tcp_status launch_project_ws(const View3& vol, const TrigTable& trig, double center, const View3& sino, void* ws,
                             cudaStream_t st) {
  const int nz = (int)vol.d0, n = (int)vol.d1, nt = (int)sino.d1, nd = (int)sino.d2;
  if (nz == 0 || nt == 0 || nd == 0) return TCP_OK;
  // slices per thread: the candidate search of a (theta, j, step) is shared by K slices
  const int K = nz >= 16 ? 16 : (nz >= 8 ? 8 : (nz >= 4 ? 4 : (nz >= 2 ? 2 : 1)));
  void (*kf)(PjArgs) = nullptr;  // blocks whose K slices all exist
  void (*kt)(PjArgs) = nullptr;  // the ragged last block
  switch (vol.dtype) {
    case TCP_F32: kf = pick_s<float>(sino.dtype, K, true); kt = pick_s<float>(sino.dtype, K, false); break;
    case TCP_F16: kf = pick_s<__half>(sino.dtype, K, true); kt = pick_s<__half>(sino.dtype, K, false); break;
    case TCP_BF16:
      kf = pick_s<__nv_bfloat16>(sino.dtype, K, true);
      kt = pick_s<__nv_bfloat16>(sino.dtype, K, false);
      break;
  }
  if (!kf || !kt) return fail(TCP_ERR_UNSUPPORTED, "project: no kernel for this dtype pair");
  PjArgs a;
  a.vol = vol.p;
  a.v_z = vol.s0;
  a.v_y = vol.s1;
  a.nz = nz;
  a.n = n;
  a.ntx = (n + kTile - 1) / kTile;
  a.sino = sino.p;
  a.s_z = sino.s0;
  a.s_t = sino.s1;
  a.ntheta = nt;
  a.ndet = nd;
  a.trig = trig.dev;
  a.center = center;
  a.half_n = 0.5 * (double)n;
  a.zbase = 0;
  const int nfull = nz / K;
  dim3 grid((unsigned)((nd + 31) / 32), (unsigned)((nt + kPjAngles - 1) / kPjAngles), (unsigned)std::max(nfull, 1));
  if (grid.y > 65535u || grid.z > 65535u)
    return fail(TCP_ERR_SHAPE, "project: too many angles or slice blocks for one launch");
  int2* orig = reinterpret_cast<int2*>(ws);
  void* volT = (char*)ws + (project_origin_bytes(nt, n) + 255) / 256 * 256;
  a.volT = volT;
  // FP32: slice groups of 16 go through the interleaved copies, the rest (if
  // any) through the plain/transposed volume
  const int G = vol.dtype == TCP_F32 ? nz / 16 : 0;
  {
    const size_t tb = ((size_t)nz * n * n * 4 + 255) / 256 * 256;
    float* I0 = (float*)((char*)volT + tb);
    a.volIy = I0;
    a.volIx = I0 + (size_t)G * 16 * n * n;
  }
  // x-major angles read the transposed copy (made unconditionally, so the
  // launch sequence does not depend on the angle set)
  if (n > 0) {
    dim3 tg((unsigned)((n + 31) / 32), (unsigned)((n + 31) / 32), (unsigned)nz);
    switch (vol.dtype) {
      case TCP_F32:
        k_transpose<float><<<tg, dim3(32, 8), 0, st>>>((const float*)vol.p, vol.s0, vol.s1, n, (float*)volT);
        break;
      case TCP_F16:
        k_transpose<__half><<<tg, dim3(32, 8), 0, st>>>((const __half*)vol.p, vol.s0, vol.s1, n, (__half*)volT);
        break;
      case TCP_BF16:
        k_transpose<__nv_bfloat16><<<tg, dim3(32, 8), 0, st>>>((const __nv_bfloat16*)vol.p, vol.s0, vol.s1, n,
                                                               (__nv_bfloat16*)volT);
        break;
    }
    TCP_CUDA_TRY(cudaGetLastError());
  }
  if (n > 0) {
    const int64_t total = (int64_t)nt * a.ntx * a.ntx;
    const int blocks = (int)std::min<int64_t>((total + 255) / 256, 4096);
    k_origin_table<<<blocks, 256, 0, st>>>(trig.dev, nt, a.ntx, a.half_n, center, orig);
  }
  a.orig = orig;
  if (G > 0) {
    const int64_t total = (int64_t)G * n * n;
    const int blocks = (int)std::min<int64_t>((total + 255) / 256, 8192);
    k_interleave16<<<blocks, 256, 0, st>>>((const float*)vol.p, vol.s0, vol.s1, n, G, (float*)a.volIy);
    k_interleave16<<<blocks, 256, 0, st>>>((const float*)volT, (int64_t)n * n, n, n, G, (float*)a.volIx);
    void (*ki)(PjArgs) = nullptr;
    switch (sino.dtype) {
      case TCP_F32: ki = k_project_i16<float>; break;
      case TCP_F16: ki = k_project_i16<__half>; break;
      case TCP_BF16: ki = k_project_i16<__nv_bfloat16>; break;
    }
    if (!ki) return fail(TCP_ERR_UNSUPPORTED, "project: no kernel for this dtype pair");
    dim3 gi(grid.x, grid.y, (unsigned)G);
    if (gi.z > 65535u) return fail(TCP_ERR_SHAPE, "project: too many slice groups for one launch");
    ki<<<gi, kPjThreads, 0, st>>>(a);
    TCP_CUDA_TRY(cudaGetLastError());
    if (nz == 16 * G) return TCP_OK;
    // the remaining slices by the plain kernel
    a.zbase = 16 * G;
    const int rem = nz - 16 * G;
    const int K2 = rem >= 8 ? 8 : (rem >= 4 ? 4 : (rem >= 2 ? 2 : 1));
    void (*k2f)(PjArgs) = pick_s<float>(sino.dtype, K2, true);
    void (*k2t)(PjArgs) = pick_s<float>(sino.dtype, K2, false);
    const int nf2 = rem / K2;
    if (nf2 > 0) {
      dim3 g2(grid.x, grid.y, (unsigned)nf2);
      k2f<<<g2, kPjThreads, 0, st>>>(a);
      TCP_CUDA_TRY(cudaGetLastError());
    }
    if (rem % K2) {
      a.zbase = 16 * G + nf2 * K2;
      dim3 g3(grid.x, grid.y, 1);
      k2t<<<g3, kPjThreads, 0, st>>>(a);
      TCP_CUDA_TRY(cudaGetLastError());
    }
    return TCP_OK;
  }
  if (nfull > 0) {
    kf<<<grid, kPjThreads, 0, st>>>(a);
    TCP_CUDA_TRY(cudaGetLastError());
  }
  if (nz % K) {
    a.zbase = nfull * K;
    grid.z = 1;
    kt<<<grid, kPjThreads, 0, st>>>(a);
    TCP_CUDA_TRY(cudaGetLastError());
  }
  return TCP_OK;
}

tcp_status launch_project(const View3& vol, const TrigTable& trig, double center, const View3& sino,
                          cudaStream_t st) {
  if (vol.d0 == 0 || sino.d1 == 0 || sino.d2 == 0) return TCP_OK;
  void* ws = nullptr;
  TCP_CUDA_TRY(cudaMallocAsync(&ws, project_workspace_bytes(sino.d1, vol.d1, vol.d0, vol.dtype), st));
  const tcp_status s = launch_project_ws(vol, trig, center, sino, ws, st);
  const cudaError_t e = cudaFreeAsync(ws, st);
  if (s == TCP_OK && e != cudaSuccess) return cuda_fail(e, "cudaFreeAsync");
  return s;
}

}  // namespace tcp
