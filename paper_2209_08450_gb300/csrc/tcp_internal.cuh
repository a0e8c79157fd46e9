// Internal declarations shared by the CUDA translation units of libtcp.
// Geometry conventions are those of include/tcp.h.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <string>
#include <type_traits>
#include <vector>

#include "tcp.h"

namespace tcp {

// ------------------------------------------------------------------ errors --

// Device error word: kernels OR bits into it instead of trapping.
enum : uint32_t {
  kErrBpWindow = 1u << 0,     // backprojector window index out of range
  kErrPjCandidate = 1u << 1,  // projector candidate outside the volume
  kErrFilterIndex = 1u << 2,  // filter shared-memory index out of range
  kErrTimeout = 1u << 3,      // bounded wait gave up
  kErrBatchItem = 1u << 4,    // batched work item out of range
};

uint32_t* device_error_word();  // device address of the word (current device)

void set_error(const std::string& msg);
tcp_status fail(tcp_status s, const std::string& msg);
tcp_status cuda_fail(cudaError_t e, const char* what);

#define TCP_CUDA_TRY(expr)                               \
  do {                                                   \
    cudaError_t e_ = (expr);                             \
    if (e_ != cudaSuccess) return cuda_fail(e_, #expr);  \
  } while (0)

bool checked_mode();

// Host-side checks shared by the entry points: a tensor descriptor (non-null,
// ndim in [lo, hi], known dtype, non-negative extents, unit innermost stride,
// data aligned to its dtype), and whether two tensors' byte ranges overlap.
tcp_status check_tensor(const tcp_tensor* t, const char* name, int ndim_lo, int ndim_hi);
bool overlap(const tcp_tensor* a, const tcp_tensor* b);

// ----------------------------------------------------------------- dtypes --

template <class T> struct Store;
template <> struct Store<float> {
  static __device__ __forceinline__ float load(const float* p) { return __ldg(p); }
  static __device__ __forceinline__ void put(float* p, float v) { *p = v; }
};
template <> struct Store<__half> {
  static __device__ __forceinline__ float load(const __half* p) { return __half2float(__ldg(p)); }
  static __device__ __forceinline__ void put(__half* p, float v) { *p = __float2half_rn(v); }
};
template <> struct Store<__nv_bfloat16> {
  static __device__ __forceinline__ float load(const __nv_bfloat16* p) {
    return __bfloat162float(__ldg(p));
  }
  static __device__ __forceinline__ void put(__nv_bfloat16* p, float v) { *p = __float2bfloat16_rn(v); }
};

// ------------------------------------------------------ normalisation math --

// Dark/flat correction and negative logarithm in FP32 (Sec. 2.2):
// r = (raw - dark)/(flat - dark), r <- 1e-6 unless finite and > 1e-6, -ln r.
__device__ __forceinline__ float neglog_ratio(float raw, float d, float f) {
  float r = (raw - d) / (f - d);
  if (!(r > 1e-6f) || isinf(r)) r = 1e-6f;
  return -logf(r);
}

// ------------------------------------------------- canonical ray geometry --
//
// The ray coordinate of voxel (ix, iy) at angle theta is
//   s = (ix - n/2) cos + (iy - n/2) sin + center.
// It is evaluated as an FP64 origin per aligned 32x32 voxel tile, split into an
// integer part and an FP32 fraction, plus FP32 in-tile offsets.  Both the
// backprojector and the projector call exactly these functions (explicit
// rounding intrinsics, no contraction freedom), so the two operators use
// bit-identical weights and are exact transposes of each other.

constexpr int kTile = 32;

struct TileOrigin {
  int i0;    // floor of the tile-origin ray coordinate
  float f0;  // fractional part in [0, 1]
  float c;   // cos(theta) rounded to FP32
  float s;   // sin(theta) rounded to FP32
};

__device__ __forceinline__ TileOrigin tile_origin(int gx, int gy, double half_n, double center,
                                                  double2 cs) {
  const double X0 = __dsub_rn((double)(gx * kTile), half_n);
  const double Y0 = __dsub_rn((double)(gy * kTile), half_n);
  const double S0 = __fma_rn(X0, cs.x, __fma_rn(Y0, cs.y, center));
  const double fl = floor(S0);
  TileOrigin o;
  o.i0 = (int)fl;
  o.f0 = __double2float_rn(__dsub_rn(S0, fl));
  o.c = __double2float_rn(cs.x);
  o.s = __double2float_rn(cs.y);
  return o;
}

// In-tile ray coordinate relative to i0 for offsets (dx, dy) in [0, 32).
__device__ __forceinline__ float rel_coord(float f0, float c, float s, float dx, float dy) {
  return __fmaf_rn(dy, s, __fmaf_rn(dx, c, f0));
}

// ------------------------------------------------------------- host side --

struct TrigTable {
  const double2* dev = nullptr;  // (cos, sin) per angle, FP64
  int64_t n = 0;
};
// Cached FP64 cos/sin table for a host angle array (first use uploads it).
tcp_status get_trig_table(const double* theta, int64_t n, TrigTable* out);
// The same table in memory owned by the caller (appended to `owned`).
tcp_status build_trig_owned(const double* theta, int64_t n, std::vector<void*>* owned, TrigTable* out);

struct FilterTable {
  const float2* response = nullptr;  // npad/2+1 complex factors (incl. 1/npad)
  // Two-level twiddles: [0, 64): exp(-2 pi i l / npad), l < 64; then
  // [64, 64 + max(1, npad / 64)): exp(-2 pi i 64 h / npad).  W^m is the
  // product of entries m % 64 and 64 + m / 64.
  const float2* twiddle = nullptr;
  int npad = 0;
};
// weight multiplies the response (pi/N_theta for FBP; any value > 0).
tcp_status get_filter_table(int64_t ndet, int32_t filter, double weight, double center, FilterTable* out,
                            bool smooth = false);
// The same response and twiddles in memory owned by the caller.
tcp_status build_filter_owned(int64_t ndet, int32_t filter, double weight, double center, bool smooth,
                              std::vector<void*>* owned, FilterTable* out);
// pad_mode: bit 0 zero padding (else edge), bit 1 smooth padded length
inline bool valid_pad_mode(int32_t m) { return m >= 0 && m <= (TCP_PAD_ZERO | TCP_PAD_SMOOTH); }
inline bool pad_smooth(int32_t m) { return (m & TCP_PAD_SMOOTH) != 0; }

// Storage scale of a sinogram that the library writes in `dtype` and reads
// back itself (pipeline, batch): FP16 keeps a 2^10 headroom so that filtered
// values stay out of the subnormal range (|filtered -log| <= 6.9 < 65504/2^10).
inline double storage_scale(int dtype) { return (dtype == TCP_F16 || dtype == TCP_F16X2) ? 1024.0 : 1.0; }

int64_t padded_length(int64_t ndet, bool smooth = false);

// Launchers (argument checks are done by the API layer).
struct View3 {  // [d0][d1][d2] with element strides s0, s1 (s2 == 1)
  void* p;
  int dtype;
  int64_t d0, d1, d2;
  int64_t s0, s1;
  int64_t plane = 0;  // TCP_F16X2: elements from the hi plane to the lo plane
};

tcp_status launch_frame_mean(const View3& frames, const View3& mean, cudaStream_t st);
tcp_status launch_normalize(const View3& raw, const View3& dark, const View3& flat, const View3& sino,
                            cudaStream_t st);
tcp_status launch_filter(const View3& sino, const FilterTable& ft, int pad_mode, cudaStream_t st);
tcp_status launch_normalize_filter(const View3& raw, const View3& dark, const View3& flat, const View3& sino,
                                   const FilterTable& ft, int pad_mode, cudaStream_t st);
tcp_status launch_backproject(const View3& sino, const TrigTable& trig, double center, const View3& vol,
                              const tcp_bp_config& cfg, cudaStream_t st, float scale = 1.0f);
tcp_status launch_project(const View3& vol, const TrigTable& trig, double center, const View3& sino,
                          cudaStream_t st);
// The projector with its per-call workspace (the tile-origin table, ntheta x
// ntx^2 int2, then the transposed volume) in caller-provided device memory of
// project_workspace_bytes.
size_t project_origin_bytes(int64_t ntheta, int64_t n);
size_t project_workspace_bytes(int64_t ntheta, int64_t n, int64_t nz, int vol_dtype);
tcp_status launch_project_ws(const View3& vol, const TrigTable& trig, double center, const View3& sino, void* ws,
                             cudaStream_t st);
// FourierRec (k_fourierrec.cu): default window width per volume dtype, the
// shape/width checks, and the launcher (sino F32/F16/BF16, vol F32/F16/BF16).
int64_t fourierrec_grid(int64_t n);  // Cartesian grid side L
int fourierrec_default_width(int vol_dtype, int64_t n);  // clamped to the grid size
void fourierrec_cache_clear();  // frees the cached twiddle, deconvolution and angle tables
tcp_status fourierrec_check(int64_t ntheta, int64_t ndet, int64_t n, int width);
tcp_status launch_fourierrec(const View3& sino, const double* theta, const TrigTable& trig, double center,
                             const View3& vol, float scale, int width, cudaStream_t st);
// The same split into tables (twiddles of the row and grid lengths, 1/Phi
// deconvolution factors, angles folded to [0, pi) and sorted) and a
// workspace (geometry, centre phase, spectra P, half-transformed H, grid G
// for nb slice pairs), so that a plan can own both.
struct FrecTables {
  const float2 *twM = nullptr, *twL = nullptr;
  const float* dec = nullptr;
  const int2* meta = nullptr;
  const float* thS = nullptr;
  const int2* order = nullptr;  // gather tiles, nearest to the zero frequency first
  // near-node sparse table (t_near = 0: none, the gather does those nodes):
  // rows of the first t_near tiles of `order`, 4096 per tile
  int t_near = 0;
  const int64_t* near_off = nullptr;  // row starts, t_near * 4096 + 1
  const int2* near_ent = nullptr;     // (P offset, weight bits)
  int64_t n_heavy = 0;                // rows with more than 4096 entries, one CTA each
  const int64_t* near_heavy = nullptr;
  const unsigned char* near_warps = nullptr;  // near flag per gather warp (512 rows each)
};
struct FrecWorkspace {
  void *geom = nullptr, *phase = nullptr, *P = nullptr, *H = nullptr, *G = nullptr;
  int nb = 1;  // slice pairs per batch
};
size_t fourierrec_workspace_bytes(int64_t nt, int64_t nd, int64_t n, int64_t nz, int* nb);
FrecWorkspace fourierrec_workspace(void* base, int64_t nt, int64_t nd, int64_t n, int64_t nz);
tcp_status fourierrec_tables_cached(const double* theta, int64_t nt, int64_t nd, int64_t n, int width,
                                    FrecTables* t);
tcp_status fourierrec_tables_owned(const double* theta, int64_t nt, int64_t nd, int64_t n, int width,
                                   std::vector<void*>* owned, FrecTables* t);
tcp_status launch_fourierrec_ws(const View3& sv, const FrecTables& tb, const FrecWorkspace& w, const TrigTable& trig,
                                double center, const View3& vv, float scale, int width, cudaStream_t st);

// Arguments of one backprojection (one dataset of a batch).
struct BpArgs {
  const void* sino;
  int64_t s_z, s_t;  // sinogram strides (elements)
  int nz, ntheta, ndet;
  void* vol;
  int64_t v_z, v_y;  // volume strides (elements)
  int n;
  int ntx;  // tiles along x (and y)
  const double2* trig;
  double center, half_n;
  float scale;  // multiplies every output voxel (1 for the plain sum)
  uint32_t* err;
};

// Work list of the persistent backprojector.
struct BpWork {
  const BpArgs* items;            // device array [nitems]
  const long long* prefix;        // device array [nitems + 1], prefix sums of units
  int nitems;
  unsigned long long* counter;    // zeroed before each launch
};

bool tc_eligible(const View3& sino);
// Launch shape of the tensor-core backprojector for nz slices: slices per
// block N, angles per stage S, blocks per SM, weight (na) and sinogram (nbb)
// ring depths, dynamic shared memory per block.  False if no ring fits.
struct TcShape {
  int N = 0, S = 0, blocks = 0, na = 0, nbb = 0;
  size_t smem = 0;
};
bool tc_shape(int64_t nz, bool split, int theta_stage, int blocks_per_sm, TcShape* sh);
// theta_stage: angles per pipeline stage (1 or 2; split mode always 1);
// blocks_per_sm: 2 sizes the shared-memory rings for two blocks per SM
// (16-bit sinograms, at most 128 slices per block), else one block.
tcp_status launch_backproject_tc(const View3& sino, const TrigTable& trig, double center, const View3& vol,
                                 float scale, int theta_stage, int blocks_per_sm, cudaStream_t st);

BpArgs make_bp_args(const View3& sino, const TrigTable& trig, double center, const View3& vol, float scale = 1.0f);
int bp_threads(const tcp_bp_config& c);
tcp_status bp_persistent_grid(int sdt, int vdt, const tcp_bp_config& cfg, int* blocks);
tcp_status launch_backproject_persistent(const BpWork& w, int sdt, int vdt, const tcp_bp_config& cfg, int blocks,
                                         cudaStream_t st);

// LpRec (k_lprec.cu): host geometry of the three angle spans (FP64), its
// device tables, the workspace of one call and the launcher.
struct LpHostSpan {
  int j0 = 0, nu = 0, p = 1, nrho = 0, npsi = 0, kpsi = 0, ext = 0, ntau = 0;
  double phi = 0, ox = 0, oy = 0, rho0 = 0, tau0 = 0, drho = 0, dpsi = 0, psi0 = 0;
  std::vector<int2> esplit, shsplit;  // (floor, FP32 fraction bits)
  std::vector<int> dbase;
  std::vector<float4> dw;
};
struct LpHostGeom {
  int64_t nt = 0, nd = 0, n = 0;
  double os = 2.0;
  LpHostSpan span[3];
};
struct LpDevGeom {
  const int2* esplit[3] = {};
  const int2* shsplit[3] = {};
  const int* dbase[3] = {};
  const float4* dw[3] = {};
};
tcp_status lprec_geometry(const double* theta, int64_t nt, int64_t nd, int64_t n, double center, double os,
                          LpHostGeom* g);
tcp_status lprec_check(const LpHostGeom& g);
int lprec_slices_per_pass(const LpHostGeom& g, int64_t nz);
size_t lprec_workspace_bytes(const LpHostGeom& g, int zpass);
tcp_status lprec_upload(const LpHostGeom& g, std::vector<void*>* owned, LpDevGeom* d, cudaStream_t st, bool async);
tcp_status lprec_cached(const double* theta, int64_t nt, int64_t nd, int64_t n, double center, double os,
                        const LpHostGeom** g, const LpDevGeom** d);
void lprec_cache_clear();
tcp_status launch_lprec_ws(const View3& sv, const LpHostGeom& g, const LpDevGeom& d, void* ws, int zpass,
                           const View3& vv, float scale, cudaStream_t st);

// ------------------------------------------------ chunked FBP (pipeline.cu) --

// Resolved options of one chunked FBP.
struct FbpParams {
  int64_t nt = 0, nz = 0, nd = 0, n = 0;
  int vdt = TCP_F32, sdt = TCP_F32;
  bool frec = false;
  bool lprec = false;
  int width = 0;       // FourierRec window width
  double os = 2.0;     // LpRec oversampling
  int64_t chunk = 0, cz = 0;  // requested chunk depth, and the deepest chunk of this run
  int B = 2;                  // ring depth for host buffers
  int filter = 0, pad = 0;
  double sscale = 1.0;        // storage scale of the filtered sinogram
  float bp_scale = 1.f;       // pi / ntheta / sscale, applied at the voxel store
  tcp_bp_config cfg{};
};
// Device resources of one chunked FBP: tables, workspace, ring buffers,
// copy streams and events (from a plan, or taken for one call).
struct FbpRes {
  TrigTable trig;
  FilterTable ft;
  FrecTables frt;
  FrecWorkspace fws;
  const LpHostGeom* lpg = nullptr;  // LpRec geometry (host copy) and its tables
  LpDevGeom lpd;
  void* lpws = nullptr;             // LpRec workspace for passes of lpz slices
  int lpz = 1;
  void* sino = nullptr;  // chunk sinogram buffer
  int64_t sino_cz = 0;   // slices it holds (F16X2: the distance between the planes)
  void* rring[3] = {nullptr, nullptr, nullptr};
  void* vring[3] = {nullptr, nullptr, nullptr};
  cudaStream_t cin = nullptr, cout = nullptr;
  cudaEvent_t raw_ready[3] = {}, raw_free[3] = {}, vol_ready[3] = {}, vol_free[3] = {};
  cudaEvent_t fork = nullptr, join_in = nullptr, join_out = nullptr;
  // optional per-chunk timeline: t0, then per chunk 6 timing events (upload
  // start/end, compute start/end, download start/end); `traced` chunks of the
  // last run, `ntrace` chunks of room
  cudaEvent_t* trace = nullptr;
  int ntrace = 0;
  int* traced = nullptr;
  int* trace_flags = nullptr;  // per chunk: bit 0 upload recorded, bit 1 download recorded
};
tcp_status fbp_resolve(const tcp_tensor* raw, const tcp_tensor* vol, const tcp_fbp_opts* opts, FbpParams* p);
tcp_status fbp_resolve_shape(int64_t nt, int64_t nz, int64_t nd, int64_t n, int vdt, const tcp_fbp_opts* opts,
                             FbpParams* p);
// dm/fm: FP32 means [nz][nd] on the device.
tcp_status fbp_run(const FbpParams& p, const FbpRes& r, const View3& dm, const View3& fm, const tcp_tensor* raw,
                   tcp_tensor* vol, bool host_raw, bool host_vol, cudaStream_t st);
bool is_device_ptr(const void* p);
bool is_pinned_ptr(const void* p);

bool tuned_bp_config(int64_t nz, int64_t nt, int64_t nd, int64_t n, int sdt, int vdt, tcp_bp_config* cfg);
tcp_bp_config bp_override();
tcp_bp_config default_bp_config(int64_t nz, int64_t ntheta, int64_t ndet, int64_t n, int sdt, int vdt);
bool valid_bp_config(const tcp_bp_config& c);

}  // namespace tcp
