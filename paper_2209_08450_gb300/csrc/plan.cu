// Reconstruction plans: everything one geometry needs besides the caller's
// buffers, allocated and uploaded once (Sec. 2.2 of the TomocuPy paper: the
// transforms and their memory are set up at start, the chunks then only
// run).  A plan owns the FP64 angle table, the filter responses and FFT
// twiddles, the FourierRec tables and workspace, the projector's tile-origin
// table, the frame-mean buffers, the chunk sinogram buffer and, for host
// input or output, the staging rings with their copy streams and events.
// Calls that take a plan allocate nothing, never synchronise and only
// enqueue work, so their first use may be captured into a CUDA graph.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <cmath>
#include <mutex>
#include <vector>

#include "tcp_internal.cuh"

struct tcp_plan {
  int dev = 0;
  tcp_plan_desc d{};
  tcp::FbpParams p;
  tcp::FbpRes r;
  tcp::FilterTable ft_pi;  // response with the pi/ntheta weight (tcp_filter_plan)
  std::vector<double> theta;
  std::vector<void*> owned;
  std::vector<cudaEvent_t> events;
  std::vector<cudaStream_t> streams;
  float* means = nullptr;       // [2][nz][ndet] FP32: dark, then flat
  void* frames = nullptr;       // staging of host U16 frames: host_frames x nz x ndet
  void* proj_orig = nullptr;    // projector workspace: tile origins and the transposed volume
  void* frec_ws = nullptr;      // FourierRec workspace
  tcp::LpHostGeom lpg;          // LpRec geometry (host copy; its tables are in `owned`)
  size_t bytes = 0;
  std::vector<cudaEvent_t> trace_events;  // timing events of the per-chunk timeline
  std::vector<int> trace_flags;
  int traced = 0;
  ~tcp_plan() {
    for (cudaEvent_t e : trace_events) cudaEventDestroy(e);
    for (void* q : owned) cudaFree(q);
    for (cudaEvent_t e : events) cudaEventDestroy(e);
    for (cudaStream_t s : streams) cudaStreamDestroy(s);
  }
};

namespace tcp {
namespace {

int esz(int dt) { return (dt == TCP_F32 || dt == TCP_F16X2) ? 4 : 2; }  // F16X2: both planes

tcp_status plan_alloc(tcp_plan* pl, void** q, size_t bytes) {
  const cudaError_t e = cudaMalloc(q, bytes ? bytes : 16);
  if (e != cudaSuccess) return cuda_fail(e, "plan: cudaMalloc");
  pl->owned.push_back(*q);
  pl->bytes += bytes;
  return TCP_OK;
}

tcp_status plan_event(tcp_plan* pl, cudaEvent_t* e) {
  const cudaError_t r = cudaEventCreateWithFlags(e, cudaEventDisableTiming);
  if (r != cudaSuccess) return cuda_fail(r, "plan: cudaEventCreate");
  pl->events.push_back(*e);
  return TCP_OK;
}

tcp_status plan_stream(tcp_plan* pl, cudaStream_t* s) {
  const cudaError_t r = cudaStreamCreateWithFlags(s, cudaStreamNonBlocking);
  if (r != cudaSuccess) return cuda_fail(r, "plan: cudaStreamCreate");
  pl->streams.push_back(*s);
  return TCP_OK;
}

// Bytes of the device allocations in `owned` (each pointer starts one
// cudaMalloc allocation), from the driver's address ranges; 0 where the entry
// point is unavailable.
size_t owned_bytes(const std::vector<void*>& owned) {
  static std::once_flag once;
  static PFN_cuMemGetAddressRange_v3020 range = nullptr;
  std::call_once(once, [] {
    cudaDriverEntryPointQueryResult q;
    void* f = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuMemGetAddressRange", &f, 3020, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      range = reinterpret_cast<PFN_cuMemGetAddressRange_v3020>(f);
  });
  size_t total = 0;
  if (!range) return 0;
  for (void* p : owned) {
    CUdeviceptr base = 0;
    size_t size = 0;
    if (p && range(&base, &size, (CUdeviceptr)p) == CUDA_SUCCESS) total += size;
  }
  return total;
}

#define PTRY(x)                    \
  do {                             \
    tcp_status s_ = (x);           \
    if (s_ != TCP_OK) return s_;   \
  } while (0)

tcp_status plan_build(tcp_plan* pl, const double* theta) {
  const tcp_plan_desc& d = pl->d;
  FbpParams& p = pl->p;
  FbpRes& r = pl->r;
  PTRY(fbp_resolve_shape(d.ntheta, d.nz, d.ndet, d.n, d.vol_dtype, &d.opts, &p));
  const int64_t nt = p.nt, nd = p.nd, n = p.n, nz = p.nz;
  pl->owned.reserve(32);
  // tables
  PTRY(build_trig_owned(theta, nt, &pl->owned, &r.trig));
  PTRY(build_filter_owned(nd, p.filter, p.sscale, d.center, pad_smooth(p.pad), &pl->owned, &r.ft));
  PTRY(build_filter_owned(nd, p.filter, nt > 0 ? M_PI / (double)nt : 1.0, d.center, pad_smooth(p.pad), &pl->owned,
                          &pl->ft_pi));
  if (p.frec) {
    PTRY(fourierrec_tables_owned(theta, nt, nd, n, p.width, &pl->owned, &r.frt));
    PTRY(plan_alloc(pl, &pl->frec_ws, fourierrec_workspace_bytes(nt, nd, n, p.cz, nullptr)));
    r.fws = fourierrec_workspace(pl->frec_ws, nt, nd, n, p.cz);
  }
  if (p.lprec) {  // the filter moves the axis to ndet/2
    PTRY(lprec_geometry(theta, nt, nd, n, 0.5 * (double)nd, p.os, &pl->lpg));
    PTRY(lprec_check(pl->lpg));
    PTRY(lprec_upload(pl->lpg, &pl->owned, &r.lpd, nullptr, false));
    r.lpg = &pl->lpg;
    r.lpz = lprec_slices_per_pass(pl->lpg, p.cz);
    PTRY(plan_alloc(pl, &r.lpws, lprec_workspace_bytes(pl->lpg, r.lpz)));
  }
  // buffers
  void* m = nullptr;
  PTRY(plan_alloc(pl, &m, sizeof(float) * 2 * (size_t)std::max<int64_t>(1, nz * nd)));
  pl->means = (float*)m;
  if (d.host_frames > 0) PTRY(plan_alloc(pl, &pl->frames, (size_t)d.host_frames * nz * nd * 2));
  PTRY(plan_alloc(pl, &pl->proj_orig, project_workspace_bytes(nt, n, nz, TCP_F32)));
  PTRY(plan_alloc(pl, &r.sino, (size_t)p.cz * nt * nd * esz(p.sdt)));
  r.sino_cz = p.cz;
  if (d.io & TCP_IO_HOST_RAW) {
    PTRY(plan_stream(pl, &r.cin));
    for (int b = 0; b < p.B; ++b) {
      PTRY(plan_alloc(pl, &r.rring[b], (size_t)nt * p.cz * nd * 2));
      PTRY(plan_event(pl, &r.raw_ready[b]));
      PTRY(plan_event(pl, &r.raw_free[b]));
    }
    PTRY(plan_event(pl, &r.join_in));
  }
  if (d.io & TCP_IO_HOST_VOL) {
    PTRY(plan_stream(pl, &r.cout));
    for (int b = 0; b < p.B; ++b) {
      PTRY(plan_alloc(pl, &r.vring[b], (size_t)p.cz * n * n * esz(p.vdt)));
      PTRY(plan_event(pl, &r.vol_ready[b]));
      PTRY(plan_event(pl, &r.vol_free[b]));
    }
    PTRY(plan_event(pl, &r.join_out));
  }
  PTRY(plan_event(pl, &r.fork));
  if (d.trace) {  // timing events for the per-chunk timeline
    const int maxc = (int)((nz + p.chunk - 1) / p.chunk) + 2;
    pl->trace_events.resize((size_t)(1 + 6 * maxc), nullptr);
    for (auto& e : pl->trace_events) TCP_CUDA_TRY(cudaEventCreate(&e));
    pl->trace_flags.assign((size_t)maxc, 0);
    r.trace = pl->trace_events.data();
    r.ntrace = maxc;
    r.traced = &pl->traced;
    r.trace_flags = pl->trace_flags.data();
  }
  // the device error word's address is looked up here, not during a capture
  if (!device_error_word()) return fail(TCP_ERR_CUDA, "plan: device error word unavailable");
  TCP_CUDA_TRY(cudaDeviceSynchronize());
  // every device allocation of the plan, its buffers (counted as they were
  // made) and its tables (angles, filters, FourierRec and LpRec geometry)
  const size_t all = owned_bytes(pl->owned);
  if (all > pl->bytes) pl->bytes = all;
  return TCP_OK;
}

// FP32 means of dark or flat (`slot` 0 or 1) for slices [0, nz) of the plan.
tcp_status plan_means(tcp_plan* pl, const tcp_tensor* t, int slot, int64_t nz, cudaStream_t st, View3* out) {
  const int64_t nd = pl->p.nd;
  float* dst = pl->means + (size_t)slot * pl->p.nz * nd;
  View3 mv;
  mv.p = dst; mv.dtype = TCP_F32; mv.d0 = 1; mv.d1 = nz; mv.d2 = nd; mv.s0 = 0; mv.s1 = nd;
  const bool dev = is_device_ptr(t->data);
  if (t->ndim == 2) {  // F32 means
    if (dev) {
      View3 v;
      v.p = t->data; v.dtype = TCP_F32; v.d0 = 1; v.d1 = nz; v.d2 = nd; v.s0 = 0; v.s1 = t->stride[0];
      *out = v;
      return TCP_OK;
    }
    TCP_CUDA_TRY(cudaMemcpy2DAsync(dst, (size_t)nd * 4, t->data, (size_t)t->stride[0] * 4, (size_t)nd * 4, (size_t)nz,
                                   cudaMemcpyHostToDevice, st));
    *out = mv;
    return TCP_OK;
  }
  View3 v;  // U16 frames
  v.dtype = TCP_U16; v.d0 = t->shape[0]; v.d1 = nz; v.d2 = nd;
  if (dev) {
    v.p = t->data; v.s0 = t->stride[0]; v.s1 = t->stride[1];
  } else {
    if (t->shape[0] > pl->d.host_frames)
      return fail(TCP_ERR_ARG, "plan: " + std::to_string(t->shape[0]) + " host frames exceed the plan's staging of " +
                                   std::to_string(pl->d.host_frames) + " (tcp_plan_desc.host_frames)");
    for (int64_t f = 0; f < t->shape[0]; ++f)
      TCP_CUDA_TRY(cudaMemcpy2DAsync((char*)pl->frames + (size_t)f * nz * nd * 2, (size_t)nd * 2,
                                     (const char*)t->data + (size_t)f * t->stride[0] * 2, (size_t)t->stride[1] * 2,
                                     (size_t)nd * 2, (size_t)nz, cudaMemcpyHostToDevice, st));
    v.p = pl->frames; v.s0 = nz * nd; v.s1 = nd;
  }
  PTRY(launch_frame_mean(v, mv, st));
  *out = mv;
  return TCP_OK;
}

View3 view_of(const tcp_tensor* t) {
  View3 v;
  v.p = t->data;
  v.dtype = t->dtype;
  v.d0 = t->shape[0];
  v.d1 = t->shape[1];
  v.d2 = t->shape[2];
  v.s0 = t->stride[0];
  v.s1 = t->stride[1];
  return v;
}

bool is_float_dt(int dt) { return dt == TCP_F32 || dt == TCP_F16 || dt == TCP_BF16; }

}  // namespace
}  // namespace tcp

using namespace tcp;

extern "C" {

tcp_status tcp_plan_create(const tcp_plan_desc* desc, const double* theta, tcp_plan** out) {
  if (!out) return fail(TCP_ERR_ARG, "plan: null output handle");
  *out = nullptr;
  if (!desc) return fail(TCP_ERR_ARG, "plan: null description");
  tcp_plan_desc d = *desc;
  if (d.n <= 0) d.n = d.ndet;
  if (d.ntheta < 1 || d.nz < 1 || d.ndet < 1 || d.n < 1)
    return fail(TCP_ERR_SHAPE, "plan: ntheta, nz, ndet and n must be positive");
  if (d.ntheta > INT32_MAX || d.nz > INT32_MAX || d.n > INT32_MAX)
    return fail(TCP_ERR_SHAPE, "plan: extent too large");
  if (!is_float_dt(d.vol_dtype)) return fail(TCP_ERR_DTYPE, "plan: vol_dtype must be F32, F16 or BF16");
  if (d.io & ~(TCP_IO_HOST_RAW | TCP_IO_HOST_VOL)) return fail(TCP_ERR_ARG, "plan: unknown io flags");
  if (d.host_frames < 0) return fail(TCP_ERR_ARG, "plan: host_frames must be >= 0");
  if (!std::isfinite(d.center)) return fail(TCP_ERR_ARG, "plan: center must be finite");
  if (!theta) return fail(TCP_ERR_ARG, "plan: theta is null");
  for (int64_t i = 0; i < d.ntheta; ++i)
    if (!std::isfinite(theta[i])) return fail(TCP_ERR_ARG, "plan: theta must be finite");
  auto* pl = new tcp_plan();
  pl->d = d;
  pl->theta.assign(theta, theta + d.ntheta);
  cudaError_t e = cudaGetDevice(&pl->dev);
  tcp_status s = e == cudaSuccess ? plan_build(pl, theta) : cuda_fail(e, "cudaGetDevice");
  if (s != TCP_OK) {
    cudaDeviceSynchronize();
    delete pl;
    return s;
  }
  *out = pl;
  return TCP_OK;
}

tcp_status tcp_plan_destroy(tcp_plan* plan) {
  if (!plan) return TCP_OK;
  int cur = 0;
  cudaGetDevice(&cur);
  if (cur != plan->dev) cudaSetDevice(plan->dev);
  const cudaError_t e = cudaDeviceSynchronize();
  const int pdev = plan->dev;
  delete plan;
  if (cur != pdev) cudaSetDevice(cur);
  if (e != cudaSuccess) return cuda_fail(e, "plan: cudaDeviceSynchronize");
  return TCP_OK;
}

tcp_status tcp_plan_info(const tcp_plan* plan, int64_t* device_bytes, tcp_fbp_opts* resolved) {
  if (!plan) return fail(TCP_ERR_ARG, "plan: null handle");
  if (device_bytes) *device_bytes = (int64_t)plan->bytes;
  if (resolved) {
    tcp_fbp_opts o = plan->d.opts;
    o.chunk_nz = (int32_t)plan->p.chunk;
    o.sino_dtype = plan->p.sdt;
    o.n_buffers = plan->p.B;
    o.width = plan->p.frec ? plan->p.width : 0;
    *resolved = o;
  }
  return TCP_OK;
}

tcp_status tcp_plan_trace(const tcp_plan* plan, double* ms, int64_t cap, int64_t* count) {
  if (!plan) return fail(TCP_ERR_ARG, "plan_trace: null plan");
  if (!plan->d.trace) return fail(TCP_ERR_ARG, "plan_trace: the plan was created without trace");
  const int nch = plan->traced;
  if (count) *count = nch;
  if (nch == 0 || !ms) return TCP_OK;
  const cudaEvent_t* e = plan->trace_events.data();
  TCP_CUDA_TRY(cudaEventSynchronize(e[1 + 6 * (nch - 1) + 3]));
  for (int k = 0; k < nch && k < cap; ++k) {
    const int fl = plan->trace_flags[(size_t)k];
    for (int w = 0; w < 6; ++w) {
      double v = -1.0;
      const bool have = (w >= 2 && w < 4) || (w < 2 && (fl & 1)) || (w >= 4 && (fl & 2));
      if (have) {
        TCP_CUDA_TRY(cudaEventSynchronize(e[1 + 6 * k + w]));
        float t = 0.f;
        TCP_CUDA_TRY(cudaEventElapsedTime(&t, e[0], e[1 + 6 * k + w]));
        v = t;
      }
      ms[6 * k + w] = v;
    }
  }
  return TCP_OK;
}

tcp_status tcp_fbp_plan(tcp_plan* plan, const tcp_tensor* raw, const tcp_tensor* dark, const tcp_tensor* flat,
                        tcp_tensor* vol, void* stream) {
  if (!plan) return fail(TCP_ERR_ARG, "fbp_plan: null plan");
  if (!raw || !dark || !flat || !vol) return fail(TCP_ERR_ARG, "fbp_plan: null tensor");
  tcp_status s;
  if ((s = check_tensor(raw, "raw", 3, 3)) != TCP_OK) return s;
  if ((s = check_tensor(vol, "vol", 3, 3)) != TCP_OK) return s;
  if ((s = check_tensor(dark, "dark", 2, 3)) != TCP_OK) return s;
  if ((s = check_tensor(flat, "flat", 2, 3)) != TCP_OK) return s;
  const FbpParams& pp = plan->p;
  if (raw->dtype != TCP_U16) return fail(TCP_ERR_DTYPE, "fbp_plan: raw must be U16");
  if (vol->dtype != pp.vdt) return fail(TCP_ERR_DTYPE, "fbp_plan: vol dtype differs from the plan's");
  const int64_t nz = raw->shape[1];
  if (raw->shape[0] != pp.nt || raw->shape[2] != pp.nd || nz < 1 || nz > pp.nz)
    return fail(TCP_ERR_SHAPE, "fbp_plan: raw must be [ntheta][nz <= plan nz][ndet] of the plan");
  if (vol->shape[0] != nz || vol->shape[1] != pp.n || vol->shape[2] != pp.n)
    return fail(TCP_ERR_SHAPE, "fbp_plan: vol must be [nz][n][n] of the plan");
  for (const tcp_tensor* df : {dark, flat}) {
    const bool ok = (df->ndim == 2 && df->dtype == TCP_F32 && df->shape[0] == nz && df->shape[1] == pp.nd) ||
                    (df->ndim == 3 && df->dtype == TCP_U16 && df->shape[0] >= 1 && df->shape[1] == nz &&
                     df->shape[2] == pp.nd);
    if (!ok) return fail(TCP_ERR_SHAPE, "fbp_plan: dark/flat must be F32 [nz][ndet] or U16 [nf][nz][ndet]");
  }
  const bool host_raw = !is_device_ptr(raw->data), host_vol = !is_device_ptr(vol->data);
  if (host_raw && !(plan->d.io & TCP_IO_HOST_RAW))
    return fail(TCP_ERR_ARG, "fbp_plan: raw is host memory but the plan has no upload ring (TCP_IO_HOST_RAW)");
  if (host_vol && !(plan->d.io & TCP_IO_HOST_VOL))
    return fail(TCP_ERR_ARG, "fbp_plan: vol is host memory but the plan has no download ring (TCP_IO_HOST_VOL)");
  if (host_raw && raw->stride[1] != pp.nd) return fail(TCP_ERR_ALIGN, "fbp_plan: host raw rows must be packed");
  if (overlap(raw, vol)) return fail(TCP_ERR_ALIAS, "fbp_plan: raw and vol overlap");
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  FbpParams p = pp;
  p.nz = nz;
  p.cz = std::max<int64_t>(1, std::min(p.chunk, nz));
  View3 dm, fm;
  if ((s = plan_means(plan, dark, 0, nz, st, &dm)) != TCP_OK) return s;
  if ((s = plan_means(plan, flat, 1, nz, st, &fm)) != TCP_OK) return s;
  return fbp_run(p, plan->r, dm, fm, raw, vol, host_raw, host_vol, st);
}

tcp_status tcp_filter_plan(const tcp_plan* plan, tcp_tensor* sino, void* stream) {
  if (!plan) return fail(TCP_ERR_ARG, "filter_plan: null plan");
  tcp_status s;
  if ((s = check_tensor(sino, "sino", 3, 3)) != TCP_OK) return s;
  if (!is_float_dt(sino->dtype)) return fail(TCP_ERR_DTYPE, "filter_plan: sino must be F32, F16 or BF16");
  if (sino->shape[1] != plan->p.nt || sino->shape[2] != plan->p.nd)
    return fail(TCP_ERR_SHAPE, "filter_plan: sino must be [nz][ntheta][ndet] of the plan");
  if (sino->shape[0] == 0) return TCP_OK;
  return launch_filter(view_of(sino), plan->ft_pi, plan->p.pad, reinterpret_cast<cudaStream_t>(stream));
}

tcp_status tcp_backproject_plan(const tcp_plan* plan, const tcp_tensor* sino, double center, tcp_tensor* vol,
                                double scale, void* stream) {
  if (!plan) return fail(TCP_ERR_ARG, "backproject_plan: null plan");
  if (!std::isfinite(scale) || !std::isfinite(center)) return fail(TCP_ERR_ARG, "backproject_plan: non-finite scalar");
  tcp_status s;
  if ((s = check_tensor(vol, "vol", 3, 3)) != TCP_OK) return s;
  if (!is_float_dt(vol->dtype)) return fail(TCP_ERR_DTYPE, "vol must be F32, F16 or BF16");
  View3 sv;
  if (sino && sino->dtype == TCP_F16X2) {
    if ((s = check_tensor(sino, "sino", 4, 4)) != TCP_OK) return s;
    if (sino->shape[0] != 2) return fail(TCP_ERR_SHAPE, "sino: F16X2 must be [2][nz][ntheta][ndet]");
    const int64_t span = (sino->shape[1] - 1) * sino->stride[1] + (sino->shape[2] - 1) * sino->stride[2] +
                         sino->shape[3];
    if (sino->stride[1] < 0 || sino->stride[2] < 0 || sino->stride[0] < span)
      return fail(TCP_ERR_ALIGN, "sino: F16X2 planes must not overlap");
    sv.p = sino->data; sv.dtype = TCP_F16X2; sv.d0 = sino->shape[1]; sv.d1 = sino->shape[2]; sv.d2 = sino->shape[3];
    sv.s0 = sino->stride[1]; sv.s1 = sino->stride[2]; sv.plane = sino->stride[0];
  } else {
    if ((s = check_tensor(sino, "sino", 3, 3)) != TCP_OK) return s;
    if (!is_float_dt(sino->dtype)) return fail(TCP_ERR_DTYPE, "sino must be F32, F16, BF16 or F16X2");
    sv = view_of(sino);
  }
  if (sv.d1 != plan->p.nt) return fail(TCP_ERR_SHAPE, "backproject_plan: angle count differs from the plan's");
  if (vol->shape[0] != sv.d0 || vol->shape[1] != vol->shape[2])
    return fail(TCP_ERR_SHAPE, "backproject_plan: vol must be [nz][n][n] with the sinogram's nz");
  if (overlap(sino, vol)) return fail(TCP_ERR_ALIAS, "sino and vol overlap");
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  if (vol->shape[0] == 0 || vol->shape[1] == 0) return TCP_OK;
  if (sv.d2 == 0) return fail(TCP_ERR_SHAPE, "backproject_plan: empty detector rows");
  tcp_bp_config cfg;
  tcp_get_backproject_config(sv.d0, sv.d1, sv.d2, vol->shape[1], sino->dtype, vol->dtype, &cfg);
  return launch_backproject(sv, plan->r.trig, center, view_of(vol), cfg, st, (float)scale);
}

tcp_status tcp_project_plan(const tcp_plan* plan, const tcp_tensor* vol, double center, tcp_tensor* sino,
                            void* stream) {
  if (!plan) return fail(TCP_ERR_ARG, "project_plan: null plan");
  if (!std::isfinite(center)) return fail(TCP_ERR_ARG, "project_plan: center must be finite");
  tcp_status s;
  if ((s = check_tensor(vol, "vol", 3, 3)) != TCP_OK) return s;
  if ((s = check_tensor(sino, "sino", 3, 3)) != TCP_OK) return s;
  if (!is_float_dt(vol->dtype) || !is_float_dt(sino->dtype))
    return fail(TCP_ERR_DTYPE, "project_plan: sino/vol must be F32, F16 or BF16");
  if (sino->shape[1] != plan->p.nt || vol->shape[1] != plan->p.n || vol->shape[2] != plan->p.n ||
      vol->shape[0] != sino->shape[0] || vol->shape[0] > plan->p.nz)
    return fail(TCP_ERR_SHAPE,
                "project_plan: vol [nz <= plan nz][n][n] and sino [nz][ntheta][ndet] must match the plan");
  if (overlap(sino, vol)) return fail(TCP_ERR_ALIAS, "sino and vol overlap");
  if (sino->shape[0] == 0 || sino->shape[2] == 0) return TCP_OK;
  return launch_project_ws(view_of(vol), plan->r.trig, center, view_of(sino), plan->proj_orig,
                           reinterpret_cast<cudaStream_t>(stream));
}

}  // extern "C"
