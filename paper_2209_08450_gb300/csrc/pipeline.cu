// Chunked asynchronous FBP (Sec. 2.3 of the TomocuPy paper): the volume is
// reconstructed by z-slabs ("chunks" of slices).  While chunk k is normalised,
// filtered and backprojected on the caller's stream, the raw slab of chunk
// k+1 is copied host->device on a copy stream and the volume slab of chunk
// k-1 is copied device->host on a third stream, through a ring of device
// buffers guarded by events.  Device-resident inputs and outputs skip the
// corresponding copies.  Every compute step is one of the library's kernels.
#include <cmath>
#include <vector>

#include "tcp_internal.cuh"

namespace tcp {
namespace {

enum Where { kDevice, kPinned, kPageable };

Where where(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return kPageable;
  }
  switch (a.type) {
    case cudaMemoryTypeDevice:
    case cudaMemoryTypeManaged: return kDevice;
    case cudaMemoryTypeHost: return kPinned;
    default: return kPageable;
  }
}

int esize(int dt) { return (dt == TCP_F32 || dt == TCP_F16X2) ? 4 : 2; }  // F16X2: both planes

// Everything created for one call; released in stream order at the end.
struct Scope {
  cudaStream_t st;
  std::vector<void*> dev;
  std::vector<cudaEvent_t> ev;
  std::vector<cudaStream_t> streams;
  tcp_status alloc(void** p, size_t bytes) {
    cudaError_t e = cudaMallocAsync(p, bytes ? bytes : 16, st);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMallocAsync");
    dev.push_back(*p);
    return TCP_OK;
  }
  tcp_status event(cudaEvent_t* e) {
    cudaError_t r = cudaEventCreateWithFlags(e, cudaEventDisableTiming);
    if (r != cudaSuccess) return cuda_fail(r, "cudaEventCreate");
    ev.push_back(*e);
    return TCP_OK;
  }
  tcp_status stream(cudaStream_t* s) {
    cudaError_t r = cudaStreamCreateWithFlags(s, cudaStreamNonBlocking);
    if (r != cudaSuccess) return cuda_fail(r, "cudaStreamCreate");
    streams.push_back(*s);
    return TCP_OK;
  }
  ~Scope() {
    // Join every side stream first, so that buffers are released in stream
    // order after their last use on any stream (also on error paths).
    for (cudaStream_t s : streams) {
      cudaEvent_t j;
      if (cudaEventCreateWithFlags(&j, cudaEventDisableTiming) == cudaSuccess) {
        cudaEventRecord(j, s);
        cudaStreamWaitEvent(st, j, 0);
        cudaEventDestroy(j);
      }
    }
    for (void* p : dev) cudaFreeAsync(p, st);
    for (cudaEvent_t e : ev) cudaEventDestroy(e);
    for (cudaStream_t s : streams) cudaStreamDestroy(s);
  }
};

#define TRY_S(x)                      \
  do {                                \
    tcp_status s_ = (x);              \
    if (s_ != TCP_OK) return s_;      \
  } while (0)

// Bring dark/flat (U16 frames or F32 means, host or device) to FP32 means on
// the device, laid out [nz][nd].
tcp_status device_means(const tcp_tensor* t, int64_t nz, int64_t nd, Scope& sc, View3* out) {
  const Where w = where(t->data);
  View3 v;
  v.dtype = t->dtype;
  if (t->ndim == 3) {
    v.d0 = t->shape[0]; v.d1 = t->shape[1]; v.d2 = t->shape[2];
    v.s0 = t->stride[0]; v.s1 = t->stride[1];
  } else {
    v.d0 = 1; v.d1 = t->shape[0]; v.d2 = t->shape[1];
    v.s0 = 0; v.s1 = t->stride[0];
  }
  v.p = t->data;
  if (w != kDevice) {  // upload packed
    const int es = esize(t->dtype == TCP_U16 ? TCP_F16 : TCP_F32);
    const size_t bytes = (size_t)v.d0 * v.d1 * v.d2 * es;
    void* d = nullptr;
    TRY_S(sc.alloc(&d, bytes));
    for (int64_t f = 0; f < v.d0; ++f)
      TCP_CUDA_TRY(cudaMemcpy2DAsync((char*)d + (size_t)f * v.d1 * v.d2 * es, (size_t)v.d2 * es,
                                     (const char*)v.p + (size_t)f * v.s0 * es, (size_t)v.s1 * es,
                                     (size_t)v.d2 * es, (size_t)v.d1, cudaMemcpyHostToDevice, sc.st));
    v.p = d;
    v.s0 = v.d1 * v.d2;
    v.s1 = v.d2;
  }
  if (t->ndim == 3) {
    void* m = nullptr;
    TRY_S(sc.alloc(&m, sizeof(float) * (size_t)(nz * nd)));
    View3 mv;
    mv.p = m; mv.dtype = TCP_F32; mv.d0 = 1; mv.d1 = nz; mv.d2 = nd; mv.s0 = 0; mv.s1 = nd;
    TRY_S(launch_frame_mean(v, mv, sc.st));
    v = mv;
  }
  *out = v;
  return TCP_OK;
}

// Chunk schedule.  With host buffers the first chunk's upload and the last
// chunk's download are not hidden behind compute, so those two chunks are
// half as deep (the middle ones, whose copies overlap compute, stay full).
std::vector<std::pair<int64_t, int64_t>> chunk_schedule(int64_t nz, int64_t chunk, bool host_io) {
  std::vector<std::pair<int64_t, int64_t>> sched;  // (z0, slices)
  int64_t z = 0;
  if (host_io && nz > chunk && chunk > 1) {
    sched.push_back({0, chunk / 2});
    z = chunk / 2;
  }
  while (nz - z > chunk + (host_io ? chunk / 2 : 0) && chunk > 0) {
    sched.push_back({z, chunk});
    z += chunk;
  }
  if (host_io && nz - z > chunk) {  // tail: one full chunk, then the short last one
    sched.push_back({z, chunk});
    z += chunk;
  }
  if (nz - z > 0) sched.push_back({z, nz - z});
  return sched;
}

}  // namespace

tcp_status fbp_resolve(const tcp_tensor* raw, const tcp_tensor* vol, const tcp_fbp_opts* opts, FbpParams* p) {
  if (!raw || !vol) return fail(TCP_ERR_ARG, "fbp: null tensor");
  if (raw->ndim != 3 || raw->dtype != TCP_U16) return fail(TCP_ERR_DTYPE, "fbp: raw must be U16 [ntheta][nz][ndet]");
  if (vol->ndim != 3 || (vol->dtype != TCP_F32 && vol->dtype != TCP_F16 && vol->dtype != TCP_BF16))
    return fail(TCP_ERR_DTYPE, "fbp: vol must be F32/F16/BF16 [nz][n][n]");
  return fbp_resolve_shape(raw->shape[0], raw->shape[1], raw->shape[2], vol->shape[1], vol->dtype, opts, p);
}

tcp_status fbp_resolve_shape(int64_t nt, int64_t nz, int64_t nd, int64_t n, int vdt, const tcp_fbp_opts* opts,
                             FbpParams* p) {
  if (nd > 4096) return fail(TCP_ERR_UNSUPPORTED, "fbp: ndet > 4096");
  tcp_fbp_opts o{};
  if (opts) o = *opts;
  if (o.algorithm != TCP_ALG_LINEREC && o.algorithm != TCP_ALG_FOURIERREC && o.algorithm != TCP_ALG_LPREC)
    return fail(TCP_ERR_ARG, "fbp: unknown algorithm");
  const bool lprec = o.algorithm == TCP_ALG_LPREC;
  const bool frec = o.algorithm == TCP_ALG_FOURIERREC;
  if (lprec && (o.width < 0 || o.width > 8)) return fail(TCP_ERR_ARG, "fbp: LpRec oversampling must be 1..8");
  // Sinogram storage: as requested, else FP16 hi/lo pairs for an FP32 volume
  // (FP32-accurate on the tensor cores; needs ndet % 8 == 0 for 16-byte rows,
  // FP32 otherwise) and the volume's own type for 16-bit volumes.
  int sdt = o.sino_dtype;
  if (sdt != TCP_F32 && sdt != TCP_F16 && sdt != TCP_BF16 && sdt != TCP_F16X2)
    sdt = vdt != TCP_F32 ? vdt : (nd % 8 == 0 && !frec && !lprec ? TCP_F16X2 : TCP_F32);
  if ((frec || lprec) && sdt == TCP_F16X2)
    return fail(TCP_ERR_DTYPE, "fbp: FourierRec and LpRec take F32, F16 or BF16 sinograms");
  const int frec_width = o.width == 0 ? fourierrec_default_width(vdt, n) : o.width;
  if (frec) {
    tcp_status sf = fourierrec_check(nt, nd, n, frec_width);
    if (sf != TCP_OK) return sf;
  }
  if (o.filter < TCP_FILTER_SHEPP || o.filter > TCP_FILTER_NONE) return fail(TCP_ERR_ARG, "fbp: unknown filter");
  if (!valid_pad_mode(o.pad_mode)) return fail(TCP_ERR_ARG, "fbp: unknown pad mode");
  p->nt = nt;
  p->nz = nz;
  p->nd = nd;
  p->n = n;
  p->vdt = vdt;
  p->sdt = sdt;
  p->frec = frec;
  p->lprec = lprec;
  p->width = frec_width;
  p->os = lprec ? (o.width > 0 ? (double)o.width : 2.0) : 2.0;
  // default chunk: 256 slices for 16-bit sinograms (the tensor-core
  // backprojector's N), 32 for FP32 sinograms (the CUDA-core kernel), 64 for
  // FourierRec (32 slice pairs)
  p->chunk = o.chunk_nz > 0 ? o.chunk_nz : lprec ? 16 : frec ? 64 : (sdt == TCP_F32 ? 32 : 256);
  p->cz = std::max<int64_t>(1, std::min(p->chunk, nz));
  p->B = o.n_buffers == 3 ? 3 : 2;
  p->filter = o.filter;
  p->pad = o.pad_mode;
  // The stored sinogram carries the band-limited ramp times storage_scale;
  // the pi/N_theta FBP weight and 1/storage_scale are applied when the
  // backprojector writes each voxel (Sec. 2.1: reorder so 16-bit values stay
  // in range).
  p->sscale = storage_scale(sdt);
  p->bp_scale = nt > 0 ? (float)(M_PI / (double)nt / p->sscale) : 1.f;
  tcp_get_backproject_config(p->cz, nt, nd, n, sdt, vdt, &p->cfg);
  return TCP_OK;
}

tcp_status fbp_run(const FbpParams& p, const FbpRes& r, const View3& dm, const View3& fm, const tcp_tensor* raw,
                   tcp_tensor* vol, bool host_raw, bool host_vol, cudaStream_t st) {
  const int64_t nt = p.nt, nz = p.nz, nd = p.nd, n = p.n, chunk = p.chunk, cz = p.cz;
  const int B = p.B, sdt = p.sdt;
  cudaStream_t cin = r.cin, cout = r.cout;
  if (host_raw || host_vol) {  // fork the copy streams off the caller's stream
    TCP_CUDA_TRY(cudaEventRecord(r.fork, st));
    if (host_raw) TCP_CUDA_TRY(cudaStreamWaitEvent(cin, r.fork, 0));
    if (host_vol) TCP_CUDA_TRY(cudaStreamWaitEvent(cout, r.fork, 0));
  }
  const auto sched = chunk_schedule(nz, chunk, host_raw || host_vol);
  const int64_t nchunks = (int64_t)sched.size();
  const bool trace = r.trace && nchunks <= r.ntrace;
  auto ev = [&](int64_t k, int which) { return r.trace[1 + 6 * k + which]; };
  if (r.traced) *r.traced = 0;
  if (trace) {
    TCP_CUDA_TRY(cudaEventRecord(r.trace[0], st));
    for (int64_t k = 0; k < nchunks; ++k) r.trace_flags[k] = 0;
  }
  auto issue_copy_in = [&](int64_t k) -> tcp_status {
    const int b = (int)(k % B);
    const int64_t z0 = sched[(size_t)k].first, c = sched[(size_t)k].second;
    if (k >= B) TCP_CUDA_TRY(cudaStreamWaitEvent(cin, r.raw_free[b], 0));
    if (trace) TCP_CUDA_TRY(cudaEventRecord(ev(k, 0), cin));
    TCP_CUDA_TRY(cudaMemcpy2DAsync(r.rring[b], (size_t)c * nd * 2,
                                   (const uint16_t*)raw->data + z0 * raw->stride[1], (size_t)raw->stride[0] * 2,
                                   (size_t)c * nd * 2, (size_t)nt, cudaMemcpyHostToDevice, cin));
    if (trace) {
      TCP_CUDA_TRY(cudaEventRecord(ev(k, 1), cin));
      r.trace_flags[k] |= 1;
    }
    TCP_CUDA_TRY(cudaEventRecord(r.raw_ready[b], cin));
    return TCP_OK;
  };
  if (host_raw)
    for (int64_t k = 0; k < std::min<int64_t>(B, nchunks); ++k) TRY_S(issue_copy_in(k));

  for (int64_t k = 0; k < nchunks; ++k) {
    const int b = (int)(k % B);
    const int64_t z0 = sched[(size_t)k].first, c = sched[(size_t)k].second;
    View3 rv;
    rv.dtype = TCP_U16;
    rv.d0 = nt; rv.d1 = c; rv.d2 = nd;
    if (host_raw) {
      TCP_CUDA_TRY(cudaStreamWaitEvent(st, r.raw_ready[b], 0));
      rv.p = r.rring[b]; rv.s0 = c * nd; rv.s1 = nd;
    } else {
      rv.p = (uint16_t*)raw->data + z0 * raw->stride[1];
      rv.s0 = raw->stride[0]; rv.s1 = raw->stride[1];
    }
    View3 dv = dm, fv = fm;
    dv.p = (float*)dm.p + z0 * dm.s1; dv.d1 = c;
    fv.p = (float*)fm.p + z0 * fm.s1; fv.d1 = c;
    if (trace) TCP_CUDA_TRY(cudaEventRecord(ev(k, 2), st));
    // the chunk sinogram is stored angle-major, [angle][slice][sample] (the
    // order of the raw frames), and passed on as a [slice][angle][sample]
    // view: one angle's rows of all the chunk's slices are then one
    // contiguous block, which is what the tensor-core backprojector's copies
    // (all slices of one angle's window at a time) read
    View3 sv;
    sv.p = r.sino; sv.dtype = sdt; sv.d0 = c; sv.d1 = nt; sv.d2 = nd; sv.s0 = nd; sv.s1 = c * nd;
    sv.plane = sdt == TCP_F16X2 ? r.sino_cz * nt * nd : 0;
    TRY_S(launch_normalize_filter(rv, dv, fv, sv, r.ft, p.pad, st));
    if (host_raw) {
      TCP_CUDA_TRY(cudaEventRecord(r.raw_free[b], st));
      if (k + B < nchunks) TRY_S(issue_copy_in(k + B));
    }
    View3 vv;
    vv.dtype = p.vdt; vv.d0 = c; vv.d1 = n; vv.d2 = n;
    if (host_vol) {
      if (k >= B) TCP_CUDA_TRY(cudaStreamWaitEvent(st, r.vol_free[b], 0));
      vv.p = r.vring[b]; vv.s0 = n * n; vv.s1 = n;
    } else {
      vv.p = (char*)vol->data + z0 * vol->stride[0] * esize(p.vdt);
      vv.s0 = vol->stride[0]; vv.s1 = vol->stride[1];
    }
    if (p.frec)
      TRY_S(launch_fourierrec_ws(sv, r.frt, r.fws, r.trig, 0.5 * (double)nd, vv, p.bp_scale, p.width, st));
    else if (p.lprec)
      TRY_S(launch_lprec_ws(sv, *r.lpg, r.lpd, r.lpws, r.lpz, vv, p.bp_scale, st));
    else
      TRY_S(launch_backproject(sv, r.trig, 0.5 * (double)nd, vv, p.cfg, st, p.bp_scale));
    if (trace) TCP_CUDA_TRY(cudaEventRecord(ev(k, 3), st));
    if (host_vol) {
      const int es = esize(p.vdt);
      TCP_CUDA_TRY(cudaEventRecord(r.vol_ready[b], st));
      TCP_CUDA_TRY(cudaStreamWaitEvent(cout, r.vol_ready[b], 0));
      if (trace) TCP_CUDA_TRY(cudaEventRecord(ev(k, 4), cout));
      if (vol->stride[1] == n && vol->stride[0] == n * n) {
        TCP_CUDA_TRY(cudaMemcpyAsync((char*)vol->data + z0 * n * n * es, r.vring[b], (size_t)c * n * n * es,
                                     cudaMemcpyDeviceToHost, cout));
      } else {
        for (int64_t z = 0; z < c; ++z)
          TCP_CUDA_TRY(cudaMemcpy2DAsync((char*)vol->data + ((z0 + z) * vol->stride[0]) * es,
                                         (size_t)vol->stride[1] * es, (char*)r.vring[b] + (size_t)z * n * n * es,
                                         (size_t)n * es, (size_t)n * es, (size_t)n, cudaMemcpyDeviceToHost, cout));
      }
      if (trace) {
        TCP_CUDA_TRY(cudaEventRecord(ev(k, 5), cout));
        r.trace_flags[k] |= 2;
      }
      TCP_CUDA_TRY(cudaEventRecord(r.vol_free[b], cout));
    }
  }
  if (trace && r.traced) *r.traced = (int)nchunks;
  (void)cz;
  // Join the side streams so that `stream` completes after every copy.
  if (host_vol) {
    TCP_CUDA_TRY(cudaEventRecord(r.join_out, cout));
    TCP_CUDA_TRY(cudaStreamWaitEvent(st, r.join_out, 0));
  }
  if (host_raw) {
    TCP_CUDA_TRY(cudaEventRecord(r.join_in, cin));
    TCP_CUDA_TRY(cudaStreamWaitEvent(st, r.join_in, 0));
  }
  return TCP_OK;
}

bool is_device_ptr(const void* p) { return where(p) == kDevice; }
bool is_pinned_ptr(const void* p) { return where(p) == kPinned; }

}  // namespace tcp

using namespace tcp;

extern "C" tcp_status tcp_fbp(const tcp_tensor* raw, const tcp_tensor* dark, const tcp_tensor* flat,
                              const double* theta, double center, tcp_tensor* vol, const tcp_fbp_opts* opts,
                              void* stream) {
  if (!raw || !dark || !flat || !vol) return fail(TCP_ERR_ARG, "fbp: null tensor");
  FbpParams p;
  tcp_status s;
  if ((s = fbp_resolve(raw, vol, opts, &p)) != TCP_OK) return s;
  const int64_t nt = p.nt, nz = p.nz, nd = p.nd, n = p.n;
  if (vol->shape[0] != nz || vol->shape[2] != n) return fail(TCP_ERR_SHAPE, "fbp: vol must be [nz][n][n]");
  if (raw->stride[2] != 1 || vol->stride[2] != 1) return fail(TCP_ERR_ALIGN, "fbp: innermost stride must be 1");
  for (const tcp_tensor* df : {dark, flat}) {
    const bool ok = (df->ndim == 2 && df->dtype == TCP_F32 && df->shape[0] == nz && df->shape[1] == nd) ||
                    (df->ndim == 3 && df->dtype == TCP_U16 && df->shape[0] >= 1 && df->shape[1] == nz &&
                     df->shape[2] == nd);
    if (!ok) return fail(TCP_ERR_SHAPE, "fbp: dark/flat must be F32 [nz][ndet] or U16 [nf][nz][ndet]");
  }
  if (!std::isfinite(center)) return fail(TCP_ERR_ARG, "fbp: center must be finite");
  if (nt > 0 && !theta) return fail(TCP_ERR_ARG, "fbp: theta is null");
  if (nz == 0 || n == 0 || nt == 0 || nd == 0) {
    if (nz * n * n > 0) return fail(TCP_ERR_SHAPE, "fbp: empty projections for a non-empty volume");
    return TCP_OK;
  }
  for (int64_t i = 0; i < nt; ++i)
    if (!std::isfinite(theta[i])) return fail(TCP_ERR_ARG, "fbp: theta must be finite");

  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const Where wraw = where(raw->data), wvol = where(vol->data);
  if (wraw != kDevice && raw->stride[1] != nd) return fail(TCP_ERR_ALIGN, "fbp: host raw rows must be packed");

  FbpRes r;
  if ((s = get_trig_table(theta, nt, &r.trig)) != TCP_OK) return s;
  if ((s = get_filter_table(nd, p.filter, p.sscale, center, &r.ft, pad_smooth(p.pad))) != TCP_OK) return s;
  Scope sc;
  sc.st = st;
  if (p.frec) {
    if ((s = fourierrec_tables_cached(theta, nt, nd, n, p.width, &r.frt)) != TCP_OK) return s;
    void* ws = nullptr;
    if ((s = sc.alloc(&ws, fourierrec_workspace_bytes(nt, nd, n, p.cz, nullptr))) != TCP_OK) return s;
    r.fws = fourierrec_workspace(ws, nt, nd, n, p.cz);
  }
  if (p.lprec) {  // the filter moved the axis to ndet/2
    const LpDevGeom* d = nullptr;
    if ((s = lprec_cached(theta, nt, nd, n, 0.5 * (double)nd, p.os, &r.lpg, &d)) != TCP_OK) return s;
    if ((s = lprec_check(*r.lpg)) != TCP_OK) return s;
    r.lpd = *d;
    r.lpz = lprec_slices_per_pass(*r.lpg, p.cz);
    if ((s = sc.alloc(&r.lpws, lprec_workspace_bytes(*r.lpg, r.lpz))) != TCP_OK) return s;
  }
  View3 dm, fm;
  if ((s = device_means(dark, nz, nd, sc, &dm)) != TCP_OK) return s;
  if ((s = device_means(flat, nz, nd, sc, &fm)) != TCP_OK) return s;
  if ((s = sc.alloc(&r.sino, (size_t)p.cz * nt * nd * esize(p.sdt))) != TCP_OK) return s;
  r.sino_cz = p.cz;
  const bool host_raw = wraw != kDevice, host_vol = wvol != kDevice;
  if (host_raw) {
    if ((s = sc.stream(&r.cin)) != TCP_OK) return s;
    for (int b = 0; b < p.B; ++b) {
      if ((s = sc.alloc(&r.rring[b], (size_t)nt * p.cz * nd * 2)) != TCP_OK) return s;
      if ((s = sc.event(&r.raw_ready[b])) != TCP_OK) return s;
      if ((s = sc.event(&r.raw_free[b])) != TCP_OK) return s;
    }
    if ((s = sc.event(&r.join_in)) != TCP_OK) return s;
  }
  if (host_vol) {
    if ((s = sc.stream(&r.cout)) != TCP_OK) return s;
    for (int b = 0; b < p.B; ++b) {
      if ((s = sc.alloc(&r.vring[b], (size_t)p.cz * n * n * esize(p.vdt))) != TCP_OK) return s;
      if ((s = sc.event(&r.vol_ready[b])) != TCP_OK) return s;
      if ((s = sc.event(&r.vol_free[b])) != TCP_OK) return s;
    }
    if ((s = sc.event(&r.join_out)) != TCP_OK) return s;
  }
  if ((s = sc.event(&r.fork)) != TCP_OK) return s;
  return fbp_run(p, r, dm, fm, raw, vol, host_raw, host_vol, st);
}

// Multi-centre "try" reconstruction (Sec. 2.4, --reconstruction-type try): one
// slice reconstructed about every candidate rotation axis.  Each candidate's
// shift lives in its own filter pass (the Fourier phase that moves the axis to
// ndet/2), so the filtered rows of all candidates form a stack that ONE
// backprojection launch reconstructs about ndet/2, candidates in place of
// slices.
extern "C" tcp_status tcp_try_centers(const tcp_tensor* raw, int64_t slice, const tcp_tensor* dark,
                                      const tcp_tensor* flat, const double* theta, const double* centers,
                                      int64_t ncenters, tcp_tensor* vol, int32_t filter, void* stream) {
  return tcp_try_centers_ex(raw, slice, dark, flat, theta, centers, ncenters, vol, filter, TCP_ALG_LINEREC, 0,
                            stream);
}

extern "C" tcp_status tcp_try_centers_ex(const tcp_tensor* raw, int64_t slice, const tcp_tensor* dark,
                                         const tcp_tensor* flat, const double* theta, const double* centers,
                                         int64_t ncenters, tcp_tensor* vol, int32_t filter, int32_t algorithm,
                                         int32_t width, void* stream) {
  if (!raw || !dark || !flat || !vol) return fail(TCP_ERR_ARG, "try_centers: null tensor");
  if (algorithm != TCP_ALG_LINEREC && algorithm != TCP_ALG_FOURIERREC)
    return fail(TCP_ERR_ARG, "try_centers: unknown algorithm");
  const bool frec = algorithm == TCP_ALG_FOURIERREC;
  if (raw->ndim != 3 || raw->dtype != TCP_U16)
    return fail(TCP_ERR_DTYPE, "try_centers: raw must be U16 [ntheta][nz][ndet]");
  if (vol->ndim != 3 || (vol->dtype != TCP_F32 && vol->dtype != TCP_F16 && vol->dtype != TCP_BF16))
    return fail(TCP_ERR_DTYPE, "try_centers: vol must be F32/F16/BF16 [ncenters][n][n]");
  const int64_t nt = raw->shape[0], nz = raw->shape[1], nd = raw->shape[2], n = vol->shape[1];
  if (ncenters < 0 || vol->shape[0] != ncenters || vol->shape[2] != n)
    return fail(TCP_ERR_SHAPE, "try_centers: vol must be [ncenters][n][n]");
  if (slice < 0 || slice >= nz) return fail(TCP_ERR_ARG, "try_centers: slice outside [0, nz)");
  if (raw->stride[2] != 1 || vol->stride[2] != 1) return fail(TCP_ERR_ALIGN, "try_centers: innermost stride must be 1");
  for (const tcp_tensor* df : {dark, flat}) {
    const bool ok = (df->ndim == 2 && df->dtype == TCP_F32 && df->shape[0] == nz && df->shape[1] == nd) ||
                    (df->ndim == 3 && df->dtype == TCP_U16 && df->shape[0] >= 1 && df->shape[1] == nz &&
                     df->shape[2] == nd);
    if (!ok) return fail(TCP_ERR_SHAPE, "try_centers: dark/flat must be F32 [nz][ndet] or U16 [nf][nz][ndet]");
  }
  if (filter < TCP_FILTER_SHEPP || filter > TCP_FILTER_NONE) return fail(TCP_ERR_ARG, "try_centers: unknown filter");
  if (nd > 4096) return fail(TCP_ERR_UNSUPPORTED, "try_centers: ndet > 4096");
  if (ncenters > 0 && !centers) return fail(TCP_ERR_ARG, "try_centers: centers is null");
  for (int64_t k = 0; k < ncenters; ++k)
    if (!std::isfinite(centers[k])) return fail(TCP_ERR_ARG, "try_centers: centers must be finite");
  if (nt > 0 && !theta) return fail(TCP_ERR_ARG, "try_centers: theta is null");
  for (int64_t i = 0; i < nt; ++i)
    if (!std::isfinite(theta[i])) return fail(TCP_ERR_ARG, "try_centers: theta must be finite");
  const int frec_width = width == 0 ? fourierrec_default_width(vol->dtype, n) : width;
  if (frec) {
    tcp_status sf = fourierrec_check(nt, nd, n, frec_width);
    if (sf != TCP_OK) return sf;
  }
  if (ncenters == 0 || n == 0) return TCP_OK;
  if (nt == 0 || nd == 0) return fail(TCP_ERR_SHAPE, "try_centers: empty projections for a non-empty volume");
  if (where(vol->data) != kDevice) return fail(TCP_ERR_ARG, "try_centers: vol must be device memory");

  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  // storage of the candidate stack: as tcp_fbp chooses for this volume dtype
  // and algorithm
  const int sdt = vol->dtype != TCP_F32 ? vol->dtype : (nd % 8 == 0 && !frec ? TCP_F16X2 : TCP_F32);
  const double sscale = storage_scale(sdt);
  TrigTable trig;
  tcp_status s;
  if ((s = get_trig_table(theta, nt, &trig)) != TCP_OK) return s;
  Scope sc;
  sc.st = st;
  View3 dm, fm;
  if ((s = device_means(dark, nz, nd, sc, &dm)) != TCP_OK) return s;
  if ((s = device_means(flat, nz, nd, sc, &fm)) != TCP_OK) return s;
  // the slice's raw rows [ntheta][1][ndet], on the device
  View3 rv;
  rv.dtype = TCP_U16;
  rv.d0 = nt; rv.d1 = 1; rv.d2 = nd;
  if (where(raw->data) == kDevice) {
    rv.p = (uint16_t*)raw->data + slice * raw->stride[1];
    rv.s0 = raw->stride[0]; rv.s1 = raw->stride[1];
  } else {
    void* d = nullptr;
    TRY_S(sc.alloc(&d, (size_t)nt * nd * 2));
    TCP_CUDA_TRY(cudaMemcpy2DAsync(d, (size_t)nd * 2, (const uint16_t*)raw->data + slice * raw->stride[1],
                                   (size_t)raw->stride[0] * 2, (size_t)nd * 2, (size_t)nt, cudaMemcpyHostToDevice, st));
    rv.p = d; rv.s0 = nd; rv.s1 = nd;
  }
  View3 dv = dm, fv = fm;
  dv.p = (float*)dm.p + slice * dm.s1; dv.d1 = 1;
  fv.p = (float*)fm.p + slice * fm.s1; fv.d1 = 1;
  void* sino = nullptr;
  TRY_S(sc.alloc(&sino, (size_t)ncenters * nt * nd * esize(sdt)));
  const int64_t plane = ncenters * nt * nd;
  for (int64_t k = 0; k < ncenters; ++k) {
    FilterTable ft;
    if ((s = get_filter_table(nd, filter, sscale, centers[k], &ft)) != TCP_OK) return s;
    View3 sv;
    sv.dtype = sdt;
    sv.p = (char*)sino + (size_t)k * nd * (sdt == TCP_F32 ? 4 : 2);  // angle-major stack
    sv.d0 = 1; sv.d1 = nt; sv.d2 = nd; sv.s0 = ncenters * nd; sv.s1 = ncenters * nd;
    sv.plane = sdt == TCP_F16X2 ? plane : 0;
    TRY_S(launch_normalize_filter(rv, dv, fv, sv, ft, TCP_PAD_EDGE, st));
  }
  View3 stack;
  stack.p = sino; stack.dtype = sdt;
  stack.d0 = ncenters; stack.d1 = nt; stack.d2 = nd; stack.s0 = nd; stack.s1 = ncenters * nd;
  stack.plane = sdt == TCP_F16X2 ? plane : 0;
  View3 vv;
  vv.p = vol->data; vv.dtype = vol->dtype; vv.d0 = ncenters; vv.d1 = n; vv.d2 = n;
  vv.s0 = vol->stride[0]; vv.s1 = vol->stride[1];
  const float bp_scale = (float)(M_PI / (double)nt / sscale);
  if (frec) return launch_fourierrec(stack, theta, trig, 0.5 * (double)nd, vv, bp_scale, frec_width, st);
  tcp_bp_config cfg;
  tcp_get_backproject_config(ncenters, nt, nd, n, sdt, vol->dtype, &cfg);
  return launch_backproject(stack, trig, 0.5 * (double)nd, vv, cfg, st, bp_scale);
}
