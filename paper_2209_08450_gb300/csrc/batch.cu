// Batched reconstruction of many datasets with uneven widths and angle
// counts (the paper's chunk pipeline, Sec. 2.3, applied to a set of stacks;
// its `try` mode of Sec. 2.4 reconstructs one slice at many centres, which
// is such a batch).  One batch object owns the per-dataset workspaces and a
// device work list.  A run is: per dataset, the fused normalise+filter
// kernel; then ONE persistent backprojection launch over the work units of
// every dataset (longest angle count first), pulled from an atomic counter.
// The whole run can be captured once into a CUDA graph and replayed.  The
// backprojector's tile configuration (slices per block, angles per stage,
// voxels per thread) is chosen by timing every instantiated configuration on
// the batch itself.  Also here: the per-shape autotuner of tcp_backproject.
#include <algorithm>
#include <cmath>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "tcp_internal.cuh"

namespace tcp {
namespace {

// CUDA-core configurations (rows_per_thread 16: 4 x 4 voxel blocks, FP32
// sinograms only), the FP32 slice-pair form (kernel 2), then the tensor-core
// kernel with 1 or 2 angles per stage (16-bit sinograms whose strides suit TMA).
const tcp_bp_config kCandidates[] = {{8, 16, 4, 0}, {4, 32, 4, 0}, {4, 16, 4, 0}, {16, 8, 2, 0}, {8, 16, 2, 0},
                                     {2, 16, 4, 0}, {1, 32, 4, 0}, {4, 16, 16, 0}, {8, 16, 16, 0}, {4, 32, 16, 0},
                                     {8, 16, 4, 2}, {16, 8, 4, 2}, {4, 16, 4, 2}, {8, 2, 4, 1}, {8, 1, 4, 1},
                                     {8, 2, 4, 3}, {8, 1, 4, 3}};

int esize(int dt) { return dt == TCP_F32 ? 4 : 2; }

View3 v3(const tcp_tensor& t) {
  View3 v;
  v.p = t.data;
  v.dtype = t.dtype;
  if (t.ndim == 3) {
    v.d0 = t.shape[0]; v.d1 = t.shape[1]; v.d2 = t.shape[2];
    v.s0 = t.stride[0]; v.s1 = t.stride[1];
  } else {
    v.d0 = 1; v.d1 = t.shape[0]; v.d2 = t.shape[1];
    v.s0 = 0; v.s1 = t.stride[0];
  }
  return v;
}

bool on_device(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

struct ItemRt {
  View3 raw, vol, sino;
  View3 dark_src, flat_src;  // frames (U16) or means (F32)
  View3 dark, flat;          // FP32 means used by the fused kernel
  bool dark_frames = false, flat_frames = false;
  TrigTable trig;
  FilterTable ft;
  double center = 0;
  int pad = 0;
};

}  // namespace
}  // namespace tcp

using namespace tcp;

struct tcp_batch {
  int dev = 0;
  int sdt = TCP_F16, vdt = TCP_F32;
  std::vector<ItemRt> items;  // in work order (longest angle count first)
  std::vector<void*> owned;
  BpArgs* d_items = nullptr;
  long long* d_prefix = nullptr;
  unsigned long long* d_counter = nullptr;
  tcp_bp_config cfg{8, 16, 4, 0};
  int blocks = 0;
  long long units = 0;
  float tuned_ms = 0.f;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  // Side streams: each dataset's chain (frame means, normalise + filter and,
  // with the tensor-core kernel, its backprojection) runs on side stream
  // i % kSide, forked from and joined back to the caller's stream by events
  // (a captured graph gets parallel branches).  Datasets touch disjoint
  // buffers, so the chains are independent; they fill each other's last waves.
  static constexpr int kSide = 3;
  cudaStream_t side[kSide] = {};
  cudaEvent_t fork = nullptr, join[kSide] = {};
  ~tcp_batch() {
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    for (int k = 0; k < kSide; ++k) {
      if (side[k]) cudaStreamDestroy(side[k]);
      if (join[k]) cudaEventDestroy(join[k]);
    }
    if (fork) cudaEventDestroy(fork);
    for (void* p : owned) cudaFree(p);
    if (d_items) cudaFree(d_items);
    if (d_prefix) cudaFree(d_prefix);
    if (d_counter) cudaFree(d_counter);
  }
};

namespace {

// The tensor-core kernel takes 16-bit sinograms with TMA-friendly strides.
bool tc_batch_ok(const tcp_batch* b) {
  if (b->sdt != TCP_F16 && b->sdt != TCP_BF16) return false;
  for (const ItemRt& it : b->items)
    if (!tc_eligible(it.sino)) return false;
  return true;
}

tcp_status set_config(tcp_batch* b, const tcp_bp_config& cfg) {
  if (cfg.kernel == 1 || cfg.kernel == 3) {  // one tensor-core launch per dataset inside the run
    if (!tc_batch_ok(b)) return fail(TCP_ERR_UNSUPPORTED, "batch: tensor-core kernel needs 16-bit TMA-friendly sinograms");
    long long units = 0;
    for (const ItemRt& it : b->items) units += ((it.vol.d1 + 15) / 16) * ((it.vol.d1 + 15) / 16);
    b->cfg = cfg;
    b->units = units;
    b->blocks = 0;
    return TCP_OK;
  }
  std::vector<BpArgs> args;
  std::vector<long long> prefix(1, 0);
  for (const ItemRt& it : b->items) {
    const float scale = (float)(M_PI / (double)it.sino.d1 / storage_scale(b->sdt));
    BpArgs a = make_bp_args(it.sino, it.trig, 0.5 * (double)it.sino.d2, it.vol, scale);
    args.push_back(a);
    const long long units = (long long)a.ntx * a.ntx * ((a.nz + cfg.k_slices - 1) / cfg.k_slices);
    prefix.push_back(prefix.back() + units);
  }
  TCP_CUDA_TRY(cudaMemcpy(b->d_items, args.data(), sizeof(BpArgs) * args.size(), cudaMemcpyHostToDevice));
  TCP_CUDA_TRY(cudaMemcpy(b->d_prefix, prefix.data(), sizeof(long long) * prefix.size(), cudaMemcpyHostToDevice));
  tcp_status s = bp_persistent_grid(b->sdt, b->vdt, cfg, &b->blocks);
  if (s != TCP_OK) return s;
  b->cfg = cfg;
  b->units = prefix.back();
  return TCP_OK;
}

tcp_status prep_item(const ItemRt& it, cudaStream_t st) {
  tcp_status s;
  if (it.dark_frames && (s = launch_frame_mean(it.dark_src, it.dark, st)) != TCP_OK) return s;
  if (it.flat_frames && (s = launch_frame_mean(it.flat_src, it.flat, st)) != TCP_OK) return s;
  return launch_normalize_filter(it.raw, it.dark, it.flat, it.sino, it.ft, it.pad, st);
}

bool tc_mode(const tcp_batch* b) { return b->cfg.kernel == 1 || b->cfg.kernel == 3; }

// The per-dataset chains on the side streams: prep (if asked) and the
// dataset's tensor-core backprojection (if asked).  The side streams are
// joined back into st even after a failed launch, so that a capture stays
// well formed.
tcp_status run_chains(tcp_batch* b, cudaStream_t st, bool with_prep, bool tc) {
  if (!with_prep && !tc) return TCP_OK;
  TCP_CUDA_TRY(cudaEventRecord(b->fork, st));
  for (int k = 0; k < tcp_batch::kSide; ++k) TCP_CUDA_TRY(cudaStreamWaitEvent(b->side[k], b->fork, 0));
  tcp_status s = TCP_OK;
  for (size_t i = 0; i < b->items.size() && s == TCP_OK; ++i) {
    const ItemRt& it = b->items[i];
    cudaStream_t si = b->side[i % tcp_batch::kSide];
    if (with_prep) s = prep_item(it, si);
    if (s == TCP_OK && tc) {
      const float scale = (float)(M_PI / (double)it.sino.d1 / storage_scale(b->sdt));
      s = launch_backproject_tc(it.sino, it.trig, 0.5 * (double)it.sino.d2, it.vol, scale, b->cfg.theta_stage,
                                b->cfg.kernel == 3 ? 2 : 1, si);
    }
  }
  for (int k = 0; k < tcp_batch::kSide; ++k) {
    cudaError_t e = cudaEventRecord(b->join[k], b->side[k]);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(st, b->join[k], 0);
    if (e != cudaSuccess && s == TCP_OK) s = cuda_fail(e, "batch: stream join");
  }
  return s;
}

// One pass over the batch: the chains, then (CUDA-core mode) the single
// persistent backprojection launch over every dataset on st.
tcp_status run_all(tcp_batch* b, cudaStream_t st, bool with_prep) {
  tcp_status s = run_chains(b, st, with_prep, tc_mode(b));
  if (s != TCP_OK || tc_mode(b)) return s;
  TCP_CUDA_TRY(cudaMemsetAsync(b->d_counter, 0, sizeof(unsigned long long), st));
  BpWork w;
  w.items = b->d_items;
  w.prefix = b->d_prefix;
  w.nitems = (int)b->items.size();
  w.counter = b->d_counter;
  return launch_backproject_persistent(w, b->sdt, b->vdt, b->cfg, b->blocks, st);
}

tcp_status time_config(tcp_batch* b, const tcp_bp_config& cfg, cudaStream_t st, float* ms) {
  tcp_status s = set_config(b, cfg);
  if (s != TCP_OK) return s;
  cudaEvent_t e0, e1;
  TCP_CUDA_TRY(cudaEventCreate(&e0));
  TCP_CUDA_TRY(cudaEventCreate(&e1));
  s = run_all(b, st, false);  // warm-up
  float best = 1e30f;
  for (int rep = 0; rep < 2 && s == TCP_OK; ++rep) {
    cudaEventRecord(e0, st);
    s = run_all(b, st, false);
    cudaEventRecord(e1, st);
    cudaError_t e = cudaEventSynchronize(e1);
    if (e != cudaSuccess) {
      s = cuda_fail(e, "autotune timing");
      break;
    }
    float t = 0.f;
    cudaEventElapsedTime(&t, e0, e1);
    best = std::min(best, t);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  *ms = best;
  return s;
}

// ------------------------------------------- per-shape autotune (single) --

std::mutex g_tune_mu;
std::map<std::tuple<int64_t, int64_t, int64_t, int64_t, int, int>, tcp_bp_config> g_tuned;

}  // namespace

namespace tcp {
bool tuned_bp_config(int64_t nz, int64_t nt, int64_t nd, int64_t n, int sdt, int vdt, tcp_bp_config* cfg) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  auto it = g_tuned.find(std::make_tuple(nz, nt, nd, n, sdt, vdt));
  if (it == g_tuned.end()) return false;
  *cfg = it->second;
  return true;
}
}  // namespace tcp

extern "C" {

tcp_status tcp_batch_create(const tcp_batch_item* items, int32_t n_items, const tcp_batch_opts* opts, void* stream,
                            tcp_batch** out) {
  if (!out) return fail(TCP_ERR_ARG, "batch: null output handle");
  *out = nullptr;
  if (!items || n_items <= 0) return fail(TCP_ERR_ARG, "batch: no items");
  tcp_batch_opts o{};
  o.sino_dtype = TCP_F16;
  if (opts) o = *opts;
  if (o.sino_dtype != TCP_F32 && o.sino_dtype != TCP_F16 && o.sino_dtype != TCP_BF16)
    return fail(TCP_ERR_DTYPE, "batch: sino dtype must be F32, F16 or BF16");
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  int dev = 0;
  TCP_CUDA_TRY(cudaGetDevice(&dev));
  auto* b = new tcp_batch();
  b->sdt = o.sino_dtype;
  b->vdt = items[0].vol.dtype;
  b->dev = dev;
  std::vector<int> order(n_items);
  for (int i = 0; i < n_items; ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(),
                   [&](int a, int c) { return items[a].raw.shape[0] > items[c].raw.shape[0]; });
  tcp_status s = TCP_OK;
  for (int oi = 0; oi < n_items && s == TCP_OK; ++oi) {
    const tcp_batch_item& in = items[order[oi]];
    const std::string tag = "batch item " + std::to_string(order[oi]) + ": ";
    if (in.raw.ndim != 3 || in.raw.dtype != TCP_U16) { s = fail(TCP_ERR_DTYPE, tag + "raw must be U16 [ntheta][nz][ndet]"); break; }
    if (in.vol.ndim != 3 || in.vol.dtype != b->vdt || (in.vol.dtype != TCP_F32 && in.vol.dtype != TCP_F16 &&
                                                         in.vol.dtype != TCP_BF16)) {
      s = fail(TCP_ERR_DTYPE, tag + "vol must be F32/F16/BF16 and one dtype for the batch");
      break;
    }
    const int64_t nt = in.raw.shape[0], nz = in.raw.shape[1], nd = in.raw.shape[2], n = in.vol.shape[1];
    if (nt < 1 || nz < 1 || nd < 1 || n < 1 || in.vol.shape[0] != nz || in.vol.shape[2] != n) {
      s = fail(TCP_ERR_SHAPE, tag + "need non-empty raw and vol [nz][n][n]");
      break;
    }
    if (nd > 4096) { s = fail(TCP_ERR_UNSUPPORTED, tag + "ndet > 4096"); break; }
    if (in.raw.stride[2] != 1 || in.vol.stride[2] != 1) { s = fail(TCP_ERR_ALIGN, tag + "innermost stride must be 1"); break; }
    if (!in.theta) { s = fail(TCP_ERR_ARG, tag + "theta is null"); break; }
    if (!std::isfinite(in.center)) { s = fail(TCP_ERR_ARG, tag + "center must be finite"); break; }
    if (in.filter < TCP_FILTER_SHEPP || in.filter > TCP_FILTER_NONE) { s = fail(TCP_ERR_ARG, tag + "unknown filter"); break; }
    if (!valid_pad_mode(in.pad_mode)) { s = fail(TCP_ERR_ARG, tag + "unknown pad mode"); break; }
    for (const void* p : {in.raw.data, in.vol.data, in.dark.data, in.flat.data})
      if (!p || !on_device(p)) { s = fail(TCP_ERR_ARG, tag + "raw, dark, flat and vol must be device buffers"); break; }
    if (s != TCP_OK) break;
    ItemRt it;
    it.raw = v3(in.raw);
    it.vol = v3(in.vol);
    it.center = in.center;
    it.pad = in.pad_mode;
    for (int k = 0; k < 2 && s == TCP_OK; ++k) {
      const tcp_tensor& df = k == 0 ? in.dark : in.flat;
      const bool frames = df.ndim == 3;
      const bool ok = (df.ndim == 2 && df.dtype == TCP_F32 && df.shape[0] == nz && df.shape[1] == nd) ||
                      (frames && df.dtype == TCP_U16 && df.shape[0] >= 1 && df.shape[1] == nz && df.shape[2] == nd);
      if (!ok) { s = fail(TCP_ERR_SHAPE, tag + "dark/flat must be F32 [nz][ndet] or U16 [nf][nz][ndet]"); break; }
      View3 src = v3(df), mean = src;
      if (frames) {
        void* m = nullptr;
        cudaError_t e = cudaMalloc(&m, sizeof(float) * (size_t)(nz * nd));
        if (e != cudaSuccess) { s = cuda_fail(e, "batch: cudaMalloc"); break; }
        b->owned.push_back(m);
        mean.p = m; mean.dtype = TCP_F32; mean.d0 = 1; mean.d1 = nz; mean.d2 = nd; mean.s0 = 0; mean.s1 = nd;
      }
      if (k == 0) { it.dark_src = src; it.dark = mean; it.dark_frames = frames; }
      else { it.flat_src = src; it.flat = mean; it.flat_frames = frames; }
    }
    if (s != TCP_OK) break;
    void* w = nullptr;
    cudaError_t e = cudaMalloc(&w, (size_t)nz * nt * nd * esize(b->sdt));
    if (e != cudaSuccess) { s = cuda_fail(e, "batch: cudaMalloc"); break; }
    b->owned.push_back(w);
    it.sino.p = w; it.sino.dtype = b->sdt; it.sino.d0 = nz; it.sino.d1 = nt; it.sino.d2 = nd;
    it.sino.s0 = nd; it.sino.s1 = nz * nd;  // angle-major storage, as in tcp_fbp's chunks
    // the batch owns its tables, so that its captured graph never depends on
    // the library's bounded caches
    if ((s = build_trig_owned(in.theta, nt, &b->owned, &it.trig)) != TCP_OK) break;
    if ((s = build_filter_owned(nd, in.filter, storage_scale(b->sdt), in.center, pad_smooth(in.pad_mode), &b->owned,
                                &it.ft)) != TCP_OK)
      break;
    b->items.push_back(it);
  }
  if (s == TCP_OK) {
    cudaError_t e = cudaMalloc(&b->d_items, sizeof(BpArgs) * b->items.size());
    if (e == cudaSuccess) e = cudaMalloc(&b->d_prefix, sizeof(long long) * (b->items.size() + 1));
    if (e == cudaSuccess) e = cudaMalloc(&b->d_counter, sizeof(unsigned long long));
    if (e != cudaSuccess) s = cuda_fail(e, "batch: cudaMalloc");
  }
  // without autotune: the configuration fixed by tcp_set_backproject_config, if any
  if (s == TCP_OK && !o.autotune && bp_override().k_slices) b->cfg = bp_override();
  if (s == TCP_OK) s = set_config(b, b->cfg);
  for (int k = 0; k < tcp_batch::kSide && s == TCP_OK; ++k) {
    cudaError_t e = cudaStreamCreateWithFlags(&b->side[k], cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->join[k], cudaEventDisableTiming);
    if (e != cudaSuccess) s = cuda_fail(e, "batch: side stream");
  }
  if (s == TCP_OK) {
    cudaError_t e = cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming);
    if (e != cudaSuccess) s = cuda_fail(e, "batch: side stream");
  }
  if (s == TCP_OK && o.autotune) {
    s = run_chains(b, st, true, false);  // the sinograms every timed configuration reads
    float best = 1e30f;
    tcp_bp_config best_cfg = b->cfg;
    for (const tcp_bp_config& c : kCandidates) {
      if (s != TCP_OK) break;
      float ms = 0.f;
      s = time_config(b, c, st, &ms);
      if (s == TCP_ERR_UNSUPPORTED) {  // not instantiated for this dtype pair: skip
        s = TCP_OK;
        continue;
      }
      if (s == TCP_OK && ms < best) {
        best = ms;
        best_cfg = c;
      }
    }
    if (s == TCP_OK) s = set_config(b, best_cfg);
    b->tuned_ms = best;
  }
  if (s != TCP_OK) {
    cudaStreamSynchronize(st);
    delete b;
    return s;
  }
  *out = b;
  return TCP_OK;
}

tcp_status tcp_batch_run(tcp_batch* b, void* stream) {
  if (!b) return fail(TCP_ERR_ARG, "batch: null handle");
  return run_all(b, reinterpret_cast<cudaStream_t>(stream), true);
}

tcp_status tcp_batch_capture(tcp_batch* b, void* stream) {
  if (!b) return fail(TCP_ERR_ARG, "batch: null handle");
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  if (!st) return fail(TCP_ERR_ARG, "batch: capture needs a non-default stream");
  if (b->exec) {
    cudaGraphExecDestroy(b->exec);
    b->exec = nullptr;
  }
  if (b->graph) {
    cudaGraphDestroy(b->graph);
    b->graph = nullptr;
  }
  TCP_CUDA_TRY(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
  tcp_status s = tcp_batch_run(b, stream);
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamEndCapture(st, &g);
  if (s != TCP_OK) {
    if (g) cudaGraphDestroy(g);
    return s;
  }
  if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
  b->graph = g;
  TCP_CUDA_TRY(cudaGraphInstantiate(&b->exec, g, 0));
  return TCP_OK;
}

tcp_status tcp_batch_replay(tcp_batch* b, void* stream) {
  if (!b) return fail(TCP_ERR_ARG, "batch: null handle");
  if (!b->exec) return fail(TCP_ERR_ARG, "batch: no captured graph (call tcp_batch_capture first)");
  TCP_CUDA_TRY(cudaGraphLaunch(b->exec, reinterpret_cast<cudaStream_t>(stream)));
  return TCP_OK;
}

tcp_status tcp_batch_info(const tcp_batch* b, tcp_bp_config* cfg, float* tuned_ms, int64_t* work_units,
                          int32_t* grid_blocks) {
  if (!b) return fail(TCP_ERR_ARG, "batch: null handle");
  if (cfg) *cfg = b->cfg;
  if (tuned_ms) *tuned_ms = b->tuned_ms;
  if (work_units) *work_units = b->units;
  if (grid_blocks) *grid_blocks = b->blocks;
  return TCP_OK;
}

tcp_status tcp_batch_destroy(tcp_batch* b) {
  if (!b) return TCP_OK;
  cudaError_t e = cudaDeviceSynchronize();
  delete b;
  if (e != cudaSuccess) return cuda_fail(e, "batch destroy");
  return TCP_OK;
}

tcp_status tcp_autotune_backproject(const tcp_tensor* sino, const double* theta, double center, tcp_tensor* vol,
                                    void* stream, tcp_bp_config* best, float* best_ms) {
  if (!sino || !vol || sino->ndim != 3 || vol->ndim != 3) return fail(TCP_ERR_ARG, "autotune: need 3-d sino and vol");
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const tcp_bp_config keep = bp_override();
  float bms = 1e30f;
  tcp_bp_config bcfg = kCandidates[0];
  cudaEvent_t e0, e1;
  TCP_CUDA_TRY(cudaEventCreate(&e0));
  TCP_CUDA_TRY(cudaEventCreate(&e1));
  tcp_status s = TCP_OK;
  std::vector<tcp_bp_config> cands;
  for (const tcp_bp_config& c : kCandidates) {
    const bool f32 = sino->dtype == TCP_F32;
    if ((c.kernel == 1 || c.kernel == 3) && f32) continue;       // tensor cores: 16-bit sinograms
    if (c.kernel == 0 && c.rows_per_thread == 16 && !f32) continue;  // 4 x 4 blocks: FP32 sinograms
    if (c.kernel == 2 && !f32) continue;                         // slice pairs: FP32 sinograms
    cands.push_back(c);
  }
  for (const tcp_bp_config& c : cands) {
    if ((s = tcp_set_backproject_config(&c)) != TCP_OK) break;
    if ((s = tcp_backproject(sino, theta, center, vol, stream)) != TCP_OK) break;  // warm-up
    cudaEventRecord(e0, st);
    s = tcp_backproject(sino, theta, center, vol, stream);
    cudaEventRecord(e1, st);
    if (s != TCP_OK) break;
    cudaError_t e = cudaEventSynchronize(e1);
    if (e != cudaSuccess) {
      s = cuda_fail(e, "autotune timing");
      break;
    }
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (ms < bms) {
      bms = ms;
      bcfg = c;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  tcp_set_backproject_config(keep.k_slices ? &keep : nullptr);
  if (s != TCP_OK) return s;
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tuned[std::make_tuple(sino->shape[0], sino->shape[1], sino->shape[2], vol->shape[1], sino->dtype, vol->dtype)] =
        bcfg;
  }
  if (best) *best = bcfg;
  if (best_ms) *best_ms = bms;
  return TCP_OK;
}

}  // extern "C"
