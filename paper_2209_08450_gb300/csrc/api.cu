// C-ABI entry points of libtcp: argument checks, views, cached device tables
// (FP64 angle tables, FP64-derived filter responses and twiddles) and error
// reporting.  Every compute step runs in the CUDA kernels of this library.
#include <cmath>
#include <complex>
#include <cstring>
#include <mutex>
#include <unordered_map>
#include <vector>

#include "tcp_internal.cuh"

namespace tcp {

// ------------------------------------------------------------ error state --

static thread_local std::string g_last_error;

void set_error(const std::string& msg) { g_last_error = msg; }
tcp_status fail(tcp_status s, const std::string& msg) {
  g_last_error = msg;
  return s;
}
tcp_status cuda_fail(cudaError_t e, const char* what) {
  g_last_error = std::string(what) + ": " + cudaGetErrorString(e);
  return e == cudaErrorMemoryAllocation ? TCP_ERR_OOM : TCP_ERR_CUDA;
}

__device__ uint32_t g_error_word;

static std::mutex g_mu;
static std::unordered_map<int, uint32_t*> g_err_ptr;

uint32_t* device_error_word() {
  int dev = 0;
  cudaGetDevice(&dev);
  std::lock_guard<std::mutex> lk(g_mu);
  auto it = g_err_ptr.find(dev);
  if (it != g_err_ptr.end()) return it->second;
  void* p = nullptr;
  if (cudaGetSymbolAddress(&p, g_error_word) != cudaSuccess) return nullptr;
  g_err_ptr[dev] = reinterpret_cast<uint32_t*>(p);
  return reinterpret_cast<uint32_t*>(p);
}

static bool g_checked = [] {
  const char* e = getenv("TCP_CHECKED");
  return e && e[0] == '1';
}();
bool checked_mode() { return g_checked; }

// ------------------------------------------------------------------ caches --

static uint64_t fnv1a(const void* p, size_t n) {
  const unsigned char* b = reinterpret_cast<const unsigned char*>(p);
  uint64_t h = 1469598103934665603ull;
  for (size_t i = 0; i < n; ++i) h = (h ^ b[i]) * 1099511628211ull;
  return h;
}

// The implicit caches below keep at most kCacheCap entries each (per kind);
// beyond that the least recently used entry is freed.  cudaFree waits for the
// device, so no queued kernel still reads a freed table; a CUDA graph captured
// with tables from these caches must not outlive them (plans own theirs).
constexpr size_t kCacheCap = 64;
static uint64_t g_stamp = 0;

struct TrigEntry {
  std::vector<double> theta;
  double2* dev = nullptr;
  uint64_t used = 0;
};
static std::unordered_map<uint64_t, std::vector<TrigEntry>> g_trig;  // key: hash ^ device
static size_t g_trig_count = 0;

static std::vector<double2> trig_host(const double* theta, int64_t n) {
  std::vector<double2> h((size_t)std::max<int64_t>(n, 1));
  for (int64_t i = 0; i < n; ++i) h[(size_t)i] = make_double2(std::cos(theta[i]), std::sin(theta[i]));
  return h;
}

static void trig_evict_lru() {
  uint64_t best = UINT64_MAX;
  uint64_t bkey = 0;
  size_t bidx = 0;
  for (auto& kv : g_trig)
    for (size_t i = 0; i < kv.second.size(); ++i)
      if (kv.second[i].used < best) {
        best = kv.second[i].used;
        bkey = kv.first;
        bidx = i;
      }
  if (best == UINT64_MAX) return;
  auto& v = g_trig[bkey];
  cudaFree(v[bidx].dev);
  v.erase(v.begin() + (long)bidx);
  if (v.empty()) g_trig.erase(bkey);
  --g_trig_count;
}

tcp_status get_trig_table(const double* theta, int64_t n, TrigTable* out) {
  int dev = 0;
  TCP_CUDA_TRY(cudaGetDevice(&dev));
  const uint64_t key = fnv1a(theta, sizeof(double) * (size_t)n) ^ ((uint64_t)(dev + 1) * 0x9e3779b97f4a7c15ull) ^
                       (uint64_t)n;
  std::lock_guard<std::mutex> lk(g_mu);
  {
    auto it = g_trig.find(key);
    if (it != g_trig.end())
      for (auto& e : it->second)
        if ((int64_t)e.theta.size() == n && std::memcmp(e.theta.data(), theta, sizeof(double) * (size_t)n) == 0) {
          e.used = ++g_stamp;
          out->dev = e.dev;
          out->n = n;
          return TCP_OK;
        }
  }
  if (g_trig_count >= kCacheCap) trig_evict_lru();
  const std::vector<double2> h = trig_host(theta, n);
  TrigEntry e;
  e.theta.assign(theta, theta + n);
  e.used = ++g_stamp;
  TCP_CUDA_TRY(cudaMalloc(&e.dev, h.size() * sizeof(double2)));
  cudaError_t err = cudaMemcpy(e.dev, h.data(), h.size() * sizeof(double2), cudaMemcpyHostToDevice);
  if (err != cudaSuccess) {
    cudaFree(e.dev);
    return cuda_fail(err, "upload angle table");
  }
  g_trig[key].push_back(e);
  ++g_trig_count;
  out->dev = e.dev;
  out->n = n;
  return TCP_OK;
}

tcp_status build_trig_owned(const double* theta, int64_t n, std::vector<void*>* owned, TrigTable* out) {
  const std::vector<double2> h = trig_host(theta, n);
  double2* d = nullptr;
  TCP_CUDA_TRY(cudaMalloc(&d, h.size() * sizeof(double2)));
  owned->push_back(d);
  TCP_CUDA_TRY(cudaMemcpy(d, h.data(), h.size() * sizeof(double2), cudaMemcpyHostToDevice));
  out->dev = d;
  out->n = n;
  return TCP_OK;
}

int64_t padded_length(int64_t ndet, bool smooth) {
  int64_t n = 1;
  while (n < 2 * ndet) n *= 2;
  if (smooth) {  // the next 3 * 2^k >= 2 ndet (from 48 on) and 5 * 2^k (from 80 on)
    for (const int64_t base : {3, 5}) {
      int64_t m = base;
      while (m < 2 * ndet || m < 16 * base) m *= 2;
      n = std::min(n, m);
    }
  }
  return n;
}

// In-place iterative radix-2 FFT in FP64 (host), forward: X_k = sum x_m e^{-2 pi i km/N}.
static void fft64(std::vector<std::complex<double>>& x) {
  const size_t N = x.size();
  for (size_t i = 1, j = 0; i < N; ++i) {
    size_t bit = N >> 1;
    for (; j & bit; bit >>= 1) j ^= bit;
    j ^= bit;
    if (i < j) std::swap(x[i], x[j]);
  }
  for (size_t len = 2; len <= N; len <<= 1) {
    for (size_t i = 0; i < N; i += len)
      for (size_t k = 0; k < len / 2; ++k) {
        const double ang = -2.0 * M_PI * (double)k / (double)len;
        const std::complex<double> w(std::cos(ang), std::sin(ang));
        const std::complex<double> u = x[i + k], v = x[i + k + len / 2] * w;
        x[i + k] = u + v;
        x[i + k + len / 2] = u - v;
      }
  }
}

// Band-limited ramp on the padded period: DFT of the spatial Ram-Lak kernel
// h[0] = 1/4, h[m] = -1/(pi^2 m^2) for odd m, 0 for even m != 0, truncated to
// -N/2 <= m < N/2.  The window multiplies it: Shepp-Logan sin(pi nu)/(pi nu),
// Parzen (1 - 2 nu)^3.
static std::vector<double> filter_response(int64_t npad, int32_t filter) {
  std::vector<double> H((size_t)npad / 2 + 1, 1.0);
  if (filter == TCP_FILTER_NONE) return H;
  std::vector<std::complex<double>> h((size_t)npad, 0.0);
  h[0] = 0.25;
  for (int64_t m = 1; m < npad / 2; m += 2) {
    const double v = -1.0 / (M_PI * M_PI * (double)m * (double)m);
    h[(size_t)m] = v;
    h[(size_t)(npad - m)] = v;
  }
  if ((npad / 2) % 2 == 1) {  // m = -npad/2 belongs to the period (odd only when npad == 2)
    const double m = (double)(npad / 2);
    h[(size_t)(npad / 2)] = -1.0 / (M_PI * M_PI * m * m);
  }
  if ((npad & (npad - 1)) == 0) {
    fft64(h);
  } else {
    // 3 * 2^k and 5 * 2^k periods: the same DFT as a direct cosine sum (h is real and even)
    std::vector<double> r((size_t)npad / 2 + 1);
    for (int64_t k = 0; k <= npad / 2; ++k) {
      double acc = 0.25;
      for (int64_t m = 1; m < npad / 2; m += 2)
        acc += 2.0 * h[(size_t)m].real() * std::cos(2.0 * M_PI * (double)((k * m) % npad) / (double)npad);
      r[(size_t)k] = acc;
    }
    for (int64_t k = 0; k <= npad / 2; ++k) h[(size_t)k] = r[(size_t)k];
  }
  for (int64_t k = 0; k <= npad / 2; ++k) {
    const double nu = (double)k / (double)npad;
    double w = 1.0;
    if (filter == TCP_FILTER_SHEPP) w = k == 0 ? 1.0 : std::sin(M_PI * nu) / (M_PI * nu);
    else if (filter == TCP_FILTER_PARZEN) w = std::pow(1.0 - 2.0 * nu, 3);
    H[(size_t)k] = h[(size_t)k].real() * w;
  }
  return H;
}

struct FiltKey {
  int dev;
  int64_t npad, ndet;
  int32_t filter;
  double weight, center;
  bool operator==(const FiltKey& o) const {
    return dev == o.dev && npad == o.npad && ndet == o.ndet && filter == o.filter &&
           std::memcmp(&weight, &o.weight, sizeof(double)) == 0 && std::memcmp(&center, &o.center, sizeof(double)) == 0;
  }
};
struct FiltKeyHash {
  size_t operator()(const FiltKey& k) const { return (size_t)fnv1a(&k, sizeof(FiltKey)); }
};
struct RespEntry {
  float2* dev = nullptr;
  uint64_t used = 0;
};
static std::unordered_map<FiltKey, RespEntry, FiltKeyHash> g_resp;
static std::unordered_map<uint64_t, float2*> g_tw;  // (dev << 32) | npad

// Two-level twiddle table: 64 low powers, then the powers of W^64.
static std::vector<float2> twiddle_host(int64_t npad) {
  const int64_t nhi = (npad + 63) / 64;
  std::vector<float2> tw((size_t)(64 + nhi));
  for (int64_t m = 0; m < 64 + nhi; ++m) {
    const double e = m < 64 ? (double)m : 64.0 * (double)(m - 64);
    const double ang = -2.0 * M_PI * e / (double)npad;
    tw[(size_t)m] = make_float2((float)std::cos(ang), (float)std::sin(ang));
  }
  return tw;
}

// Response bins 0..npad/2: H(k) * weight / npad * e^{2 pi i (k/npad)(center - ndet/2)}.
static std::vector<float2> response_host(int64_t npad, int64_t ndet, int32_t filter, double weight, double center) {
  const std::vector<double> H = filter_response(npad, filter);
  const double shift = center - 0.5 * (double)ndet;
  const double scale = weight / (double)npad;
  std::vector<float2> F(H.size());
  for (int64_t k = 0; k <= npad / 2; ++k) {
    const double ph = 2.0 * M_PI * ((double)k / (double)npad) * shift;
    double re = H[(size_t)k] * scale * std::cos(ph), im = H[(size_t)k] * scale * std::sin(ph);
    if (k == npad / 2) im = 0.0;  // Hermitian Nyquist bin: real part only
    F[(size_t)k] = make_float2((float)re, (float)im);
  }
  return F;
}

tcp_status get_filter_table(int64_t ndet, int32_t filter, double weight, double center, FilterTable* out,
                            bool smooth) {
  int dev = 0;
  TCP_CUDA_TRY(cudaGetDevice(&dev));
  const int64_t npad = padded_length(ndet, smooth);
  FiltKey key;
  std::memset(&key, 0, sizeof(key));
  key.dev = dev;
  key.npad = npad;
  key.ndet = ndet;
  key.weight = weight;
  key.filter = filter;
  key.center = center;
  std::lock_guard<std::mutex> lk(g_mu);
  out->npad = (int)npad;
  const uint64_t twkey = ((uint64_t)(uint32_t)dev << 32) | (uint64_t)npad;
  auto tit = g_tw.find(twkey);
  if (tit == g_tw.end()) {  // one small table per padded length: not evicted
    const std::vector<float2> tw = twiddle_host(npad);
    float2* d = nullptr;
    TCP_CUDA_TRY(cudaMalloc(&d, tw.size() * sizeof(float2)));
    cudaError_t e = cudaMemcpy(d, tw.data(), tw.size() * sizeof(float2), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
      cudaFree(d);
      return cuda_fail(e, "upload twiddles");
    }
    tit = g_tw.emplace(twkey, d).first;
  }
  out->twiddle = tit->second;
  auto rit = g_resp.find(key);
  if (rit == g_resp.end()) {
    if (g_resp.size() >= kCacheCap) {
      auto lru = g_resp.begin();
      for (auto it = g_resp.begin(); it != g_resp.end(); ++it)
        if (it->second.used < lru->second.used) lru = it;
      cudaFree(lru->second.dev);
      g_resp.erase(lru);
    }
    const std::vector<float2> F = response_host(npad, ndet, filter, weight, center);
    float2* d = nullptr;
    TCP_CUDA_TRY(cudaMalloc(&d, F.size() * sizeof(float2)));
    cudaError_t e = cudaMemcpy(d, F.data(), F.size() * sizeof(float2), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
      cudaFree(d);
      return cuda_fail(e, "upload filter response");
    }
    rit = g_resp.emplace(key, RespEntry{d, 0}).first;
  }
  rit->second.used = ++g_stamp;
  out->response = rit->second.dev;
  return TCP_OK;
}

tcp_status build_filter_owned(int64_t ndet, int32_t filter, double weight, double center, bool smooth,
                              std::vector<void*>* owned, FilterTable* out) {
  const int64_t npad = padded_length(ndet, smooth);
  const std::vector<float2> tw = twiddle_host(npad);
  const std::vector<float2> F = response_host(npad, ndet, filter, weight, center);
  float2 *dt = nullptr, *dr = nullptr;
  TCP_CUDA_TRY(cudaMalloc(&dt, tw.size() * sizeof(float2)));
  owned->push_back(dt);
  TCP_CUDA_TRY(cudaMalloc(&dr, F.size() * sizeof(float2)));
  owned->push_back(dr);
  TCP_CUDA_TRY(cudaMemcpy(dt, tw.data(), tw.size() * sizeof(float2), cudaMemcpyHostToDevice));
  TCP_CUDA_TRY(cudaMemcpy(dr, F.data(), F.size() * sizeof(float2), cudaMemcpyHostToDevice));
  out->npad = (int)npad;
  out->twiddle = dt;
  out->response = dr;
  return TCP_OK;
}

static tcp_status cache_clear() {
  std::lock_guard<std::mutex> lk(g_mu);
  TCP_CUDA_TRY(cudaDeviceSynchronize());
  for (auto& kv : g_trig)
    for (auto& e : kv.second) cudaFree(e.dev);
  g_trig.clear();
  g_trig_count = 0;
  for (auto& kv : g_resp) cudaFree(kv.second.dev);
  g_resp.clear();
  for (auto& kv : g_tw) cudaFree(kv.second);
  g_tw.clear();
  fourierrec_cache_clear();
  lprec_cache_clear();
  return TCP_OK;
}

// --------------------------------------------------------- argument checks --

static int dtype_size(int dt) {
  switch (dt) {
    case TCP_U16: case TCP_F16: case TCP_BF16: case TCP_F16X2: return 2;
    case TCP_F32: return 4;
  }
  return 0;
}

tcp_status check_tensor(const tcp_tensor* t, const char* name, int ndim_lo, int ndim_hi) {
  if (!t) return fail(TCP_ERR_ARG, std::string(name) + ": null tensor");
  if (t->ndim < ndim_lo || t->ndim > ndim_hi)
    return fail(TCP_ERR_SHAPE, std::string(name) + ": wrong number of dimensions");
  if (dtype_size(t->dtype) == 0) return fail(TCP_ERR_DTYPE, std::string(name) + ": unknown dtype");
  int64_t numel = 1;
  for (int i = 0; i < t->ndim; ++i) {
    if (t->shape[i] < 0) return fail(TCP_ERR_SHAPE, std::string(name) + ": negative extent");
    if (t->shape[i] > (int64_t)INT32_MAX) return fail(TCP_ERR_SHAPE, std::string(name) + ": extent too large");
    numel *= t->shape[i];
  }
  if (numel > 0) {
    if (!t->data) return fail(TCP_ERR_ARG, std::string(name) + ": null data");
    if (t->shape[t->ndim - 1] > 1 && t->stride[t->ndim - 1] != 1)
      return fail(TCP_ERR_ALIGN, std::string(name) + ": innermost stride must be 1");
    if ((uintptr_t)t->data % dtype_size(t->dtype) != 0)
      return fail(TCP_ERR_ALIGN, std::string(name) + ": data not aligned to its dtype");
  }
  return TCP_OK;
}

// View of a 2- or 3-d tensor as [d0][d1][d2].
static View3 view3(const tcp_tensor* t) {
  View3 v;
  v.p = t->data;
  v.dtype = t->dtype;
  if (t->ndim == 3) {
    v.d0 = t->shape[0];
    v.d1 = t->shape[1];
    v.d2 = t->shape[2];
    v.s0 = t->stride[0];
    v.s1 = t->stride[1];
  } else if (t->ndim == 2) {
    v.d0 = 1;
    v.d1 = t->shape[0];
    v.d2 = t->shape[1];
    v.s0 = 0;
    v.s1 = t->stride[0];
  } else {
    v.d0 = 1;
    v.d1 = 1;
    v.d2 = t->shape[0];
    v.s0 = 0;
    v.s1 = 0;
  }
  return v;
}

static int64_t numel(const tcp_tensor* t) {
  int64_t n = 1;
  for (int i = 0; i < t->ndim; ++i) n *= t->shape[i];
  return n;
}

// Byte range [lo, hi) covered by a tensor.
static void extent(const tcp_tensor* t, uintptr_t* lo, uintptr_t* hi) {
  int64_t last = 0;
  for (int i = 0; i < t->ndim; ++i) last += (t->shape[i] - 1) * t->stride[i];
  *lo = (uintptr_t)t->data;
  *hi = (uintptr_t)t->data + (uintptr_t)(last + 1) * dtype_size(t->dtype);
}
bool overlap(const tcp_tensor* a, const tcp_tensor* b) {
  if (numel(a) == 0 || numel(b) == 0) return false;
  uintptr_t al, ah, bl, bh;
  extent(a, &al, &ah);
  extent(b, &bl, &bh);
  return al < bh && bl < ah;
}

static bool is_float(int dt) { return dt == TCP_F32 || dt == TCP_F16 || dt == TCP_BF16; }

// A sinogram argument: 3-d F32/F16/BF16 [nz][ntheta][ndet], or (where
// `split_ok`) a 4-d TCP_F16X2 [2][nz][ntheta][ndet] pair of FP16 planes.
static tcp_status check_sino(const tcp_tensor* t, const char* name, bool split_ok) {
  if (t && t->dtype == TCP_F16X2) {
    if (!split_ok) return fail(TCP_ERR_DTYPE, std::string(name) + ": F16X2 is accepted only by normalize_filter and backproject");
    tcp_status s = check_tensor(t, name, 4, 4);
    if (s != TCP_OK) return s;
    if (t->shape[0] != 2) return fail(TCP_ERR_SHAPE, std::string(name) + ": F16X2 must be [2][nz][ntheta][ndet]");
    const int64_t span = (t->shape[1] - 1) * t->stride[1] + (t->shape[2] - 1) * t->stride[2] + t->shape[3];
    if (numel(t) > 0 && (t->stride[1] < 0 || t->stride[2] < 0 || t->stride[0] < span))
      return fail(TCP_ERR_ALIGN, std::string(name) + ": F16X2 planes must not overlap (stride[0] >= one plane)");
    return TCP_OK;
  }
  tcp_status s = check_tensor(t, name, 3, 3);
  if (s != TCP_OK) return s;
  if (!is_float(t->dtype)) return fail(TCP_ERR_DTYPE, std::string(name) + ": sino must be F32, F16 or BF16");
  return TCP_OK;
}

// [nz][ntheta][ndet] view of a sinogram (the hi plane plus the plane offset
// for F16X2).
static View3 sino_view(const tcp_tensor* t) {
  if (t->dtype != TCP_F16X2) return view3(t);
  View3 v;
  v.p = t->data;
  v.dtype = TCP_F16X2;
  v.d0 = t->shape[1];
  v.d1 = t->shape[2];
  v.d2 = t->shape[3];
  v.s0 = t->stride[1];
  v.s1 = t->stride[2];
  v.plane = t->stride[0];
  return v;
}

static tcp_bp_config g_bp_override{0, 0, 0, 0};

tcp_bp_config bp_override() { return g_bp_override; }

}  // namespace tcp

using namespace tcp;

extern "C" {

const char* tcp_status_string(tcp_status s) {
  switch (s) {
    case TCP_OK: return "ok";
    case TCP_ERR_ARG: return "invalid argument";
    case TCP_ERR_SHAPE: return "invalid shape";
    case TCP_ERR_DTYPE: return "invalid dtype";
    case TCP_ERR_ALIGN: return "invalid stride or alignment";
    case TCP_ERR_CUDA: return "CUDA error";
    case TCP_ERR_OOM: return "out of memory";
    case TCP_ERR_TIMEOUT: return "device wait timed out";
    case TCP_ERR_DEVICE_CHECK: return "device index check failed";
    case TCP_ERR_UNSUPPORTED: return "unsupported";
    case TCP_ERR_ALIAS: return "overlapping input and output";
  }
  return "unknown status";
}

const char* tcp_last_error(void) { return g_last_error.c_str(); }

int tcp_version(void) { return TCP_VERSION; }

int64_t tcp_padded_length(int64_t ndet, int32_t pad_mode) {
  if (ndet < 1) return -1;
  return padded_length(ndet, pad_smooth(pad_mode));
}

tcp_status tcp_set_checked(int32_t on) {
  g_checked = on != 0;
  return TCP_OK;
}

tcp_status tcp_cache_clear(void) { return cache_clear(); }

tcp_status tcp_device_check(void* stream, uint32_t* word) {
  uint32_t* p = device_error_word();
  if (!p) return fail(TCP_ERR_CUDA, "device error word unavailable");
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  uint32_t h = 0;
  TCP_CUDA_TRY(cudaMemcpyAsync(&h, p, sizeof(h), cudaMemcpyDeviceToHost, st));
  TCP_CUDA_TRY(cudaMemsetAsync(p, 0, sizeof(uint32_t), st));
  TCP_CUDA_TRY(cudaStreamSynchronize(st));
  if (word) *word = h;
  if (h) return fail(TCP_ERR_DEVICE_CHECK, "device error word set: " + std::to_string(h));
  return TCP_OK;
}

tcp_status tcp_frame_mean(const tcp_tensor* frames, tcp_tensor* mean, void* stream) {
  tcp_status s;
  if ((s = check_tensor(frames, "frames", 3, 3)) != TCP_OK) return s;
  if ((s = check_tensor(mean, "mean", 2, 2)) != TCP_OK) return s;
  if (frames->dtype != TCP_U16) return fail(TCP_ERR_DTYPE, "frames must be U16");
  if (mean->dtype != TCP_F32) return fail(TCP_ERR_DTYPE, "mean must be F32");
  if (mean->shape[0] != frames->shape[1] || mean->shape[1] != frames->shape[2])
    return fail(TCP_ERR_SHAPE, "mean must be [nz][ndet] of frames [nf][nz][ndet]");
  if (frames->shape[0] < 1 && numel(mean) > 0) return fail(TCP_ERR_SHAPE, "need at least one frame");
  return launch_frame_mean(view3(frames), view3(mean), reinterpret_cast<cudaStream_t>(stream));
}

static tcp_status normalize_impl(const tcp_tensor* raw, const tcp_tensor* dark, const tcp_tensor* flat,
                                 tcp_tensor* sino, const FilterTable* ft, int32_t pad_mode, void* stream);

tcp_status tcp_normalize(const tcp_tensor* raw, const tcp_tensor* dark, const tcp_tensor* flat, tcp_tensor* sino,
                         void* stream) {
  return normalize_impl(raw, dark, flat, sino, nullptr, TCP_PAD_EDGE, stream);
}

tcp_status tcp_normalize_filter_ex(const tcp_tensor* raw, const tcp_tensor* dark, const tcp_tensor* flat,
                                   tcp_tensor* sino, int32_t filter, double center, int32_t pad_mode, double weight,
                                   void* stream) {
  if (filter < TCP_FILTER_SHEPP || filter > TCP_FILTER_NONE) return fail(TCP_ERR_ARG, "unknown filter");
  if (!valid_pad_mode(pad_mode)) return fail(TCP_ERR_ARG, "unknown pad mode");
  if (!std::isfinite(center)) return fail(TCP_ERR_ARG, "center must be finite");
  if (!std::isfinite(weight)) return fail(TCP_ERR_ARG, "weight must be finite");
  FilterTable ft;
  tcp_status s;
  if ((s = check_sino(sino, "sino", true)) != TCP_OK) return s;
  const View3 sv = sino_view(sino);
  if (sv.d2 > 4096) return fail(TCP_ERR_UNSUPPORTED, "filter: ndet > 4096 (padded length > 8192)");
  if (raw && raw->ndim == 3 && numel(sino) > 0 && numel(raw) > 0) {
    const double w = weight > 0 ? weight : M_PI / (double)sv.d1;
    if ((s = get_filter_table(sv.d2, filter, w, center, &ft, pad_smooth(pad_mode))) != TCP_OK) return s;
  } else {
    ft.npad = 0;
  }
  return normalize_impl(raw, dark, flat, sino, &ft, pad_mode, stream);
}

tcp_status tcp_normalize_filter(const tcp_tensor* raw, const tcp_tensor* dark, const tcp_tensor* flat,
                                tcp_tensor* sino, int32_t filter, double center, int32_t pad_mode, void* stream) {
  return tcp_normalize_filter_ex(raw, dark, flat, sino, filter, center, pad_mode, 0.0, stream);
}

static tcp_status normalize_impl(const tcp_tensor* raw, const tcp_tensor* dark, const tcp_tensor* flat,
                                 tcp_tensor* sino, const FilterTable* ft, int32_t pad_mode, void* stream) {
  tcp_status s;
  if ((s = check_tensor(raw, "raw", 3, 3)) != TCP_OK) return s;
  if ((s = check_tensor(dark, "dark", 2, 3)) != TCP_OK) return s;
  if ((s = check_tensor(flat, "flat", 2, 3)) != TCP_OK) return s;
  if ((s = check_sino(sino, "sino", ft != nullptr)) != TCP_OK) return s;
  if (raw->dtype != TCP_U16) return fail(TCP_ERR_DTYPE, "raw must be U16");
  const int64_t nt = raw->shape[0], nz = raw->shape[1], nd = raw->shape[2];
  const View3 sview = sino_view(sino);
  if (sview.d0 != nz || sview.d1 != nt || sview.d2 != nd)
    return fail(TCP_ERR_SHAPE, "sino must be [nz][ntheta][ndet] of raw [ntheta][nz][ndet]");
  for (const tcp_tensor* df : {dark, flat}) {
    if (df->ndim == 2) {
      if (df->dtype != TCP_F32) return fail(TCP_ERR_DTYPE, "2-d dark/flat must be F32 means");
      if (df->shape[0] != nz || df->shape[1] != nd) return fail(TCP_ERR_SHAPE, "dark/flat means must be [nz][ndet]");
    } else {
      if (df->dtype != TCP_U16) return fail(TCP_ERR_DTYPE, "3-d dark/flat must be U16 frames");
      if (df->shape[1] != nz || df->shape[2] != nd) return fail(TCP_ERR_SHAPE, "dark/flat frames must be [nf][nz][ndet]");
      if (df->shape[0] < 1 && nz * nd > 0) return fail(TCP_ERR_SHAPE, "dark/flat need at least one frame");
    }
  }
  if (overlap(raw, sino)) return fail(TCP_ERR_ALIAS, "raw and sino overlap");
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  if (numel(sino) == 0) return TCP_OK;
  float* scratch = nullptr;
  View3 dv = view3(dark), fv = view3(flat);
  const bool need = dark->ndim == 3 || flat->ndim == 3;
  if (need) {
    TCP_CUDA_TRY(cudaMallocAsync((void**)&scratch, sizeof(float) * 2 * (size_t)(nz * nd), st));
    View3 m;
    m.dtype = TCP_F32;
    m.d0 = 1;
    m.d1 = nz;
    m.d2 = nd;
    m.s0 = 0;
    m.s1 = nd;
    if (dark->ndim == 3) {
      m.p = scratch;
      if ((s = launch_frame_mean(dv, m, st)) != TCP_OK) { cudaFreeAsync(scratch, st); return s; }
      dv = m;
    }
    if (flat->ndim == 3) {
      m.p = scratch + nz * nd;
      if ((s = launch_frame_mean(fv, m, st)) != TCP_OK) { cudaFreeAsync(scratch, st); return s; }
      fv = m;
    }
  }
  s = ft ? launch_normalize_filter(view3(raw), dv, fv, sview, *ft, pad_mode, st)
         : launch_normalize(view3(raw), dv, fv, sview, st);
  if (scratch) {
    cudaError_t e = cudaFreeAsync(scratch, st);
    if (s == TCP_OK && e != cudaSuccess) return cuda_fail(e, "cudaFreeAsync");
  }
  return s;
}

tcp_status tcp_filter_ex(tcp_tensor* sino, int32_t filter, double center, int32_t pad_mode, int64_t ntheta,
                         void* stream) {
  tcp_status s;
  if ((s = check_tensor(sino, "sino", 2, 3)) != TCP_OK) return s;
  if (!is_float(sino->dtype)) return fail(TCP_ERR_DTYPE, "sino must be F32, F16 or BF16");
  if (filter < TCP_FILTER_SHEPP || filter > TCP_FILTER_NONE) return fail(TCP_ERR_ARG, "unknown filter");
  if (!valid_pad_mode(pad_mode)) return fail(TCP_ERR_ARG, "unknown pad mode");
  if (!std::isfinite(center)) return fail(TCP_ERR_ARG, "center must be finite");
  View3 v = view3(sino);
  if (v.d2 > 4096) return fail(TCP_ERR_UNSUPPORTED, "filter: ndet > 4096 (padded length > 8192)");
  const int64_t nt = ntheta > 0 ? ntheta : v.d1;
  if (numel(sino) == 0) return TCP_OK;
  FilterTable ft;
  if ((s = get_filter_table(v.d2, filter, M_PI / (double)nt, center, &ft, pad_smooth(pad_mode))) != TCP_OK)
    return s;
  return launch_filter(v, ft, pad_mode, reinterpret_cast<cudaStream_t>(stream));
}

tcp_status tcp_filter(tcp_tensor* sino, int32_t filter, double center, void* stream) {
  return tcp_filter_ex(sino, filter, center, TCP_PAD_EDGE, 0, stream);
}

tcp_status tcp_set_backproject_config(const tcp_bp_config* cfg) {
  if (!cfg) {
    g_bp_override = tcp_bp_config{0, 0, 0, 0};
    return TCP_OK;
  }
  if (!valid_bp_config(*cfg)) return fail(TCP_ERR_UNSUPPORTED, "no backprojector instantiated for this config");
  g_bp_override = *cfg;
  return TCP_OK;
}

tcp_status tcp_get_backproject_config(int64_t nz, int64_t ntheta, int64_t ndet, int64_t n, int32_t sdt, int32_t vdt,
                                      tcp_bp_config* cfg) {
  if (!cfg) return fail(TCP_ERR_ARG, "null config");
  if (g_bp_override.k_slices) *cfg = g_bp_override;
  else if (!tuned_bp_config(nz, ntheta, ndet, n, sdt, vdt, cfg)) *cfg = default_bp_config(nz, ntheta, ndet, n, sdt, vdt);
  return TCP_OK;
}

tcp_status tcp_backproject(const tcp_tensor* sino, const double* theta, double center, tcp_tensor* vol,
                           void* stream) {
  return tcp_backproject_ex(sino, theta, center, vol, 1.0, stream);
}

tcp_status tcp_backproject_ex(const tcp_tensor* sino, const double* theta, double center, tcp_tensor* vol,
                              double scale, void* stream) {
  tcp_status s;
  if (!std::isfinite(scale)) return fail(TCP_ERR_ARG, "scale must be finite");
  if ((s = check_sino(sino, "sino", true)) != TCP_OK) return s;
  if ((s = check_tensor(vol, "vol", 3, 3)) != TCP_OK) return s;
  if (!is_float(vol->dtype)) return fail(TCP_ERR_DTYPE, "vol must be F32, F16 or BF16");
  const View3 sv = sino_view(sino);
  if (vol->shape[0] != sv.d0) return fail(TCP_ERR_SHAPE, "vol and sino must have the same slice count");
  if (vol->shape[1] != vol->shape[2]) return fail(TCP_ERR_SHAPE, "vol slices must be square [n][n]");
  if (!std::isfinite(center)) return fail(TCP_ERR_ARG, "center must be finite");
  const int64_t nt = sv.d1;
  if (nt > 0 && !theta) return fail(TCP_ERR_ARG, "theta is null");
  for (int64_t i = 0; i < nt; ++i)
    if (!std::isfinite(theta[i])) return fail(TCP_ERR_ARG, "theta must be finite");
  if (overlap(sino, vol)) return fail(TCP_ERR_ALIAS, "sino and vol overlap");
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  if (numel(vol) == 0) return TCP_OK;
  if (nt == 0 || sv.d2 == 0) {  // no rays: the sum is zero
    for (int64_t z = 0; z < vol->shape[0]; ++z)
      TCP_CUDA_TRY(cudaMemset2DAsync((char*)vol->data + z * vol->stride[0] * dtype_size(vol->dtype),
                                     vol->stride[1] * dtype_size(vol->dtype), 0,
                                     vol->shape[2] * dtype_size(vol->dtype), vol->shape[1], st));
    return TCP_OK;
  }
  TrigTable trig;
  if ((s = get_trig_table(theta, nt, &trig)) != TCP_OK) return s;
  tcp_bp_config cfg;
  tcp_get_backproject_config(sv.d0, nt, sv.d2, vol->shape[1], sino->dtype, vol->dtype, &cfg);
  return launch_backproject(sv, trig, center, view3(vol), cfg, st, (float)scale);
}

tcp_status tcp_fourierrec(const tcp_tensor* sino, const double* theta, double center, tcp_tensor* vol,
                          double scale, int32_t width, void* stream) {
  tcp_status s;
  if (!std::isfinite(scale)) return fail(TCP_ERR_ARG, "scale must be finite");
  if ((s = check_tensor(sino, "sino", 3, 4)) != TCP_OK) return s;
  if (!is_float(sino->dtype)) return fail(TCP_ERR_DTYPE, "fourierrec: sino must be F32, F16 or BF16");
  if (sino->ndim != 3) return fail(TCP_ERR_SHAPE, "fourierrec: sino must be [nz][ntheta][ndet]");
  if ((s = check_tensor(vol, "vol", 3, 3)) != TCP_OK) return s;
  if (!is_float(vol->dtype)) return fail(TCP_ERR_DTYPE, "vol must be F32, F16 or BF16");
  if (vol->shape[0] != sino->shape[0]) return fail(TCP_ERR_SHAPE, "vol and sino must have the same slice count");
  if (vol->shape[1] != vol->shape[2]) return fail(TCP_ERR_SHAPE, "vol slices must be square [n][n]");
  if (!std::isfinite(center)) return fail(TCP_ERR_ARG, "center must be finite");
  const int64_t nt = sino->shape[1], nd = sino->shape[2], n = vol->shape[1];
  if (nt > 0 && !theta) return fail(TCP_ERR_ARG, "theta is null");
  for (int64_t i = 0; i < nt; ++i)
    if (!std::isfinite(theta[i])) return fail(TCP_ERR_ARG, "theta must be finite");
  const int w = width == 0 ? fourierrec_default_width(vol->dtype, n) : width;
  if ((s = fourierrec_check(nt, nd, n, w)) != TCP_OK) return s;
  if (overlap(sino, vol)) return fail(TCP_ERR_ALIAS, "sino and vol overlap");
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  if (numel(vol) == 0) return TCP_OK;
  if (nt == 0 || nd == 0) {  // no rays: the sum is zero
    for (int64_t z = 0; z < vol->shape[0]; ++z)
      TCP_CUDA_TRY(cudaMemset2DAsync((char*)vol->data + z * vol->stride[0] * dtype_size(vol->dtype),
                                     vol->stride[1] * dtype_size(vol->dtype), 0,
                                     vol->shape[2] * dtype_size(vol->dtype), vol->shape[1], st));
    return TCP_OK;
  }
  TrigTable trig;
  if ((s = get_trig_table(theta, nt, &trig)) != TCP_OK) return s;
  return launch_fourierrec(view3(sino), theta, trig, center, view3(vol), (float)scale, w, st);
}

tcp_status tcp_lprec(const tcp_tensor* sino, const double* theta, double center, tcp_tensor* vol, double scale,
                     double oversampling, void* stream) {
  tcp_status s;
  if (!std::isfinite(scale)) return fail(TCP_ERR_ARG, "scale must be finite");
  if ((s = check_tensor(sino, "sino", 3, 4)) != TCP_OK) return s;
  if (!is_float(sino->dtype) || sino->ndim != 3)
    return fail(TCP_ERR_DTYPE, "lprec: sino must be F32, F16 or BF16 [nz][ntheta][ndet]");
  if ((s = check_tensor(vol, "vol", 3, 3)) != TCP_OK) return s;
  if (!is_float(vol->dtype)) return fail(TCP_ERR_DTYPE, "vol must be F32, F16 or BF16");
  if (vol->shape[0] != sino->shape[0]) return fail(TCP_ERR_SHAPE, "vol and sino must have the same slice count");
  if (vol->shape[1] != vol->shape[2]) return fail(TCP_ERR_SHAPE, "vol slices must be square [n][n]");
  if (!std::isfinite(center)) return fail(TCP_ERR_ARG, "center must be finite");
  const int64_t nt = sino->shape[1], nd = sino->shape[2], n = vol->shape[1];
  if (nt > 0 && !theta) return fail(TCP_ERR_ARG, "theta is null");
  for (int64_t i = 0; i < nt; ++i)
    if (!std::isfinite(theta[i])) return fail(TCP_ERR_ARG, "theta must be finite");
  const double os = oversampling > 0 ? oversampling : 2.0;
  if (overlap(sino, vol)) return fail(TCP_ERR_ALIAS, "sino and vol overlap");
  LpHostGeom probe;
  if (nt >= 1 && (s = lprec_geometry(theta, nt, nd, std::max<int64_t>(n, 1), center, os, &probe)) != TCP_OK) return s;
  if (nt >= 1 && (s = lprec_check(probe)) != TCP_OK) return s;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  if (numel(vol) == 0) return TCP_OK;
  if (nt == 0 || nd == 0) return fail(TCP_ERR_SHAPE, "lprec: empty projections for a non-empty volume");
  const LpHostGeom* g = nullptr;
  const LpDevGeom* d = nullptr;
  if ((s = lprec_cached(theta, nt, nd, n, center, os, &g, &d)) != TCP_OK) return s;
  const int zpass = lprec_slices_per_pass(*g, vol->shape[0]);
  void* ws = nullptr;
  TCP_CUDA_TRY(cudaMallocAsync(&ws, lprec_workspace_bytes(*g, zpass), st));
  s = launch_lprec_ws(view3(sino), *g, *d, ws, zpass, view3(vol), (float)scale, st);
  const cudaError_t e = cudaFreeAsync(ws, st);
  if (s == TCP_OK && e != cudaSuccess) return cuda_fail(e, "cudaFreeAsync");
  return s;
}

tcp_status tcp_project(const tcp_tensor* vol, const double* theta, double center, tcp_tensor* sino, void* stream) {
  tcp_status s;
  if ((s = check_tensor(vol, "vol", 3, 3)) != TCP_OK) return s;
  if ((s = check_tensor(sino, "sino", 3, 3)) != TCP_OK) return s;
  if (!is_float(sino->dtype) || !is_float(vol->dtype)) return fail(TCP_ERR_DTYPE, "sino/vol must be F32, F16 or BF16");
  if (vol->shape[0] != sino->shape[0]) return fail(TCP_ERR_SHAPE, "vol and sino must have the same slice count");
  if (vol->shape[1] != vol->shape[2]) return fail(TCP_ERR_SHAPE, "vol slices must be square [n][n]");
  if (!std::isfinite(center)) return fail(TCP_ERR_ARG, "center must be finite");
  const int64_t nt = sino->shape[1];
  if (nt > 0 && !theta) return fail(TCP_ERR_ARG, "theta is null");
  for (int64_t i = 0; i < nt; ++i)
    if (!std::isfinite(theta[i])) return fail(TCP_ERR_ARG, "theta must be finite");
  if (overlap(sino, vol)) return fail(TCP_ERR_ALIAS, "sino and vol overlap");
  if (numel(sino) == 0) return TCP_OK;
  TrigTable trig;
  if ((s = get_trig_table(theta, nt, &trig)) != TCP_OK) return s;
  return launch_project(view3(vol), trig, center, view3(sino), reinterpret_cast<cudaStream_t>(stream));
}

}  // extern "C"
