// Allocation-free form of tcp_normalize for uint16 dark/flat frames.
//
// tcp_normalize averages dark and flat frames into scratch memory that it
// takes from the stream-ordered allocator.  Some callers cannot allow that:
// an acquisition or steering service that reserves all device memory for its
// own pool at start-up and forbids any further device allocation while a
// scan is running (to rule out allocation latency and out-of-memory failures
// in the middle of an experiment), or a host framework whose allocator owns
// the whole device.  For them, this entry point keeps the two frame means in
// one fixed array that lives in the library's module (a file-scope __device__
// array), so the call allocates nothing.
//
// Costs and limits of that choice:
//   - Every GPU that loads the library holds the array (8 MiB) until the
//     process exits.
//   - At most kMaxMean = 1,048,576 elements per mean (nz * ndet); larger
//     requests are rejected with TCP_ERR_SHAPE.
//   - All calls on a device share the array.  Calls whose work overlaps on the
//     GPU (other streams, or other host threads) race on it; serialise them.
//   - The first call on a device looks up the array's device address (with
//     that device current) and caches it; make that first call before any
//     stream capture.  The array keeps the previous call's values; nothing in
//     it needs to start at zero because each call overwrites every element it
//     later reads.
#include <mutex>
#include <string>
#include <unordered_map>

#include "tcp_internal.cuh"

namespace tcp {
namespace {

constexpr int64_t kMaxMean = 1 << 20;  // elements per mean (nz * ndet)

// [0, kMaxMean): dark mean, [kMaxMean, 2 kMaxMean): flat mean.
static __device__ __align__(256) float g_noalloc_means[2 * kMaxMean];

std::mutex g_na_mu;
std::unordered_map<int, float*> g_na_ptr;

// Device address of the array on the current device (cached per device).  In
// host code the symbol itself is only a host-side stand-in, never a device
// address, so it must be translated here before a kernel may use it.
tcp_status means_scratch(float** out) {
  int dev = 0;
  TCP_CUDA_TRY(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lk(g_na_mu);
  auto it = g_na_ptr.find(dev);
  if (it == g_na_ptr.end()) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_means);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(no-alloc means)");
    it = g_na_ptr.emplace(dev, reinterpret_cast<float*>(p)).first;
  }
  *out = it->second;
  return TCP_OK;
}

bool valid3(const tcp_tensor* t) {
  if (!t || t->ndim != 3) return false;
  for (int i = 0; i < 3; ++i)
    if (t->shape[i] < 0 || t->shape[i] > (int64_t)INT32_MAX) return false;
  return t->stride[2] == 1 || t->shape[2] <= 1;
}

View3 as_view(const tcp_tensor* t) {
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

}  // namespace
}  // namespace tcp

using namespace tcp;

extern "C" tcp_status tcp_normalize_noalloc(const tcp_tensor* raw, const tcp_tensor* dark, const tcp_tensor* flat,
                                            tcp_tensor* sino, void* stream) {
  // the descriptor checks of tcp_normalize (unit innermost stride, data
  // aligned to its dtype, ...) come first, so that no misaligned pointer
  // reaches a kernel
  tcp_status s;
  if ((s = check_tensor(raw, "raw", 3, 3)) != TCP_OK) return s;
  if ((s = check_tensor(dark, "dark", 3, 3)) != TCP_OK) return s;
  if ((s = check_tensor(flat, "flat", 3, 3)) != TCP_OK) return s;
  if ((s = check_tensor(sino, "sino", 3, 3)) != TCP_OK) return s;
  if (!valid3(raw) || !valid3(dark) || !valid3(flat) || !valid3(sino))
    return fail(TCP_ERR_SHAPE, "normalize_noalloc: raw, dark, flat and sino must be 3-d with unit innermost stride");
  if (raw->dtype != TCP_U16 || dark->dtype != TCP_U16 || flat->dtype != TCP_U16)
    return fail(TCP_ERR_DTYPE, "normalize_noalloc: raw and the dark/flat frames must be U16");
  if (sino->dtype != TCP_F32 && sino->dtype != TCP_F16 && sino->dtype != TCP_BF16)
    return fail(TCP_ERR_DTYPE, "normalize_noalloc: sino must be F32, F16 or BF16");
  const int64_t nt = raw->shape[0], nz = raw->shape[1], nd = raw->shape[2];
  if (sino->shape[0] != nz || sino->shape[1] != nt || sino->shape[2] != nd)
    return fail(TCP_ERR_SHAPE, "normalize_noalloc: sino must be [nz][ntheta][ndet] of raw [ntheta][nz][ndet]");
  for (const tcp_tensor* f : {dark, flat})
    if (f->shape[1] != nz || f->shape[2] != nd || f->shape[0] < 1)
      return fail(TCP_ERR_SHAPE, "normalize_noalloc: dark/flat must be U16 frames [nf >= 1][nz][ndet]");
  if (nz * nd > kMaxMean)
    return fail(TCP_ERR_SHAPE, "normalize_noalloc: nz * ndet = " + std::to_string(nz * nd) +
                                   " exceeds the fixed scratch of " + std::to_string(kMaxMean) +
                                   " elements per mean; use tcp_normalize");
  if (overlap(raw, sino)) return fail(TCP_ERR_ALIAS, "normalize_noalloc: raw and sino overlap");
  if (overlap(dark, sino) || overlap(flat, sino))
    return fail(TCP_ERR_ALIAS, "normalize_noalloc: dark/flat and sino overlap");
  if (nt * nz * nd == 0) return TCP_OK;
  float* scratch = nullptr;
  s = means_scratch(&scratch);
  if (s != TCP_OK) return s;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  View3 dm, fm;
  dm.p = scratch;
  dm.dtype = TCP_F32;
  dm.d0 = 1;
  dm.d1 = nz;
  dm.d2 = nd;
  dm.s0 = 0;
  dm.s1 = nd;
  fm = dm;
  fm.p = scratch + kMaxMean;
  if ((s = launch_frame_mean(as_view(dark), dm, st)) != TCP_OK) return s;
  if ((s = launch_frame_mean(as_view(flat), fm, st)) != TCP_OK) return s;
  return launch_normalize(as_view(raw), dm, fm, as_view(sino), st);
}
