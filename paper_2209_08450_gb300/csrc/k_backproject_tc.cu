// LineRec backprojection on the 5th-generation tensor cores, for 16-bit
// sinograms (Sec. 2.2 / Sec. 3 of the TomocuPy paper; 16-bit storage with
// FP32 accumulation, Sec. 2.1).
//
// For one angle, the backprojection of a voxel tile into K slices is a matrix
// product: vol[v][z] += sum_j W[v][j] q[z][j], where row v of W holds the
// two linear-interpolation weights (1 - w, w) at the detector samples floor(s)
// and floor(s) + 1 of that voxel's ray, inside a 32-sample window that covers
// the tile.  Only 2 of 32 entries per row are non-zero, but the tensor pipe
// runs ~30x the FP32 FMA rate, and the slice dimension (N = 256) reuses every
// weight 256 times.
//
//   A = W      two 128 x 32 halves (a 16 x 16 voxel tile: rows 0-7 and 8-15)
//              built by 8 warps in shared memory (64-byte-swizzled K-major);
//   B = q      N slices x 32 samples of one sinogram row, one TMA tile copy
//              (64-byte swizzle, zero fill outside the detector), shared by
//              both halves: the footprint of a 16 x 16 tile spans at most
//              15 sqrt(2) < 22 samples, so 32 still cover it after the window
//              start is rounded down to 16 bytes;
//   D          two 128 x N FP32 accumulators in tensor memory (2N columns)
//              for the whole angle loop; read back once with tcgen05.ld.
//
// Split mode (below) swaps the operands: D[z][v] = q W^T with the CTA's 128
// sinogram rows (slices) as the MMA's M and the 256 weight rows of both
// halves as its N, one MMA per K step and product.  The copy of one angle's window for all N slices reads one
// contiguous block when the sinogram is stored angle-major ([theta][z][j],
// the layout tcp_fbp's chunks use); the tensor map follows whichever of the
// slice and angle strides is smaller.
//
// Pipeline per CTA: warp-specialised roles (weight builders, TMA producer,
// MMA issuer) exchange stages of two angles through rings of shared buffers
// guarded by mbarriers, so weight building, copies and MMAs overlap.  The
// rings normally fill the shared memory (one CTA per SM); with few slices per
// weight matrix the builders bind, and 16-bit launches can size the rings for
// half of it so that two CTAs share an SM (their accumulators then take at
// most 256 TMEM columns each).
// Every mbarrier wait is bounded by a clock budget; on timeout the kernel
// records kErrTimeout, every role stops, the issued MMAs are drained (bounded)
// and the tensor memory is freed.
//
// The ray coordinate and the weights come from the same canonical geometry as
// the CUDA-core backprojector (FP64 tile origin + FP32 in-tile offsets), the
// weights rounded to the sinogram's 16-bit type.
//
// Split mode (TCP_F16X2 sinograms, FP32 accuracy): every sample is stored as
// FP16 hi + lo and every weight is split the same way, so each angle runs
// three products per accumulator, A_hi B_hi + A_hi B_lo + A_lo B_hi (the
// dropped A_lo B_lo is below 2^-22 of the term); the FP16 x FP16 products are
// exact, but the tensor core's accumulation into TMEM does not round to
// nearest: its error grows linearly with the number of accumulation steps
// (measured: 1.2e-4 relative after 2048 angles).  Split mode therefore
// accumulates segments of kTcSeg angles on the tensor cores and adds each
// segment into FP32 running sums held in TMEM next to the accumulators, with
// round-to-nearest FP32 adds on the CUDA cores (N <= 128 leaves room for
// both: 2N accumulator columns + 2N sum columns).
#include <cuda.h>
#include <cudaTypedefs.h>

#include <mutex>

#include "tcp_internal.cuh"

namespace tcp {
namespace {

constexpr int kTcM = 128;          // voxels per MMA (16 x 8)
constexpr int kTcH = 2;            // MMAs (accumulators) per tile: 16 x 16 voxels
constexpr int kTcK = 32;           // detector samples per angle window
constexpr int kTcRowBytes = 64;    // one K-major row of 32 x 16-bit
constexpr int kTcHalfA = kTcM * kTcRowBytes;   // 8 KB of weights per half
constexpr int kTcAngleA = kTcH * kTcHalfA;     // 16 KB of weights per angle
constexpr int kTcBuilders = 4 * kTcH;          // builder warps (one voxel row per thread)
constexpr int kTcThreads = 32 * (kTcBuilders + 2);
constexpr long long kTcBudget = 4000000000ll;  // clock cycles per wait (~2 s)
constexpr size_t kTcSmemLimit = 232448;        // opt-in shared memory per block
constexpr size_t kTcSmemPerSM = 233472;        // shared memory per SM (228 KB; 1 KB reserved per block)
// Blocks per SM at most: two at 68 registers.  Three or four (48 registers,
// shallower rings) measured slower at 2048^2 x 2048 angles: 41.5 against
// 40.9 ms for 32 slices.
constexpr int kTcMaxBlocks = 2;

struct TcArgs {
  int nz, ntheta, ndet, n;
  int nsub_x, nsub_y;  // 16 x 16 sub-tiles along x and y
  int N;               // slices per CTA (multiple of 16, <= 256)
  void* vol;
  int vdt;
  int64_t v_z, v_y;
  const double2* trig;
  double center, half_n;
  float scale;
  uint32_t idesc;
  uint32_t* err;
  int check;
  int na, nbb;  // A and B ring depths (stages)
  int vec4;     // FP32 volume with 16-byte aligned rows: 16-byte stores in the epilogue
  int zfirst;   // tensor map dimensions (sample, slice, angle) instead of (sample, angle, slice)
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}

__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap* map, uint32_t bar, int x, int y, int z) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4, %5}], [%2];"
      ::"r"(dst), "l"(reinterpret_cast<uint64_t>(map)), "r"(bar), "r"(x), "r"(y), "r"(z)
      : "memory");
}

// Shared-memory matrix descriptor: K-major, 64-byte swizzle, 8-row groups 512 B apart.
__device__ __forceinline__ uint64_t sw64_desc(uint32_t addr) {
  uint64_t d = 0;
  d |= (uint64_t)((addr >> 4) & 0x3fff);      // start address
  d |= (uint64_t)1 << 16;                      // leading byte offset (unused for swizzled K-major)
  d |= (uint64_t)(512 >> 4) << 32;             // stride byte offset
  d |= (uint64_t)1 << 46;                      // descriptor version
  d |= (uint64_t)4 << 61;                      // layout: 64-byte swizzle
  return d;
}

__device__ __forceinline__ void mma_f16(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n"
      ::"r"(tmem_d), "l"(a), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}
__device__ __forceinline__ void mma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}

template <class TS> __device__ __forceinline__ uint16_t weight_bits(float w);
template <> __device__ __forceinline__ uint16_t weight_bits<__half>(float w) {
  return __half_as_ushort(__float2half_rn(w));
}
template <> __device__ __forceinline__ uint16_t weight_bits<__nv_bfloat16>(float w) {
  return __bfloat16_as_ushort(__float2bfloat16_rn(w));
}

template <class TV>
__device__ __forceinline__ void put(void* base, int64_t off, float v) {
  Store<TV>::put(reinterpret_cast<TV*>(base) + off, v);
}

// Warp roles (320 threads):
//   warps 0-7  build the weight matrices A (one voxel row per thread; warps
//              4h .. 4h+3 own half h) and, at the end, read D out of tensor
//              memory (warp w reads lanes 32 (w % 4) .. of accumulator w / 4)
//              and store the tile;
//   warp 8     producer: tile geometry (32 angles per pass) and the TMA
//              copies of B;
//   warp 9     issues the MMAs (one elected thread) and commits them.
// A stage is S angles (1 or 2).  A (built in the SM, cheap) cycles through NA
// buffers; B (copied from L2, microseconds away) through NBB buffers, as many
// as the remaining shared memory holds, so that up to ~180 KB of copies are
// in flight.  Each cross-role hand-off costs the MMA thread a wake-up, so a
// stage has one barrier for "ready" and one for "consumed":
//   geo_full[s % NBB] producer -> builders: geometry of stage s is written
//   full    [s % NBB] builders (8 warp arrivals) + producer (expect_tx and the
//                     TMA bytes) -> MMA: A and B of stage s are in place
//   empty   [s % NBB] MMA commit -> producer (B slot s % NBB free) and
//                     builders (A slot s % NA free once stage s - NA is
//                     consumed; NA <= NBB)
// Stage s waits the phase (s / NBB) & 1 of its ring slot.
constexpr int kTcSeg = 32;      // split mode: angles per tensor-core accumulation segment
constexpr int kTcMaxNA = 4;     // A stage buffers (at most)
constexpr int kTcMaxNBB = 32;   // B stage buffers (at most)
constexpr int kTcGeoRing = 64;  // geometry ring (two chunks of 32 angles)
// The geometry of chunk c overwrites that of chunk c - 2 once empty of
// stage c * 32 / S - NBB has completed; the builders are then done with
// every stage up to there, which covers chunk c - 2 if NBB <= 32 / S + 1.
__host__ __device__ constexpr int tc_max_nbb(int S) { return 32 / S < kTcMaxNBB ? 32 / S : kTcMaxNBB; }

struct TcGeoP {  // packed geometry of one angle (16 bytes)
  int bj;        // low 16 bits: i0 - j0, high 16 bits: j0 (both signed)
  float f0, c, s;
};

struct TcBars {
  uint64_t geo_full[kTcMaxNBB], full[kTcMaxNBB], empty[kTcMaxNBB], done;
  uint64_t seg_done, seg_free;  // split mode: segment accumulated / accumulators read
  uint32_t tmem;
  int abort;
};

__device__ __forceinline__ bool wait_or_abort(uint32_t bar, uint32_t parity, volatile int* abort, uint32_t* err) {
  const long long t0 = clock64();
  while (!mbar_try(bar, parity)) {
    if (*abort) return false;
    if (clock64() - t0 > kTcBudget) {
      *abort = 1;
      atomicOr(err, kErrTimeout);
      return false;
    }
  }
  return true;
}
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

// 16 consecutive TMEM columns of this warp's 32 lanes (one per thread).
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, "
      "%14, %15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
}
__device__ __forceinline__ void tmem_st16(uint32_t taddr, const uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15, %16};" ::"r"(taddr),
      "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]), "r"(r[8]), "r"(r[9]),
      "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]), "r"(r[15])
      : "memory");
}

// shared memory: [A: NA x S x P x 16 KB][B: NBB x S x P x N*64 B][geo ring]
// [barriers], P = 2 planes (hi, lo) in split mode, else 1.
template <class TS, int kTcS2, bool SPLIT>
__global__ void __launch_bounds__(kTcThreads, 1) k_backproject_tc(const __grid_constant__ CUtensorMap tmap,
                                                                   const __grid_constant__ CUtensorMap tmap_lo,
                                                                   TcArgs a) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* smem = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  constexpr int kParts = SPLIT ? 2 : 1;
  // Split mode swaps the operands: the sinogram rows (slices) are the MMA's
  // M side and both weight halves its N = 256 side, so one MMA covers the
  // whole tile and each K step reads 12 KB of operands instead of 16 KB.
  // Its sinogram stages then hold 128 rows whatever N is (rows past N are
  // never copied; their results are never stored).
  constexpr bool SWAP = SPLIT;
  const int N = a.N;
  const int rowsB = SWAP ? kTcM : N;       // sinogram rows per angle and plane in shared memory
  const int bBytes = rowsB * kTcRowBytes;  // B bytes per angle and plane
  const int angleB = kParts * bBytes;      // B bytes per angle
  const int txB = kParts * N * kTcRowBytes;  // bytes the copies of one angle deliver
  constexpr int angleA = kParts * kTcAngleA;
  unsigned char* Abuf = smem;
  const int NA = a.na, NBB = a.nbb;  // ring depths (stages)
  unsigned char* Bbuf = smem + NA * kTcS2 * angleA;
  TcGeoP* geo = reinterpret_cast<TcGeoP*>(Bbuf + NBB * kTcS2 * angleB);  // angle th -> geo[th % 64]
  TcBars* bars = reinterpret_cast<TcBars*>(geo + kTcGeoRing);
  volatile int* abort = &bars->abort;

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  // CTAs run in blocks of 8 x 8 sub-tiles (128 x 128 voxels) for L2 reuse
  const int per_blk = 8 * 8;
  const int blk = blockIdx.x / per_blk, inblk = blockIdx.x % per_blk;
  const int blocks_x = (a.nsub_x + 7) / 8;
  const int sub_x = (blk % blocks_x) * 8 + (inblk % 8);
  const int sub_y = (blk / blocks_x) * 8 + (inblk / 8);
  const int z0 = blockIdx.y * N;
  const bool live_tile = sub_x < a.nsub_x && sub_y < a.nsub_y;
  const int gx = sub_x >> 1, gy = sub_y >> 1;
  const int ox = (sub_x & 1) * 16, oy = (sub_y & 1) * 16;
  // columns: [accumulator half 0][half 1], then in split mode [sum 0][sum 1]
  // (split mode: 128 voxel columns per half, lanes = slices; else N slice
  // columns per half, lanes = voxels)
  const int colsH = SWAP ? kTcM : N;  // accumulator columns per half
  const int ncols = (SPLIT ? 2 : 1) * kTcH * colsH;
  const uint32_t tmem_cols = ncols <= 32 ? 32 : (ncols <= 64 ? 64 : (ncols <= 128 ? 128 : (ncols <= 256 ? 256 : 512)));
  const int nstages = (a.ntheta + kTcS2 - 1) / kTcS2;

  if (tid == 0) {
    bars->abort = 0;
    for (int i = 0; i < NBB; ++i) {
      mbar_init(smem_u32(&bars->geo_full[i]), 1);
      mbar_init(smem_u32(&bars->full[i]), kTcBuilders + 1);
      mbar_init(smem_u32(&bars->empty[i]), 1);
    }
    mbar_init(smem_u32(&bars->done), 1);
    mbar_init(smem_u32(&bars->seg_done), 1);
    mbar_init(smem_u32(&bars->seg_free), kTcBuilders);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&bars->tmem)),
                 "r"(tmem_cols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem_d = bars->tmem;
  int mma_stages = 0;  // MMA thread: stages whose MMAs were issued

  if (live_tile) {
    if (warp == kTcBuilders) {
      // ---- producer.  Ring slot th % 64 of chunk c (angles 32c .. 32c+31)
      // is rewritten only after empty of stage 32c / S - NBB completed,
      // which is after the builders finished every stage of chunk c - 2.
      constexpr int kStagesPerChunk = 32 / kTcS2;
      int ib = 0;
      uint32_t ph = 0;  // phase of slot ib for this pass over the ring
      for (int s = 0; s < nstages; ++s) {
        if (s >= NBB && !wait_or_abort(smem_u32(&bars->empty[ib]), ph ^ 1u, abort, a.err)) break;
        if (s % kStagesPerChunk == 0) {
          const int th = s * kTcS2 + lane;
          if (th < a.ntheta) {
            const TileOrigin o = tile_origin(gx, gy, a.half_n, a.center, a.trig[th]);
            const float lo = o.f0 + fminf((float)ox * o.c, (float)(ox + 15) * o.c) +
                             fminf((float)oy * o.s, (float)(oy + 15) * o.s);
            const int jl = o.i0 + (int)floorf(lo) - 1;
            const int j0 = jl >= 0 ? (jl & ~7) : -((-jl + 7) & ~7);
            TcGeoP g;
            g.bj = ((o.i0 - j0) & 0xffff) | (j0 << 16);
            g.f0 = o.f0;
            g.c = o.c;
            g.s = o.s;
            geo[th % kTcGeoRing] = g;
          }
          __syncwarp();
        }
        const int nt = min(kTcS2, a.ntheta - s * kTcS2);
        if (lane == 0) {
          mbar_arrive(smem_u32(&bars->geo_full[ib]));
          const uint32_t fb = smem_u32(&bars->full[ib]);
          mbar_expect_tx(fb, (uint32_t)(nt * txB));
          for (int t = 0; t < nt; ++t) {
            const int th = s * kTcS2 + t;
            const int jb = geo[th % kTcGeoRing].bj >> 16;
            unsigned char* dst = Bbuf + (ib * kTcS2 + t) * angleB;
            const int cy = a.zfirst ? z0 : th, cz = a.zfirst ? th : z0;
            tma_load_3d(smem_u32(dst), &tmap, fb, jb, cy, cz);
            if (SPLIT) tma_load_3d(smem_u32(dst + bBytes), &tmap_lo, fb, jb, cy, cz);
          }
        }
        __syncwarp();
        if (++ib == NBB) {
          ib = 0;
          ph ^= 1u;
        }
      }
    } else if (warp == kTcBuilders + 1) {
      // ---- MMA issuer.  One thread issues every MMA, so its own instruction
      // count per MMA bounds the tensor pipe: the descriptors are built once
      // and advanced by adding byte offsets / 16 to their start-address
      // field, and consecutive MMAs alternate between the two accumulators so
      // that no MMA waits for the previous one's accumulation.
      if (lane == 0) {
        const uint64_t dA0 = sw64_desc(smem_u32(Abuf)), dB0 = sw64_desc(smem_u32(Bbuf));
        const uint32_t bStage = (uint32_t)(kTcS2 * angleB) >> 4, bAngle = (uint32_t)angleB >> 4;
        const uint32_t bPlane = (uint32_t)bBytes >> 4;
        int ia = 0, ib = 0;
        uint32_t ph = 0;
        for (int s = 0; s < nstages; ++s) {
          if (!wait_or_abort(smem_u32(&bars->full[ib]), ph, abort, a.err)) break;
          // split mode: a new segment overwrites the accumulators once the
          // builders have added the previous segment into the sums
          const bool seg0 = SPLIT ? (s % kTcSeg == 0) : (s == 0);
          if (SPLIT && s > 0 && seg0 &&
              !wait_or_abort(smem_u32(&bars->seg_free), (uint32_t)((s / kTcSeg - 1) & 1), abort, a.err))
            break;
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          const int nt = min(kTcS2, a.ntheta - s * kTcS2);
          const uint64_t dA = dA0 + (uint64_t)((uint32_t)(ia * kTcS2 * angleA) >> 4);
          const uint64_t dB = dB0 + (uint64_t)((uint32_t)ib * bStage);
#pragma unroll
          for (int t = 0; t < kTcS2; ++t) {
            if (t < nt) {
#pragma unroll
              for (int kk = 0; kk < 2; ++kk)
#pragma unroll
                for (int pr = 0; pr < (SPLIT ? 3 : 1); ++pr) {  // (W_hi,q_hi), (W_hi,q_lo), (W_lo,q_hi)
                  const uint64_t dq = dB + (uint32_t)(t * bAngle + (pr == 1 ? bPlane : 0u) + ((32 * kk) >> 4));
                  if (SWAP) {  // D[slice][voxel] = q (M = 128) x W^T (N = 256)
                    mma_f16(tmem_d, dq, dA + (uint32_t)((t * angleA + (pr == 2 ? kTcAngleA : 0) + 32 * kk) >> 4),
                            a.idesc, (seg0 && (t | kk | pr) == 0) ? 0u : 1u);
                  } else {  // D[voxel][slice] = W (M = 128 per half) x q^T (N slices)
#pragma unroll
                    for (int h = 0; h < kTcH; ++h)
                      mma_f16(tmem_d + (uint32_t)(h * N),
                              dA + (uint32_t)((t * angleA + (pr == 2 ? kTcAngleA : 0) + h * kTcHalfA + 32 * kk) >> 4),
                              dq, a.idesc, (seg0 && (t | kk | pr) == 0) ? 0u : 1u);
                  }
                }
            }
          }
          mma_commit(smem_u32(&bars->empty[ib]));
          if (SPLIT && (s + 1) % kTcSeg == 0 && s + 1 < nstages) mma_commit(smem_u32(&bars->seg_done));
          ++mma_stages;
          if (++ia == NA) ia = 0;
          if (++ib == NBB) {
            ib = 0;
            ph ^= 1u;
          }
        }
        // every issued MMA completes before `done` arrives
        mma_commit(smem_u32(&bars->done));
      }
      __syncwarp();
    } else {
      // ---- builders: one voxel row of A per thread; warps 4h .. 4h+3 build half h
      const int h = warp >> 2, m = tid & (kTcM - 1);
      const float fdx = (float)(ox + (m & 15)), fdy = (float)(oy + 8 * h + (m >> 4));
      const int swz = (m & 7) >> 1;
      int ia = 0, ib = 0, ie = NBB - NA;  // ie: ring slot of stage s - NA
      uint32_t ph = 0, phe = 1;           // phases of slots ib and ie
      for (int s = 0; s < nstages; ++s) {
        if (!wait_or_abort(smem_u32(&bars->geo_full[ib]), ph, abort, a.err)) break;
        if (s >= NA && !wait_or_abort(smem_u32(&bars->empty[ie]), phe, abort, a.err)) break;
        const int nt = min(kTcS2, a.ntheta - s * kTcS2);
        for (int t = 0; t < nt; ++t) {
          const TcGeoP g = geo[(s * kTcS2 + t) % kTcGeoRing];
          const float sr = rel_coord(g.f0, g.c, g.s, fdx, fdy);
          const float fl = floorf(sr);
          const float w = sr - fl;
          int idx = (int)fl + (int)(short)(g.bj & 0xffff);
          if (a.check && (idx < 0 || idx > kTcK - 2)) {
            atomicOr(a.err, kErrBpWindow);
            idx = 0;
          }
          unsigned char* row =
              Abuf + (ia * kTcS2 + t) * angleA + h * kTcHalfA + (m >> 3) * 512 + (m & 7) * kTcRowBytes;
          const int k1 = idx + 1;
          const int o0 = (((idx >> 3) ^ swz) << 4) + (idx & 7) * 2, o1 = (((k1 >> 3) ^ swz) << 4) + (k1 & 7) * 2;
#pragma unroll
          for (int c = 0; c < 4; ++c) *reinterpret_cast<uint4*>(row + ((c ^ swz) << 4)) = make_uint4(0, 0, 0, 0);
          if (SPLIT) {
            // FP16 hi/lo of both weights; the lo matrix sits one plane later
            const float u = 1.f - w;
            const __half uh = __float2half_rn(u), wh = __float2half_rn(w);
            const __half ul = __float2half_rn(u - __half2float(uh)), wl = __float2half_rn(w - __half2float(wh));
            unsigned char* lrow = row + kTcAngleA;
#pragma unroll
            for (int c = 0; c < 4; ++c) *reinterpret_cast<uint4*>(lrow + ((c ^ swz) << 4)) = make_uint4(0, 0, 0, 0);
            *reinterpret_cast<uint16_t*>(row + o0) = __half_as_ushort(uh);
            *reinterpret_cast<uint16_t*>(row + o1) = __half_as_ushort(wh);
            *reinterpret_cast<uint16_t*>(lrow + o0) = __half_as_ushort(ul);
            *reinterpret_cast<uint16_t*>(lrow + o1) = __half_as_ushort(wl);
          } else {
            *reinterpret_cast<uint16_t*>(row + o0) = weight_bits<TS>(1.f - w);
            *reinterpret_cast<uint16_t*>(row + o1) = weight_bits<TS>(w);
          }
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncwarp();
        if (lane == 0) mbar_arrive(smem_u32(&bars->full[ib]));
        if (SPLIT && s > 0 && s % kTcSeg == 0) {
          // segment k = s / kTcSeg - 1 is complete: sums (+)= accumulators,
          // round-to-nearest FP32 on the CUDA cores
          const int k = s / kTcSeg - 1;
          if (!wait_or_abort(smem_u32(&bars->seg_done), (uint32_t)(k & 1), abort, a.err)) break;
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          const uint32_t lanes = (uint32_t)((warp & 3) * 32) << 16;
          for (int c0 = 0; c0 < colsH; c0 += 16) {
            uint32_t acc[16], sum[16];
            tmem_ld16(tmem_d + lanes + (uint32_t)(h * colsH + c0), acc);
            if (k > 0) tmem_ld16(tmem_d + lanes + (uint32_t)(kTcH * colsH + h * colsH + c0), sum);
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
            for (int q = 0; q < 16; ++q)
              sum[q] = k > 0 ? __float_as_uint(__fadd_rn(__uint_as_float(sum[q]), __uint_as_float(acc[q]))) : acc[q];
            tmem_st16(tmem_d + lanes + (uint32_t)(kTcH * colsH + h * colsH + c0), sum);
          }
          asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
          asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
          __syncwarp();
          if (lane == 0) mbar_arrive(smem_u32(&bars->seg_free));
        }
        if (++ia == NA) ia = 0;
        if (++ib == NBB) {
          ib = 0;
          ph ^= 1u;
        }
        if (++ie == NBB) {
          ie = 0;
          phe ^= 1u;
        }
      }
    }
  }

  // ---- epilogue (builder warps): wait for the last MMAs, read D, store
  __syncthreads();
  if (live_tile && warp < kTcBuilders) {
    bool ok = !*abort && wait_or_abort(smem_u32(&bars->done), 0, abort, a.err);
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (ok && SWAP) {
      // TMEM lane = slice, column = voxel (half h: columns 128 h ..): warp w
      // reads slices 32 (w % 4) .. and the voxels of half w / 4, 16 columns
      // (one row of 16 voxels) at a time
      const int h = warp >> 2, zl = (warp & 3) * 32 + lane;
      const int z = z0 + zl;
      const bool zin = zl < N && z < a.nz;
      const bool add_sums = (nstages + kTcSeg - 1) / kTcSeg > 1;
      const int ix0 = gx * kTile + ox;
      for (int c0 = 0; c0 < kTcM; c0 += 16) {
        uint32_t r[16];
        const uint32_t taddr = tmem_d + ((uint32_t)((warp & 3) * 32) << 16) + (uint32_t)(h * kTcM + c0);
        tmem_ld16(taddr, r);
        if (add_sums) {
          uint32_t sm[16];
          tmem_ld16(taddr + (uint32_t)(kTcH * kTcM), sm);
          asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
          for (int q = 0; q < 16; ++q) r[q] = __float_as_uint(__fadd_rn(__uint_as_float(sm[q]), __uint_as_float(r[q])));
        }
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        const int iy = gy * kTile + oy + 8 * h + (c0 >> 4);
        if (zin && iy < a.n) {
          const int64_t off = (int64_t)z * a.v_z + (int64_t)iy * a.v_y + ix0;
          if (a.vdt == TCP_F32 && ix0 + 16 <= a.n && a.vec4) {
            float4* dst = reinterpret_cast<float4*>(reinterpret_cast<float*>(a.vol) + off);
#pragma unroll
            for (int q = 0; q < 4; ++q)
              dst[q] = make_float4(__uint_as_float(r[4 * q]) * a.scale, __uint_as_float(r[4 * q + 1]) * a.scale,
                                   __uint_as_float(r[4 * q + 2]) * a.scale, __uint_as_float(r[4 * q + 3]) * a.scale);
          } else {
#pragma unroll
            for (int q = 0; q < 16; ++q) {
              if (ix0 + q < a.n) {
                const float v = __uint_as_float(r[q]) * a.scale;
                if (a.vdt == TCP_F32) put<float>(a.vol, off + q, v);
                else if (a.vdt == TCP_F16) put<__half>(a.vol, off + q, v);
                else put<__nv_bfloat16>(a.vol, off + q, v);
              }
            }
          }
        }
      }
    } else if (ok) {
      // TMEM lane = voxel row of a half; warp w reads lanes 32 (w % 4) .. of half w / 4
      const int h = warp >> 2, m = tid & (kTcM - 1);
      const int ix = gx * kTile + ox + (m & 15), iy = gy * kTile + oy + 8 * h + (m >> 4);
      const bool inside = ix < a.n && iy < a.n;
      // split mode: segments 0 .. nseg-2 are in the sums, the last one in the accumulators
      const bool add_sums = SPLIT && (nstages + kTcSeg - 1) / kTcSeg > 1;
      for (int c0 = 0; c0 < N; c0 += 16) {
        uint32_t r[16];
        const uint32_t taddr = tmem_d + ((uint32_t)((warp & 3) * 32) << 16) + (uint32_t)(h * N + c0);
        tmem_ld16(taddr, r);
        if (add_sums) {
          uint32_t sm[16];
          tmem_ld16(taddr + (uint32_t)(kTcH * N), sm);
          asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
          for (int q = 0; q < 16; ++q) r[q] = __float_as_uint(__fadd_rn(__uint_as_float(sm[q]), __uint_as_float(r[q])));
        }
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        if (inside) {
#pragma unroll
          for (int q = 0; q < 16; ++q) {
            const int z = z0 + c0 + q;
            if (z < a.nz) {
              const int64_t off = (int64_t)z * a.v_z + (int64_t)iy * a.v_y + ix;
              const float v = __uint_as_float(r[q]) * a.scale;
              if (a.vdt == TCP_F32) put<float>(a.vol, off, v);
              else if (a.vdt == TCP_F16) put<__half>(a.vol, off, v);
              else put<__nv_bfloat16>(a.vol, off, v);
            }
          }
        }
      }
    }
  }
  // On an abort, MMAs already issued may still run: wait (bounded) for them
  // before the tensor memory is released.
  if (live_tile && warp == kTcBuilders + 1 && lane == 0 && *abort && mma_stages > 0) {
    const long long t0 = clock64();
    while (!mbar_try(smem_u32(&bars->done), 0) && clock64() - t0 < kTcBudget) {
    }
  }
  // Also on an abort, sinogram copies the producer issued may still be
  // landing in shared memory.  They complete only the stage barriers, which
  // also wait for builder arrivals that an abort cancels, so the producer
  // holds the block for a fixed interval (~50k cycles, far above a copy's
  // latency) before the shared memory is given up.
  if (live_tile && warp == kTcBuilders && lane == 0 && *abort) {
    const long long t0 = clock64();
    while (clock64() - t0 < 50000) {
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_d), "r"(tmem_cols) : "memory");
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static std::once_flag once;
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  std::call_once(once, [] {
    cudaDriverEntryPointQueryResult q;
    void* p = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  });
  return fn;
}

}  // namespace

size_t tc_smem_bytes(int N, int S, int parts, int na, int nbb) {
  return 1024 + (size_t)na * S * parts * kTcAngleA + (size_t)nbb * S * parts * N * kTcRowBytes +
         (size_t)kTcGeoRing * sizeof(TcGeoP) + sizeof(TcBars);
}

// Ring depths for N slices and S angles per stage: NA weight buffers, 4 in
// split mode (measured at 2048^2 x 256 slices x 2048 angles: 271, 258 and
// 231 ms for NA = 2, 3, 4; the builders then run further ahead of the MMAs
// and absorb the segment-sum pauses), else 3 (S = 1) or 2 (S = 2); then as
// many B buffers as fit in `limit` bytes (at most the geometry ring's bound).
void tc_rings(int N, int S, int parts, size_t limit, int* na, int* nbb) {
  *na = parts == 2 ? kTcMaxNA : ((S == 1) ? 3 : 2);
  const size_t fixed = tc_smem_bytes(N, S, parts, *na, 0);
  const size_t per = (size_t)S * parts * N * kTcRowBytes;
  const size_t avail = limit > fixed ? limit - fixed : 0;
  *nbb = (int)std::min<size_t>((size_t)tc_max_nbb(S), avail / per);
  if (*na > *nbb) *na = *nbb;  // the builders wait on the empty barrier of stage s - NA
}

int tc_slices(int64_t nz, bool split) {
  const int64_t r = ((nz + 15) / 16) * 16;
  return (int)std::min<int64_t>(split ? 128 : 256, std::max<int64_t>(16, r));
}

// Launch shape of one call: slices per block N, angles per stage S, blocks
// per SM and ring depths, and the dynamic shared memory per block.  Two
// blocks per SM (16-bit sinograms; split mode takes all 512 TMEM columns)
// where both blocks' accumulators (2N columns each, allocated in powers of
// two) fit in the SM's 512 TMEM columns and their rings (at least two B
// stages) in half the shared memory.  False if no ring of two B stages fits.
bool tc_shape(int64_t nz, bool split, int theta_stage, int blocks_per_sm, TcShape* sh) {
  sh->N = tc_slices(nz, split);
  sh->S = (split || theta_stage == 1) ? 1 : 2;  // split mode: one angle per stage (its A and B are twice as large)
  const int parts = split ? 2 : 1;
  const int rowsB = split ? kTcM : sh->N;  // sinogram rows per angle and plane in shared memory
  sh->blocks = 1;
  if (!split && blocks_per_sm > 1) {
    const int ncols = kTcH * sh->N;
    const int tcols = ncols <= 32 ? 32 : (ncols <= 64 ? 64 : (ncols <= 128 ? 128 : (ncols <= 256 ? 256 : 512)));
    sh->blocks = std::min(std::min(blocks_per_sm, kTcMaxBlocks), 512 / tcols);
    for (; sh->blocks > 1; --sh->blocks) {
      tc_rings(rowsB, sh->S, parts, kTcSmemPerSM / sh->blocks - 1024, &sh->na, &sh->nbb);
      if (sh->nbb >= 2) break;
    }
  }
  if (sh->blocks == 1) tc_rings(rowsB, sh->S, parts, kTcSmemLimit, &sh->na, &sh->nbb);
  sh->smem = tc_smem_bytes(rowsB, sh->S, parts, sh->na, sh->nbb);
  return sh->nbb >= 2;
}

bool tc_eligible(const View3& sino) {
  if (sino.dtype != TCP_F16 && sino.dtype != TCP_BF16 && sino.dtype != TCP_F16X2) return false;
  if ((uintptr_t)sino.p % 16 != 0) return false;
  if ((sino.s1 * 2) % 16 != 0 || (sino.s0 * 2) % 16 != 0) return false;
  if (sino.dtype == TCP_F16X2 && (sino.plane * 2) % 16 != 0) return false;
  if (sino.d1 < 1 || sino.d2 < 1 || sino.d0 < 1) return false;
  return encode_fn() != nullptr;
}

tcp_status launch_backproject_tc(const View3& sino, const TrigTable& trig, double center, const View3& vol,
                                 float scale, int theta_stage, int blocks_per_sm, cudaStream_t st) {
  if (!tc_eligible(sino)) return fail(TCP_ERR_UNSUPPORTED, "tensor-core backprojector: sinogram not eligible");
  const int nz = (int)sino.d0, nt = (int)sino.d1, nd = (int)sino.d2, n = (int)vol.d1;
  if (nz == 0 || n == 0) return TCP_OK;
  const bool split = sino.dtype == TCP_F16X2;
  TcShape sh;
  if (!tc_shape(nz, split, theta_stage, blocks_per_sm, &sh))
    return fail(TCP_ERR_UNSUPPORTED, "tensor-core backprojector: shared memory too small for its rings");
  const int N = sh.N, S = sh.S;
  CUtensorMap map, map_lo;
  // The map's outer dimensions follow the memory order: an angle-major chunk
  // ([angle][slice][sample], slice stride < angle stride) keeps the N rows of
  // one copy within one angle's contiguous block instead of N slice planes.
  const bool zfirst = sino.s0 < sino.s1;
  const cuuint64_t dims[3] = {(cuuint64_t)nd, (cuuint64_t)(zfirst ? nz : nt), (cuuint64_t)(zfirst ? nt : nz)};
  const cuuint64_t strides[2] = {(cuuint64_t)(zfirst ? sino.s0 : sino.s1) * 2, (cuuint64_t)(zfirst ? sino.s1 : sino.s0) * 2};
  const cuuint32_t box[3] = {(cuuint32_t)kTcK, zfirst ? (cuuint32_t)N : 1u, zfirst ? 1u : (cuuint32_t)N};
  const cuuint32_t estr[3] = {1, 1, 1};
  const CUtensorMapDataType tdt = sino.dtype == TCP_BF16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT16;
  for (int pl = 0; pl < (split ? 2 : 1); ++pl) {
    void* base = pl == 0 ? sino.p : (void*)((__half*)sino.p + sino.plane);
    const CUresult r = encode_fn()(pl == 0 ? &map : &map_lo, tdt, 3, base, dims, strides, box, estr,
                                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B,
                                   CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return fail(TCP_ERR_CUDA, "cuTensorMapEncodeTiled failed: " + std::to_string((int)r));
  }
  if (!split) map_lo = map;
  TcArgs a;
  a.nz = nz;
  a.ntheta = nt;
  a.ndet = nd;
  a.n = n;
  // 16 x 16 sub-tiles are taken inside whole 32 x 32 canonical tiles
  a.nsub_x = ((n + kTile - 1) / kTile) * 2;
  a.nsub_y = ((n + kTile - 1) / kTile) * 2;
  a.N = N;
  a.vol = vol.p;
  a.vdt = vol.dtype;
  a.v_z = vol.s0;
  a.v_y = vol.s1;
  a.trig = trig.dev;
  a.center = center;
  a.half_n = 0.5 * (double)n;
  a.scale = scale;
  a.zfirst = zfirst ? 1 : 0;
  a.vec4 = vol.dtype == TCP_F32 && (uintptr_t)vol.p % 16 == 0 && vol.s0 % 4 == 0 && vol.s1 % 4 == 0;
  // instruction descriptor: D FP32, A/B F16 or BF16, K-major, N >> 3, M >> 4
  const uint32_t fmt = sino.dtype == TCP_BF16 ? 1u : 0u;
  // split mode: M = 128 slices, N = 256 voxels (both halves); else M = 128
  // voxels of one half, N = the CTA's slices
  const uint32_t mmaN = split ? (uint32_t)(kTcH * kTcM) : (uint32_t)N;
  a.idesc = (1u << 4) | (fmt << 7) | (fmt << 10) | ((mmaN >> 3) << 17) | ((uint32_t)(kTcM >> 4) << 24);
  a.err = device_error_word();
  a.check = checked_mode() ? 1 : 0;
  a.na = sh.na;
  a.nbb = sh.nbb;
  const int blocks = sh.blocks;
  const size_t smem = sh.smem;
  void (*k)(const CUtensorMap, const CUtensorMap, TcArgs) =
      split ? k_backproject_tc<__half, 1, true>
      : sino.dtype == TCP_F16
          ? (S == 1 ? k_backproject_tc<__half, 1, false> : k_backproject_tc<__half, 2, false>)
          : (S == 1 ? k_backproject_tc<__nv_bfloat16, 1, false> : k_backproject_tc<__nv_bfloat16, 2, false>);
  TCP_CUDA_TRY(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  if (blocks > 1)
    TCP_CUDA_TRY(cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout,
                                      (int)cudaSharedmemCarveoutMaxShared));
  const int blocks_x = (a.nsub_x + 7) / 8, blocks_y = (a.nsub_y + 7) / 8;
  dim3 grid((unsigned)(blocks_x * blocks_y * 8 * 8), (unsigned)((nz + N - 1) / N));
  if (grid.y > 65535u) return fail(TCP_ERR_SHAPE, "backproject (tensor cores): too many slice blocks");
  k<<<grid, kTcThreads, smem, st>>>(map, map_lo, a);
  TCP_CUDA_TRY(cudaGetLastError());
  return TCP_OK;
}

}  // namespace tcp
