/*
 * tcp.h -- C ABI of the GB300 (sm_103a) chunked parallel-beam FBP library.
 *
 * The operations follow the problem statement of Nikitin, "TomocuPy: efficient
 * GPU-based tomographic reconstruction with asynchronous data processing"
 * (arXiv 2209.08450):
 *   Sec. 2.2  dark-flat field correction and negative logarithm (tcp_normalize),
 *             one-dimensional Shepp-Logan / Parzen filtering of each detector
 *             row in Fourier space with padding (tcp_filter), and backprojection
 *             by direct discretisation of the line integral with linear
 *             interpolation, the method called LineRec in Sec. 3
 *             (tcp_backproject);
 *   Sec. 2.3  asynchronous chunk processing with host-device copies overlapped
 *             with GPU computation (tcp_fbp);
 *   Sec. 2.1  16-bit storage with wider arithmetic where 16 bits would lose
 *             accuracy (every call accepts FP16/BF16 storage and accumulates in
 *             FP32).
 * tcp_project, the adjoint Radon projector, is not in the paper; it is the exact
 * transpose of tcp_backproject.
 *
 * Geometry (pixel units):
 *   projections  raw[theta][z][j]   uint16, projection-major as acquired
 *   sinograms    sino[z][theta][j]  detector pixel j has its centre at j
 *   volume       vol[z][iy][ix]     voxel centre (x, y) = (ix - n/2, iy - n/2)
 *   ray coordinate  s = x cos(theta) + y sin(theta) + center
 *   interpolation   q(s) = (1-w) q[floor(s)] + w q[floor(s)+1], w = s - floor(s),
 *                   q[j] = 0 outside [0, ndet)
 *
 * Conventions shared by every call:
 *   - Buffers are described by tcp_tensor: a pointer, a dtype, up to 4 dims and
 *     element strides.  The innermost stride (the detector or x axis) must be 1.
 *     The caller allocates and frees every input and output buffer; the library
 *     never frees caller memory.
 *   - Device-compute calls are asynchronous on the caller's CUDA stream `stream`
 *     (a cudaStream_t; NULL means the legacy default stream).  Arguments are
 *     checked on the host before anything is launched; a rejected call launches
 *     nothing and returns a non-zero tcp_status.  Errors of kernels already
 *     queued surface at a later call or through tcp_device_check.
 *   - The library never synchronises the device inside a compute call, except
 *     where a call says so (first use of an angle set or filter, see below).
 *   - Angle arrays `theta` are HOST pointers to FP64 radians.  The calls
 *     without a plan build, on first use of an angle set, its FP64 cos/sin
 *     table in device memory with a synchronous copy; later calls with the
 *     same contents reuse the cached table.  The same holds for filter
 *     responses (keyed by padded length, filter, weight and centre) and the
 *     FourierRec tables.  Each cache keeps at most 64 entries and frees the
 *     least recently used one beyond that (cudaFree, which waits for the
 *     device).  Make the first such call outside CUDA-graph capture, and do
 *     not let a captured graph outlive its tables.  Plans (tcp_plan_create)
 *     own their tables and workspace instead: calls that take a plan
 *     allocate nothing and never synchronise.
 *   - Scratch memory that a call without a plan needs is taken from the CUDA
 *     stream-ordered allocator on `stream` and released on it.
 *   - No call aborts or throws across the ABI; failures return a tcp_status and
 *     record a message retrievable with tcp_last_error (thread-local).
 */
#ifndef TCP_H_
#define TCP_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define TCP_VERSION 1

typedef enum {
  TCP_OK = 0,
  TCP_ERR_ARG = 1,          /* null pointer, unknown enum, non-finite scalar */
  TCP_ERR_SHAPE = 2,        /* inconsistent, empty-with-data or unsupported sizes */
  TCP_ERR_DTYPE = 3,        /* dtype not accepted by this argument */
  TCP_ERR_ALIGN = 4,        /* innermost stride not 1 or a required alignment */
  TCP_ERR_CUDA = 5,         /* a CUDA runtime call failed */
  TCP_ERR_OOM = 6,          /* device or host allocation failed */
  TCP_ERR_TIMEOUT = 7,      /* a bounded device-side wait gave up */
  TCP_ERR_DEVICE_CHECK = 8, /* a kernel recorded an index violation (checked mode) */
  TCP_ERR_UNSUPPORTED = 9,  /* valid request outside what this build implements */
  TCP_ERR_ALIAS = 10        /* input and output overlap where they must not */
} tcp_status;

/* TCP_F16X2: an FP32 value v kept as two FP16 planes, hi = fp16(v) and
 * lo = fp16(v - hi), so that |v - hi - lo| <= 2^-22 |v| while lo is a normal
 * FP16 number (|v| >= 2^-3; below that the error is at most 2^-25 absolute).
 * A tensor of this dtype is 4-d [2][nz][ntheta][ndet] FP16: plane 0 = hi,
 * plane 1 = lo, stride[0] = distance between the planes.  Only the fused
 * normalise + filter writes it and only the backprojector reads it; products
 * hi*hi + hi*lo + lo*hi of the split samples and split weights, accumulated in
 * FP32 on the tensor cores, reproduce the FP32 backprojection.  Scale the
 * values into [2^-3, 65504] with `weight` (the pipeline stores the ramp-
 * filtered -log times 2^10 and applies pi/N_theta/2^10 when writing voxels). */
typedef enum { TCP_U16 = 0, TCP_F16 = 1, TCP_BF16 = 2, TCP_F32 = 3, TCP_F16X2 = 4 } tcp_dtype;

/* Filters of Sec. 2.2 ("Shepp-Logan, Parzen or other").  Every ramp is the
 * band-limited Ram-Lak response on the padded period; SHEPP multiplies it by
 * sin(pi nu)/(pi nu), PARZEN by (1 - 2|nu|)^3, NONE applies no filter (only the
 * pi/N_theta weight and the centre shift). */
typedef enum {
  TCP_FILTER_SHEPP = 0,
  TCP_FILTER_PARZEN = 1,
  TCP_FILTER_RAMP = 2,
  TCP_FILTER_NONE = 3
} tcp_filter_kind;

/* Padding of each row before the filter FFT (Sec. 2.2 pads to FFT-friendly
 * sizes; Sec. 3 pads to suppress artefacts from objects wider than the field
 * of view).  The padded length is the next power of two >= 2*ndet; with the
 * TCP_PAD_SMOOTH flag set (e.g. TCP_PAD_EDGE | TCP_PAD_SMOOTH) it is the
 * smallest of that, the next 3 * 2^k >= 2*ndet (counted from 48 on) and the
 * next 5 * 2^k >= 2*ndet (from 80 on), e.g. 3072 instead of 4096 for
 * ndet = 1536 and 5120 instead of 8192 for 2560. */
typedef enum { TCP_PAD_EDGE = 0, TCP_PAD_ZERO = 1, TCP_PAD_SMOOTH = 2 } tcp_pad_mode;

/* Padded row length the filter uses for ndet detector pixels and this
 * padding mode (only the TCP_PAD_SMOOTH bit matters); -1 for ndet < 1. */
int64_t tcp_padded_length(int64_t ndet, int32_t pad_mode);

typedef struct {
  void* data;         /* device pointer unless the call says host */
  int32_t dtype;      /* tcp_dtype */
  int32_t ndim;       /* 1..4 */
  int64_t shape[4];   /* outermost first */
  int64_t stride[4];  /* in elements; stride[ndim-1] must be 1 */
} tcp_tensor;

/* ---------------------------------------------------------------- status -- */

const char* tcp_status_string(tcp_status s);
/* Message of the last failing call on this host thread ("" if none). */
const char* tcp_last_error(void);
int tcp_version(void);

/* Reads and clears the device error word that kernels set in checked mode
 * (and on bounded-wait timeouts).  Synchronises `stream`.  *word receives the
 * raw bits (0 = clean).  Returns TCP_ERR_DEVICE_CHECK if bits were set. */
tcp_status tcp_device_check(void* stream, uint32_t* word);

/* Turn per-access index checks on (1) or off (0) for later launches. */
tcp_status tcp_set_checked(int32_t on);

/* Free every cached angle table, filter response, FourierRec table
 * (twiddles, deconvolution factors, sorted angles, near-node weight tables)
 * and LpRec geometry; synchronises the device. */
tcp_status tcp_cache_clear(void);

/* ------------------------------------------------------------- normalise -- */

/* Mean over frames of uint16 frames[f][z][j] -> FP32 mean[z][j]
 * (Sec. 2.2 dark-flat field correction; the paper does not say how frames are
 * reduced, the arithmetic mean is used).  frames: U16, ndim 3.  mean: F32,
 * ndim 2, shape [nz][ndet].  nf >= 1. */
tcp_status tcp_frame_mean(const tcp_tensor* frames, tcp_tensor* mean, void* stream);

/* Dark/flat correction and negative logarithm (Sec. 2.2), computed in FP32:
 *   r = (raw - dark) / (flat - dark);  r <- 1e-6 if r is not finite or r <= 1e-6;
 *   sino[z][theta][j] = -ln(r).
 * raw:  U16 [ntheta][nz][ndet] (any outer strides; a z-chunk of a larger stack
 *       is a view with the full stack's strides).
 * dark, flat: F32 [nz][ndet] pre-averaged means, or U16 frames [nf][nz][ndet]
 *       (then averaged on the device in stream-ordered scratch).
 * sino: F32, F16 or BF16 [nz][ntheta][ndet]; must not overlap raw.
 * The transposition from projection-major to sinogram-major is part of the
 * call. */
tcp_status tcp_normalize(const tcp_tensor* raw, const tcp_tensor* dark, const tcp_tensor* flat,
                         tcp_tensor* sino, void* stream);

/* Allocation-free tcp_normalize for U16 dark/flat frames.  The paper has no
 * counterpart: it is for callers that may not allocate device memory once
 * they are running, such as an acquisition service that reserved all device
 * memory for its own pool at start-up, or a framework whose allocator owns
 * the device.  The frame means live in one fixed 8 MiB array inside the
 * library (held on every GPU that loads it until exit); nz * ndet may not
 * exceed 1,048,576 (else TCP_ERR_SHAPE).  No allocation of any kind is made.
 * All calls on a device share that array: calls that overlap on the GPU race,
 * so serialise them.  The first call on a device caches the array's device
 * address; make it before any stream capture.  raw: U16 [ntheta][nz][ndet];
 * dark, flat: U16 [nf][nz][ndet]; sino: F32/F16/BF16 [nz][ntheta][ndet].
 * Result equals tcp_normalize with the same frames. */
tcp_status tcp_normalize_noalloc(const tcp_tensor* raw, const tcp_tensor* dark, const tcp_tensor* flat,
                                 tcp_tensor* sino, void* stream);

/* ---------------------------------------------------------------- filter -- */

/* One-dimensional FBP filter of every detector row, in place (Sec. 2.2).
 * Per row: pad to npad = next power of two >= 2*ndet, or the smooth length
 * of tcp_pad_mode (L = (npad-ndet)/2 on the left, edge-replicated unless
 * TCP_PAD_ZERO), FFT, multiply bin k by
 *   H(k) * pi/ntheta * exp(2 pi i (k/npad) (center - ndet/2))
 * (Hermitian: the Nyquist bin takes the real part), inverse FFT, crop
 * [L, L+ndet).  The phase factor moves the rotation axis from `center` to
 * ndet/2, so the filtered stack is backprojected with center = ndet/2.
 * Passing center = ndet/2 applies no shift.  sino: F32/F16/BF16
 * [nz][ntheta][ndet] or [rows][ndet] (then ntheta = rows), FFT math in FP32
 * with FP64-derived twiddles and responses.  ndet <= 4096 (npad <= 8192). */
tcp_status tcp_filter(tcp_tensor* sino, int32_t filter, double center, void* stream);

/* tcp_filter with an explicit padding mode (TCP_PAD_EDGE or TCP_PAD_ZERO) and
 * an explicit angle count for the pi/ntheta weight (ntheta <= 0: take it from
 * the sinogram shape). */
tcp_status tcp_filter_ex(tcp_tensor* sino, int32_t filter, double center, int32_t pad_mode,
                         int64_t ntheta, void* stream);

/* Normalisation fused with the filter (Sec. 2.2 steps in order, one pass over
 * HBM): -ln((raw - dark)/(flat - dark)) is computed in FP32 straight into the
 * padded row in shared memory, filtered as tcp_filter_ex does, and the
 * filtered sinogram is stored once in its dtype.  16-bit outputs are rounded
 * after filtering only (rounding the unfiltered sinogram to BF16 loses
 * accuracy to the ramp's removal of its low-frequency content, Sec. 2.1).
 * raw: U16 [ntheta][nz][ndet]; dark, flat: F32 means [nz][ndet] or U16 frames
 * [nf][nz][ndet]; sino: F32/F16/BF16 [nz][ntheta][ndet] or F16X2
 * [2][nz][ntheta][ndet] (hi and lo FP16 planes of the FP32 result), must not
 * overlap raw.  ndet <= 4096. */
tcp_status tcp_normalize_filter(const tcp_tensor* raw, const tcp_tensor* dark, const tcp_tensor* flat,
                                tcp_tensor* sino, int32_t filter, double center, int32_t pad_mode,
                                void* stream);

/* tcp_normalize_filter with the response multiplied by `weight` instead of
 * pi/ntheta (weight <= 0: pi/ntheta).  A weight that is a power of two times
 * 1 (e.g. 1024 for FP16 storage) keeps small filtered values out of the FP16
 * subnormal range; apply pi/ntheta/weight afterwards with
 * tcp_backproject_ex (Sec. 2.1: reorder operations to stay in range).
 * |filtered -log| <= 6.9 for every filter, so weight <= 2^13 cannot overflow
 * FP16. */
tcp_status tcp_normalize_filter_ex(const tcp_tensor* raw, const tcp_tensor* dark, const tcp_tensor* flat,
                                   tcp_tensor* sino, int32_t filter, double center, int32_t pad_mode,
                                   double weight, void* stream);

/* ----------------------------------------------------------- backproject -- */

/* LineRec backprojection (Sec. 2.2, Sec. 3): for every voxel,
 *   vol[z][iy][ix] = sum over theta of q_{z,theta}(s(x, y, theta)),
 * linear interpolation, zero outside the detector.  The FBP weight pi/ntheta
 * belongs to tcp_filter, so this is the plain sum (the transpose of
 * tcp_project).  Output is overwritten, not accumulated.
 * sino:  F32/F16/BF16 [nz][ntheta][ndet], or F16X2 [2][nz][ntheta][ndet]
 *        (always on the tensor cores; planes, slices and rows must start on
 *        16-byte boundaries, else TCP_ERR_ALIGN); theta: HOST FP64 [ntheta];
 * vol:   F32/F16/BF16 [nz][n][n] (n is taken from vol), accumulation in FP32.
 * The ray coordinate is formed from an FP64 origin per 32x32 voxel tile and
 * FP32 in-tile offsets (|error| < 1e-5 px).
 * Layout: any element strides with the detector innermost.  The tensor-core
 * kernel copies one angle's window of all of a block's slices at a time, so a
 * sinogram stored angle-major (slice stride ndet, angle stride nz * ndet, the
 * layout of tcp_fbp's chunks) is read 1.4-2x faster at 2048^2 than a
 * slice-major one; the results are identical. */
tcp_status tcp_backproject(const tcp_tensor* sino, const double* theta, double center,
                           tcp_tensor* vol, void* stream);

/* tcp_backproject with every output voxel multiplied by `scale` (applied to
 * the FP32 accumulator before the store). */
tcp_status tcp_backproject_ex(const tcp_tensor* sino, const double* theta, double center,
                              tcp_tensor* vol, double scale, void* stream);

/* Adjoint Radon projector (not in the paper): the exact transpose of
 * tcp_backproject with the same interpolation weights,
 *   sino[z][theta][j] = sum over voxels of vol * (weight of j in q(s)).
 * vol: F32/F16/BF16 [nz][n][n]; theta: HOST FP64 [ntheta];
 * sino: F32/F16/BF16 [nz][ntheta][ndet] (ndet from sino), overwritten.
 * A gather per (theta, j): no atomics, deterministic. */
tcp_status tcp_project(const tcp_tensor* vol, const double* theta, double center,
                       tcp_tensor* sino, void* stream);

/* FourierRec backprojection (Sec. 1, Sec. 2.2, Sec. 3: the Fourier-slice
 * theorem with transforms on unequally spaced frequencies, exponential-type
 * interpolation in the frequency domain, oversampling by 2, controlled
 * accuracy).  Each filtered row q[j] (j < ndet), extended by zeros to the
 * period M = the next power of two >= 2 ndet, is replaced by its
 * trigonometric interpolant
 *   q~(s) = (1/M) sum_{k=-M/2..M/2} w_k Q[k] e^{2 pi i k s / M},
 *   Q[k] = sum_j q[j] e^{-2 pi i k j / M}, w_{+-M/2} = 1/2, else 1,
 * and, for every voxel,
 *   vol[z][iy][ix] = scale * sum over theta of q~_{z,theta}(s(x, y, theta))
 * with the ray coordinate of tcp_backproject.  The sum is evaluated on an
 * L x L Cartesian frequency grid (L = the next power of two >= 2n, at least
 * 16) with the
 * "exponential of semicircle" window of `width` grid points (2..16; 0 picks
 * 7 for an F32 volume, 5 for F16/BF16): relative error about 1e-6 at 7 and
 * tenfold smaller per extra point.  Two slices share one complex transform.
 * sino:  F32/F16/BF16 [nz][ntheta][ndet], ndet <= 8192, ntheta <= 2^24;
 * theta: HOST FP64 [ntheta]; vol: F32/F16/BF16 [nz][n][n], n even, n <= 8192,
 * overwritten.  Works in about 1.5 GiB of stream-ordered workspace
 * (cudaMallocAsync on `stream`).  Errors: TCP_ERR_SHAPE for odd n or sizes
 * over the limits, TCP_ERR_ARG for a width outside 2..16,
 * TCP_ERR_DTYPE for F16X2 or U16 sinograms.
 * The first call for a new size, width or angle set builds cached tables
 * (twiddles, deconvolution factors, sorted angles, and the sparse table of
 * window weights of the grid nodes within 128 points of the zero frequency:
 * about 0.2 GB at 2048^2 and 2048 angles, four geometries kept, least
 * recently used freed beyond that) with synchronous uploads, so that call
 * must not be inside CUDA graph capture. */
tcp_status tcp_fourierrec(const tcp_tensor* sino, const double* theta, double center,
                          tcp_tensor* vol, double scale, int32_t width, void* stream);

/* LpRec backprojection (Sec. 1, Sec. 3: the backprojection evaluated in
 * log-polar coordinates, where it is a convolution, with cubic B-splines, for
 * equally spaced angles).  Each filtered row is replaced by its interpolating
 * cubic B-spline q~ (zero samples outside the detector) and, per voxel,
 *   vol[z][iy][ix] = scale * sum over theta of q~_{z,theta}(s(x, y, theta))
 * with the ray coordinate of tcp_backproject, evaluated as: three spans of a
 * third of the angles each; per span the log-polar origin at 4 R outside the
 * object (R = n/sqrt(2) + 2) on the span's middle direction, G_theta(tau) =
 * q~_theta(center - a cos(theta - phi) + e^tau) sampled on a uniform
 * log-radius grid and turned into B-spline coefficients, the span's sum as a
 * convolution on the uniform (log-radius, angle) grid, its 2-D B-spline
 * coefficients, and the 4 x 4 cubic interpolation at every voxel.  Grid steps
 * are 1/oversampling pixel at the far radius (oversampling <= 0: 2; the error
 * to the direct cubic-spline sums falls with it, about 6e-3, 6e-4, 5e-5 at
 * 2, 4, 8 on white-noise rows).
 * theta: HOST FP64 [ntheta], ntheta >= 3, equally spaced (to 1e-9) over a
 * half turn [theta0, theta0 + pi), else TCP_ERR_ARG; sino: F32/F16/BF16
 * [nz][ntheta][ndet]; vol: F32/F16/BF16 [nz][n][n], overwritten.  Works in
 * stream-ordered workspace (about 0.9 GiB per slice of a pass at n = 2048,
 * oversampling 2, passes of at most 16 slices) and caches the slice-independent
 * geometry (8 sets, least recently used freed beyond that) built on first use
 * with synchronous uploads: make that call outside CUDA-graph capture. */
tcp_status tcp_lprec(const tcp_tensor* sino, const double* theta, double center, tcp_tensor* vol, double scale,
                     double oversampling, void* stream);

/* Backprojector launch configuration.  k_slices: slices per thread block
 * (1, 2, 4, 8 or 16); theta_stage: angles staged in shared memory per step
 * (8, 16 or 32); rows_per_thread: voxels per thread (2 or 4).
 * kernel: 0 = FP32 pipes (every dtype; rows_per_thread 16 on FP32 sinograms:
 * 4 x 4 voxel blocks reusing samples along the walk); 1 = tensor cores
 * (tcgen05.mma with TMEM accumulators, FP16/BF16 sinograms whose row and
 * slice strides are multiples of 8 elements; other inputs fall back to
 * kernel 0; theta_stage 1 or 2 sets the angles per pipeline stage, the other
 * fields are ignored); 2 = FP32 pipes for FP32 sinograms with slice pairs
 * (packed FP32x2 FMAs, one 8-byte shared load per slice pair and voxel after
 * the first of each column; k_slices even); 3 = kernel 1 with two thread
 * blocks per SM, its shared-memory rings sized for half the shared memory
 * (FP16/BF16 sinograms with at most 128 slices per block, where two blocks'
 * TMEM accumulators fit; otherwise exactly kernel 1).
 * The automatic choice is kernel 3 for 16-bit sinograms with at least 32
 * slices.  F16X2 sinograms always use the tensor cores. */
typedef struct {
  int32_t k_slices;
  int32_t theta_stage;
  int32_t rows_per_thread;
  int32_t kernel;
} tcp_bp_config;

/* Fix the backprojector configuration for later calls (NULL: automatic). */
tcp_status tcp_set_backproject_config(const tcp_bp_config* cfg);
/* Configuration the next call with this shape and dtype pair would use. */
tcp_status tcp_get_backproject_config(int64_t nz, int64_t ntheta, int64_t ndet, int64_t n,
                                      int32_t sino_dtype, int32_t vol_dtype, tcp_bp_config* cfg);

/* Launch shape of the tensor-core backprojector (kernels 1 and 3) for nz
 * slices of FP16, BF16 or F16X2 sinograms: host arithmetic only, no device
 * work.  theta_stage 1 or 2 (angles per pipeline stage; F16X2 always 1),
 * blocks_per_sm 1 or 2 (kernel 1 or 3).  Fills slices_per_block (the MMA's
 * slice dimension, a multiple of 16, at most 256, 128 for F16X2),
 * angles_per_stage, blocks_per_sm (2 only where two blocks' TMEM
 * accumulators, 2 x slices_per_block columns each, fit in 512 columns and
 * their rings in half the shared memory), weight_stages, sinogram_stages and
 * smem_bytes (dynamic shared memory per block).  TCP_ERR_ARG for a null
 * shape or nz < 1, TCP_ERR_DTYPE for other sinogram dtypes. */
typedef struct {
  int32_t slices_per_block;
  int32_t angles_per_stage;
  int32_t blocks_per_sm;
  int32_t weight_stages;
  int32_t sinogram_stages;
  int64_t smem_bytes;
} tcp_tc_shape;
tcp_status tcp_tc_launch_shape(int64_t nz, int32_t sino_dtype, int32_t theta_stage, int32_t blocks_per_sm,
                               tcp_tc_shape* shape);

/* ------------------------------------------------------------- pipeline -- */

typedef struct {
  int32_t chunk_nz;     /* slices per chunk (<= 0: 256 for 16-bit and F16X2 sinograms, 32 for FP32) */
  int32_t sino_dtype;   /* storage of the intermediate sinogram chunk: F32, F16, BF16 or F16X2;
                           any other value: F16X2 for an FP32 volume when ndet % 8 == 0 (else
                           F32), the volume's dtype for 16-bit volumes */
  int32_t filter;       /* tcp_filter_kind */
  int32_t pad_mode;     /* tcp_pad_mode */
  int32_t n_buffers;    /* device ring depth, 2 or 3 (default 2) */
  int32_t algorithm;    /* tcp_algorithm: backprojector (0 = LineRec) */
  int32_t width;        /* FourierRec window width (0: the tcp_fourierrec default); LpRec
                           oversampling, an integer 1..8 (0: 2) */
  int32_t reserved[1];
} tcp_fbp_opts;

/* Backprojector of tcp_fbp (Sec. 3 names all three): LineRec, the direct
 * linear-interpolation sum (tcp_backproject); FourierRec, the Fourier-slice
 * evaluation with band-limited interpolation (tcp_fourierrec; F32/F16/BF16
 * sinogram chunks, the default F32 for FP32 volumes; chunk_nz <= 0 gives 64;
 * n must be even); or LpRec, the log-polar evaluation with cubic B-splines
 * (tcp_lprec; F32/F16/BF16 chunks as FourierRec; chunk_nz <= 0 gives 16;
 * equally spaced angles over a half turn). */
typedef enum { TCP_ALG_LINEREC = 0, TCP_ALG_FOURIERREC = 1, TCP_ALG_LPREC = 2 } tcp_algorithm;

/* Chunked FBP (Sec. 2.3): for each chunk of chunk_nz slices, copy the raw
 * z-slab in, normalise, filter (axis moved to ndet/2) and backproject into
 * vol[z0:z1].  raw may be a HOST buffer (page-locked for overlap) or a device
 * buffer; vol likewise.  Host inputs are copied on an internal copy stream into
 * a ring of device buffers while the previous chunk computes on `stream`; host
 * outputs are copied back on a third stream.  dark/flat: U16 frames or F32
 * means, on the device or the host.  The intermediate sinogram holds the
 * ramp-filtered -log times 2^10 for FP16 and F16X2 storage (times 1 otherwise); the
 * pi/ntheta weight and the inverse storage scale are applied by the
 * backprojector, so small values never fall into the FP16 subnormal range.  Returns after queueing the work; the
 * result is complete when `stream` is.  Device buffers of the ring are taken
 * from the stream-ordered allocator. */
tcp_status tcp_fbp(const tcp_tensor* raw, const tcp_tensor* dark, const tcp_tensor* flat,
                   const double* theta, double center, tcp_tensor* vol, const tcp_fbp_opts* opts,
                   void* stream);

/* Multi-centre "try" reconstruction (Sec. 2.4, --reconstruction-type try):
 * slice `slice` of the projections reconstructed about each of `ncenters`
 * candidate rotation axes (Sec. 2.4: one image per centre, from which the
 * axis is picked before the full reconstruction).  Each candidate's shift is
 * applied in its own filter pass (the axis moves to ndet/2), and one
 * backprojection launch reconstructs the stack of candidates as if they were
 * slices.  raw: U16 [ntheta][nz][ndet], host or device; dark/flat as for
 * tcp_fbp; theta: HOST FP64 [ntheta]; centers: HOST FP64 [ncenters];
 * vol: DEVICE F32/F16/BF16 [ncenters][n][n], overwritten (FP32 volumes are
 * reconstructed from FP16 hi/lo pairs when ndet % 8 == 0, as tcp_fbp does).
 * slice outside [0, nz) or a non-finite centre: TCP_ERR_ARG. */
tcp_status tcp_try_centers(const tcp_tensor* raw, int64_t slice, const tcp_tensor* dark, const tcp_tensor* flat,
                           const double* theta, const double* centers, int64_t ncenters, tcp_tensor* vol,
                           int32_t filter, void* stream);

/* tcp_try_centers with the backprojector chosen: algorithm TCP_ALG_LINEREC
 * (as tcp_try_centers) or TCP_ALG_FOURIERREC (the candidate stack stored as
 * F32, or as the volume's 16-bit type, and backprojected by tcp_fourierrec
 * with window `width`, 0 for its default; n must be even). */
tcp_status tcp_try_centers_ex(const tcp_tensor* raw, int64_t slice, const tcp_tensor* dark, const tcp_tensor* flat,
                              const double* theta, const double* centers, int64_t ncenters, tcp_tensor* vol,
                              int32_t filter, int32_t algorithm, int32_t width, void* stream);

/* Time every instantiated backprojector configuration on these tensors (the
 * output is overwritten) and keep the fastest for later calls with the same
 * shapes and dtypes (an explicit tcp_set_backproject_config still wins).
 * Synchronises `stream`.  best / best_ms may be NULL. */
tcp_status tcp_autotune_backproject(const tcp_tensor* sino, const double* theta, double center,
                                    tcp_tensor* vol, void* stream, tcp_bp_config* best, float* best_ms);

/* -------------------------------------------------------------- batching -- */

/* A batch reconstructs many datasets of uneven width and angle count: per
 * dataset the fused normalise+filter kernel, then either ONE persistent
 * CUDA-core backprojection launch whose blocks pull (dataset, slice block,
 * 32x32 tile) work units from an atomic counter, longest angle count first,
 * or (tensor-core configurations, kernels 1 and 3) one tensor-core launch per
 * dataset.  Each dataset's chain (frame means, normalise+filter and, on the
 * tensor cores, its backprojection) runs on one of three side streams the
 * batch owns, forked from and joined back to the caller's stream by events,
 * so datasets overlap; results do not depend on the overlap.  No block waits
 * on another.  The run can be captured into a CUDA graph (the chains become
 * parallel branches; the counter is reset by a memset node) and replayed. */
typedef struct tcp_batch tcp_batch;

typedef struct {
  tcp_tensor raw;       /* U16 [ntheta][nz][ndet], device */
  tcp_tensor dark;      /* U16 frames [nf][nz][ndet] or F32 means [nz][ndet], device */
  tcp_tensor flat;      /* same forms as dark */
  tcp_tensor vol;       /* F32/F16/BF16 [nz][n][n], device; one dtype per batch */
  const double* theta;  /* host FP64 [ntheta]; read during tcp_batch_create only */
  double center;        /* rotation axis of this dataset */
  int32_t filter;       /* tcp_filter_kind */
  int32_t pad_mode;     /* tcp_pad_mode */
} tcp_batch_item;

typedef struct {
  int32_t sino_dtype;   /* storage of the filtered sinograms (F16 when opts is NULL) */
  int32_t autotune;     /* 1: time every backprojector configuration on this batch (CUDA-core
                           configurations in one persistent launch, and for 16-bit sinograms the
                           tensor-core kernel at one and two blocks per SM, one launch per
                           dataset) and keep the fastest;
                           0: the configuration fixed by tcp_set_backproject_config, if any, else
                           {8, 16, 4, 0} */
  int32_t reserved[2];
} tcp_batch_opts;

/* Validate the items, allocate the batch's device workspaces (one filtered
 * sinogram per dataset, FP32 means for frame inputs, the work list) with
 * cudaMalloc, build the angle and filter tables and, with autotune, run the
 * batch once per configuration on `stream` (synchronising it).  The tensors'
 * memory must stay valid while the batch is used.  *out is NULL on failure. */
tcp_status tcp_batch_create(const tcp_batch_item* items, int32_t n_items, const tcp_batch_opts* opts,
                            void* stream, tcp_batch** out);
/* Launch one run on `stream` (asynchronous). */
tcp_status tcp_batch_run(tcp_batch* b, void* stream);
/* Capture one run on `stream` (a non-default stream) into the batch's CUDA
 * graph and instantiate it; nothing executes during capture. */
tcp_status tcp_batch_capture(tcp_batch* b, void* stream);
/* Launch the captured graph on `stream`. */
tcp_status tcp_batch_replay(tcp_batch* b, void* stream);
/* Chosen configuration, autotune time of the winner (ms, 0 without autotune),
 * work units and persistent grid size.  Any output may be NULL. */
tcp_status tcp_batch_info(const tcp_batch* b, tcp_bp_config* cfg, float* tuned_ms, int64_t* work_units,
                          int32_t* grid_blocks);
/* Synchronise the device and free the batch (NULL is accepted). */
tcp_status tcp_batch_destroy(tcp_batch* b);

/* ----------------------------------------------------------------- plans -- */

/* A plan holds everything the reconstruction of one geometry needs besides
 * the caller's buffers, set up once (Sec. 2.2: the transforms and their
 * memory are prepared at start; Sec. 2.3: the chunks then run through fixed
 * device buffers): the FP64 angle table, the filter responses and FFT
 * twiddles, the FourierRec tables and workspace, the projector's tile-origin
 * table, the FP32 frame-mean buffers, the chunk sinogram buffer and, for
 * host input or output, the staging rings with their copy streams and events.
 *
 * tcp_plan_create allocates all of it with cudaMalloc on the current device,
 * uploads the tables and synchronises the device once.  The calls that take
 * a plan then allocate nothing, never synchronise, read no cached table and
 * only enqueue work on `stream` (and, for host buffers, on the plan's copy
 * streams, forked from and joined back to `stream` by events), so their
 * first use may be captured into a CUDA graph; host buffers must then be
 * page-locked.  A plan is used by one stream at a time: calls on different
 * streams that overlap race on its buffers.  tcp_plan_destroy synchronises
 * the device and frees everything (NULL is accepted). */
typedef struct tcp_plan tcp_plan;

#define TCP_IO_HOST_RAW 1 /* tcp_fbp_plan's raw may be host memory: allocate the upload ring */
#define TCP_IO_HOST_VOL 2 /* tcp_fbp_plan's vol may be host memory: allocate the download ring */

typedef struct {
  int64_t ntheta;       /* projection angles (>= 1) */
  int64_t nz;           /* slices: the most a tcp_fbp_plan call reconstructs */
  int64_t ndet;         /* detector pixels per row (<= 4096) */
  int64_t n;            /* volume side (<= 0: ndet) */
  double center;        /* rotation axis in detector pixels (filter phase of tcp_fbp_plan/tcp_filter_plan) */
  int32_t vol_dtype;    /* F32, F16 or BF16 */
  int32_t io;           /* TCP_IO_HOST_RAW | TCP_IO_HOST_VOL, 0 for device buffers only */
  int32_t host_frames;  /* U16 dark/flat frames that may come from host memory (0: device frames or means) */
  int32_t trace;        /* 1: time every chunk's upload, compute and download (tcp_plan_trace) */
  tcp_fbp_opts opts;    /* chunk, sinogram storage, filter, padding, ring depth, algorithm, width (as tcp_fbp) */
} tcp_plan_desc;

/* theta: HOST FP64 [ntheta], copied.  *out is NULL on failure.  Errors:
 * TCP_ERR_SHAPE/DTYPE/ARG for an invalid description, TCP_ERR_OOM when the
 * device memory does not fit. */
tcp_status tcp_plan_create(const tcp_plan_desc* desc, const double* theta, tcp_plan** out);
tcp_status tcp_plan_destroy(tcp_plan* plan);
/* Device bytes the plan holds, and the options it resolved (chunk depth,
 * sinogram storage, ring depth, FourierRec width).  Either output may be NULL. */
tcp_status tcp_plan_info(const tcp_plan* plan, int64_t* device_bytes, tcp_fbp_opts* resolved);

/* Per-chunk timeline of the last tcp_fbp_plan call of a plan created with
 * trace = 1 (Sec. 2.3: the asynchronous pipeline hides the copies of chunk
 * k+1 and k-1 behind the computation of chunk k).  Waits for that call to
 * finish.  ms receives up to `cap` rows of 6 values, in milliseconds from
 * the start of the call: upload start/end, compute start/end (normalise +
 * filter + backprojection), download start/end; -1 where a chunk had no such
 * copy.  *count = the number of chunks.  The events are CUDA events with
 * timing (resolution about 0.5 us); a traced call must not be captured. */
tcp_status tcp_plan_trace(const tcp_plan* plan, double* ms, int64_t cap, int64_t* count);

/* tcp_fbp through a plan: raw U16 [ntheta][nz][ndet] with nz <= the plan's,
 * vol [nz][n][n] of the plan's dtype; raw and vol on the device, or in host
 * memory where the plan's io flags allow it; dark/flat as for tcp_fbp (host
 * U16 frames at most host_frames of them).  Same result as tcp_fbp with the
 * plan's options. */
tcp_status tcp_fbp_plan(tcp_plan* plan, const tcp_tensor* raw, const tcp_tensor* dark, const tcp_tensor* flat,
                        tcp_tensor* vol, void* stream);
/* tcp_filter through a plan (the plan's filter, padding and centre, weight
 * pi/ntheta): sino F32/F16/BF16 [nz][ntheta][ndet] in place. */
tcp_status tcp_filter_plan(const tcp_plan* plan, tcp_tensor* sino, void* stream);
/* tcp_backproject_ex through a plan (its angle table): sino [nz][ntheta][ndet]
 * (or F16X2 pairs), vol [nz][n][n]. */
tcp_status tcp_backproject_plan(const tcp_plan* plan, const tcp_tensor* sino, double center, tcp_tensor* vol,
                                double scale, void* stream);
/* tcp_project through a plan (its angle table and tile-origin buffer): vol
 * [nz][n][n] of the plan's n, sino [nz][ntheta][ndet].  Calls that overlap on
 * the GPU share the origin buffer: serialise them. */
tcp_status tcp_project_plan(const tcp_plan* plan, const tcp_tensor* vol, double center, tcp_tensor* sino,
                            void* stream);

#ifdef __cplusplus
}
#endif

#endif /* TCP_H_ */
