// LpRec backprojection (Sec. 1 and Sec. 3 of the TomocuPy paper: the
// backprojection evaluated in log-polar coordinates, where it is a
// convolution, with cubic B-spline interpolation, for equally spaced angles).
//
// What it evaluates: every filtered row q[j] is replaced by its interpolating
// cubic B-spline q~ (zero samples outside the detector) and, per voxel,
//   vol = scale * sum_theta q~_theta(x cos(theta) + y sin(theta) + center).
// How (the paper names the method only; the steps below are this library's
// reading, the same as its FP64 reference):
//   the angles are split into three spans of a third each; for the span
//   centred on phi the log-polar origin is O = -a (cos phi, sin phi) with
//   a = 4 R (R covers the voxel grid), a voxel is O + e^rho (cos psi, sin psi),
//   and the span's sum is f(rho, psi) = sum_theta G_theta(rho + ln cos(psi -
//   theta)) with G_theta(tau) = q~_theta(sh_theta + e^tau),
//   sh_theta = center - a cos(theta - phi):
//   (1) G_theta on a uniform tau grid (step drho) and its B-spline
//       coefficients;
//   (2) f on the uniform (rho, psi) grid (steps drho, dpsi = dtheta / p):
//       for a fixed angle and grid column the shift ln cos(psi - theta) is the
//       same for every rho, so each column of f is a sum over angles of
//       4-tap filters of G's coefficient columns, whose base and weights depend
//       only on k - p u (a convolution in (rho, psi));
//   (3) the 2-D B-spline coefficients of f;
//   (4) f interpolated at every voxel (4 x 4 taps) and the three spans added.
// Grid steps are 1/os pixel at the far radius (os = oversampling, default 2).
//
// GB300 design.  Geometry that does not depend on the slice (the split
// positions of step 1, the per-(k - p u) bases and weights of step 2, the
// per-voxel log-polar coordinates of step 4) is computed once in FP64 and
// stored as an integer index plus an FP32 fraction, so every per-slice step
// runs in FP32.  Cubic B-spline prefilters (the inverse of the (1, 4, 1)/6
// filter) are applied as 49-tap symmetric FIR filters sqrt(3) z1^|m|,
// z1 = sqrt(3) - 2, |m| <= 24 (the omitted tail is below 3e-14 relative;
// every prefiltered signal carries 24 zero samples on each side, as the
// reference's finite system does).  Step (2), the dominant one, runs with one
// thread per (psi column, run of 32 rho rows): per angle it reads the
// (base, weights) pair of its column once and slides a 4-sample register
// window down G's coefficient column: 35 loads and 128 FMAs per angle.
#include <cmath>
#include <cstring>
#include <map>
#include <mutex>
#include <vector>

#include "tcp_internal.cuh"

namespace tcp {
namespace {

constexpr int kPad = 24;  // zero samples on each side of a prefiltered signal
constexpr int kFir = 24;  // prefilter half-length
constexpr int kRun = 32;  // rho rows per thread in step (2)

__constant__ float c_fir[kFir + 1];  // sqrt(3) z1^m, m = 0..24

// Cubic B-spline weights at offsets 0..3 from floor(t) - 1, u = frac(t).
__device__ __forceinline__ float4 bspline_w(float u) {
  const float v = 1.f - u, u2 = u * u, u3 = u2 * u;
  return make_float4(v * v * v * (1.f / 6.f), (3.f * u3 - 6.f * u2 + 4.f) * (1.f / 6.f),
                     (-3.f * u3 + 3.f * u2 + 3.f * u + 1.f) * (1.f / 6.f), u3 * (1.f / 6.f));
}

// Prefilter of a zero-extended signal held in shared memory s[0, len):
// c[k] = sum_{|m| <= 24} c_fir[|m|] s[k - m].
__device__ __forceinline__ float fir_at(const float* s, int len, int k) {
  float acc = c_fir[0] * s[k];
#pragma unroll
  for (int m = 1; m <= kFir; ++m) {
    const float a = (k - m >= 0) ? s[k - m] : 0.f;
    const float b = (k + m < len) ? s[k + m] : 0.f;
    acc = __fmaf_rn(c_fir[m], a + b, acc);
  }
  return acc;
}

// Row coefficients: C[z][t][k], k in [0, nd + 48), of q[z][t][0, nd) padded
// by 24 zeros each side.  One block per (t, z).
template <class TS>
__global__ void k_lp_rowcoef(const TS* q, int64_t q_z, int64_t q_t, int nd, float* C, int64_t c_z, int64_t c_t) {
  extern __shared__ float s[];
  const int t = blockIdx.x, z = blockIdx.y;
  const int len = nd + 2 * kPad;
  const TS* row = q + z * q_z + t * q_t;
  for (int k = threadIdx.x; k < len; k += blockDim.x) {
    const int j = k - kPad;
    s[k] = (j >= 0 && j < nd) ? Store<TS>::load(row + j) : 0.f;
  }
  __syncthreads();
  float* out = C + z * c_z + t * c_t;
  for (int k = threadIdx.x; k < len; k += blockDim.x) out[k] = fir_at(s, len, k);
}

struct LpSpanDev {
  int j0, nu, p, nrho, npsi, ntau;
  int L;     // ntau + 48: G coefficient length per (slice, angle)
  int nr;    // npsi + p (nu - 1): step-(2) table length
  int frow;  // npsi + 48: row length of the padded f grid
  int fcol;  // nrho + 48: rows of the padded f grid
  const int2* esplit;   // [ntau]: floor and FP32 fraction (bits) of e^{tau_l}
  const int2* shsplit;  // [nu]: floor and fraction of sh_u + 24
  const int* dbase;     // [nr]: floor(delta) - 1
  const float4* dw;     // [nr]: cubic weights at frac(delta)
};

// Step (1): G[z][u][k] = B-spline coefficients (along tau) of
// g[l] = q~_{j0+u}(sh_u + e^{tau_l}) for l < ntau, padded by 24 zeros.
// One block per (u, z); g lives in shared memory.
__global__ void k_lp_g(LpSpanDev sp, const float* C, int64_t c_z, int64_t c_t, int clen, float* G, int64_t g_z) {
  extern __shared__ float s[];
  const int u = blockIdx.x, z = blockIdx.y;
  const float* crow = C + z * c_z + (int64_t)(sp.j0 + u) * c_t;
  const int2 sh = sp.shsplit[u];
  const float fsh = __int_as_float(sh.y);
  for (int k = threadIdx.x; k < sp.L; k += blockDim.x) {
    const int l = k - kPad;
    float v = 0.f;
    if (l >= 0 && l < sp.ntau) {
      const int2 e = __ldg(sp.esplit + l);
      float fr = fsh + __int_as_float(e.y);
      int fl = sh.x + e.x;
      if (fr >= 1.f) {
        fr -= 1.f;
        fl += 1;
      }
      const int b = fl - 1;
      const float4 w = bspline_w(fr);
      const float c0 = (b >= 0 && b < clen) ? __ldg(crow + b) : 0.f;
      const float c1 = (b + 1 >= 0 && b + 1 < clen) ? __ldg(crow + b + 1) : 0.f;
      const float c2 = (b + 2 >= 0 && b + 2 < clen) ? __ldg(crow + b + 2) : 0.f;
      const float c3 = (b + 3 >= 0 && b + 3 < clen) ? __ldg(crow + b + 3) : 0.f;
      v = __fmaf_rn(w.w, c3, __fmaf_rn(w.z, c2, __fmaf_rn(w.y, c1, w.x * c0)));
    }
    s[k] = v;
  }
  __syncthreads();
  float* out = G + z * g_z + (int64_t)u * sp.L;
  for (int k = threadIdx.x; k < sp.L; k += blockDim.x) out[k] = fir_at(s, sp.L, k);
}

// Step (2): F[z][24 + i][24 + k] = sum_u sum_d w_d(r) G[z][u][i + base(r) + d],
// r = k - p u + p (nu - 1).  Thread: one column k, rows i0 .. i0 + 31.
__global__ void __launch_bounds__(256) k_lp_span(LpSpanDev sp, const float* G, int64_t g_z, float* F, int64_t f_z) {
  const int k = blockIdx.x * 32 + (threadIdx.x & 31);
  const int i0 = (blockIdx.y * 8 + (threadIdx.x >> 5)) * kRun;
  const int z = blockIdx.z;
  if (k >= sp.npsi || i0 >= sp.nrho) return;
  const float* Gz = G + z * g_z;
  float acc[kRun];
#pragma unroll
  for (int ii = 0; ii < kRun; ++ii) acc[ii] = 0.f;
  const int rofs = k + sp.p * (sp.nu - 1);
  for (int u = 0; u < sp.nu; ++u) {
    const int r = rofs - sp.p * u;
    const int base = __ldg(sp.dbase + r);
    const float4 w = __ldg(sp.dw + r);
    const float* g = Gz + (int64_t)u * sp.L;
    const int lo = i0 + base;
    if (lo >= 0 && lo + kRun + 3 <= sp.L) {
      float a0 = __ldg(g + lo), a1 = __ldg(g + lo + 1), a2 = __ldg(g + lo + 2);
#pragma unroll
      for (int ii = 0; ii < kRun; ++ii) {
        const float a3 = __ldg(g + lo + ii + 3);
        acc[ii] = __fmaf_rn(w.w, a3, __fmaf_rn(w.z, a2, __fmaf_rn(w.y, a1, __fmaf_rn(w.x, a0, acc[ii]))));
        a0 = a1;
        a1 = a2;
        a2 = a3;
      }
    } else {  // near the ends of G: zero outside [0, L)
#pragma unroll 4
      for (int ii = 0; ii < kRun; ++ii) {
        float v = 0.f;
        const float wd[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
        for (int d = 0; d < 4; ++d) {
          const int idx = lo + ii + d;
          if (idx >= 0 && idx < sp.L) v = __fmaf_rn(wd[d], __ldg(g + idx), v);
        }
        acc[ii] += v;
      }
    }
  }
  float* out = F + z * f_z + (int64_t)(kPad + i0) * sp.frow + kPad + k;
#pragma unroll
  for (int ii = 0; ii < kRun; ++ii)
    if (i0 + ii < sp.nrho) out[(int64_t)ii * sp.frow] = acc[ii];
}

// Zero the 24-wide borders of the padded f grid [fcol][frow] of each slice.
__global__ void k_lp_border(float* F, int64_t f_z, int nrho, int npsi, int frow, int fcol) {
  const int z = blockIdx.y;
  float* Fz = F + z * f_z;
  const int64_t total = (int64_t)fcol * frow;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int row = (int)(e / frow), col = (int)(e - (int64_t)row * frow);
    if (row < kPad || row >= kPad + nrho || col < kPad || col >= kPad + npsi) Fz[e] = 0.f;
  }
}

// Step (3a): prefilter along psi (rows): F2[z][row][:] = fir(F[z][row][:]).
__global__ void k_lp_fir_rows(const float* F, float* F2, int64_t f_z, int frow) {
  extern __shared__ float s[];
  const int row = blockIdx.x, z = blockIdx.y;
  const float* in = F + z * f_z + (int64_t)row * frow;
  for (int k = threadIdx.x; k < frow; k += blockDim.x) s[k] = in[k];
  __syncthreads();
  float* out = F2 + z * f_z + (int64_t)row * frow;
  for (int k = threadIdx.x; k < frow; k += blockDim.x) out[k] = fir_at(s, frow, k);
}

// Step (3b): prefilter along rho (columns), tiles of 32 columns x 128 rows.
constexpr int kColTile = 32, kRowTile = 128;
__global__ void __launch_bounds__(256) k_lp_fir_cols(const float* F2, float* F, int64_t f_z, int frow, int fcol) {
  __shared__ float s[kRowTile + 2 * kFir][kColTile + 1];
  const int c0 = blockIdx.x * kColTile, r0 = blockIdx.y * kRowTile, z = blockIdx.z;
  const float* in = F2 + z * f_z;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  for (int rr = ty; rr < kRowTile + 2 * kFir; rr += 8) {
    const int row = r0 - kFir + rr, col = c0 + tx;
    s[rr][tx] = (row >= 0 && row < fcol && col < frow) ? in[(int64_t)row * frow + col] : 0.f;
  }
  __syncthreads();
  float* out = F + z * f_z;
  for (int rr = ty; rr < kRowTile; rr += 8) {
    const int row = r0 + rr, col = c0 + tx;
    if (row >= fcol || col >= frow) continue;
    float acc = c_fir[0] * s[rr + kFir][tx];
#pragma unroll
    for (int m = 1; m <= kFir; ++m) acc = __fmaf_rn(c_fir[m], s[rr + kFir - m][tx] + s[rr + kFir + m][tx], acc);
    out[(int64_t)row * frow + col] = acc;
  }
}

// Step (4) geometry, FP64 once per call: per voxel and span the index and
// fraction of its log-polar coordinates (rho, psi) on the padded f grid.
struct LpVoxGeo {
  double ox, oy, phi, rho0, drho, psi0, dpsi;
};
struct LpVoxArgs {
  LpVoxGeo g[3];
  int n;
  int4* out;  // [3][n][n]: (floor(ti) - 1, frac bits, floor(tk) - 1, frac bits)
};
__global__ void k_lp_voxgeo(LpVoxArgs a) {
  const int64_t total = (int64_t)a.n * a.n;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int iy = (int)(e / a.n), ix = (int)(e - (int64_t)iy * a.n);
    const double X = (double)ix - 0.5 * a.n, Y = (double)iy - 0.5 * a.n;
#pragma unroll
    for (int m = 0; m < 3; ++m) {
      const LpVoxGeo& g = a.g[m];
      const double dx = X - g.ox, dy = Y - g.oy;
      const double vr = log(hypot(dx, dy));
      double vpsi = atan2(dy, dx) - g.phi;  // wrapped to (-pi, pi] about phi
      vpsi = atan2(sin(vpsi), cos(vpsi)) + g.phi;
      const double ti = (vr - g.rho0) / g.drho + kPad, tk = (vpsi - g.psi0) / g.dpsi + kPad;
      const double fi = floor(ti), fk = floor(tk);
      a.out[m * total + e] = make_int4((int)fi - 1, __float_as_int((float)(ti - fi)), (int)fk - 1,
                                       __float_as_int((float)(tk - fk)));
    }
  }
}

// Step (4): vol[z][iy][ix] = scale * sum over spans of the 4 x 4 B-spline sum
// of the span's coefficient grid at the voxel's log-polar coordinates.
template <class TV>
__global__ void k_lp_vox(const float* F0, const float* F1, const float* F2, int64_t f_z, int frow0, int fcol0,
                         int frow1, int fcol1, int frow2, int fcol2, const int4* geo, int n, TV* vol, int64_t v_z,
                         int64_t v_y, float scale) {
  const int64_t total = (int64_t)n * n;
  const int z = blockIdx.y;
  const float* Fs[3] = {F0 + z * f_z, F1 + z * f_z, F2 + z * f_z};
  const int rows[3] = {fcol0, fcol1, fcol2}, cols[3] = {frow0, frow1, frow2};
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    float acc = 0.f;
#pragma unroll
    for (int m = 0; m < 3; ++m) {
      const int4 t = __ldg(geo + m * total + e);
      const float4 wi = bspline_w(__int_as_float(t.y)), wk = bspline_w(__int_as_float(t.w));
      const float wiv[4] = {wi.x, wi.y, wi.z, wi.w}, wkv[4] = {wk.x, wk.y, wk.z, wk.w};
      const float* F = Fs[m];
#pragma unroll
      for (int a = 0; a < 4; ++a) {
        const int row = t.x + a;
        if (row < 0 || row >= rows[m]) continue;
        float racc = 0.f;
#pragma unroll
        for (int b = 0; b < 4; ++b) {
          const int col = t.z + b;
          if (col >= 0 && col < cols[m]) racc = __fmaf_rn(wkv[b], __ldg(F + (int64_t)row * cols[m] + col), racc);
        }
        acc = __fmaf_rn(wiv[a], racc, acc);
      }
    }
    const int iy = (int)(e / n), ix = (int)(e - (int64_t)iy * n);
    Store<TV>::put(vol + z * v_z + (int64_t)iy * v_y + ix, acc * scale);
  }
}

// ------------------------------------------------------------- host side --

int f2i_host(float f) {
  int i;
  std::memcpy(&i, &f, sizeof(i));
  return i;
}

// The prefilter taps, once per device (every device that loads the module
// holds its own copy of the constant).
tcp_status upload_fir() {
  int dev = 0;
  TCP_CUDA_TRY(cudaGetDevice(&dev));
  static std::mutex mu;
  static std::map<int, bool> done;
  std::lock_guard<std::mutex> lk(mu);
  if (!done[dev]) {
    const double z1 = std::sqrt(3.0) - 2.0;
    float h[kFir + 1];
    for (int m = 0; m <= kFir; ++m) h[m] = (float)(std::sqrt(3.0) * std::pow(z1, m));
    const cudaError_t e = cudaMemcpyToSymbol(c_fir, h, sizeof(h));
    if (e != cudaSuccess) return cuda_fail(e, "lprec: upload prefilter taps");
    done[dev] = true;
  }
  return TCP_OK;
}

}  // namespace

// Host geometry of the three spans (FP64), as in the library's reading above.
tcp_status lprec_geometry(const double* theta, int64_t nt, int64_t nd, int64_t n, double center, double os,
                          LpHostGeom* g) {
  if (nt < 3) return fail(TCP_ERR_SHAPE, "lprec: needs at least 3 angles");
  const double dth = theta[1] - theta[0];
  for (int64_t j = 1; j < nt; ++j)
    if (std::fabs((theta[j] - theta[j - 1]) - dth) > 1e-9)
      return fail(TCP_ERR_ARG, "lprec: angles must be equally spaced");
  if (std::fabs(dth * (double)nt - M_PI) > 1e-9)
    return fail(TCP_ERR_ARG, "lprec: angles must cover a half turn [theta0, theta0 + pi)");
  if (!(os >= 0.5 && os <= 16.0)) return fail(TCP_ERR_ARG, "lprec: oversampling must be in [0.5, 16]");
  const int margin = 12;
  const double R = (double)n / std::sqrt(2.0) + 2.0, a = 4.0 * R;
  const double drho = 1.0 / (os * (a + R));
  const int p = (int)std::ceil(os * (a + R) * dth);
  const double dpsi = dth / p;
  g->nt = nt;
  g->nd = nd;
  g->n = n;
  g->os = os;
  for (int m = 0; m < 3; ++m) {
    LpHostSpan& s = g->span[m];
    const int64_t b0 = std::llround((double)m * nt / 3.0), b1 = std::llround((double)(m + 1) * nt / 3.0);
    s.j0 = (int)b0;
    s.nu = (int)(b1 - b0);
    s.p = p;
    s.drho = drho;
    s.dpsi = dpsi;
    if (s.nu <= 0) return fail(TCP_ERR_SHAPE, "lprec: empty angle span");
    s.phi = 0.5 * (theta[b0] + theta[b1 - 1]);
    s.ox = -a * std::cos(s.phi);
    s.oy = -a * std::sin(s.phi);
    s.rho0 = std::log(a - R) - margin * drho;
    s.nrho = (int)std::ceil((std::log(a + R) - std::log(a - R)) / drho) + 2 * margin + 1;
    const double half = std::asin(R / a) + margin * dpsi;
    s.kpsi = (int)std::ceil(half / dpsi);
    s.npsi = 2 * s.kpsi + 1;
    s.psi0 = s.phi - s.kpsi * dpsi;
    double span = 0.0;
    for (int k = 0; k < s.npsi; k += std::max(1, s.npsi - 1))
      for (int64_t j = b0; j < b1; j += std::max<int64_t>(1, b1 - b0 - 1))
        span = std::max(span, std::fabs(s.psi0 + k * dpsi - theta[j]));
    s.ext = (int)std::ceil(-std::log(std::cos(span)) / drho) + margin;
    s.tau0 = s.rho0 - s.ext * drho;
    s.ntau = s.nrho + s.ext;
    // step (1): split e^{tau_l} and sh_u + 24
    s.esplit.resize((size_t)s.ntau);
    for (int l = 0; l < s.ntau; ++l) {
      const double e = std::exp(s.tau0 + drho * l);
      const double f = std::floor(e);
      s.esplit[(size_t)l] = make_int2((int)f, f2i_host((float)(e - f)));
    }
    s.shsplit.resize((size_t)s.nu);
    for (int u = 0; u < s.nu; ++u) {
      const double sh = center - a * std::cos(theta[b0 + u] - s.phi) + kPad;
      const double f = std::floor(sh);
      s.shsplit[(size_t)u] = make_int2((int)f, f2i_host((float)(sh - f)));
    }
    // step (2): per r = k - p u + p (nu - 1): delta = ext + 24 + ln cos(psi_k - theta_u) / drho
    const int nr = s.npsi + p * (s.nu - 1);
    s.dbase.resize((size_t)nr);
    s.dw.resize((size_t)nr);
    for (int r = 0; r < nr; ++r) {
      // psi_k - theta_u with k - p u = r - p (nu - 1): the angle of u = 0 and column r - p (nu - 1)
      const int kk = r - p * (s.nu - 1);
      const double ang = s.psi0 + kk * dpsi - theta[b0];
      const double delta = s.ext + kPad + std::log(std::cos(ang)) / drho;
      const double f = std::floor(delta);
      const double fr = delta - f;
      s.dbase[(size_t)r] = (int)f - 1;
      const double v = 1.0 - fr;
      s.dw[(size_t)r] = make_float4((float)(v * v * v / 6.0), (float)((3 * fr * fr * fr - 6 * fr * fr + 4) / 6.0),
                                    (float)((-3 * fr * fr * fr + 3 * fr * fr + 3 * fr + 1) / 6.0),
                                    (float)(fr * fr * fr / 6.0));
    }
  }
  return TCP_OK;
}

namespace {
int lp_L(const LpHostSpan& s) { return s.ntau + 2 * kPad; }
int lp_frow(const LpHostSpan& s) { return s.npsi + 2 * kPad; }
int lp_fcol(const LpHostSpan& s) { return s.nrho + 2 * kPad; }
size_t up256(size_t b) { return (b + 255) / 256 * 256; }
}  // namespace

int lprec_slices_per_pass(const LpHostGeom& g, int64_t nz) {
  // f grids of three spans (twice: coefficients and the row-filtered copy
  // share one), G coefficients of the largest span and the row coefficients,
  // about 6 GiB per pass at most
  size_t per = 0;
  for (int m = 0; m < 3; ++m) per += (size_t)lp_frow(g.span[m]) * lp_fcol(g.span[m]) * 4;
  size_t gmax = 0;
  for (int m = 0; m < 3; ++m) gmax = std::max(gmax, (size_t)g.span[m].nu * lp_L(g.span[m]) * 4);
  per += std::max<size_t>(gmax, (size_t)lp_frow(g.span[0]) * lp_fcol(g.span[0]) * 4);
  per += (size_t)g.nt * (g.nd + 2 * kPad) * 4;
  const int64_t zmax = std::max<int64_t>(1, (int64_t)((size_t(6) << 30) / std::max<size_t>(per, 1)));
  return (int)std::max<int64_t>(1, std::min<int64_t>(nz, std::min<int64_t>(zmax, 16)));
}

size_t lprec_workspace_bytes(const LpHostGeom& g, int zpass) {
  size_t b = up256((size_t)3 * g.n * g.n * sizeof(int4));
  for (int m = 0; m < 3; ++m) b += up256((size_t)zpass * lp_frow(g.span[m]) * lp_fcol(g.span[m]) * 4);
  size_t gmax = 0;
  for (int m = 0; m < 3; ++m) gmax = std::max(gmax, (size_t)g.span[m].nu * lp_L(g.span[m]) * 4);
  gmax = std::max<size_t>(gmax, (size_t)lp_frow(g.span[0]) * lp_fcol(g.span[0]) * 4);
  for (int m = 1; m < 3; ++m) gmax = std::max<size_t>(gmax, (size_t)lp_frow(g.span[m]) * lp_fcol(g.span[m]) * 4);
  b += up256((size_t)zpass * gmax);
  b += up256((size_t)zpass * g.nt * (g.nd + 2 * kPad) * 4);
  return b;
}

tcp_status lprec_upload(const LpHostGeom& g, std::vector<void*>* owned, LpDevGeom* d, cudaStream_t st,
                        bool async) {
  tcp_status s = upload_fir();
  if (s != TCP_OK) return s;
  auto up = [&](const void* h, size_t bytes, const void** out) -> tcp_status {
    void* p = nullptr;
    TCP_CUDA_TRY(cudaMalloc(&p, bytes ? bytes : 16));
    owned->push_back(p);
    if (bytes) {
      if (async) TCP_CUDA_TRY(cudaMemcpyAsync(p, h, bytes, cudaMemcpyHostToDevice, st));
      else TCP_CUDA_TRY(cudaMemcpy(p, h, bytes, cudaMemcpyHostToDevice));
    }
    *out = p;
    return TCP_OK;
  };
  for (int m = 0; m < 3; ++m) {
    const LpHostSpan& hs = g.span[m];
    if ((s = up(hs.esplit.data(), hs.esplit.size() * sizeof(int2), (const void**)&d->esplit[m])) != TCP_OK) return s;
    if ((s = up(hs.shsplit.data(), hs.shsplit.size() * sizeof(int2), (const void**)&d->shsplit[m])) != TCP_OK)
      return s;
    if ((s = up(hs.dbase.data(), hs.dbase.size() * sizeof(int), (const void**)&d->dbase[m])) != TCP_OK) return s;
    if ((s = up(hs.dw.data(), hs.dw.size() * sizeof(float4), (const void**)&d->dw[m])) != TCP_OK) return s;
  }
  return TCP_OK;
}

tcp_status launch_lprec_ws(const View3& sv, const LpHostGeom& g, const LpDevGeom& d, void* ws, int zpass,
                           const View3& vv, float scale, cudaStream_t st) {
  const int64_t nz = sv.d0, nt = sv.d1, nd = sv.d2, n = vv.d1;
  if (nt != g.nt || nd != g.nd || n != g.n) return fail(TCP_ERR_SHAPE, "lprec: geometry differs from the call");
  if (nz == 0 || n == 0) return TCP_OK;
  tcp_status s = upload_fir();
  if (s != TCP_OK) return s;
  // workspace layout
  char* p = (char*)ws;
  int4* geo = (int4*)p;
  p += up256((size_t)3 * n * n * sizeof(int4));
  float* Fm[3];
  int64_t fz[3];
  for (int m = 0; m < 3; ++m) {
    fz[m] = (int64_t)lp_frow(g.span[m]) * lp_fcol(g.span[m]);
    Fm[m] = (float*)p;
    p += up256((size_t)zpass * fz[m] * 4);
  }
  size_t gmax = 0;
  for (int m = 0; m < 3; ++m) {
    gmax = std::max(gmax, (size_t)g.span[m].nu * lp_L(g.span[m]) * 4);
    gmax = std::max<size_t>(gmax, (size_t)fz[m] * 4);
  }
  float* Gbuf = (float*)p;  // G coefficients, then the row-filtered f of one span
  p += up256((size_t)zpass * gmax);
  const int clen = (int)nd + 2 * kPad;
  float* C = (float*)p;
  // step (4) geometry (FP64, once per call)
  {
    LpVoxArgs a;
    for (int m = 0; m < 3; ++m) {
      const LpHostSpan& hs = g.span[m];
      a.g[m] = LpVoxGeo{hs.ox, hs.oy, hs.phi, hs.rho0, hs.drho, hs.psi0, hs.dpsi};
    }
    a.n = (int)n;
    a.out = geo;
    const int64_t total = n * n;
    k_lp_voxgeo<<<(unsigned)std::min<int64_t>((total + 255) / 256, 8192), 256, 0, st>>>(a);
    TCP_CUDA_TRY(cudaGetLastError());
  }
  for (int64_t z0 = 0; z0 < nz; z0 += zpass) {
    const int zc = (int)std::min<int64_t>(zpass, nz - z0);
    // row coefficients
    {
      const size_t sm = sizeof(float) * clen;
      const char* base = (const char*)sv.p + z0 * sv.s0 * (sv.dtype == TCP_F32 ? 4 : 2);
      dim3 grid((unsigned)nt, (unsigned)zc);
      switch (sv.dtype) {
        case TCP_F32:
          cudaFuncSetAttribute(k_lp_rowcoef<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
          k_lp_rowcoef<float><<<grid, 256, sm, st>>>((const float*)base, sv.s0, sv.s1, (int)nd, C,
                                                     (int64_t)nt * clen, clen);
          break;
        case TCP_F16:
          cudaFuncSetAttribute(k_lp_rowcoef<__half>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
          k_lp_rowcoef<__half><<<grid, 256, sm, st>>>((const __half*)base, sv.s0, sv.s1, (int)nd, C,
                                                      (int64_t)nt * clen, clen);
          break;
        case TCP_BF16:
          cudaFuncSetAttribute(k_lp_rowcoef<__nv_bfloat16>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
          k_lp_rowcoef<__nv_bfloat16><<<grid, 256, sm, st>>>((const __nv_bfloat16*)base, sv.s0, sv.s1, (int)nd, C,
                                                             (int64_t)nt * clen, clen);
          break;
        default: return fail(TCP_ERR_DTYPE, "lprec: sino must be F32, F16 or BF16");
      }
      TCP_CUDA_TRY(cudaGetLastError());
    }
    for (int m = 0; m < 3; ++m) {
      const LpHostSpan& hs = g.span[m];
      LpSpanDev sp;
      sp.j0 = hs.j0; sp.nu = hs.nu; sp.p = hs.p; sp.nrho = hs.nrho; sp.npsi = hs.npsi; sp.ntau = hs.ntau;
      sp.L = lp_L(hs); sp.nr = hs.npsi + hs.p * (hs.nu - 1); sp.frow = lp_frow(hs); sp.fcol = lp_fcol(hs);
      sp.esplit = d.esplit[m]; sp.shsplit = d.shsplit[m]; sp.dbase = d.dbase[m]; sp.dw = d.dw[m];
      // (1)
      const size_t smg = sizeof(float) * sp.L;
      cudaFuncSetAttribute(k_lp_g, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smg);
      const int64_t g_z = (int64_t)sp.nu * sp.L;
      k_lp_g<<<dim3((unsigned)sp.nu, (unsigned)zc), 256, smg, st>>>(sp, C, (int64_t)nt * clen, clen, clen, Gbuf,
                                                                     g_z);
      TCP_CUDA_TRY(cudaGetLastError());
      // (2)
      k_lp_border<<<dim3(256, (unsigned)zc), 256, 0, st>>>(Fm[m], fz[m], sp.nrho, sp.npsi, sp.frow, sp.fcol);
      dim3 gs((unsigned)((sp.npsi + 31) / 32), (unsigned)((sp.nrho + 8 * kRun - 1) / (8 * kRun)), (unsigned)zc);
      k_lp_span<<<gs, 256, 0, st>>>(sp, Gbuf, g_z, Fm[m], fz[m]);
      TCP_CUDA_TRY(cudaGetLastError());
      // (3): rows into the scratch buffer, columns back into Fm
      const size_t smr = sizeof(float) * sp.frow;
      cudaFuncSetAttribute(k_lp_fir_rows, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smr);
      k_lp_fir_rows<<<dim3((unsigned)sp.fcol, (unsigned)zc), 256, smr, st>>>(Fm[m], Gbuf, fz[m], sp.frow);
      TCP_CUDA_TRY(cudaGetLastError());
      k_lp_fir_cols<<<dim3((unsigned)((sp.frow + kColTile - 1) / kColTile),
                           (unsigned)((sp.fcol + kRowTile - 1) / kRowTile), (unsigned)zc),
                      256, 0, st>>>(Gbuf, Fm[m], fz[m], sp.frow, sp.fcol);
      TCP_CUDA_TRY(cudaGetLastError());
    }
    // (4)
    const int64_t total = n * n;
    dim3 gv((unsigned)std::min<int64_t>((total + 255) / 256, 4096), (unsigned)zc);
    const int fr0 = lp_frow(g.span[0]), fc0 = lp_fcol(g.span[0]), fr1 = lp_frow(g.span[1]), fc1 = lp_fcol(g.span[1]),
              fr2 = lp_frow(g.span[2]), fc2 = lp_fcol(g.span[2]);
    const int64_t fzc = std::max(fz[0], std::max(fz[1], fz[2]));
    (void)fzc;
    // each span's grid has its own slice stride
    auto launch_vox = [&](auto* tv) -> tcp_status {
      using TV = std::remove_pointer_t<decltype(tv)>;
      TV* vol = (TV*)vv.p + z0 * vv.s0;
      if (fz[0] == fz[1] && fz[1] == fz[2]) {
        k_lp_vox<TV><<<gv, 256, 0, st>>>(Fm[0], Fm[1], Fm[2], fz[0], fr0, fc0, fr1, fc1, fr2, fc2, geo, (int)n, vol,
                                         vv.s0, vv.s1, scale);
      } else {
        for (int zz = 0; zz < zc; ++zz)  // spans of unequal size: one slice per launch
          k_lp_vox<TV><<<dim3(gv.x, 1), 256, 0, st>>>(Fm[0] + zz * fz[0], Fm[1] + zz * fz[1], Fm[2] + zz * fz[2], 0,
                                                      fr0, fc0, fr1, fc1, fr2, fc2, geo, (int)n, vol + zz * vv.s0,
                                                      vv.s0, vv.s1, scale);
      }
      TCP_CUDA_TRY(cudaGetLastError());
      return TCP_OK;
    };
    switch (vv.dtype) {
      case TCP_F32: s = launch_vox((float*)nullptr); break;
      case TCP_F16: s = launch_vox((__half*)nullptr); break;
      case TCP_BF16: s = launch_vox((__nv_bfloat16*)nullptr); break;
      default: return fail(TCP_ERR_DTYPE, "lprec: vol must be F32, F16 or BF16");
    }
    if (s != TCP_OK) return s;
  }
  return TCP_OK;
}

// Geometry of one (angle set, detector, grid, centre, oversampling), cached
// for the calls without a plan (at most 8 sets; the least recently used one
// is freed beyond that, cudaFree waiting for the device).
struct LpCacheEntry {
  std::vector<double> theta;
  int64_t nd, n;
  double center, os;
  int dev;
  uint64_t used;
  LpHostGeom* g;
  LpDevGeom d;
  std::vector<void*> owned;
};
namespace {
std::mutex g_lp_mu;
std::vector<LpCacheEntry> g_lp;
uint64_t g_lp_stamp = 0;
}  // namespace

tcp_status lprec_cached(const double* theta, int64_t nt, int64_t nd, int64_t n, double center, double os,
                        const LpHostGeom** g, const LpDevGeom** d) {
  int dev = 0;
  TCP_CUDA_TRY(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lk(g_lp_mu);
  for (auto& e : g_lp)
    if (e.dev == dev && e.nd == nd && e.n == n && e.center == center && e.os == os && (int64_t)e.theta.size() == nt &&
        std::equal(e.theta.begin(), e.theta.end(), theta)) {
      e.used = ++g_lp_stamp;
      *g = e.g;
      *d = &e.d;
      return TCP_OK;
    }
  if (g_lp.size() >= 8) {
    auto lru = std::min_element(g_lp.begin(), g_lp.end(),
                                [](const LpCacheEntry& a, const LpCacheEntry& b) { return a.used < b.used; });
    for (void* q : lru->owned) cudaFree(q);
    delete lru->g;
    g_lp.erase(lru);
  }
  LpCacheEntry e;
  e.theta.assign(theta, theta + nt);
  e.nd = nd;
  e.n = n;
  e.center = center;
  e.os = os;
  e.dev = dev;
  e.used = ++g_lp_stamp;
  e.g = new LpHostGeom();
  tcp_status s = lprec_geometry(theta, nt, nd, n, center, os, e.g);
  if (s == TCP_OK) s = lprec_upload(*e.g, &e.owned, &e.d, nullptr, false);
  if (s != TCP_OK) {
    for (void* q : e.owned) cudaFree(q);
    delete e.g;
    return s;
  }
  g_lp.push_back(std::move(e));
  *g = g_lp.back().g;
  *d = &g_lp.back().d;
  return TCP_OK;
}

void lprec_cache_clear() {
  std::lock_guard<std::mutex> lk(g_lp_mu);
  for (auto& e : g_lp) {
    for (void* q : e.owned) cudaFree(q);
    delete e.g;
  }
  g_lp.clear();
}

// Shared-memory limits of the kernels for this geometry.
tcp_status lprec_check(const LpHostGeom& g) {
  const size_t lim = 227 * 1024;
  for (int m = 0; m < 3; ++m) {
    if ((size_t)lp_L(g.span[m]) * 4 > lim || (size_t)lp_frow(g.span[m]) * 4 > lim)
      return fail(TCP_ERR_UNSUPPORTED, "lprec: log-polar grid too large for shared memory (lower the oversampling)");
  }
  if ((size_t)(g.nd + 2 * kPad) * 4 > lim) return fail(TCP_ERR_UNSUPPORTED, "lprec: ndet too large");
  return TCP_OK;
}

}  // namespace tcp
