/*
 * FP64 CPU oracle for chunked parallel-beam filtered backprojection.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow, obviously correct
 * definition that the CUDA path is checked against.  It shares no code, header,
 * table or constant with the CUDA library; only tests, the smoke check and the
 * benchmark's CPU-baseline leg may load it.  Nothing in the product path links
 * or calls it.
 *
 * Paper: Nikitin, "TomocuPy: efficient GPU-based tomographic reconstruction
 * with asynchronous data processing" (arXiv 2209.08450).
 *   - Sec. 2.2: dark-flat field correction, negative logarithm, 1-D filtering
 *     along detector rows, and backprojection by direct discretisation of the
 *     line integral with linear interpolation (the method called LineRec in
 *     Sec. 3).
 *   - The projector (adjoint) is not in the paper; it is the exact transpose of
 *     the backprojector defined here.
 *
 * Conventions (all in pixel units, FP64 throughout):
 *   raw[theta][z][j]  uint16, projection-major as acquired.
 *   sino[z][theta][j] detector pixel j has its centre at coordinate j.
 *   vol[z][iy][ix]    voxel centre (x, y) = (ix - n/2, iy - n/2).
 *   ray coordinate    s(x, y, theta) = x cos(theta) + y sin(theta) + center.
 *   interpolation     q(s) = (1 - w) q[floor(s)] + w q[floor(s) + 1],
 *                     w = s - floor(s), q[j] = 0 outside [0, ndet).
 *
 * Parallelism: an OpenMP loop over independent (slice, row) pairs; each output
 * is still the plain sum the definition states, in angle order.
 */
#include <math.h>
#include <stdint.h>
#include <string.h>

/* Arithmetic mean of a stack of frames[f][z][j] over f (Sec. 2.2 names the
 * dark-flat correction without its formula; the mean is the reading used). */
void or_frame_mean(const uint16_t* frames, int64_t nframes, int64_t nz, int64_t ndet,
                   double* mean) {
    for (int64_t z = 0; z < nz; ++z)
        for (int64_t j = 0; j < ndet; ++j) {
            double acc = 0.0;
            for (int64_t f = 0; f < nframes; ++f) acc += (double)frames[(f * nz + z) * ndet + j];
            mean[z * ndet + j] = acc / (double)nframes;
        }
}

/* Dark/flat correction and negative logarithm (Sec. 2.2):
 *   r = (raw - dark) / (flat - dark),  p = -ln(max(r, eps)),
 * with r replaced by eps when it is not a finite number greater than eps.
 * Output is transposed to the sinogram layout sino[z][theta][j]. */
void or_normalize(const uint16_t* raw, int64_t ntheta, int64_t nz, int64_t ndet,
                  const double* dark, const double* flat, double eps, double* sino) {
    for (int64_t t = 0; t < ntheta; ++t)
        for (int64_t z = 0; z < nz; ++z)
            for (int64_t j = 0; j < ndet; ++j) {
                double d = dark[z * ndet + j], f = flat[z * ndet + j];
                double r = ((double)raw[(t * nz + z) * ndet + j] - d) / (f - d);
                if (!(r > eps) || isinf(r)) r = eps;
                sino[(z * ntheta + t) * ndet + j] = -log(r);
            }
}

/* Linear interpolation of one detector row at ray coordinate s, zero outside
 * the detector (Sec. 2.2 / Sec. 3, LineRec). */
static double lerp_row(const double* q, int64_t ndet, double s) {
    double fl = floor(s);
    double w = s - fl;
    int64_t i = (int64_t)fl;
    double a = (i >= 0 && i < ndet) ? q[i] : 0.0;
    double b = (i + 1 >= 0 && i + 1 < ndet) ? q[i + 1] : 0.0;
    return (1.0 - w) * a + w * b;
}

/* Backprojection by direct discretisation of the line integral (Sec. 2.2,
 * LineRec): vol[z][iy][ix] = sum over theta of q_{z,theta}(s(x, y, theta)).
 * The FBP angular weight belongs to the filter, so this is the plain sum, the
 * exact transpose of or_project. */
void or_backproject(const double* sino, int64_t nz, int64_t ntheta, int64_t ndet,
                    const double* theta, double center, int64_t n, double* vol) {
    const double half = 0.5 * (double)n;
#pragma omp parallel for collapse(2) schedule(static)
    for (int64_t z = 0; z < nz; ++z)
        for (int64_t iy = 0; iy < n; ++iy) {
            double* row = vol + (z * n + iy) * n;
            for (int64_t ix = 0; ix < n; ++ix) row[ix] = 0.0;
            const double y = (double)iy - half;
            for (int64_t t = 0; t < ntheta; ++t) {
                const double c = cos(theta[t]), s = sin(theta[t]);
                const double* q = sino + (z * ntheta + t) * ndet;
                for (int64_t ix = 0; ix < n; ++ix) {
                    const double x = (double)ix - half;
                    row[ix] += lerp_row(q, ndet, x * c + y * s + center);
                }
            }
        }
}

/* The same sum evaluated at listed voxels of one slice: out[p] is the
 * backprojection at (ix[p], iy[p]).  Used to check sampled outputs of very
 * large volumes one voxel at a time. */
void or_backproject_points(const double* sino_slice, int64_t ntheta, int64_t ndet,
                           const double* theta, double center, int64_t n,
                           const int64_t* ix, const int64_t* iy, int64_t npts, double* out) {
    const double half = 0.5 * (double)n;
#pragma omp parallel for schedule(static)
    for (int64_t p = 0; p < npts; ++p) {
        const double x = (double)ix[p] - half, y = (double)iy[p] - half;
        double acc = 0.0;
        for (int64_t t = 0; t < ntheta; ++t)
            acc += lerp_row(sino_slice + t * ndet, ndet, x * cos(theta[t]) + y * sin(theta[t]) + center);
        out[p] = acc;
    }
}

/* Radon projector, the adjoint of or_backproject (not in the paper; it is the
 * transpose of the LineRec matrix):
 *   sino[z][theta][j] = sum over voxels of vol * max(0, 1 - |s - j|).
 * Written as the scatter of each voxel into its two neighbouring detector
 * pixels floor(s) and floor(s) + 1 with weights 1 - w and w, which are the
 * only j where the hat function is non-zero. */
void or_project(const double* vol, int64_t nz, int64_t n, const double* theta, int64_t ntheta,
                double center, int64_t ndet, double* sino) {
    const double half = 0.5 * (double)n;
#pragma omp parallel for collapse(2) schedule(static)
    for (int64_t z = 0; z < nz; ++z)
        for (int64_t t = 0; t < ntheta; ++t) {
            double* q = sino + (z * ntheta + t) * ndet;
            for (int64_t j = 0; j < ndet; ++j) q[j] = 0.0;
            const double c = cos(theta[t]), s = sin(theta[t]);
            for (int64_t iy = 0; iy < n; ++iy) {
                const double y = (double)iy - half;
                const double* row = vol + (z * n + iy) * n;
                for (int64_t ix = 0; ix < n; ++ix) {
                    const double sv = ((double)ix - half) * c + y * s + center;
                    const double fl = floor(sv);
                    const double w = sv - fl;
                    const int64_t i = (int64_t)fl;
                    if (i >= 0 && i < ndet) q[i] += (1.0 - w) * row[ix];
                    if (i + 1 >= 0 && i + 1 < ndet) q[i + 1] += w * row[ix];
                }
            }
        }
}
