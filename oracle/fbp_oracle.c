/*
 * FP64 CPU oracle for parallel-beam filtered backprojection (FBP).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU
 * baseline leg of the benchmark may load this library.  The GPU library
 * shares no code, header, table or constant with it.
 *
 * It is plain and slow on purpose: every function is the definition it cites,
 * written out with explicit loops in double precision, no blocking and no
 * reordering.  Paper: "Performance evaluation in the reconstruction of 2D
 * images of computed tomography using massively parallel programming CUDA"
 * (arXiv 2109.02174).
 *
 * Conventions (the paper fixes none of them; these are the readings used by
 * the whole project):
 *   - pixel (row r, column c) of an n x n image has centre
 *       x = c - (n-1)/2,  y = r - (n-1)/2            (pixel size 1)
 *   - detector bin k of n_det bins has centre t_k = (k - (n_det-1)/2) * tau
 *   - a ray at angle theta is the line x cos(theta) + y sin(theta) = t
 *     (section "Computed tomography", the line equation before Eq. 2)
 *   - the filtered projection is read between bins by linear interpolation
 *     with zero outside [0, n_det)
 *   - Eq. 2 sums over the angles; the angular step pi/n_angles is applied so
 *     that the result approximates the attenuation density.
 */
#include <math.h>
#include <pthread.h>
#include <stdlib.h>
#include <string.h>

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

enum { ORACLE_RAM_LAK = 0, ORACLE_SHEPP_LOGAN = 1, ORACLE_NONE = 2 };

/*
 * Lambert-Beer (Eq. 1): a ray of incident intensity i0 leaves the object with
 * I = i0 exp(-integral of mu), so the line integral the filter takes is
 * p = -ln(I / i0).  A measured count of zero has no logarithm; one count is
 * the floor (p = -ln(max(I, 1) / i0)).  n values, in order.
 */
void oracle_lambert_beer(const double *I, long n, double i0, double *p)
{
    for (long k = 0; k < n; ++k) {
        const double v = I[k] > 1.0 ? I[k] : 1.0;
        p[k] = -log(v / i0);
    }
}

/*
 * Spatial filter taps H (the convolution kernel of Q = P * H, text after
 * Eq. 2).  The paper does not name H; the band-limited ramp kernels of
 * Kak & Slaney ("Principles of Computerized Tomographic Imaging", ch. 3) are
 * used:
 *   Ram-Lak:     h(0) = 1/(4 tau^2), h(m) = 0 for even m != 0,
 *                h(m) = -1/(pi^2 m^2 tau^2) for odd m
 *   Shepp-Logan: h(m) = 2 / (pi^2 tau^2 (1 - 4 m^2))
 *   none:        h(0) = 1/tau, else 0   (so that Q = P)
 * Output: h[m + n_det - 1] = h(m) for m = -(n_det-1) .. n_det-1
 * (2*n_det - 1 values).  Returns 0, or -1 on a bad argument.
 */
int oracle_taps(int kind, int n_det, double tau, double *h)
{
    if (n_det < 1 || !(tau > 0.0) || h == NULL) return -1;
    for (int m = -(n_det - 1); m <= n_det - 1; ++m) {
        double v;
        if (kind == ORACLE_RAM_LAK) {
            if (m == 0)
                v = 1.0 / (4.0 * tau * tau);
            else if (m % 2 == 0)
                v = 0.0;
            else
                v = -1.0 / (M_PI * M_PI * (double)m * (double)m * tau * tau);
        } else if (kind == ORACLE_SHEPP_LOGAN) {
            v = 2.0 / (M_PI * M_PI * tau * tau * (1.0 - 4.0 * (double)m * (double)m));
        } else if (kind == ORACLE_NONE) {
            v = (m == 0) ? 1.0 / tau : 0.0;
        } else {
            return -1;
        }
        h[m + n_det - 1] = v;
    }
    return 0;
}

/*
 * Filtered projections Q_theta = P_theta * H (text after Eq. 2), as the
 * discrete linear convolution of each sinogram row with the taps, the row
 * being zero outside the detector:
 *   Q[i][k] = tau * sum_{j=0}^{n_det-1} h(k - j) * P[i][j],   k in [0, n_det)
 * P has row stride ld (>= n_det); Q has row stride n_det.
 */
static void filter_row(const double *p, int n_det, const double *h, double tau, double *q)
{
    for (int k = 0; k < n_det; ++k) {
        double s = 0.0;
        for (int j = 0; j < n_det; ++j) s += h[(k - j) + n_det - 1] * p[j];
        q[k] = tau * s;
    }
}

typedef struct {
    const double *P, *h;
    double tau;
    double *Q;
    int n_det, ld, i0, i1;
} filt_job;

static void *filter_rows_job(void *arg)
{
    filt_job *j = (filt_job *)arg;
    for (int i = j->i0; i < j->i1; ++i)
        filter_row(j->P + (size_t)i * j->ld, j->n_det, j->h, j->tau, j->Q + (size_t)i * j->n_det);
    return NULL;
}

/* nthreads > 1 splits the rows over POSIX threads (each row is independent). */
void oracle_filter_mt(const double *P, int n_angles, int n_det, int ld, const double *h,
                      double tau, double *Q, int nthreads)
{
    if (nthreads < 1) nthreads = 1;
    if (nthreads > n_angles) nthreads = n_angles;
    pthread_t *th = (pthread_t *)malloc(sizeof(pthread_t) * (size_t)nthreads);
    filt_job *jobs = (filt_job *)malloc(sizeof(filt_job) * (size_t)nthreads);
    for (int t = 0; t < nthreads; ++t) {
        jobs[t].P = P;
        jobs[t].h = h;
        jobs[t].tau = tau;
        jobs[t].Q = Q;
        jobs[t].n_det = n_det;
        jobs[t].ld = ld;
        jobs[t].i0 = (int)((long)n_angles * t / nthreads);
        jobs[t].i1 = (int)((long)n_angles * (t + 1) / nthreads);
    }
    if (nthreads == 1) {
        filter_rows_job(&jobs[0]);
    } else {
        for (int t = 0; t < nthreads; ++t) pthread_create(&th[t], NULL, filter_rows_job, &jobs[t]);
        for (int t = 0; t < nthreads; ++t) pthread_join(th[t], NULL);
    }
    free(jobs);
    free(th);
}

void oracle_filter(const double *P, int n_angles, int n_det, int ld, const double *h, double tau,
                   double *Q)
{
    oracle_filter_mt(P, n_angles, n_det, ld, h, tau, Q, 1);
}

/* Q_i read at fractional bin u: linear interpolation, zero outside [0,n_det). */
static double interp(const double *q, int n_det, double u)
{
    double fk = floor(u);
    double w = u - fk;
    long k = (long)fk;
    double q0 = (k >= 0 && k < n_det) ? q[k] : 0.0;
    double q1 = (k + 1 >= 0 && k + 1 < n_det) ? q[k + 1] : 0.0;
    return (1.0 - w) * q0 + w * q1;
}

/*
 * One pixel of Eq. 2: f(x,y) = (pi/n_angles) * sum_i Q_i(x cos th_i + y sin th_i),
 * the angles summed in order i = 0 .. n_angles-1.
 */
static double pixel_value(const double *Q, int n_angles, int n_det,
                          const double *theta, double tau, int n, int r, int c)
{
    double x = (double)c - 0.5 * (double)(n - 1);
    double y = (double)r - 0.5 * (double)(n - 1);
    double s = 0.0;
    for (int i = 0; i < n_angles; ++i) {
        double t = x * cos(theta[i]) + y * sin(theta[i]);
        double u = t / tau + 0.5 * (double)(n_det - 1);
        s += interp(Q + (size_t)i * n_det, n_det, u);
    }
    return s * (M_PI / (double)n_angles);
}

typedef struct {
    const double *Q;
    const double *theta;
    double tau;
    double *f;
    int n_angles, n_det, n, r0, r1;
} bp_job;

static void *bp_rows(void *arg)
{
    bp_job *j = (bp_job *)arg;
    for (int r = j->r0; r < j->r1; ++r)
        for (int c = 0; c < j->n; ++c)
            j->f[(size_t)r * j->n + c] =
                pixel_value(j->Q, j->n_angles, j->n_det, j->theta, j->tau, j->n, r, c);
    return NULL;
}

/*
 * Backprojection (Eq. 2) of filtered rows Q [n_angles][n_det] into the image
 * f [n][n] (row-major, f[r][c]).  nthreads > 1 splits the image rows over
 * POSIX threads; every pixel is computed the same way whatever the split.
 */
void oracle_backproject(const double *Q, int n_angles, int n_det,
                        const double *theta, double tau, int n, double *f,
                        int nthreads)
{
    if (nthreads < 1) nthreads = 1;
    if (nthreads > n) nthreads = n;
    pthread_t *th = (pthread_t *)malloc(sizeof(pthread_t) * (size_t)nthreads);
    bp_job *jobs = (bp_job *)malloc(sizeof(bp_job) * (size_t)nthreads);
    for (int t = 0; t < nthreads; ++t) {
        jobs[t].Q = Q;
        jobs[t].theta = theta;
        jobs[t].tau = tau;
        jobs[t].f = f;
        jobs[t].n_angles = n_angles;
        jobs[t].n_det = n_det;
        jobs[t].n = n;
        jobs[t].r0 = (int)((long)n * t / nthreads);
        jobs[t].r1 = (int)((long)n * (t + 1) / nthreads);
    }
    if (nthreads == 1) {
        bp_rows(&jobs[0]);
    } else {
        for (int t = 0; t < nthreads; ++t) pthread_create(&th[t], NULL, bp_rows, &jobs[t]);
        for (int t = 0; t < nthreads; ++t) pthread_join(th[t], NULL);
    }
    free(jobs);
    free(th);
}

/* Eq. 2 at selected pixels only (for spot checks of large images). */
void oracle_backproject_pixels(const double *Q, int n_angles, int n_det,
                               const double *theta, double tau, int n,
                               const int *rows, const int *cols, int count,
                               double *out)
{
    for (int p = 0; p < count; ++p)
        out[p] = pixel_value(Q, n_angles, n_det, theta, tau, n, rows[p], cols[p]);
}

/*
 * Discrete projection of an image (the Radon transform of the section
 * "Computed tomography", Fig. 1) in the form that is the exact transpose of
 * the interpolation above: each pixel adds its value to the two bins around
 * its detector coordinate with the linear-interpolation weights,
 *   P[i][k] = sum_{pixels} f(x,y) * max(0, 1 - |u_i(x,y) - k|),
 * with u_i(x,y) = (x cos th_i + y sin th_i)/tau + (n_det-1)/2 and the pi/n_angles
 * factor left out.  P is [n_angles][n_det].
 */
void oracle_forward(const double *f, int n, int n_angles, int n_det,
                    const double *theta, double tau, double *P)
{
    memset(P, 0, sizeof(double) * (size_t)n_angles * (size_t)n_det);
    for (int i = 0; i < n_angles; ++i) {
        double *p = P + (size_t)i * n_det;
        for (int r = 0; r < n; ++r) {
            for (int c = 0; c < n; ++c) {
                double x = (double)c - 0.5 * (double)(n - 1);
                double y = (double)r - 0.5 * (double)(n - 1);
                double t = x * cos(theta[i]) + y * sin(theta[i]);
                double u = t / tau + 0.5 * (double)(n_det - 1);
                double fk = floor(u);
                double w = u - fk;
                long k = (long)fk;
                double v = f[(size_t)r * n + c];
                if (k >= 0 && k < n_det) p[k] += (1.0 - w) * v;
                if (k + 1 >= 0 && k + 1 < n_det) p[k + 1] += w * v;
            }
        }
    }
}

/*
 * Whole FBP: taps, row filter, backprojection.  P has row stride ld.
 * Returns 0, or -1 on a bad argument or allocation failure.
 */
int oracle_fbp(const double *P, int n_angles, int n_det, int ld,
               const double *theta, double tau, int kind, int n, double *f,
               int nthreads)
{
    if (n_angles < 1 || n_det < 1 || n < 1 || ld < n_det) return -1;
    double *h = (double *)malloc(sizeof(double) * (size_t)(2 * n_det - 1));
    double *Q = (double *)malloc(sizeof(double) * (size_t)n_angles * (size_t)n_det);
    if (h == NULL || Q == NULL || oracle_taps(kind, n_det, tau, h) != 0) {
        free(h);
        free(Q);
        return -1;
    }
    oracle_filter_mt(P, n_angles, n_det, ld, h, tau, Q, nthreads);
    oracle_backproject(Q, n_angles, n_det, theta, tau, n, f, nthreads);
    free(h);
    free(Q);
    return 0;
}

/*
 * PSNR (Eq. 3): 20 log10(MAX / sqrt(MSE)) of an image x against a reference
 * y, both rows x cols (row-major, contiguous).  The paper leaves MAX open;
 * here MAX = max |y|.  Identical images give +inf (MSE = 0), as the paper
 * notes.  out[0] = PSNR in dB, out[1] = MSE, out[2] = MAX.
 */
void oracle_psnr(const double *x, const double *y, int rows, int cols, double *out)
{
    double se = 0.0, mx = 0.0;
    const long n = (long)rows * cols;
    for (long k = 0; k < n; ++k) {
        const double d = x[k] - y[k];
        se += d * d;
        if (fabs(y[k]) > mx) mx = fabs(y[k]);
    }
    const double mse = se / (double)n;
    out[0] = mse > 0.0 ? 20.0 * log10(mx / sqrt(mse)) : INFINITY;
    out[1] = mse;
    out[2] = mx;
}

/*
 * SSIM (Eq. 4) with the constants and window the paper leaves open taken from
 * Wang, Bovik, Sheikh & Simoncelli (2004): an 11 x 11 circular Gaussian window
 * of standard deviation 1.5 (weights normalised to sum 1), C1 = (0.01 L)^2,
 * C2 = (0.03 L)^2, and the image SSIM is the mean over every window that lies
 * inside the image.  L is the dynamic range; L <= 0 takes max(y) - min(y) of
 * the reference.  Per window:
 *     mu_x = sum w x,  sigma_x^2 = sum w (x - mu_x)^2,
 *     sigma_xy = sum w (x - mu_x)(y - mu_y),
 *     SSIM = (2 mu_x mu_y + C1)(2 sigma_xy + C2)
 *            / ((mu_x^2 + mu_y^2 + C1)(sigma_x^2 + sigma_y^2 + C2)).
 * Returns the mean SSIM (NaN if the image is smaller than the window).
 */
double oracle_ssim(const double *x, const double *y, int rows, int cols, double L)
{
    enum { W = 11, R = 5 };
    if (rows < W || cols < W) return NAN;
    if (L <= 0.0) {
        double lo = y[0], hi = y[0];
        for (long k = 1; k < (long)rows * cols; ++k) {
            if (y[k] < lo) lo = y[k];
            if (y[k] > hi) hi = y[k];
        }
        L = hi - lo;
    }
    const double c1 = (0.01 * L) * (0.01 * L), c2 = (0.03 * L) * (0.03 * L);
    double w[W][W], wsum = 0.0;
    for (int a = 0; a < W; ++a)
        for (int b = 0; b < W; ++b) {
            const double d2 = (double)((a - R) * (a - R) + (b - R) * (b - R));
            w[a][b] = exp(-d2 / (2.0 * 1.5 * 1.5));
            wsum += w[a][b];
        }
    for (int a = 0; a < W; ++a)
        for (int b = 0; b < W; ++b) w[a][b] /= wsum;
    double total = 0.0;
    long count = 0;
    for (int i = 0; i + W <= rows; ++i) {
        for (int j = 0; j + W <= cols; ++j) {
            double mx = 0.0, my = 0.0;
            for (int a = 0; a < W; ++a)
                for (int b = 0; b < W; ++b) {
                    mx += w[a][b] * x[(long)(i + a) * cols + (j + b)];
                    my += w[a][b] * y[(long)(i + a) * cols + (j + b)];
                }
            double vx = 0.0, vy = 0.0, cxy = 0.0;
            for (int a = 0; a < W; ++a)
                for (int b = 0; b < W; ++b) {
                    const double dx = x[(long)(i + a) * cols + (j + b)] - mx;
                    const double dy = y[(long)(i + a) * cols + (j + b)] - my;
                    vx += w[a][b] * dx * dx;
                    vy += w[a][b] * dy * dy;
                    cxy += w[a][b] * dx * dy;
                }
            total += ((2.0 * mx * my + c1) * (2.0 * cxy + c2)) /
                     ((mx * mx + my * my + c1) * (vx + vy + c2));
            ++count;
        }
    }
    return total / (double)count;
}

/*
 * A 3D volume from a stack of reconstructed 2D slices by interpolation along
 * z (section "Introduction": 3D images from the interpolation of a stack of
 * 2D images; the paper gives no rule, linear interpolation is read here).
 * K slices of n x n pixels at strictly increasing positions z[k]; M output
 * planes at zo[m], each inside [z[0], z[K-1]]: plane m = (1 - t) S_k + t S_{k+1}
 * with z[k] <= zo[m] <= z[k+1] and t = (zo[m] - z[k]) / (z[k+1] - z[k]).
 * Returns 0, or -1 for a plane outside the stack or non-increasing z.
 */
int oracle_volume(const double *slices, int K, const double *z, int n, const double *zo, int M,
                  double *out)
{
    for (int k = 1; k < K; ++k)
        if (!(z[k] > z[k - 1])) return -1;
    const long np = (long)n * n;
    for (int m = 0; m < M; ++m) {
        if (zo[m] < z[0] || zo[m] > z[K - 1]) return -1;
        int k = 0;
        while (k + 1 < K - 1 && zo[m] > z[k + 1]) ++k;
        if (K == 1) {
            for (long p = 0; p < np; ++p) out[(long)m * np + p] = slices[p];
            continue;
        }
        const double t = (zo[m] - z[k]) / (z[k + 1] - z[k]);
        for (long p = 0; p < np; ++p)
            out[(long)m * np + p] = (1.0 - t) * slices[(long)k * np + p] +
                                    t * slices[(long)(k + 1) * np + p];
    }
    return 0;
}

/*
 * FDK cone-beam reconstruction (Feldkamp, Davis & Kress 1984), the 3D
 * extension the paper names as its future work (section "Conclusion").  The
 * paper fixes no cone-beam geometry; the one read here:
 *   - the source circles the z axis at radius R, at (R cos b, R sin b, 0) for
 *     projection angle b, over a full turn (b_a given, 2 pi / A apart);
 *   - projections live on a virtual flat detector through the rotation axis,
 *     perpendicular to the central ray, with axes u along (-sin b, cos b, 0)
 *     and v along z: P[a][i][j] at u_j = (j - (nu-1)/2) du, v_i = (i - (nv-1)/2) dv;
 *   - voxel (ix, iy, iz) of an nx x ny x nz volume (f[iz][iy][ix]) has centre
 *     (ix - (nx-1)/2, iy - (ny-1)/2, iz - (nz-1)/2), voxel size 1.
 * Steps, in the order of the algorithm:
 *   1. weight: P~ = P R / sqrt(R^2 + u^2 + v^2);
 *   2. filter every detector row along u with the ramp taps (oracle_taps with
 *      spacing du): Q[a][i][k] = du sum_j h(k - j) P~[a][i][j];
 *   3. backproject: for every voxel and angle, s = x cos b + y sin b,
 *      t = -x sin b + y cos b, U = R - s, the voxel projects to
 *      u = R t / U, v = R z / U; Q is read there by bilinear interpolation
 *      (zero outside the detector) and weighted by (R / U)^2; the sum over the
 *      angles (in order) is scaled by (1/2)(2 pi / A) = pi / A, the 1/2 for the
 *      two passes of a full turn over every line.
 * As R grows the rays turn parallel, every weight tends to 1, u -> t and
 * v -> z: the result tends to the parallel-beam FBP (Eq. 2) of each detector
 * row at angles b + pi/2.  Returns 0, or -1 on a bad argument.
 */
typedef struct {
    const double *Q;
    const double *beta;
    int A, nv, nu, nx, ny, nz, z0, z1;
    double R, du, dv;
    double *f;
} fdk_job;

static double fdk_sample(const double *row0, const double *row1, double w1, int nu, double ku)
{
    /* row0/row1: the two detector rows around v (NULL when outside);
     * ku: column coordinate; linear in u then in v. */
    const double fk = floor(ku);
    const int k = (int)fk;
    const double w = ku - fk;
    double a = 0.0, b = 0.0;
    if (row0) {
        const double q0 = (k >= 0 && k < nu) ? row0[k] : 0.0;
        const double q1 = (k + 1 >= 0 && k + 1 < nu) ? row0[k + 1] : 0.0;
        a = (1.0 - w) * q0 + w * q1;
    }
    if (row1) {
        const double q0 = (k >= 0 && k < nu) ? row1[k] : 0.0;
        const double q1 = (k + 1 >= 0 && k + 1 < nu) ? row1[k + 1] : 0.0;
        b = (1.0 - w) * q0 + w * q1;
    }
    return (1.0 - w1) * a + w1 * b;
}

static void *fdk_slices(void *arg)
{
    fdk_job *J = (fdk_job *)arg;
    const long row_len = J->nu;
    for (int iz = J->z0; iz < J->z1; ++iz) {
        const double z = (double)iz - 0.5 * (double)(J->nz - 1);
        for (int iy = 0; iy < J->ny; ++iy) {
            const double y = (double)iy - 0.5 * (double)(J->ny - 1);
            for (int ix = 0; ix < J->nx; ++ix) {
                const double x = (double)ix - 0.5 * (double)(J->nx - 1);
                double sum = 0.0;
                for (int a = 0; a < J->A; ++a) {
                    const double cb = cos(J->beta[a]), sb = sin(J->beta[a]);
                    const double s = x * cb + y * sb, t = -x * sb + y * cb;
                    const double U = J->R - s;
                    const double u = J->R * t / U, v = J->R * z / U;
                    const double ku = u / J->du + 0.5 * (double)(J->nu - 1);
                    const double kv = v / J->dv + 0.5 * (double)(J->nv - 1);
                    const double fv = floor(kv);
                    const int i = (int)fv;
                    const double wv = kv - fv;
                    const double *base = J->Q + (long)a * J->nv * row_len;
                    const double *r0 = (i >= 0 && i < J->nv) ? base + (long)i * row_len : NULL;
                    const double *r1 = (i + 1 >= 0 && i + 1 < J->nv) ? base + (long)(i + 1) * row_len : NULL;
                    const double q = fdk_sample(r0, r1, wv, J->nu, ku);
                    sum += (J->R / U) * (J->R / U) * q;
                }
                J->f[((long)iz * J->ny + iy) * J->nx + ix] = sum * (M_PI / (double)J->A);
            }
        }
    }
    return NULL;
}

int oracle_fdk(const double *P, int A, int nv, int nu, const double *beta, double R, double du,
               double dv, int kind, int nx, int ny, int nz, double *f, int nthreads)
{
    if (A < 1 || nv < 1 || nu < 1 || nx < 1 || ny < 1 || nz < 1 || !(R > 0.0) || !(du > 0.0) ||
        !(dv > 0.0))
        return -1;
    const long rows = (long)A * nv;
    double *h = (double *)malloc(sizeof(double) * (size_t)(2 * nu - 1));
    double *Pw = (double *)malloc(sizeof(double) * (size_t)rows * (size_t)nu);
    double *Q = (double *)malloc(sizeof(double) * (size_t)rows * (size_t)nu);
    if (h == NULL || Pw == NULL || Q == NULL || oracle_taps(kind, nu, du, h) != 0) {
        free(h);
        free(Pw);
        free(Q);
        return -1;
    }
    /* 1. cosine weight */
    for (int a = 0; a < A; ++a)
        for (int i = 0; i < nv; ++i) {
            const double v = ((double)i - 0.5 * (double)(nv - 1)) * dv;
            for (int j = 0; j < nu; ++j) {
                const double u = ((double)j - 0.5 * (double)(nu - 1)) * du;
                const long k = ((long)a * nv + i) * nu + j;
                Pw[k] = P[k] * R / sqrt(R * R + u * u + v * v);
            }
        }
    /* 2. ramp filter along u, row by row */
    oracle_filter_mt(Pw, (int)rows, nu, nu, h, du, Q, nthreads);
    /* 3. weighted backprojection, slabs of z over threads */
    if (nthreads < 1) nthreads = 1;
    if (nthreads > nz) nthreads = nz;
    pthread_t *th = (pthread_t *)malloc(sizeof(pthread_t) * (size_t)nthreads);
    fdk_job *jobs = (fdk_job *)malloc(sizeof(fdk_job) * (size_t)nthreads);
    for (int t = 0; t < nthreads; ++t) {
        fdk_job J = {Q, beta, A, nv, nu, nx, ny, nz, (int)((long)nz * t / nthreads),
                     (int)((long)nz * (t + 1) / nthreads), R, du, dv, f};
        jobs[t] = J;
        if (nthreads == 1)
            fdk_slices(&jobs[t]);
        else
            pthread_create(&th[t], NULL, fdk_slices, &jobs[t]);
    }
    if (nthreads > 1)
        for (int t = 0; t < nthreads; ++t) pthread_join(th[t], NULL);
    free(th);
    free(jobs);
    free(h);
    free(Pw);
    free(Q);
    return 0;
}
