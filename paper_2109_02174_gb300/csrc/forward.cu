// Test-only discrete projector (the Radon projection of section "Computed
// tomography", Fig. 1) in the form that is the transpose of the interpolating
// backprojection:
//   sino[i][k] = sum_{r,c} image[r][c] * max(0, 1 - |u_i(r,c) - k|).
// Gather form: one thread per (angle, bin) walks the image along its dominant
// axis and visits only the pixels with |u - k| < 1.  No atomics; positions and
// the running sum are FP64.
#include "fbp_internal.h"

namespace fbp {
namespace {

__global__ void radon_forward_f32_kernel(const float *__restrict__ img, float *__restrict__ sino,
                                         const double2 *__restrict__ trig, int n, int A, int D,
                                         double half_n, double half_d)
{
    const int k = blockIdx.y * blockDim.x + threadIdx.x;
    const int i = blockIdx.x;  // angles on x: up to 2^31 - 1 of them
    if (k >= D || i >= A) return;
    const double c = trig[i].x;  // cos / tau
    const double s = trig[i].y;  // sin / tau
    const double kk = (double)k - half_d;  // u - half_d at the bin centre
    double acc = 0.0;
    if (fabs(c) >= fabs(s)) {
        for (int r = 0; r < n; ++r) {
            const double ys = ((double)r - half_n) * s;
            double xa = (kk - 1.0 - ys) / c;
            double xb = (kk + 1.0 - ys) / c;
            if (xa > xb) { const double t = xa; xa = xb; xb = t; }
            const int c0 = max(0, (int)ceil(xa + half_n));
            const int c1 = min(n - 1, (int)floor(xb + half_n));
            for (int col = c0; col <= c1; ++col) {
                const double w = 1.0 - fabs(((double)col - half_n) * c + ys - kk);
                if (w > 0.0) acc += w * (double)img[(size_t)r * n + col];
            }
        }
    } else {
        for (int col = 0; col < n; ++col) {
            const double xc = ((double)col - half_n) * c;
            double ya = (kk - 1.0 - xc) / s;
            double yb = (kk + 1.0 - xc) / s;
            if (ya > yb) { const double t = ya; ya = yb; yb = t; }
            const int r0 = max(0, (int)ceil(ya + half_n));
            const int r1 = min(n - 1, (int)floor(yb + half_n));
            for (int r = r0; r <= r1; ++r) {
                const double w = 1.0 - fabs(xc + ((double)r - half_n) * s - kk);
                if (w > 0.0) acc += w * (double)img[(size_t)r * n + col];
            }
        }
    }
    sino[(size_t)i * D + k] = (float)acc;
}

}  // namespace

cudaError_t launch_radon_forward_f32(const Plan &p, const float *image, float *sino,
                                     cudaStream_t s)
{
    dim3 grid(p.A, (p.D + 127) / 128);
    radon_forward_f32_kernel<<<grid, 128, 0, s>>>(image, sino, p.d_trig64, p.n, p.A, p.D,
                                                 0.5 * (double)(p.n - 1),
                                                 0.5 * (double)(p.D - 1));
    return cudaGetLastError();
}

}  // namespace fbp
