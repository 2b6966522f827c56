// Eq. 1 (Lambert-Beer) on load.  The filter routes take line integrals p; a
// plan with an incident intensity i0 > 0 reads measured intensities (or photon
// counts) I instead and converts each value as it loads it,
//     p = -ln(max(I, 1) / i0) = ln(i0) - ln(max(I, 1)),
// one count being the floor (zero counts have no logarithm).  The FP32 routes
// take the difference form with ln(i0) computed once per plan in FP64 (no
// division per value); the FP64 path takes the ratio form.  i0 = 0 passes the
// value through.  Values outside the detector are zero padding and are not
// converted.
#pragma once

namespace fbp {

__device__ __forceinline__ float line_integral(float v, float i0, float ln_i0)
{
    return i0 > 0.0f ? ln_i0 - logf(fmaxf(v, 1.0f)) : v;
}

__device__ __forceinline__ double line_integral(double v, double i0)
{
    return i0 > 0.0 ? -log(fmax(v, 1.0) / i0) : v;
}

}  // namespace fbp
