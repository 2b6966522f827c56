// Ramp filter Q = P * H (the convolution stated after Eq. 2), FFT route.
//
// With N >= 2*n_det - 1 the circular convolution of the zero-padded row with
// the circularly arranged taps equals the linear convolution on [0, n_det),
// so Q_i = IDFT_N( DFT_N(P_i) . H ) restricted to the first n_det bins, where
// H = DFT_N of the taps tau*h(m) placed at m mod N.  H is real and even (the
// taps are symmetric), so two real rows can share one complex transform:
// z = P_i + i P_{i+1} gives IDFT(DFT(z) . H) = Q_i + i Q_{i+1} exactly.
//
// One CTA per row pair; the N-point complex transform is a radix-4 Stockham
// autosort FFT (one radix-2 pass first when log2 N is odd) ping-ponging
// between two shared-memory buffers; twiddles exp(-2 pi i t / N) come from a
// plan table computed in FP64.  The 1/N of the inverse is folded into H.
// One launch can cover the row pairs of many slices (their plans may differ),
// so a batch fills the GPU instead of running slice after slice.
#include "fbp_internal.h"
#include "pairs.cuh"

namespace fbp {
namespace {

__device__ __forceinline__ float2 cmul(float2 a, float2 b)
{
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 conj_if(float2 a, bool inv) { return inv ? make_float2(a.x, -a.y) : a; }

// Radix-2 pass, sub-transform size ns -> 2 ns.
__device__ void pass2(const float2 *x, float2 *y, const float2 *__restrict__ tw, int N, int ns,
                      bool inv)
{
    const int half = N >> 1;
    const int stride = N / (2 * ns);
    for (int j = threadIdx.x; j < half; j += blockDim.x) {
        const int k = j & (ns - 1);
        const float2 w = conj_if(__ldg(&tw[k * stride]), inv);
        const float2 a0 = x[j];
        const float2 a1 = cmul(x[j + half], w);
        const int o = ((j - k) << 1) + k;
        y[o] = cadd(a0, a1);
        y[o + ns] = csub(a0, a1);
    }
}

// Radix-4 pass, sub-transform size ns -> 4 ns.
__device__ void pass4(const float2 *x, float2 *y, const float2 *__restrict__ tw, int N, int ns,
                      bool inv)
{
    const int q = N >> 2;
    const int stride = N / (4 * ns);
    for (int j = threadIdx.x; j < q; j += blockDim.x) {
        const int k = j & (ns - 1);
        const float2 w1 = conj_if(__ldg(&tw[k * stride]), inv);
        const float2 w2 = conj_if(__ldg(&tw[2 * k * stride]), inv);
        const float2 w3 = conj_if(__ldg(&tw[3 * k * stride]), inv);
        const float2 a0 = x[j];
        const float2 a1 = cmul(x[j + q], w1);
        const float2 a2 = cmul(x[j + 2 * q], w2);
        const float2 a3 = cmul(x[j + 3 * q], w3);
        const float2 b0 = cadd(a0, a2);
        const float2 b1 = csub(a0, a2);
        const float2 b2 = cadd(a1, a3);
        const float2 d = csub(a1, a3);
        // forward: multiply by -i; inverse: by +i
        const float2 b3 = inv ? make_float2(-d.y, d.x) : make_float2(d.y, -d.x);
        const int o = ((j - k) << 2) + k;
        y[o] = cadd(b0, b2);
        y[o + ns] = cadd(b1, b3);
        y[o + 2 * ns] = csub(b0, b2);
        y[o + 3 * ns] = csub(b1, b3);
    }
}

// Full transform; returns the buffer holding the result.
__device__ float2 *fft(float2 *x, float2 *y, const float2 *__restrict__ tw, int N, int log2n,
                       bool inv)
{
    int ns = 1;
    if (log2n & 1) {
        pass2(x, y, tw, N, ns, inv);
        __syncthreads();
        float2 *t = x; x = y; y = t;
        ns = 2;
    }
    for (; ns < N; ns <<= 2) {
        pass4(x, y, tw, N, ns, inv);
        __syncthreads();
        float2 *t = x; x = y; y = t;
    }
    return x;
}

// One slice's part of a launch; pair_end is the inclusive prefix sum of the
// slices' row-pair counts, so CTA b works on the slice s with
// pair_end[s-1] <= b < pair_end[s].
struct FftSlice {
    const float *sino;
    void *q;
    const float2 *tw;
    const float *h;
    int ld;
    int pitch;
    int A;
    int D;
    int N;
    int log2n;
    int pair_end;
    int pad_;
};

template <int MAXS>
struct FftLaunch {
    FftSlice s[MAXS];
    int n;
};

template <typename OutT, int MAXS>
__global__ void __launch_bounds__(256) filter_fft_kernel(const __grid_constant__ FftLaunch<MAXS> L)
{
    extern __shared__ float2 buf[];
    int lo = 0, hi = L.n - 1;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if ((int)blockIdx.x < L.s[mid].pair_end) hi = mid; else lo = mid + 1;
    }
    const FftSlice &S = L.s[lo];
    const int pair = (int)blockIdx.x - (lo > 0 ? L.s[lo - 1].pair_end : 0);
    const int N = S.N, D = S.D;
    float2 *x = buf;
    float2 *y = buf + N;
    const int i0 = 2 * pair;
    const bool two = i0 + 1 < S.A;
    const float *p0 = S.sino + (size_t)i0 * S.ld;
    const float *p1 = S.sino + (size_t)(two ? i0 + 1 : i0) * S.ld;
    for (int j = threadIdx.x; j < N; j += blockDim.x) {
        float2 v = make_float2(0.0f, 0.0f);
        if (j < D) {
            v.x = p0[j];
            v.y = two ? p1[j] : 0.0f;
        }
        x[j] = v;
    }
    __syncthreads();
    float2 *z = fft(x, y, S.tw, N, S.log2n, false);
    for (int j = threadIdx.x; j < N; j += blockDim.x) {
        const float hv = __ldg(&S.h[j]);
        z[j] = make_float2(z[j].x * hv, z[j].y * hv);
    }
    __syncthreads();
    float2 *other = (z == x) ? y : x;
    z = fft(z, other, S.tw, N, S.log2n, true);
    // z[k] = (Q_i0[k], Q_i0+1[k]) for k < n_det; write (mid, slope) pairs.
    OutT *r0 = static_cast<OutT *>(S.q) + (size_t)i0 * S.pitch;
    OutT *r1 = static_cast<OutT *>(S.q) + (size_t)(i0 + 1) * S.pitch;
    for (int p = threadIdx.x; p < S.pitch / 2; p += blockDim.x) {
        float2 a = make_float2(0.0f, 0.0f), b = make_float2(0.0f, 0.0f);
        if (p <= D) {
            if (p >= 1) a = z[p - 1];
            if (p < D) b = z[p];
        }
        store_pair(r0, p, a.x, b.x);
        if (two) store_pair(r1, p, a.y, b.y);
    }
}

template <typename OutT, int MAXS>
cudaError_t launch_set(const FftLaunch<MAXS> &L, int total, int nmax, cudaStream_t s)
{
    const size_t smem = sizeof(float2) * (size_t)(2 * nmax);
    cudaError_t e = cudaFuncSetAttribute(filter_fft_kernel<OutT, MAXS>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    filter_fft_kernel<OutT, MAXS><<<total, 256, smem, s>>>(L);
    return cudaGetLastError();
}

FftSlice fft_slice(const Plan &p, const float *sino, int ld, void *q)
{
    FftSlice f;
    f.sino = sino;
    f.q = q;
    f.tw = p.d_fft_tw;
    f.h = p.d_fft_h;
    f.ld = ld;
    f.pitch = p.pitch;
    f.A = p.A;
    f.D = p.D;
    f.N = p.fft_len;
    int log2n = 0;
    while ((1 << log2n) < p.fft_len) ++log2n;
    f.log2n = log2n;
    f.pair_end = 0;
    f.pad_ = 0;
    return f;
}

}  // namespace

size_t filter_fft_smem_bytes(int N) { return sizeof(float2) * (size_t)(2 * N); }

cudaError_t launch_filter_fft(const Plan &p, const float *sino, int ld, void *q, cudaStream_t s)
{
    FftLaunch<1> L;
    L.s[0] = fft_slice(p, sino, ld, q);
    L.s[0].pair_end = (p.A + 1) / 2;
    L.n = 1;
    if (p.q_storage == FBP_F16) return launch_set<__half, 1>(L, L.s[0].pair_end, p.fft_len, s);
    return launch_set<float, 1>(L, L.s[0].pair_end, p.fft_len, s);
}

cudaError_t launch_filter_fft_many(const Plan *const *plans, const float *const *sinos,
                                   const int *lds, void *const *qs, int n, cudaStream_t s)
{
    // one launch per (storage type, up to kFftMaxSlices slices)
    for (int half = 0; half < 2; ++half) {
        FftLaunch<kFftMaxSlices> L;
        int cnt = 0, total = 0, nmax = 16;
        auto flush = [&]() -> cudaError_t {
            if (cnt == 0) return cudaSuccess;
            L.n = cnt;
            cudaError_t e = half ? launch_set<__half, kFftMaxSlices>(L, total, nmax, s)
                                 : launch_set<float, kFftMaxSlices>(L, total, nmax, s);
            cnt = 0;
            total = 0;
            nmax = 16;
            return e;
        };
        for (int i = 0; i < n; ++i) {
            const Plan &p = *plans[i];
            if (p.filter_path != FBP_PATH_FFT || (p.q_storage == FBP_F16) != (half == 1)) continue;
            L.s[cnt] = fft_slice(p, sinos[i], lds[i], qs[i]);
            total += (p.A + 1) / 2;
            L.s[cnt].pair_end = total;
            nmax = p.fft_len > nmax ? p.fft_len : nmax;
            if (++cnt == kFftMaxSlices) {
                cudaError_t e = flush();
                if (e != cudaSuccess) return e;
            }
        }
        cudaError_t e = flush();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace fbp
