// Ramp filter Q = P * H (the convolution stated after Eq. 2), FFT route.
//
// With N >= 2*n_det - 1 the circular convolution of the zero-padded row with
// the circularly arranged taps equals the linear convolution on [0, n_det),
// so Q_i = IDFT_N( DFT_N(P_i) . H ) restricted to the first n_det bins, where
// H = DFT_N of the taps tau*h(m) placed at m mod N.  H is real and even (the
// taps are symmetric), so two real rows can share one complex transform:
// z = P_i + i P_{i+1} gives IDFT(DFT(z) . H) = Q_i + i Q_{i+1} exactly.
//
// One CTA of N/16 threads per row pair.  The transform is a Stockham autosort
// FFT whose butterflies run in registers: thread t always holds 16 elements,
// those at positions t + q N/16 (q = 0..15).  log2 N = 4a + b is done as a
// radix-16 passes and, when b > 0, one last radix-2^b pass; between passes the
// elements go through shared memory once (index padded by one slot per 16,
// which keeps every pass's stores and loads free of bank conflicts).  The last
// pass of a Stockham transform leaves each thread's results at the same
// positions it read, so the product with H and the first pass of the inverse
// follow in registers, without a shared-memory exchange.  Twiddles
// exp(-2 pi i t / N) come from a plan table computed in FP64: a radix-16 pass
// loads w^k, w^2k, w^4k, w^8k and forms the other eleven powers with at most
// three complex products.  The 1/N of the inverse is folded into H.
// One launch covers the row pairs of many slices with the same N (their plans
// may differ otherwise), so a batch fills the GPU instead of running slice
// after slice.
#include "fbp_internal.h"
#include "pairs.cuh"

#include <vector>

namespace fbp {
namespace {

__device__ __forceinline__ float2 cmul(float2 a, float2 b)
{
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }

// a times exp(-i pi/2) (forward) or exp(+i pi/2) (inverse).
template <bool INV>
__device__ __forceinline__ float2 rot90(float2 a)
{
    return INV ? make_float2(-a.y, a.x) : make_float2(a.y, -a.x);
}

// cos(pi e / 8) for e in [0, 16).
constexpr float kCosPi8[16] = {
    1.0f,  0.92387953251128674f,  0.70710678118654752f,  0.38268343236508977f,
    0.0f,  -0.38268343236508977f, -0.70710678118654752f, -0.92387953251128674f,
    -1.0f, -0.92387953251128674f, -0.70710678118654752f, -0.38268343236508977f,
    0.0f,  0.38268343236508977f,  0.70710678118654752f,  0.92387953251128674f};

// a times exp(-+ 2 pi i E / 16).
template <bool INV, int E>
__device__ __forceinline__ float2 twiddle16(float2 a)
{
    static_assert(E >= 0 && E < 16, "exponent in [0, 16)");
    if constexpr (E == 0) {
        return a;
    } else if constexpr (E == 4) {
        return rot90<INV>(a);
    } else {
        constexpr float c = kCosPi8[E], s = kCosPi8[(E + 12) % 16];  // sin(x) = cos(x - pi/2)
        return cmul(a, make_float2(c, INV ? s : -s));
    }
}

template <bool INV>
__device__ __forceinline__ void dft2(float2 &a0, float2 &a1)
{
    const float2 b = csub(a0, a1);
    a0 = cadd(a0, a1);
    a1 = b;
}

// 4-point DFT, inputs and outputs in natural order.
template <bool INV>
__device__ __forceinline__ void dft4(float2 &a0, float2 &a1, float2 &a2, float2 &a3)
{
    const float2 b0 = cadd(a0, a2), b1 = csub(a0, a2), b2 = cadd(a1, a3);
    const float2 b3 = rot90<INV>(csub(a1, a3));
    a0 = cadd(b0, b2);
    a1 = cadd(b1, b3);
    a2 = csub(b0, b2);
    a3 = csub(b1, b3);
}

// 8-point DFT as 2 x 4: q = q1 + 2 q2, m = m2 + 4 m1.
template <bool INV>
__device__ __forceinline__ void dft8(float2 (&a)[8])
{
    dft4<INV>(a[0], a[2], a[4], a[6]);  // q1 = 0: A[0][m2] in a[2 m2]
    dft4<INV>(a[1], a[3], a[5], a[7]);  // q1 = 1: A[1][m2] in a[2 m2 + 1]
    a[3] = twiddle16<INV, 2>(a[3]);     // exp(-+ 2 pi i m2 / 8), m2 = 1..3
    a[5] = twiddle16<INV, 4>(a[5]);
    a[7] = twiddle16<INV, 6>(a[7]);
    float2 x[8];
#pragma unroll
    for (int m2 = 0; m2 < 4; ++m2) {
        x[m2] = cadd(a[2 * m2], a[2 * m2 + 1]);
        x[m2 + 4] = csub(a[2 * m2], a[2 * m2 + 1]);
    }
#pragma unroll
    for (int m = 0; m < 8; ++m) a[m] = x[m];
}

// 16-point DFT as 4 x 4: q = q1 + 4 q2, m = m2 + 4 m1.
template <bool INV>
__device__ __forceinline__ void dft16(float2 (&v)[16])
{
#pragma unroll
    for (int q1 = 0; q1 < 4; ++q1) dft4<INV>(v[q1], v[q1 + 4], v[q1 + 8], v[q1 + 12]);
    // v[q1 + 4 m2] = A[q1][m2]; twiddle by exp(-+ 2 pi i q1 m2 / 16)
    v[5] = twiddle16<INV, 1>(v[5]);
    v[9] = twiddle16<INV, 2>(v[9]);
    v[13] = twiddle16<INV, 3>(v[13]);
    v[6] = twiddle16<INV, 2>(v[6]);
    v[10] = twiddle16<INV, 4>(v[10]);
    v[14] = twiddle16<INV, 6>(v[14]);
    v[7] = twiddle16<INV, 3>(v[7]);
    v[11] = twiddle16<INV, 6>(v[11]);
    v[15] = twiddle16<INV, 9>(v[15]);
#pragma unroll
    for (int m2 = 0; m2 < 4; ++m2) dft4<INV>(v[4 * m2], v[4 * m2 + 1], v[4 * m2 + 2], v[4 * m2 + 3]);
    // X[m2 + 4 m1] sits in v[m1 + 4 m2]: transpose
    float2 x[16];
#pragma unroll
    for (int m2 = 0; m2 < 4; ++m2)
#pragma unroll
        for (int m1 = 0; m1 < 4; ++m1) x[m2 + 4 * m1] = v[m1 + 4 * m2];
#pragma unroll
    for (int m = 0; m < 16; ++m) v[m] = x[m];
}

__device__ __forceinline__ int pad16(int i) { return i + (i >> 4); }

template <bool INV>
__device__ __forceinline__ float2 tw_at(const float2 *__restrict__ tw, int i)
{
    float2 w = __ldg(&tw[i]);
    if (INV) w.y = -w.y;
    return w;
}

// Full N-point transform of the elements the block holds (thread t: positions
// t + q N/16 in v[q]); on return v[q] holds output position t + q N/16.
template <bool INV>
__device__ void fft_regs(float2 (&v)[16], float2 *buf, const float2 *__restrict__ tw, int N,
                         int log2n)
{
    const int t = threadIdx.x;
    const int T = N >> 4;
    const int n16 = log2n >> 2;
    const int rem = log2n & 3;
    int ns = 1, log2ns = 0;
    for (int p = 0; p < n16; ++p) {
        const bool last = rem == 0 && p == n16 - 1;
        const int k = t & (ns - 1);
        if (ns > 1) {
            const int i1 = k << (log2n - 4 - log2ns);  // k N / (16 ns)
            const float2 w1 = tw_at<INV>(tw, i1), w2 = tw_at<INV>(tw, 2 * i1);
            const float2 w4 = tw_at<INV>(tw, 4 * i1), w8 = tw_at<INV>(tw, 8 * i1);
            const float2 w3 = cmul(w1, w2);
            const float2 w5 = cmul(w4, w1), w6 = cmul(w4, w2), w7 = cmul(w4, w3);
            v[1] = cmul(v[1], w1);
            v[2] = cmul(v[2], w2);
            v[3] = cmul(v[3], w3);
            v[4] = cmul(v[4], w4);
            v[5] = cmul(v[5], w5);
            v[6] = cmul(v[6], w6);
            v[7] = cmul(v[7], w7);
            v[8] = cmul(v[8], w8);
            v[9] = cmul(v[9], cmul(w8, w1));
            v[10] = cmul(v[10], cmul(w8, w2));
            v[11] = cmul(v[11], cmul(w8, w3));
            v[12] = cmul(v[12], cmul(w8, w4));
            v[13] = cmul(v[13], cmul(w8, w5));
            v[14] = cmul(v[14], cmul(w8, w6));
            v[15] = cmul(v[15], cmul(w8, w7));
        }
        dft16<INV>(v);
        if (!last) {
            const int o = ((t - k) << 4) + k;
#pragma unroll
            for (int m = 0; m < 16; ++m) buf[pad16(o + m * ns)] = v[m];
            __syncthreads();
#pragma unroll
            for (int q = 0; q < 16; ++q) v[q] = buf[pad16(t + q * T)];
            __syncthreads();
        }
        ns <<= 4;
        log2ns += 4;
    }
    if (rem == 0) return;
    // last pass, radix R = 2^rem, ns = N / R: butterfly j = t + m T (m < 16/R)
    // takes positions j + s N/R = t + (m + s 16/R) T, twiddles exp(-+ 2 pi i s j / N)
    if (rem == 3) {
#pragma unroll
        for (int m = 0; m < 2; ++m) {
            const int j = t + m * T;
            float2 a[8];
#pragma unroll
            for (int s = 0; s < 8; ++s) a[s] = s ? cmul(v[m + 2 * s], tw_at<INV>(tw, s * j)) : v[m];
            dft8<INV>(a);
#pragma unroll
            for (int s = 0; s < 8; ++s) v[m + 2 * s] = a[s];
        }
    } else if (rem == 2) {
#pragma unroll
        for (int m = 0; m < 4; ++m) {
            const int j = t + m * T;
            float2 a1 = cmul(v[m + 4], tw_at<INV>(tw, j));
            float2 a2 = cmul(v[m + 8], tw_at<INV>(tw, 2 * j));
            float2 a3 = cmul(v[m + 12], tw_at<INV>(tw, 3 * j));
            dft4<INV>(v[m], a1, a2, a3);
            v[m + 4] = a1;
            v[m + 8] = a2;
            v[m + 12] = a3;
        }
    } else {
#pragma unroll
        for (int m = 0; m < 8; ++m) {
            const int j = t + m * T;
            float2 a1 = cmul(v[m + 8], tw_at<INV>(tw, j));
            dft2<INV>(v[m], a1);
            v[m + 8] = a1;
        }
    }
}

// One slice's part of a launch; pair_end is the inclusive prefix sum of the
// slices' row-pair counts, so CTA b works on the slice s with
// pair_end[s-1] <= b < pair_end[s].  All slices of a launch share N.
struct FftSlice {
    const float *sino;
    void *q;
    const float2 *tw;
    const float *h;
    int ld;
    int pitch;
    int A;
    int D;
    int pair_end;
    int pad_;
};

template <int MAXS>
struct FftLaunch {
    FftSlice s[MAXS];
    int n;
    int N;
    int log2n;
};

template <typename OutT, int MAXS>
__global__ void __launch_bounds__(kMaxFftLen / 16) filter_fft_kernel(const __grid_constant__ FftLaunch<MAXS> L)
{
    extern __shared__ float2 buf[];
    int lo = 0, hi = L.n - 1;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if ((int)blockIdx.x < L.s[mid].pair_end) hi = mid; else lo = mid + 1;
    }
    const FftSlice &S = L.s[lo];
    const int pair = (int)blockIdx.x - (lo > 0 ? L.s[lo - 1].pair_end : 0);
    const int N = L.N, D = S.D, T = N >> 4, t = threadIdx.x;
    const int i0 = 2 * pair;
    const bool two = i0 + 1 < S.A;
    const float *p0 = S.sino + (size_t)i0 * S.ld;
    const float *p1 = S.sino + (size_t)(two ? i0 + 1 : i0) * S.ld;
    float2 v[16];
#pragma unroll
    for (int q = 0; q < 16; ++q) {
        const int j = t + q * T;
        v[q] = make_float2(0.0f, 0.0f);
        if (j < D) {
            v[q].x = p0[j];
            v[q].y = two ? p1[j] : 0.0f;
        }
    }
    fft_regs<false>(v, buf, S.tw, N, L.log2n);
#pragma unroll
    for (int q = 0; q < 16; ++q) {
        const float hv = __ldg(&S.h[t + q * T]);
        v[q] = make_float2(v[q].x * hv, v[q].y * hv);
    }
    fft_regs<true>(v, buf, S.tw, N, L.log2n);
    // every thread is past its last read of buf (the final pass of the inverse
    // reads none; the one before ends with a barrier)
#pragma unroll
    for (int q = 0; q < 16; ++q) buf[pad16(t + q * T)] = v[q];
    __syncthreads();
    // buf[k] = (Q_i0[k], Q_i0+1[k]) for k < n_det; write (mid, slope) pairs.
    OutT *r0 = static_cast<OutT *>(S.q) + (size_t)i0 * S.pitch;
    OutT *r1 = static_cast<OutT *>(S.q) + (size_t)(i0 + 1) * S.pitch;
    for (int p = t; p < S.pitch / 2; p += T) {
        float2 a = make_float2(0.0f, 0.0f), b = make_float2(0.0f, 0.0f);
        if (p <= D) {
            if (p >= 1) a = buf[pad16(p - 1)];
            if (p < D) b = buf[pad16(p)];
        }
        store_pair(r0, p, a.x, b.x);
        if (two) store_pair(r1, p, a.y, b.y);
    }
}

int log2_of(int N)
{
    int l = 0;
    while ((1 << l) < N) ++l;
    return l;
}

template <typename OutT, int MAXS>
cudaError_t launch_set(FftLaunch<MAXS> &L, int total, int N, cudaStream_t s)
{
    L.N = N;
    L.log2n = log2_of(N);
    const size_t smem = filter_fft_smem_bytes(N);
    cudaError_t e = cudaFuncSetAttribute(filter_fft_kernel<OutT, MAXS>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    filter_fft_kernel<OutT, MAXS><<<total, N / 16, smem, s>>>(L);
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
    f.pair_end = 0;
    f.pad_ = 0;
    return f;
}

}  // namespace

size_t filter_fft_smem_bytes(int N) { return sizeof(float2) * (size_t)(N + N / 16); }

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
    // one launch per (storage type, FFT length, up to kFftMaxSlices slices)
    std::vector<int> lens;
    for (int i = 0; i < n; ++i) {
        const Plan &p = *plans[i];
        if (p.filter_path != FBP_PATH_FFT) continue;
        bool seen = false;
        for (int v : lens) seen = seen || v == p.fft_len;
        if (!seen) lens.push_back(p.fft_len);
    }
    for (int N : lens) {
        for (int half = 0; half < 2; ++half) {
            FftLaunch<kFftMaxSlices> L;
            int cnt = 0, total = 0;
            auto flush = [&]() -> cudaError_t {
                if (cnt == 0) return cudaSuccess;
                L.n = cnt;
                cudaError_t e = half ? launch_set<__half, kFftMaxSlices>(L, total, N, s)
                                     : launch_set<float, kFftMaxSlices>(L, total, N, s);
                cnt = 0;
                total = 0;
                return e;
            };
            for (int i = 0; i < n; ++i) {
                const Plan &p = *plans[i];
                if (p.filter_path != FBP_PATH_FFT || p.fft_len != N ||
                    (p.q_storage == FBP_F16) != (half == 1))
                    continue;
                L.s[cnt] = fft_slice(p, sinos[i], lds[i], qs[i]);
                total += (p.A + 1) / 2;
                L.s[cnt].pair_end = total;
                if (++cnt == kFftMaxSlices) {
                    cudaError_t e = flush();
                    if (e != cudaSuccess) return e;
                }
            }
            cudaError_t e = flush();
            if (e != cudaSuccess) return e;
        }
    }
    return cudaSuccess;
}

}  // namespace fbp
