// Ramp filter Q = P * H (the convolution stated after Eq. 2), FFT route.
//
// With N >= 2*n_det - 1 the circular convolution of the zero-padded row with
// the circularly arranged taps equals the linear convolution on [0, n_det),
// so Q_i = IDFT_N( DFT_N(P_i) . H ) restricted to the first n_det bins, where
// H = DFT_N of the taps tau*h(m) placed at m mod N.  H is real and even (the
// taps are symmetric), so two real rows can share one complex transform:
// z = P_i + i P_{i+1} gives IDFT(DFT(z) . H) = Q_i + i Q_{i+1} exactly.
//
// One CTA of N/16 threads per block of four rows: two complex transforms
// (rows i, i+1 and rows i+2, i+3) computed in lockstep with packed f32x2
// arithmetic, lane .x of every register pair belonging to the first transform
// and lane .y to the second, so each complex add is one packed instruction
// and each product two.  The transform is a Stockham autosort FFT whose
// butterflies run in registers: thread t always holds the 16 elements at
// positions t + q N/16 (q = 0..15).  log2 N = 4a + b is done as a radix-16
// passes and, when b > 0, one last radix-2^b pass; between passes the elements
// go through shared memory once (index padded by one slot per 16, which keeps
// every pass's 16-byte stores and loads free of bank conflicts).  The last pass
// of a Stockham transform leaves each thread's results at the positions it
// read, so the product with H and the first pass of the inverse follow in
// registers, without a shared-memory exchange.  Twiddles exp(-2 pi i t / N)
// come from a plan table computed in FP64 and stored as broadcast pairs: a
// radix-16 pass loads w^k, w^2k, w^4k, w^8k and forms the other eleven powers
// with at most three complex products; the last pass loads w^t, w^2t, w^4t,
// forms the other powers the same way and the other butterflies' twiddles by
// constant rotations exp(-+2 pi i s m / 16).  Each pass's entries are loaded
// during the exchange before it (after the stores, before the barrier), so
// the load latency hides behind the exchange.  The 1/N of the inverse is
// folded into H.  One launch covers the row blocks of many slices with the same N (their
// plans may differ otherwise), so a batch fills the GPU instead of running
// slice after slice.
#include "fbp_internal.h"
#include "lambert.cuh"
#include "pairs.cuh"

#include <cstring>
#include <vector>

namespace fbp {
namespace {

// Two complex numbers, one per transform: .x of each pair is the first
// transform's, .y the second's.
struct C2 {
    float2 re, im;
};

__device__ __forceinline__ float2 padd(float2 a, float2 b) { return __fadd2_rn(a, b); }
// a - b with one rounding (b * -1 is exact)
__device__ __forceinline__ float2 psub(float2 a, float2 b)
{
    return __ffma2_rn(b, make_float2(-1.0f, -1.0f), a);
}
__device__ __forceinline__ float2 pmul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 pfma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 pneg(float2 a) { return pmul(a, make_float2(-1.0f, -1.0f)); }

__device__ __forceinline__ C2 cadd(const C2 &a, const C2 &b)
{
    return {padd(a.re, b.re), padd(a.im, b.im)};
}
__device__ __forceinline__ C2 csub(const C2 &a, const C2 &b)
{
    return {psub(a.re, b.re), psub(a.im, b.im)};
}

// A twiddle r + i s for both transforms, with n = -s kept beside it.
struct Tw {
    float2 r, s, n;
};

// a * w
__device__ __forceinline__ C2 cmul(const C2 &a, const Tw &w)
{
    return {pfma(a.im, w.n, pmul(a.re, w.r)), pfma(a.re, w.s, pmul(a.im, w.r))};
}

// a * b of two twiddles
__device__ __forceinline__ Tw tmul(const Tw &a, const Tw &b)
{
    Tw w;
    w.r = pfma(a.n, b.s, pmul(a.r, b.r));  // ar br - as bs
    w.s = pfma(a.s, b.r, pmul(a.r, b.s));  // ar bs + as br
    w.n = pfma(a.n, b.r, pmul(a.r, b.n));  // -(ar bs + as br)
    return w;
}

// A table entry through a volatile load, so it is issued where it is written.
__device__ __forceinline__ float4 tw_raw(const float4 *__restrict__ tw, int t)
{
    float4 v;
    asm volatile("ld.global.nc.v4.f32 {%0, %1, %2, %3}, [%4];"
                 : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
                 : "l"(tw + t));
    return v;
}

// Plan twiddle t, exp(-2 pi i t / N) (forward) or its conjugate (inverse),
// from its table entry (cos, cos, sin, sin).
template <bool INV>
__device__ __forceinline__ Tw tw_from_raw(const float4 &v)
{
    const float2 s = make_float2(v.z, v.w);
    const float2 n = pneg(s);
    Tw w;
    w.r = make_float2(v.x, v.y);
    w.s = INV ? n : s;
    w.n = INV ? s : n;
    return w;
}

// cos(pi e / 8) for e in [0, 16).
constexpr float kCosPi8[16] = {
    1.0f,  0.92387953251128674f,  0.70710678118654752f,  0.38268343236508977f,
    0.0f,  -0.38268343236508977f, -0.70710678118654752f, -0.92387953251128674f,
    -1.0f, -0.92387953251128674f, -0.70710678118654752f, -0.38268343236508977f,
    0.0f,  0.38268343236508977f,  0.70710678118654752f,  0.92387953251128674f};

// a times exp(-+ 2 pi i E / 16).
template <bool INV, int E>
__device__ __forceinline__ C2 twiddle16(const C2 &a)
{
    static_assert(E >= 0 && E < 16, "exponent in [0, 16)");
    if constexpr (E == 0) {
        return a;
    } else if constexpr (E == 4) {
        // times -i (forward) or +i (inverse)
        return INV ? C2{pneg(a.im), a.re} : C2{a.im, pneg(a.re)};
    } else {
        constexpr float c = kCosPi8[E], s = kCosPi8[(E + 12) % 16];  // sin(x) = cos(x - pi/2)
        const float2 C = make_float2(c, c), S = make_float2(s, s), NS = make_float2(-s, -s);
        // forward w = c - i s; inverse w = c + i s
        return INV ? C2{pfma(a.im, NS, pmul(a.re, C)), pfma(a.re, S, pmul(a.im, C))}
                   : C2{pfma(a.im, S, pmul(a.re, C)), pfma(a.re, NS, pmul(a.im, C))};
    }
}

template <bool INV>
__device__ __forceinline__ void dft2(C2 &a0, C2 &a1)
{
    const C2 b = csub(a0, a1);
    a0 = cadd(a0, a1);
    a1 = b;
}

// 4-point DFT, inputs and outputs in natural order.
template <bool INV>
__device__ __forceinline__ void dft4(C2 &a0, C2 &a1, C2 &a2, C2 &a3)
{
    const C2 b0 = cadd(a0, a2), b1 = csub(a0, a2), b2 = cadd(a1, a3), d = csub(a1, a3);
    a0 = cadd(b0, b2);
    a2 = csub(b0, b2);
    // forward: b1 - i d and b1 + i d; inverse: b1 + i d and b1 - i d
    if (INV) {
        a1 = {psub(b1.re, d.im), padd(b1.im, d.re)};
        a3 = {padd(b1.re, d.im), psub(b1.im, d.re)};
    } else {
        a1 = {padd(b1.re, d.im), psub(b1.im, d.re)};
        a3 = {psub(b1.re, d.im), padd(b1.im, d.re)};
    }
}

// 8-point DFT as 2 x 4: q = q1 + 2 q2, m = m2 + 4 m1.
template <bool INV>
__device__ __forceinline__ void dft8(C2 (&a)[8])
{
    dft4<INV>(a[0], a[2], a[4], a[6]);  // q1 = 0: A[0][m2] in a[2 m2]
    dft4<INV>(a[1], a[3], a[5], a[7]);  // q1 = 1: A[1][m2] in a[2 m2 + 1]
    a[3] = twiddle16<INV, 2>(a[3]);     // exp(-+ 2 pi i m2 / 8), m2 = 1..3
    a[5] = twiddle16<INV, 4>(a[5]);
    a[7] = twiddle16<INV, 6>(a[7]);
    C2 x[8];
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
__device__ __forceinline__ void dft16(C2 (&v)[16])
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
    C2 x[16];
#pragma unroll
    for (int m2 = 0; m2 < 4; ++m2)
#pragma unroll
        for (int m1 = 0; m1 < 4; ++m1) x[m2 + 4 * m1] = v[m1 + 4 * m2];
#pragma unroll
    for (int m = 0; m < 16; ++m) v[m] = x[m];
}

// 4-point DFT of (a0, a1, 0, 0): the first stage of a transform whose upper
// half of inputs is zero padding (the same values dft4 gives for those inputs).
template <bool INV>
__device__ __forceinline__ void dft4_z23(C2 &a0, C2 &a1, C2 &a2, C2 &a3)
{
    const C2 b = a0, d = a1;
    a0 = cadd(b, d);
    a2 = csub(b, d);
    if (INV) {
        a1 = {psub(b.re, d.im), padd(b.im, d.re)};
        a3 = {padd(b.re, d.im), psub(b.im, d.re)};
    } else {
        a1 = {padd(b.re, d.im), psub(b.im, d.re)};
        a3 = {psub(b.re, d.im), padd(b.im, d.re)};
    }
}

// 4-point DFT computing outputs 0 and 1 only (2 and 3 are not needed).
template <bool INV>
__device__ __forceinline__ void dft4_out01(C2 &a0, C2 &a1, const C2 &a2, const C2 &a3)
{
    const C2 b0 = cadd(a0, a2), b1 = csub(a0, a2), b2 = cadd(a1, a3), d = csub(a1, a3);
    a0 = cadd(b0, b2);
    a1 = INV ? C2{psub(b1.re, d.im), padd(b1.im, d.re)} : C2{padd(b1.re, d.im), psub(b1.im, d.re)};
}

// 16-point DFT (as dft16) with two prunings: ZHI, inputs 8..15 are zero;
// OLO, only outputs 0..7 are needed (8..15 are left unspecified).
template <bool INV, bool ZHI, bool OLO>
__device__ __forceinline__ void dft16p(C2 (&v)[16])
{
#pragma unroll
    for (int q1 = 0; q1 < 4; ++q1) {
        if constexpr (ZHI)
            dft4_z23<INV>(v[q1], v[q1 + 4], v[q1 + 8], v[q1 + 12]);
        else
            dft4<INV>(v[q1], v[q1 + 4], v[q1 + 8], v[q1 + 12]);
    }
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
    for (int m2 = 0; m2 < 4; ++m2) {
        if constexpr (OLO)
            dft4_out01<INV>(v[4 * m2], v[4 * m2 + 1], v[4 * m2 + 2], v[4 * m2 + 3]);
        else
            dft4<INV>(v[4 * m2], v[4 * m2 + 1], v[4 * m2 + 2], v[4 * m2 + 3]);
    }
    // X[m2 + 4 m1] sits in v[m1 + 4 m2]: transpose
    C2 x[16];
#pragma unroll
    for (int m2 = 0; m2 < 4; ++m2)
#pragma unroll
        for (int m1 = 0; m1 < (OLO ? 2 : 4); ++m1) x[m2 + 4 * m1] = v[m1 + 4 * m2];
#pragma unroll
    for (int m = 0; m < (OLO ? 8 : 16); ++m) v[m] = x[m];
}

// 8-point DFT computing outputs 0..3 only.
template <bool INV>
__device__ __forceinline__ void dft8_lo4(C2 (&a)[8])
{
    dft4<INV>(a[0], a[2], a[4], a[6]);
    dft4<INV>(a[1], a[3], a[5], a[7]);
    a[3] = twiddle16<INV, 2>(a[3]);
    a[5] = twiddle16<INV, 4>(a[5]);
    a[7] = twiddle16<INV, 6>(a[7]);
    C2 x[4];
#pragma unroll
    for (int m2 = 0; m2 < 4; ++m2) x[m2] = cadd(a[2 * m2], a[2 * m2 + 1]);
#pragma unroll
    for (int m = 0; m < 4; ++m) a[m] = x[m];
}

// Last pass of radix R: element m + S (16/R) (butterfly j = t + m T) times
// w^{S j} = w^{S t} exp(-+ 2 pi i S m / 16), from the one twiddle w^{S t}.
template <bool INV, int R, int S, int M>
__device__ __forceinline__ void last_scale(C2 (&v)[16], const Tw &w)
{
    constexpr int idx = M + S * (16 / R);
    v[idx] = twiddle16<INV, (S * M) % 16>(cmul(v[idx], w));
    if constexpr (M + 1 < 16 / R) last_scale<INV, R, S, M + 1>(v, w);
}

__device__ __forceinline__ int pad16(int i) { return i + (i >> 4); }

__device__ __forceinline__ void put(float4 *buf, int i, const C2 &a)
{
    buf[pad16(i)] = make_float4(a.re.x, a.re.y, a.im.x, a.im.y);
}
__device__ __forceinline__ C2 get(const float4 *buf, int i)
{
    const float4 f = buf[pad16(i)];
    return {make_float2(f.x, f.y), make_float2(f.z, f.w)};
}

// Full N-point transform (N = 2^L, T = N/16 threads) of the elements the
// block holds (thread t: positions t + q T in v[q]); on return v[q] holds
// output position t + q T.  Compile-time N: every shared-memory and table
// index below is a per-thread base plus a constant.  Prunings (values equal
// to the unpruned transform's): FIRST_HALF_ZERO, inputs q >= 8 are zero (a
// row zero-padded to N >= 2 n_det - 1 has n_det <= N/2); LAST_LO8, only
// outputs q < 8 are needed (the bins 0..n_det-1 of the inverse).
template <bool INV, int L, bool FIRST_HALF_ZERO, bool LAST_LO8>
__device__ __forceinline__ void fft_regs(C2 (&v)[16], float4 *buf, const float4 *__restrict__ tw)
{
    constexpr int N = 1 << L;
    constexpr int T = N >> 4;
    constexpr int NP = L >> 2;   // radix-16 passes
    constexpr int REM = L & 3;   // bits of the last pass (radix 2^REM), 0: none
    const int t = threadIdx.x;
    int np = NP;
    asm volatile("" : "+r"(np));
    // the next pass's table entries, loaded during the exchange before it
    // (after the stores, before the barrier: the data registers are free)
    float4 x1, x2, x4, x8;
    auto preload = [&](int pn) {
        if (pn < np) {
            const int log2ns = 4 * pn;
            const int k = t & ((1 << log2ns) - 1);
            const int i1 = k << (L - 4 - log2ns);  // k N / (16 ns)
            x1 = tw_raw(tw, i1);
            x2 = tw_raw(tw, 2 * i1);
            x4 = tw_raw(tw, 4 * i1);
            x8 = tw_raw(tw, 8 * i1);
        } else {
            // last pass: w^{t}, w^{2t}, w^{4t} (the other butterflies' and
            // powers' twiddles follow from these)
            if constexpr (REM >= 1) x1 = tw_raw(tw, t);
            if constexpr (REM >= 2) x2 = tw_raw(tw, 2 * t);
            if constexpr (REM == 3) x4 = tw_raw(tw, 4 * t);
        }
    };
    // the exchange after a radix-16 pass: write positions o + m ns from wb with
    // stride ws (padded), read t + q T
    auto exchange = [&](int wb, int ws, int pn) {
#pragma unroll
        for (int m = 0; m < 16; ++m) {
            const C2 &a = v[m];
            buf[wb + m * ws] = make_float4(a.re.x, a.re.y, a.im.x, a.im.y);
        }
        preload(pn);
        __syncthreads();
        if constexpr (T >= 16) {
            const int rb = t + (t >> 4);
#pragma unroll
            for (int q = 0; q < 16; ++q) {
                const float4 f = buf[rb + q * (T + T / 16)];
                v[q] = {make_float2(f.x, f.y), make_float2(f.z, f.w)};
            }
        } else {
#pragma unroll
            for (int q = 0; q < 16; ++q) v[q] = get(buf, t + q * T);
        }
        __syncthreads();
    };
    // pass 0 (ns = 1): no twiddles; outputs o + m, o = 16 t: padded 17 t + m
    constexpr bool LAST0 = REM == 0 && NP == 1;
    if constexpr (FIRST_HALF_ZERO && LAST0 && LAST_LO8) dft16p<INV, true, true>(v);
    else if constexpr (FIRST_HALF_ZERO) dft16p<INV, true, false>(v);
    else if constexpr (LAST0 && LAST_LO8) dft16p<INV, false, true>(v);
    else dft16<INV>(v);
    if constexpr (!LAST0) exchange(17 * t, 1, 1);
    // passes 1 .. NP-1 (ns = 16^p), kept as a loop whose trip count the
    // compiler cannot see: straight-line (one middle pass, N = 2^9 .. 2^11), its
    // schedule overlaps the passes and spills registers
#pragma unroll 1
    for (int p = 1; p < np; ++p) {
        const int log2ns = 4 * p;
        const int ns = 1 << log2ns;
        const bool last = REM == 0 && p == NP - 1;
        const int k = t & (ns - 1);
        const Tw w1 = tw_from_raw<INV>(x1), w2 = tw_from_raw<INV>(x2);
        const Tw w4 = tw_from_raw<INV>(x4), w8 = tw_from_raw<INV>(x8);
        const Tw w3 = tmul(w1, w2);
        v[1] = cmul(v[1], w1);
        v[2] = cmul(v[2], w2);
        v[3] = cmul(v[3], w3);
        v[4] = cmul(v[4], w4);
        v[5] = cmul(v[5], tmul(w4, w1));
        v[6] = cmul(v[6], tmul(w4, w2));
        v[7] = cmul(v[7], tmul(w4, w3));
        v[8] = cmul(v[8], w8);
        v[9] = cmul(v[9], tmul(w8, w1));
        v[10] = cmul(v[10], tmul(w8, w2));
        v[11] = cmul(v[11], tmul(w8, w3));
        const Tw w12 = tmul(w8, w4);
        v[12] = cmul(v[12], w12);
        v[13] = cmul(v[13], tmul(w12, w1));
        v[14] = cmul(v[14], tmul(w12, w2));
        v[15] = cmul(v[15], tmul(w12, w3));
        if (LAST_LO8 && last) {
            dft16p<INV, false, true>(v);
        } else {
            dft16<INV>(v);
        }
        if (!last) {
            // outputs o + m ns, o = 16 (t - k) + k; padded pad16(o) + m (ns + ns/16)
            const int o = ((t - k) << 4) + k;
            exchange(pad16(o), ns + (ns >> 4), p + 1);
        }
    }
    if constexpr (REM == 0) return;
    // last pass, radix R = 2^REM, ns = N / R: butterfly j = t + m T (m < 16/R)
    // takes positions j + s N/R = t + (m + s 16/R) T, twiddles exp(-+ 2 pi i s j / N);
    // with LAST_LO8 only the outputs at q = m + s 16/R < 8 are formed
    if constexpr (REM == 3) {
        {
            const Tw w1 = tw_from_raw<INV>(x1), w2 = tw_from_raw<INV>(x2);
            const Tw w4 = tw_from_raw<INV>(x4);
            last_scale<INV, 8, 1, 0>(v, w1);
            last_scale<INV, 8, 2, 0>(v, w2);
            last_scale<INV, 8, 4, 0>(v, w4);
            last_scale<INV, 8, 5, 0>(v, tmul(w4, w1));
            last_scale<INV, 8, 6, 0>(v, tmul(w4, w2));
            const Tw w3 = tmul(w1, w2);
            last_scale<INV, 8, 3, 0>(v, w3);
            last_scale<INV, 8, 7, 0>(v, tmul(w4, w3));
        }
#pragma unroll
        for (int m = 0; m < 2; ++m) {
            C2 a[8];
#pragma unroll
            for (int s = 0; s < 8; ++s) a[s] = v[m + 2 * s];
            if constexpr (LAST_LO8) {
                dft8_lo4<INV>(a);
#pragma unroll
                for (int s = 0; s < 4; ++s) v[m + 2 * s] = a[s];
            } else {
                dft8<INV>(a);
#pragma unroll
                for (int s = 0; s < 8; ++s) v[m + 2 * s] = a[s];
            }
        }
    } else if constexpr (REM == 2) {
        {
            const Tw w1 = tw_from_raw<INV>(x1), w2 = tw_from_raw<INV>(x2);
            last_scale<INV, 4, 1, 0>(v, w1);
            last_scale<INV, 4, 2, 0>(v, w2);
            last_scale<INV, 4, 3, 0>(v, tmul(w1, w2));
        }
#pragma unroll
        for (int m = 0; m < 4; ++m) {
            C2 a1 = v[m + 4], a2 = v[m + 8], a3 = v[m + 12];
            if constexpr (LAST_LO8) {
                dft4_out01<INV>(v[m], a1, a2, a3);
                v[m + 4] = a1;
            } else {
                dft4<INV>(v[m], a1, a2, a3);
                v[m + 4] = a1;
                v[m + 8] = a2;
                v[m + 12] = a3;
            }
        }
    } else {
        last_scale<INV, 2, 1, 0>(v, tw_from_raw<INV>(x1));
#pragma unroll
        for (int m = 0; m < 8; ++m) {
            if constexpr (LAST_LO8) {
                v[m] = cadd(v[m], v[m + 8]);
            } else {
                C2 a1 = v[m + 8];
                dft2<INV>(v[m], a1);
                v[m + 8] = a1;
            }
        }
    }
}

// One slice's part of a launch; block_end is the inclusive prefix sum of the
// slices' four-row block counts, so CTA b works on the slice s with
// block_end[s-1] <= b < block_end[s].  All slices of a launch share N.
struct FftSlice {
    const float *sino;
    void *q;
    const float4 *tw;
    const float2 *h;
    int ld;
    int pitch;
    int A;
    int D;
    int block_end;
    float i0;  // > 0: intensity input, converted on load (lambert.cuh)
    float ln_i0;
    int wt_rows;       // > 0: row r's values are multiplied by wt[(r mod wt_rows)][j] on load
    const float *wt;
};

template <int MAXS>
struct FftLaunch {
    FftSlice s[MAXS];
    int n;
    int N;
    int log2n;
};

// Blocks per SM the register budget is sized for: 128 registers a thread.
constexpr int fft_min_blocks(int L)
{
    return ((1 << L) / 16) >= 32 ? 512 / ((1 << L) / 16) : 16;
}

template <typename OutT, int MAXS, int L>
__global__ void __launch_bounds__((1 << L) / 16, fft_min_blocks(L))
    filter_fft_kernel(const __grid_constant__ FftLaunch<MAXS> P)
{
    constexpr int N = 1 << L;
    constexpr int T = N / 16;
    extern __shared__ float4 buf[];
    int lo = 0, hi = P.n - 1;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if ((int)blockIdx.x < P.s[mid].block_end) hi = mid; else lo = mid + 1;
    }
    const FftSlice &S = P.s[lo];
    const int blk = (int)blockIdx.x - (lo > 0 ? P.s[lo - 1].block_end : 0);
    const int D = S.D, t = threadIdx.x;
    const int i0 = 4 * blk;
    const int rows = min(4, S.A - i0);  // 1..4 rows in this block
    // rows i0, i0+1 -> transform 0 (re, im); rows i0+2, i0+3 -> transform 1;
    // a row past the slice is never read
    const float *p0 = S.sino + (size_t)i0 * S.ld;
    const float *p1 = p0 + (rows > 1 ? S.ld : 0);
    const float *p2 = p0 + (rows > 2 ? 2 * (size_t)S.ld : 0);
    const float *p3 = p0 + (rows > 3 ? 3 * (size_t)S.ld : 0);
    // n_det <= N/2: positions t + q T with q >= 8 are zero padding
    C2 v[16];
#pragma unroll
    for (int q = 0; q < 16; ++q) {
        const int j = t + q * T;
        v[q].re = make_float2(0.0f, 0.0f);
        v[q].im = make_float2(0.0f, 0.0f);
        if (q < 8 && j < D) {
            v[q].re.x = p0[j];
            if (rows > 1) v[q].im.x = p1[j];
            if (rows > 2) v[q].re.y = p2[j];
            if (rows > 3) v[q].im.y = p3[j];
        }
    }
    if (S.i0 > 0.0f) {
        // intensities: convert after all loads are in flight (the padding stays zero)
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            if (t + q * T < D) {
                v[q].re.x = line_integral(v[q].re.x, S.i0, S.ln_i0);
                if (rows > 1) v[q].im.x = line_integral(v[q].im.x, S.i0, S.ln_i0);
                if (rows > 2) v[q].re.y = line_integral(v[q].re.y, S.i0, S.ln_i0);
                if (rows > 3) v[q].im.y = line_integral(v[q].im.y, S.i0, S.ln_i0);
            }
        }
    }
    if (S.wt != nullptr) {
        // per-element weights of the row (a cone-beam cosine weight), applied to the
        // line integrals
        const float *w0 = S.wt + (size_t)(i0 % S.wt_rows) * D;
        const float *w1 = S.wt + (size_t)((i0 + 1) % S.wt_rows) * D;
        const float *w2 = S.wt + (size_t)((i0 + 2) % S.wt_rows) * D;
        const float *w3 = S.wt + (size_t)((i0 + 3) % S.wt_rows) * D;
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const int j = t + q * T;
            if (j < D) {
                v[q].re.x *= __ldg(&w0[j]);
                v[q].im.x *= __ldg(&w1[j]);
                v[q].re.y *= __ldg(&w2[j]);
                v[q].im.y *= __ldg(&w3[j]);
            }
        }
    }
    fft_regs<false, L, true, false>(v, buf, S.tw);
#pragma unroll
    for (int q = 0; q < 16; ++q) {
        const float2 hv = __ldg(&S.h[t + q * T]);
        v[q].re = pmul(v[q].re, hv);
        v[q].im = pmul(v[q].im, hv);
    }
    fft_regs<true, L, false, true>(v, buf, S.tw);
    // v[q], q < 8, holds Q of the four rows at bin t + q T (bins past n_det are
    // not zero: they are cleared below).  Every thread is past its last read of
    // buf (the final pass of the inverse reads none; the one before ends with
    // a barrier): publish the values so each thread can read its left
    // neighbour's.  Layout (row 0, row 2, row 1, row 3).
#pragma unroll
    for (int q = 0; q < 8; ++q) put(buf, t + q * T, v[q]);
    __syncthreads();
    // the pair at p = t + q T is (Q[p-1], Q[p]) -> (mid, slope), Q zero outside
    // [0, n_det); p runs to pitch/2 - 1 <= n_det + 3 (<= N/2 + 3)
    OutT *r0 = static_cast<OutT *>(S.q) + (size_t)i0 * S.pitch;
    const int P2 = S.pitch / 2;
#pragma unroll
    for (int q = 0; q < 16; ++q) {
        if (q * T >= P2) break;
        const int p = t + q * T;
        if (p < P2) {
            float4 a = make_float4(0.0f, 0.0f, 0.0f, 0.0f), b = a;
            if (q < 8 && p < D) b = make_float4(v[q].re.x, v[q].re.y, v[q].im.x, v[q].im.y);
            if (p >= 1 && p - 1 < D) a = buf[pad16(p - 1)];
            store_pair(r0, p, a.x, b.x);
            if (rows > 1) store_pair(r0 + S.pitch, p, a.z, b.z);
            if (rows > 2) store_pair(r0 + 2 * (size_t)S.pitch, p, a.y, b.y);
            if (rows > 3) store_pair(r0 + 3 * (size_t)S.pitch, p, a.w, b.w);
        }
    }
}

int log2_of(int N)
{
    int l = 0;
    while ((1 << l) < N) ++l;
    return l;
}

template <typename OutT, int MAXS, int L>
cudaError_t launch_one_len(const FftLaunch<MAXS> &P, int total, cudaStream_t s, bool prepare)
{
    const size_t smem = filter_fft_smem_bytes(1 << L);
    cudaError_t e = cudaFuncSetAttribute(filter_fft_kernel<OutT, MAXS, L>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess || prepare) return e;
    filter_fft_kernel<OutT, MAXS, L><<<total, (1 << L) / 16, smem, s>>>(P);
    return cudaGetLastError();
}

// N = 16 .. 8192 (the plan keeps N within kMaxFftLen)
template <typename OutT, int MAXS>
cudaError_t launch_set(FftLaunch<MAXS> &P, int total, int N, cudaStream_t s, bool prepare = false)
{
    P.N = N;
    P.log2n = log2_of(N);
    switch (P.log2n) {
    case 4: return launch_one_len<OutT, MAXS, 4>(P, total, s, prepare);
    case 5: return launch_one_len<OutT, MAXS, 5>(P, total, s, prepare);
    case 6: return launch_one_len<OutT, MAXS, 6>(P, total, s, prepare);
    case 7: return launch_one_len<OutT, MAXS, 7>(P, total, s, prepare);
    case 8: return launch_one_len<OutT, MAXS, 8>(P, total, s, prepare);
    case 9: return launch_one_len<OutT, MAXS, 9>(P, total, s, prepare);
    case 10: return launch_one_len<OutT, MAXS, 10>(P, total, s, prepare);
    case 11: return launch_one_len<OutT, MAXS, 11>(P, total, s, prepare);
    case 12: return launch_one_len<OutT, MAXS, 12>(P, total, s, prepare);
    case 13: return launch_one_len<OutT, MAXS, 13>(P, total, s, prepare);
    default: return cudaErrorInvalidValue;
    }
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
    f.block_end = 0;
    f.i0 = p.i0f;
    f.ln_i0 = p.ln_i0f;
    f.wt = p.d_row_weight;
    f.wt_rows = p.row_weight_rows;
    return f;
}

}  // namespace

size_t filter_fft_smem_bytes(int N) { return sizeof(float4) * (size_t)(N + N / 16); }

cudaError_t launch_filter_fft(const Plan &p, const float *sino, int ld, void *q, cudaStream_t s)
{
    FftLaunch<1> L;
    L.s[0] = fft_slice(p, sino, ld, q);
    L.s[0].block_end = (p.A + 3) / 4;
    L.n = 1;
    if (p.q_storage == FBP_F16) return launch_set<__half, 1>(L, L.s[0].block_end, p.fft_len, s);
    return launch_set<float, 1>(L, L.s[0].block_end, p.fft_len, s);
}

cudaError_t prepare_filter_fft(const Plan &p)
{
    FftLaunch<1> L;
    std::memset(&L, 0, sizeof L);
    if (p.q_storage == FBP_F16) return launch_set<__half, 1>(L, 0, p.fft_len, nullptr, true);
    return launch_set<float, 1>(L, 0, p.fft_len, nullptr, true);
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
                total += (p.A + 3) / 4;
                L.s[cnt].block_end = total;
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
