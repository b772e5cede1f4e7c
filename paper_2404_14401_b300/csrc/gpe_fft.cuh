// gpe_fft.cuh -- register/shared-memory Stockham FFT for one pencil (a row or
// a column of the grid) per group of threads, for sm_103a.
//
// The split-step of Sec. 3.1 (Eqs. 3-4) needs F and F^-1 along x and y.  A
// pencil of N = 2^n complex64 points is spread over TP = N/E threads, thread
// j holding elements j + r*TP (r < E) in registers -- the natural order that
// both the first and the last Stockham stage read and write, so a pencil can
// be loaded from global memory, transformed, multiplied by a phase and
// transformed back without leaving registers at the ends.  Stages are
// radix-R Stockham steps (R = 2^(n mod 4, or 4) for the first, 16 after),
// each thread doing E/R butterflies per stage; between stages the pencil is
// exchanged through shared memory in a layout padded by one slot per 16
// elements, which keeps 64-bit accesses of every stage free of bank
// conflicts.  Twiddles come from a per-stage table (consecutive lanes read
// consecutive entries) computed in double precision and stored as two-float
// (hi + lo) pairs.
#pragma once

#include <cuda_runtime.h>

namespace gpe {

__host__ __device__ constexpr int ilog2(int n) { return n <= 1 ? 0 : 1 + ilog2(n / 2); }

__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b)
{
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// multiply by -i (forward transform) or +i (inverse)
template <bool INV> __device__ __forceinline__ float2 mul_mi(float2 a)
{
    return INV ? make_float2(-a.y, a.x) : make_float2(a.y, -a.x);
}

// cos(2 pi j / 16) split as hi + lo (two floats, |hi + lo - cos| < 1e-15).
// Twiddles whose stored modulus differs from 1 by a rounding error of one
// float would scale every transformed value the same way each step and make
// the real-time norm drift; with the pair the modulus is 1 to 1e-15 and the
// remaining roundings are unbiased.
__host__ __device__ constexpr float cos16_hi(int j)
{
    constexpr float C1 = 0x1.d906bcp-1f, C2 = 0x1.6a09e6p-1f, C3 = 0x1.87de2ap-2f;
    switch (j & 15) {
    case 0: return 1.f;  case 1: return C1;  case 2: return C2;  case 3: return C3;
    case 4: return 0.f;  case 5: return -C3; case 6: return -C2; case 7: return -C1;
    case 8: return -1.f; case 9: return -C1; case 10: return -C2; case 11: return -C3;
    case 12: return 0.f; case 13: return C3; case 14: return C2; default: return C1;
    }
}
__host__ __device__ constexpr float cos16_lo(int j)
{
    constexpr float L1 = 0x1.e651a8p-26f, L2 = 0x1.9fcef4p-27f, L3 = 0x1.abaa58p-28f;
    switch (j & 15) {
    case 1: return L1;   case 2: return L2;   case 3: return L3;
    case 5: return -L3;  case 6: return -L2;  case 7: return -L1;
    case 9: return -L1;  case 10: return -L2; case 11: return -L3;
    case 13: return L3;  case 14: return L2;  case 15: return L1;
    default: return 0.f;
    }
}
__host__ __device__ constexpr float sin16_hi(int j) { return cos16_hi(j - 4); }
__host__ __device__ constexpr float sin16_lo(int j) { return cos16_lo(j - 4); }

// a * (w.x + w.z + i (w.y + w.w)): complex product with a two-float twiddle
__device__ __forceinline__ float2 cmul_df(float2 a, float4 w)
{
    const float re_lo = fmaf(-a.y, w.w, a.x * w.z);
    const float im_lo = fmaf(a.y, w.z, a.x * w.w);
    return make_float2(fmaf(a.x, w.x, fmaf(-a.y, w.y, re_lo)), fmaf(a.x, w.y, fmaf(a.y, w.x, im_lo)));
}

// a * W16^J with W16 = exp(-2 pi i/16) (forward) or its conjugate (inverse)
template <int J, bool INV> __device__ __forceinline__ float2 tw16(float2 a)
{
    constexpr int j = J & 15;
    if constexpr (j == 0) return a;
    else if constexpr (j == 4) return mul_mi<INV>(a);
    else if constexpr (j == 8) return make_float2(-a.x, -a.y);
    else if constexpr (j == 12) return mul_mi<!INV>(a);
    else if constexpr ((j & 3) == 2) {
        // (+-1 +- i) sqrt(1/2): exact sign combination, then one scaling by the pair
        constexpr float sr = cos16_hi(j) > 0.f ? 1.f : -1.f;
        constexpr float si = (INV ? sin16_hi(j) : -sin16_hi(j)) > 0.f ? 1.f : -1.f;
        constexpr float h = cos16_hi(2), l = cos16_lo(2);
        const float u = sr * a.x - si * a.y, v = si * a.x + sr * a.y;
        return make_float2(fmaf(u, h, u * l), fmaf(v, h, v * l));
    } else {
        constexpr float wr = cos16_hi(j), wi = INV ? sin16_hi(j) : -sin16_hi(j);
        constexpr float lr = cos16_lo(j), li = INV ? sin16_lo(j) : -sin16_lo(j);
        return cmul_df(a, make_float4(wr, wi, lr, li));
    }
}

// packed two-lane float add / subtract (one f32x2 instruction for a complex add)
__device__ __forceinline__ float2 add2(float2 a, float2 b)
{
    float2 r;
    asm("{.reg .b64 ra, rb, rd;\n\t"
        "mov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\t"
        "add.rn.f32x2 rd, ra, rb;\n\tmov.b64 {%0, %1}, rd;}"
        : "=f"(r.x), "=f"(r.y)
        : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return r;
}
__device__ __forceinline__ float2 sub2(float2 a, float2 b)
{
    float2 r;
    asm("{.reg .b64 ra, rb, rd;\n\t"
        "mov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\t"
        "sub.rn.f32x2 rd, ra, rb;\n\tmov.b64 {%0, %1}, rd;}"
        : "=f"(r.x), "=f"(r.y)
        : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return r;
}

template <bool INV> __device__ __forceinline__ void dft2(float2 &a0, float2 &a1)
{
    const float2 t = a0;
    a0 = add2(t, a1);
    a1 = sub2(t, a1);
}

template <bool INV> __device__ __forceinline__ void dft4(float2 &a0, float2 &a1, float2 &a2, float2 &a3)
{
    const float2 t0 = add2(a0, a2), t1 = sub2(a0, a2), t2 = add2(a1, a3);
    const float2 t3 = mul_mi<INV>(sub2(a1, a3));
    a0 = add2(t0, t2);
    a2 = sub2(t0, t2);
    a1 = cadd(t1, t3);
    a3 = csub(t1, t3);
}

// 8-point DFT as 4 x 2: n = 2 n1 + n2, k = k1 + 4 k2
template <bool INV> __device__ __forceinline__ void dft8(float2 (&a)[8])
{
    dft4<INV>(a[0], a[2], a[4], a[6]);
    dft4<INV>(a[1], a[3], a[5], a[7]);
    a[3] = tw16<2, INV>(a[3]);
    a[5] = tw16<4, INV>(a[5]);
    a[7] = tw16<6, INV>(a[7]);
    const float2 y0[4] = {a[0], a[2], a[4], a[6]};
    const float2 y1[4] = {a[1], a[3], a[5], a[7]};
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        a[k] = add2(y0[k], y1[k]);
        a[k + 4] = sub2(y0[k], y1[k]);
    }
}

// 16-point DFT as 4 x 4: n = 4 n1 + n2, k = k1 + 4 k2
template <bool INV> __device__ __forceinline__ void dft16(float2 (&a)[16])
{
#pragma unroll
    for (int n2 = 0; n2 < 4; ++n2) dft4<INV>(a[n2], a[n2 + 4], a[n2 + 8], a[n2 + 12]);
    a[5] = tw16<1, INV>(a[5]);
    a[6] = tw16<2, INV>(a[6]);
    a[7] = tw16<3, INV>(a[7]);
    a[9] = tw16<2, INV>(a[9]);
    a[10] = tw16<4, INV>(a[10]);
    a[11] = tw16<6, INV>(a[11]);
    a[13] = tw16<3, INV>(a[13]);
    a[14] = tw16<6, INV>(a[14]);
    a[15] = tw16<9, INV>(a[15]);
#pragma unroll
    for (int k1 = 0; k1 < 4; ++k1) dft4<INV>(a[4 * k1], a[4 * k1 + 1], a[4 * k1 + 2], a[4 * k1 + 3]);
    float2 t[16];
#pragma unroll
    for (int k1 = 0; k1 < 4; ++k1)
#pragma unroll
        for (int k2 = 0; k2 < 4; ++k2) t[k1 + 4 * k2] = a[4 * k1 + k2];
#pragma unroll
    for (int i = 0; i < 16; ++i) a[i] = t[i];
}

template <int R, bool INV> __device__ __forceinline__ void dft(float2 (&a)[R])
{
    if constexpr (R == 2) dft2<INV>(a[0], a[1]);
    else if constexpr (R == 4) dft4<INV>(a[0], a[1], a[2], a[3]);
    else if constexpr (R == 8) dft8<INV>(a);
    else dft16<INV>(a);
}

// padded shared-memory slot of pencil element e: one spare slot per 16
__device__ __forceinline__ int padx(int e) { return e + (e >> 4); }

// Radix schedule of an N-point transform: stage 0 has radix 2^(n mod 4) (16
// when n is a multiple of 4), the others 16; NS = points combined before a stage.
__host__ __device__ constexpr int fft_stages(int n) { return (ilog2(n) + 3) / 4; }
__host__ __device__ constexpr int fft_radix(int n, int s)
{
    return s == 0 ? (1 << (ilog2(n) - 4 * (fft_stages(n) - 1))) : 16;
}
__host__ __device__ constexpr int fft_ns(int n, int s) { return s == 0 ? 1 : fft_ns(n, s - 1) * fft_radix(n, s - 1); }
// Twiddle table layout: stage s >= 1 owns (R - 1) NS consecutive entries,
// entry (r - 1) NS + k = W_{NS R}^{r k}, so the lanes of a warp (consecutive k)
// read consecutive entries.  Offset of stage s; the total is below n.
__host__ __device__ constexpr int fft_tw_offset(int n, int s)
{
    return s <= 1 ? 0 : fft_tw_offset(n, s - 1) + (fft_radix(n, s - 1) - 1) * fft_ns(n, s - 1);
}
// entries of the whole table
__host__ __device__ constexpr int fft_tw_count(int n) { return fft_tw_offset(n, fft_stages(n)); }

// The same schedule and table layout for a main radix of 2^LR: LR = 4 is the
// schedule above; LR = 3 (radix-8 stages after a first stage of radix
// 2^(n mod 3)) serves transforms with 8 elements per thread, twice the
// threads per pencil and half the serial work of each.
template <int LR> __host__ __device__ constexpr int fftg_stages(int n) { return (ilog2(n) + LR - 1) / LR; }
template <int LR> __host__ __device__ constexpr int fftg_radix(int n, int s)
{
    return s == 0 ? (1 << (ilog2(n) - LR * (fftg_stages<LR>(n) - 1))) : (1 << LR);
}
template <int LR> __host__ __device__ constexpr int fftg_ns(int n, int s)
{
    return s == 0 ? 1 : fftg_ns<LR>(n, s - 1) * fftg_radix<LR>(n, s - 1);
}
template <int LR> __host__ __device__ constexpr int fftg_tw_offset(int n, int s)
{
    return s <= 1 ? 0 : fftg_tw_offset<LR>(n, s - 1) + (fftg_radix<LR>(n, s - 1) - 1) * fftg_ns<LR>(n, s - 1);
}
template <int LR> __host__ __device__ constexpr int fftg_tw_count(int n)
{
    return fftg_tw_offset<LR>(n, fftg_stages<LR>(n));
}
static_assert(fftg_tw_count<4>(2048) == fft_tw_count(2048) && fftg_radix<4>(512, 0) == fft_radix(512, 0),
              "the radix-16 instance is the schedule above");

// One Stockham stage of radix R after NS points have been combined.
// Butterfly jp takes x[jp + r N/R], multiplies input r by W_{NS R}^{r (jp mod NS)}
// and writes output p to y[(jp / NS) NS R + jp mod NS + p NS].
// sb: this pencil's shared buffer, es: element stride in float2 units,
// tws: this stage's twiddle block (shared or read-only global memory).
template <int N, int E, int R, int NS, bool INV, bool LAST, class Sync>
__device__ __forceinline__ void fft_stage(float2 (&v)[E], float2 *__restrict__ sb, int j, int es,
                                          const float4 *__restrict__ tws, const Sync &sync)
{
    constexpr int TP = N / E, B = E / R;
#pragma unroll
    for (int q = 0; q < B; ++q) {
        const int jp = j + q * TP;
        const int k = jp & (NS - 1);
        float2 a[R];
#pragma unroll
        for (int r = 0; r < R; ++r) a[r] = v[q + B * r];
        if constexpr (NS > 1) {
#pragma unroll
            for (int r = 1; r < R; ++r) {
                float4 w = tws[(r - 1) * NS + k];
                if constexpr (INV) {
                    w.y = -w.y;
                    w.w = -w.w;
                }
                a[r] = cmul_df(a[r], w);
            }
        }
        dft<R, INV>(a);
        if constexpr (LAST) {
#pragma unroll
            for (int p = 0; p < R; ++p) v[q + B * p] = a[p];
        } else {
            const int base = (jp - k) * R + k;
#pragma unroll
            for (int p = 0; p < R; ++p) sb[padx(base + p * NS) * es] = a[p];
        }
    }
    if constexpr (!LAST) {
        sync();
#pragma unroll
        for (int r = 0; r < E; ++r) v[r] = sb[padx(j + r * TP) * es];
        sync();
    }
}

// Barrier between the scatter and the gather of an exchange: the whole CTA
// (the default) or one named barrier of a group of warps that owns its
// pencil buffers (id >= 1; n threads, a multiple of 32).
struct CtaSync {
    __device__ __forceinline__ void operator()() const { __syncthreads(); }
};
struct GroupSync {
    int id, n;
    __device__ __forceinline__ void operator()() const
    {
        asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(n) : "memory");
    }
};

// Full transform of one pencil: natural order in v (element j + r TP) in and
// out.  Forward: X_k = sum_n x_n e^{-2 pi i nk/N}; INV: the conjugate sum,
// without the 1/N factor.  Every thread that `sync` covers must call it
// together.  tw: the per-stage twiddle table of this axis (fft_tw_offset layout).
template <int N, int E, bool INV, int S = 0, class Sync = CtaSync>
__device__ __forceinline__ void fft_pencil(float2 (&v)[E], float2 *__restrict__ sb, int j, int es,
                                           const float4 *__restrict__ tw, const Sync &sync = Sync())
{
    constexpr int R = fft_radix(N, S), NS = fft_ns(N, S);
    constexpr bool LAST = (S == fft_stages(N) - 1);
    static_assert(E % R == 0, "radix must divide the elements per thread");
    fft_stage<N, E, R, NS, INV, LAST>(v, sb, j, es, tw + fft_tw_offset(N, S), sync);
    if constexpr (!LAST) fft_pencil<N, E, INV, S + 1>(v, sb, j, es, tw, sync);
}

}  // namespace gpe
