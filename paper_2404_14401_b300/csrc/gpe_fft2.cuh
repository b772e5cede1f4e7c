// gpe_fft2.cuh -- Stockham FFT of a pair of pencils in packed f32x2 registers,
// for sm_103a.
//
// Two pencils that undergo identical arithmetic (the two columns of a column
// tile, or two rows of the same grid) are transformed together: every value
// is a packed pair whose lane 0 belongs to pencil A and lane 1 to pencil B,
// and a complex element is two such pairs, X = (re_A, re_B) and
// Y = (im_A, im_B).  Each butterfly add, constant multiply and twiddle
// multiply is then one f32x2 instruction (add/sub/mul/fma.rn.f32x2) for both
// pencils, where the one-pencil transform of gpe_fft.cuh issues one scalar
// instruction per pencil for every multiply and for the additions that
// multiplication by -i turns into mixed-component adds.  Multiplication by
// +-i is a renaming of X and Y with the sign folded into the following add
// or subtract.  Each rounding is the one the scalar transform makes for the
// same operation, lane by lane.
//
// Layout: a pencil pair of N points is spread over TP = N/16 threads, 16
// elements of each pencil per thread in natural order (element j + r TP),
// in the stages of the one-pencil transform (radix 2^(n mod 4) first, 16
// after) and with its twiddle table: 32 complex values (64 registers) per
// thread.  Between stages the pair is exchanged through shared memory as
// 16-byte slots {re_A, re_B, im_A, im_B}, padded by one slot per 8, which
// keeps every stage's 128-bit accesses free of bank conflicts.  One
// twiddle entry, loaded once, serves both pencils.
#pragma once

#include "gpe_fft.cuh"

namespace gpe {

// ---------------------------------------------------------------- packed ops
__device__ __forceinline__ float2 mul2(float2 a, float2 b)
{
    float2 r;
    asm("{.reg .b64 ra, rb, rd;\n\t"
        "mov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\t"
        "mul.rn.f32x2 rd, ra, rb;\n\tmov.b64 {%0, %1}, rd;}"
        : "=f"(r.x), "=f"(r.y)
        : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return r;
}
// a * b + c, one rounding per lane
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c)
{
    float2 r;
    asm("{.reg .b64 ra, rb, rc, rd;\n\t"
        "mov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\tmov.b64 rc, {%6, %7};\n\t"
        "fma.rn.f32x2 rd, ra, rb, rc;\n\tmov.b64 {%0, %1}, rd;}"
        : "=f"(r.x), "=f"(r.y)
        : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y), "f"(c.x), "f"(c.y));
    return r;
}
__device__ __forceinline__ float2 bc2(float v) { return make_float2(v, v); }

// padded 16-byte slot of element e: one spare slot per 8
__device__ __forceinline__ int pad8(int e) { return e + (e >> 3); }
__host__ __device__ constexpr int pad8_len(int n) { return n + n / 8; }

// ---------------------------------------------------------------- butterflies
// (X, Y) *= hi + lo for a real two-float constant (both lanes)
__device__ __forceinline__ void scale_df(float2 &x, float2 &y, float h, float l)
{
    x = fma2(x, bc2(h), mul2(x, bc2(l)));
    y = fma2(y, bc2(h), mul2(y, bc2(l)));
}

// complex product with a two-float constant (wr + lr) + i (wi + li), in the
// rounding order of cmul_df
__device__ __forceinline__ void cmul_df2(float2 &x, float2 &y, float wr, float wi, float lr, float li)
{
    const float2 re_lo = fma2(y, bc2(-li), mul2(x, bc2(lr)));
    const float2 im_lo = fma2(y, bc2(lr), mul2(x, bc2(li)));
    const float2 nx = fma2(x, bc2(wr), fma2(y, bc2(-wi), re_lo));
    y = fma2(x, bc2(wi), fma2(y, bc2(wr), im_lo));
    x = nx;
}

// (X, Y) *= W16^J (forward) or its conjugate (INV), the product tw16 forms
template <int J, bool INV> __device__ __forceinline__ void tw16_2(float2 &x, float2 &y)
{
    constexpr int j = J & 15;
    if constexpr (j == 0) {
    } else if constexpr (j == 4 || j == 12) {
        // times -i (forward j = 4) or +i: (x, y) -> (y, -x) or (-y, x)
        constexpr bool minus_i = (j == 4) != INV;
        const float2 t = x;
        x = minus_i ? y : make_float2(-y.x, -y.y);
        y = minus_i ? make_float2(-t.x, -t.y) : t;
    } else if constexpr (j == 8) {
        x = make_float2(-x.x, -x.y);
        y = make_float2(-y.x, -y.y);
    } else if constexpr ((j & 3) == 2) {
        // (+-1 +- i) sqrt(1/2): u = sr x - si y, v = si x + sr y, each then
        // scaled by the two-float sqrt(1/2); a negative sum is carried in the
        // sign of the constant (negation commutes with rounding)
        constexpr float sr = cos16_hi(j) > 0.f ? 1.f : -1.f;
        constexpr float si = (INV ? sin16_hi(j) : -sin16_hi(j)) > 0.f ? 1.f : -1.f;
        constexpr float h = cos16_hi(2), l = cos16_lo(2);
        // u = sr x - si y
        const float2 u = (sr > 0.f) ? (si > 0.f ? sub2(x, y) : add2(x, y)) : (si > 0.f ? add2(x, y) : sub2(y, x));
        constexpr float su = (sr < 0.f && si > 0.f) ? -1.f : 1.f;
        // v = si x + sr y
        const float2 v = (si > 0.f) ? (sr > 0.f ? add2(x, y) : sub2(x, y)) : (sr > 0.f ? sub2(y, x) : add2(x, y));
        constexpr float sv = (si < 0.f && sr < 0.f) ? -1.f : 1.f;
        x = fma2(u, bc2(su * h), mul2(u, bc2(su * l)));
        y = fma2(v, bc2(sv * h), mul2(v, bc2(sv * l)));
    } else {
        constexpr float wr = cos16_hi(j), wi = INV ? sin16_hi(j) : -sin16_hi(j);
        constexpr float lr = cos16_lo(j), li = INV ? sin16_lo(j) : -sin16_lo(j);
        cmul_df2(x, y, wr, wi, lr, li);
    }
}

template <bool INV> __device__ __forceinline__ void dft2_2(float2 &x0, float2 &y0, float2 &x1, float2 &y1)
{
    const float2 tx = x0, ty = y0;
    x0 = add2(tx, x1);
    y0 = add2(ty, y1);
    x1 = sub2(tx, x1);
    y1 = sub2(ty, y1);
}

// 4-point DFT of (a0, a1, a2, a3); a1 - a3 times -i (forward) or +i is a
// renaming whose sign goes into the final add / subtract
template <bool INV>
__device__ __forceinline__ void dft4_2(float2 &x0, float2 &y0, float2 &x1, float2 &y1, float2 &x2, float2 &y2,
                                       float2 &x3, float2 &y3)
{
    const float2 t0x = add2(x0, x2), t0y = add2(y0, y2);
    const float2 t1x = sub2(x0, x2), t1y = sub2(y0, y2);
    const float2 t2x = add2(x1, x3), t2y = add2(y1, y3);
    const float2 dx = sub2(x1, x3), dy = sub2(y1, y3);
    x0 = add2(t0x, t2x);
    y0 = add2(t0y, t2y);
    x2 = sub2(t0x, t2x);
    y2 = sub2(t0y, t2y);
    if constexpr (!INV) {
        // t3 = -i d = (dy, -dx): a1 = t1 + t3, a3 = t1 - t3
        x1 = add2(t1x, dy);
        y1 = sub2(t1y, dx);
        x3 = sub2(t1x, dy);
        y3 = add2(t1y, dx);
    } else {
        // t3 = +i d = (-dy, dx)
        x1 = sub2(t1x, dy);
        y1 = add2(t1y, dx);
        x3 = add2(t1x, dy);
        y3 = sub2(t1y, dx);
    }
}

// 8-point DFT as 4 x 2 (n = 2 n1 + n2, k = k1 + 4 k2), as dft8
template <bool INV> __device__ __forceinline__ void dft8_2(float2 (&x)[8], float2 (&y)[8])
{
    dft4_2<INV>(x[0], y[0], x[2], y[2], x[4], y[4], x[6], y[6]);
    dft4_2<INV>(x[1], y[1], x[3], y[3], x[5], y[5], x[7], y[7]);
    tw16_2<2, INV>(x[3], y[3]);
    tw16_2<6, INV>(x[7], y[7]);
    // element 5 times W8^2 = -i (forward) or +i: folded into its add / subtract
    const float2 p0x = add2(x[0], x[1]), p0y = add2(y[0], y[1]);
    const float2 p4x = sub2(x[0], x[1]), p4y = sub2(y[0], y[1]);
    const float2 p1x = add2(x[2], x[3]), p1y = add2(y[2], y[3]);
    const float2 p5x = sub2(x[2], x[3]), p5y = sub2(y[2], y[3]);
    float2 p2x, p2y, p6x, p6y;
    if constexpr (!INV) {
        // y1[2] = (y5, -x5)
        p2x = add2(x[4], y[5]);
        p2y = sub2(y[4], x[5]);
        p6x = sub2(x[4], y[5]);
        p6y = add2(y[4], x[5]);
    } else {
        // y1[2] = (-y5, x5)
        p2x = sub2(x[4], y[5]);
        p2y = add2(y[4], x[5]);
        p6x = add2(x[4], y[5]);
        p6y = sub2(y[4], x[5]);
    }
    const float2 p3x = add2(x[6], x[7]), p3y = add2(y[6], y[7]);
    const float2 p7x = sub2(x[6], x[7]), p7y = sub2(y[6], y[7]);
    x[0] = p0x; y[0] = p0y;
    x[1] = p1x; y[1] = p1y;
    x[2] = p2x; y[2] = p2y;
    x[3] = p3x; y[3] = p3y;
    x[4] = p4x; y[4] = p4y;
    x[5] = p5x; y[5] = p5y;
    x[6] = p6x; y[6] = p6y;
    x[7] = p7x; y[7] = p7y;
}

// 16-point DFT as 4 x 4 (n = 4 n1 + n2, k = k1 + 4 k2), as dft16
template <bool INV> __device__ __forceinline__ void dft16_2(float2 (&x)[16], float2 (&y)[16])
{
#pragma unroll
    for (int n2 = 0; n2 < 4; ++n2)
        dft4_2<INV>(x[n2], y[n2], x[n2 + 4], y[n2 + 4], x[n2 + 8], y[n2 + 8], x[n2 + 12], y[n2 + 12]);
    tw16_2<1, INV>(x[5], y[5]);
    tw16_2<2, INV>(x[6], y[6]);
    tw16_2<3, INV>(x[7], y[7]);
    tw16_2<2, INV>(x[9], y[9]);
    tw16_2<4, INV>(x[10], y[10]);
    tw16_2<6, INV>(x[11], y[11]);
    tw16_2<3, INV>(x[13], y[13]);
    tw16_2<6, INV>(x[14], y[14]);
    tw16_2<9, INV>(x[15], y[15]);
#pragma unroll
    for (int k1 = 0; k1 < 4; ++k1)
        dft4_2<INV>(x[4 * k1], y[4 * k1], x[4 * k1 + 1], y[4 * k1 + 1], x[4 * k1 + 2], y[4 * k1 + 2], x[4 * k1 + 3],
                    y[4 * k1 + 3]);
    float2 tx[16], ty[16];
#pragma unroll
    for (int k1 = 0; k1 < 4; ++k1)
#pragma unroll
        for (int k2 = 0; k2 < 4; ++k2) {
            tx[k1 + 4 * k2] = x[4 * k1 + k2];
            ty[k1 + 4 * k2] = y[4 * k1 + k2];
        }
#pragma unroll
    for (int i = 0; i < 16; ++i) {
        x[i] = tx[i];
        y[i] = ty[i];
    }
}

template <int R, bool INV> __device__ __forceinline__ void dft_2(float2 (&x)[R], float2 (&y)[R])
{
    if constexpr (R == 2) dft2_2<INV>(x[0], y[0], x[1], y[1]);
    else if constexpr (R == 4) dft4_2<INV>(x[0], y[0], x[1], y[1], x[2], y[2], x[3], y[3]);
    else if constexpr (R == 8) dft8_2<INV>(x, y);
    else dft16_2<INV>(x, y);
}

// (X, Y) *= w (forward) or conj(w) (INV) for a table entry {re_hi, im_hi,
// re_lo, im_lo}, in the rounding order of cmul_df
template <bool INV> __device__ __forceinline__ void twmul2(float2 &x, float2 &y, float4 w)
{
    cmul_df2(x, y, w.x, INV ? -w.y : w.y, w.z, INV ? -w.w : w.w);
}

// ---------------------------------------------------------------- stages
// One Stockham stage of radix R after NS points have been combined, for the
// pair (X, Y): butterfly jp takes element jp + r N/R of both pencils,
// multiplies input r by W_{NS R}^{r (jp mod NS)} and writes output p to
// element (jp / NS) NS R + jp mod NS + p NS.  sb: the pair's exchange buffer
// of pad8_len(N) 16-byte slots; tws: this stage's twiddle block.
template <int N, int E, int R, int NS, bool INV, bool LAST, class Sync>
__device__ __forceinline__ void pair_stage(float2 (&X)[E], float2 (&Y)[E], float4 *__restrict__ sb, int j,
                                           const float4 *__restrict__ tws, const Sync &sync)
{
    constexpr int TP = N / E, B = E / R;
#pragma unroll
    for (int q = 0; q < B; ++q) {
        const int jp = j + q * TP;
        const int k = jp & (NS - 1);
        float2 ax[R], ay[R];
#pragma unroll
        for (int r = 0; r < R; ++r) {
            ax[r] = X[q + B * r];
            ay[r] = Y[q + B * r];
        }
        if constexpr (NS > 1) {
#pragma unroll
            for (int r = 1; r < R; ++r) twmul2<INV>(ax[r], ay[r], tws[(r - 1) * NS + k]);
        }
        dft_2<R, INV>(ax, ay);
        if constexpr (LAST) {
#pragma unroll
            for (int p = 0; p < R; ++p) {
                X[q + B * p] = ax[p];
                Y[q + B * p] = ay[p];
            }
        } else {
            const int base = (jp - k) * R + k;
#pragma unroll
            for (int p = 0; p < R; ++p) sb[pad8(base + p * NS)] = make_float4(ax[p].x, ax[p].y, ay[p].x, ay[p].y);
        }
    }
    if constexpr (!LAST) {
        sync();
#pragma unroll
        for (int r = 0; r < E; ++r) {
            const float4 t = sb[pad8(j + r * TP)];
            X[r] = make_float2(t.x, t.y);
            Y[r] = make_float2(t.z, t.w);
        }
        sync();
    }
}

// Full transform of a pencil pair, natural order in and out (element j + r TP
// of both pencils in X[r], Y[r]), in the radix schedule of main radix E
// (fftg_radix<log2 E>: with E = 16 the one-pencil transform's schedule and
// twiddle table, with E = 8 the radix-8 schedule and its table).
// Forward: X_k = sum_n x_n e^{-2 pi i nk/N}; INV: the conjugate sum without
// 1/N.  Every thread that `sync` covers calls it together.
template <int N, int E, bool INV, int S = 0, class Sync = CtaSync>
__device__ __forceinline__ void fft_pair(float2 (&X)[E], float2 (&Y)[E], float4 *__restrict__ sb, int j,
                                         const float4 *__restrict__ tw, const Sync &sync = Sync())
{
    static_assert(E == 16 || E == 8, "8 or 16 elements per pencil per thread");
    constexpr int LR = E == 16 ? 4 : 3;
    constexpr int R = fftg_radix<LR>(N, S), NS = fftg_ns<LR>(N, S);
    constexpr bool LAST = (S == fftg_stages<LR>(N) - 1);
    static_assert(E % R == 0, "radix must divide the elements per thread");
    pair_stage<N, E, R, NS, INV, LAST>(X, Y, sb, j, tw + fftg_tw_offset<LR>(N, S), sync);
    if constexpr (!LAST) fft_pair<N, E, INV, S + 1>(X, Y, sb, j, tw, sync);
}

}  // namespace gpe
