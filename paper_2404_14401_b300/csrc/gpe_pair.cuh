// gpe_pair.cuh -- device pieces of the pencil-pair passes (sm_103a), shared by
// the one-pass-per-launch pair kernels (gpe_pair.cu) and the cooperative
// persistent kernel (gpe_coop.cu): the potential at two pencils, the
// potential phase of a thread's packed elements, the conjugated kinetic
// factor and T = F^-1 K F of one pencil pair (Sec. 3.1, Eqs. 3-4).
#pragma once

#include <cuda_runtime.h>
#include <math.h>

#include "gpe_device.cuh"
#include "gpe_fft2.cuh"
#include "gpe_internal.h"

namespace gpe {

// V at the same y of two columns (coefficients pa, pb; y-table entry t), in
// the order of pot_at
__device__ __forceinline__ float2 pot_at2(const PotCoefs &pa, const PotCoefs &pb, float4 t)
{
    const float2 f = add2(make_float2(pa.F, pb.F), bc2(t.x));
    const float2 u = fma2(bc2(pa.A), bc2(t.y), f);
    const float2 w = fma2(bc2(pa.B), bc2(t.z), make_float2(pa.C, pb.C));
    return fma2(w, bc2(t.z), u);
}

// (X, Y) <- exp(-i theta) (X, Y) on a packed pair, in phase_mul's 1 + d form
// with the Taylor series of sin and cos of theta/2 (|theta| <= 1)
__device__ __forceinline__ void rot2_taylor(float2 &X, float2 &Y, float2 th)
{
    const float2 w = mul2(bc2(0.5f), th);
    const float2 v = mul2(w, w);
    float2 ps = fma2(v, bc2(1.f / 362880.f), bc2(-1.f / 5040.f));
    ps = fma2(v, ps, bc2(1.f / 120.f));
    ps = fma2(v, ps, bc2(-1.f / 6.f));
    const float2 s = fma2(mul2(w, v), ps, w);
    float2 pc = fma2(v, bc2(1.f / 40320.f), bc2(-1.f / 720.f));
    pc = fma2(v, pc, bc2(1.f / 24.f));
    pc = fma2(v, pc, bc2(-0.5f));
    const float2 c = fma2(v, pc, bc2(1.f));
    const float2 m2s = mul2(bc2(-2.f), s);
    const float2 dr = mul2(m2s, s), di = mul2(m2s, c);
    const float2 nx = add2(X, fma2(X, dr, mul2(Y, make_float2(-di.x, -di.y))));
    Y = add2(Y, fma2(X, di, mul2(Y, dr)));
    X = nx;
}

// phase_adjoint on a packed pair: lambda (LX, LY) <- mu + 2 h g Im(conj(mu)
// psi) psi with mu = exp(+i theta) lambda, theta = (V + g |psi|^2) h given;
// (PX, PY) is the phase's input psi.  Returns Im(conj(mu) psi) per lane.
// The rotation in rot2_taylor's form (|theta| <= 1).
__device__ __forceinline__ float2 adjoint2_taylor(float2 &LX, float2 &LY, float2 PX, float2 PY, float2 th, float g,
                                                  float h)
{
    float2 MX = LX, MY = LY;
    rot2_taylor(MX, MY, make_float2(-th.x, -th.y));
    const float2 q = fma2(MX, PY, mul2(make_float2(-MY.x, -MY.y), PX));
    const float2 f = mul2(bc2(2.f * h * g), q);
    LX = fma2(f, PX, MX);
    LY = fma2(f, PY, MY);
    return q;
}

// phase_mul (exp(-i theta) in the 1 + d form with the Taylor series of sin
// and cos of theta/2, or exp(-theta) in imaginary time; theta = (V + g
// |psi|^2) h) on all E packed pairs of a thread: every theta first, then one
// branch for the whole thread -- the packed Taylor path unless some |theta|
// exceeds 1 -- so that the per-element code is one straight line (the rare
// sincosf path sits in a block of its own instead of beside every element)
template <int E>
__device__ __forceinline__ void phase_all2(float2 (&X)[E], float2 (&Y)[E], float2 (&V)[E], float g, float h,
                                           int imag)
{
    bool small = true;
#pragma unroll
    for (int r = 0; r < E; ++r) {
        const float2 n = fma2(X[r], X[r], mul2(Y[r], Y[r]));
        V[r] = mul2(fma2(bc2(g), n, V[r]), bc2(h));           // V[r] now holds theta
        small = small && fabsf(V[r].x) <= 1.f && fabsf(V[r].y) <= 1.f;
    }
    if (imag) {
#pragma unroll
        for (int r = 0; r < E; ++r) {
            const float2 f = make_float2(expf(-V[r].x), expf(-V[r].y));
            X[r] = mul2(X[r], f);
            Y[r] = mul2(Y[r], f);
        }
    } else if (small) {
#pragma unroll
        for (int r = 0; r < E; ++r) rot2_taylor(X[r], Y[r], V[r]);
    } else {
#pragma unroll
        for (int r = 0; r < E; ++r) {
            const float2 r0 = phase_rot(make_float2(X[r].x, Y[r].x), V[r].x);
            const float2 r1 = phase_rot(make_float2(X[r].y, Y[r].y), V[r].y);
            X[r] = make_float2(r0.x, r1.x);
            Y[r] = make_float2(r0.y, r1.y);
        }
    }
}

// T's kinetic factor on the pair, conjugated: (X, Y) <- conj(K (X, Y)) with
// K = (1 + d) s in real time (the 1 + D form of the table) and e^{-k^2
// dt/2m} s in imaginary time, s the 1/N of the inverse transform.  KCONJ:
// the adjoint propagator's factor, d -> conj(d) (real time).
template <int E, int TP, bool KCONJ = false>
__device__ __forceinline__ void kinetic_conj_pair(float2 (&X)[E], float2 (&Y)[E], const float2 *__restrict__ D,
                                                  int j, float s, int imag)
{
    if (imag) {
#pragma unroll
        for (int r = 0; r < E; ++r) {
            const float k = __ldg(&D[j + r * TP]).x;
            X[r] = mul2(X[r], bc2(k * s));
            Y[r] = mul2(Y[r], bc2(-k * s));
        }
    } else {
#pragma unroll
        for (int r = 0; r < E; ++r) {
            float2 d = __ldg(&D[j + r * TP]);
            if constexpr (KCONJ) d.y = -d.y;
            const float2 pdx = fma2(X[r], bc2(d.x), mul2(Y[r], bc2(-d.y)));
            const float2 pdy = fma2(X[r], bc2(d.y), mul2(Y[r], bc2(d.x)));
            X[r] = mul2(add2(X[r], pdx), bc2(s));
            Y[r] = mul2(add2(Y[r], pdy), bc2(-s));
        }
    }
}

// F^-1 K F on the pencil pair, with the inverse taken as conj(F(conj(.))):
// one loop runs the forward transform twice, the kinetic factor and the
// first conjugation between the two runs, so that the unrolled transform is
// in the code once.  Half the instruction footprint of writing out both
// directions: the row pass at 2048 points ran 34.0 -> 33.6 us per pass (its
// instruction-cache hit rate 74 -> 85%), 4096 133 -> 125 us and 8192 918 ->
// 814 us; the column pass at 8192 points 886 -> 798 us.
template <int N, int E, int TP, class Sync = CtaSync, bool KCONJ = false>
__device__ __forceinline__ void transform_pair(float2 (&X)[E], float2 (&Y)[E], float4 *__restrict__ sb, int j,
                                               const float4 *__restrict__ tw, const float2 *__restrict__ D, float s,
                                               int imag, const Sync &sync = Sync())
{
#pragma unroll 1
    for (int pass = 0; pass < 2; ++pass) {
        fft_pair<N, E, false, 0, Sync>(X, Y, sb, j, tw, sync);
        if (pass == 0) kinetic_conj_pair<E, TP, KCONJ>(X, Y, D, j, s, imag);
    }
#pragma unroll
    for (int r = 0; r < E; ++r) Y[r] = mul2(Y[r], bc2(-1.f));      // the second conjugation
}

}  // namespace gpe
