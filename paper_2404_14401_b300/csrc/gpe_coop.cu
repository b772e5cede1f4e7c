// gpe_coop.cu -- cooperative persistent kernel (sm_103a): every split step of
// one gpe_step call (Sec. 3.1, Eqs. 3-4; imaginary time Sec. 3.3; cavity
// Sec. 5.3, Eqs. 10-15) on one grid that fits on chip, in one launch.
//
// The per-pass path launches two or three kernels per step; on a 512^2 grid
// each of them is a few hundred small CTAs whose time is mostly launch,
// ramp-up and the latency of one FFT chain.  Here one or two CTAs per SM stay
// resident for all n steps and run the host scheduler's pass program itself:
// a row pass (potential phase, T_x) on pairs of rows, a column pass (T_y
// [+ closing phase] [+ reductions]) on pairs of columns, and the pointwise
// prologue / epilogue passes, each pass separated from the next by a grid
// barrier.  psi stays in L2 between passes (2 MB at 512^2): loads and stores
// go through L2 (ld.global.cg / st.global.cg), never the non-coherent L1.
//
// A group of N/8 threads owns one pencil pair at a time and transforms it
// with the pair code of the pair passes (gpe_pair.cuh): the two rows (or
// columns) in packed f32x2 registers, exchanges through the group's own
// shared-memory slots, synchronised with a named barrier of the group.
// Reducing passes: each CTA sums its threads' partials in FP64 (fixed tree),
// stores them, and after the grid barrier every CTA sums all CTAs' partials in
// the same fixed order and finalises the norm, 1/sqrt(norm) and alpha (Eqs.
// 14-15) itself, so no second barrier is needed to share them; CTA 0 also
// writes them to the context's scalars.  Row-pass and column-pass partials use
// separate arrays, so a reduction's partials are never overwritten before
// every CTA has read them.
//
// The grid barrier: thread 0 of each CTA adds its arrival to a counter that
// only grows and polls it until every CTA has arrived, with a bounded number
// of polls.  A wait that runs out latches GPE_ETIMEOUT and raises an abort
// flag that ends every CTA at its next barrier.  The cooperative launch
// guarantees that all CTAs are resident, so every wait ends.
//
// A pass takes about the time one group needs to transform its pencil pair,
// which is why 512-point pairs are transformed in the radix-8 schedule (8
// elements per thread, two warps per pair) rather than the per-pass kernels'
// radix-16 one.  Measured on a B300, per step against the per-pass path:
// 512^2 lattice (real time) 10.9 against 13.3 us, the 512^2 cavity ramp 17.8
// against 24.6 us, a 512^2 trap in imaginary time 16.2 against 23.8 us.  At
// 1024^2: real time 24.2 against 21.4 us, imaginary time 31.6 against 33.6
// us, the cavity 33.4 against 35.2 us.  At 512^2 with 256-thread CTAs it was
// 11.1, 20.2 and 18.0 us; with 16 elements per thread (one warp per pair)
// 14.7, 24.0 and 22.6 us; with 512-thread CTAs 12.6, 25.3 and 23.3 us.  At
// 1024^2 with the radix-8 schedule, real time took 26.6 us (two CTAs per SM)
// and 28.7 us (one).
#include <cuda.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <atomic>

#include "../../include/gpe.h"
#include "gpe_ctrl.cuh"
#include "gpe_device.cuh"
#include "gpe_fft2.cuh"
#include "gpe_internal.h"
#include "gpe_pair.cuh"

namespace gpe {

// Elements of each pencil per thread, and CTA shape, by the longer axis.
// 512 points: the radix-8 schedule (8 elements, a pencil pair over two
// warps), CTAs of two such groups (128 threads), one per SM -- a 512^2 pass
// keeps one or two groups per SM busy, and fewer idle warps make every CTA
// barrier and reduction shorter.  1024 points: the radix-16 schedule (16
// elements, two warps per pair; the radix-8 one needs a fourth stage and a
// third exchange there, 208 against about 170 instructions per point-step),
// two groups per CTA, two CTAs per SM so that each group has one pair per
// pass.  The exchange slots of a CTA's groups, (CT / TP) groups of
// pad8_len(N) 16-byte slots, are CT * E * 18 bytes whatever the length.
template <int NX, int NY> struct CoopCfg {
    static constexpr int NMAX = NX > NY ? NX : NY;
    static constexpr int E = NMAX >= 1024 ? 16 : 8;
    static constexpr int CT = 2 * (NMAX / E);
    static constexpr int CPS = NMAX >= 1024 ? 2 : 1;       // CTAs per SM
    static constexpr size_t SLOT_BYTES = (size_t)CT * E * 18;
    static constexpr size_t SMEM = SLOT_BYTES + 128;
};

// The tables and the potential array, read by the passes through a copy in
// shared memory: a pointer loaded from shared memory after a barrier is new
// to the compiler at every pass, so it cannot hoist the passes' table loads
// out of the step loop (which it did from the launch arguments, keeping the
// kinetic factors and coordinates of every pass live across the whole loop
// and spilling them).
struct CoopPtrs {
    Tables T;
    const float *V;
};

template <int N, int CT, int E_> struct CoopAxis {
    static constexpr int E = E_, TP = N / E, GPB = CT / TP, SLOTS = pad8_len(N);
    static_assert((size_t)GPB * SLOTS * 16 == (size_t)CT * E * 18, "group slots");
    static_assert(TP % 32 == 0 && GPB <= 15, "groups of whole warps, one named barrier each");
};

// ------------------------------------------------------------------ grid barrier
// Every thread of every CTA calls it, the same number of times (k counts this
// CTA's barriers in shared memory).  Writes made before it (by any thread of
// any CTA) are visible, through L2, to reads after it.  The arrival counter
// only grows: barrier k is complete when it reaches k * gridDim.x, so there
// is no reset and no second word to release.  Returns false once a wait has
// run out anywhere (the launch is being abandoned).
__device__ bool coop_sync(const CoopArgs &a, int *s_ok, unsigned int *k)
{
    __syncthreads();
    if (threadIdx.x == 0) {
        DevScalars *sc = a.T.sc;
        const unsigned int target = (++*k) * gridDim.x;
        __threadfence();                           // this CTA's writes before the arrival
        int ok = 1;
        if (atomicAdd(&sc->bar_count, 1u) + 1u < target) {
            const int limit = a.spins < (1 << 22) ? a.spins : (1 << 22);
            int polls = 0;
            unsigned int ns = 32;
            while (ld_acquire(&sc->bar_count) < target) {
                if (polls++ >= limit || ld_acquire(&sc->bar_abort)) {
                    ok = 0;
                    break;
                }
                if (polls > 64) {                  // back off once the wait is long
                    __nanosleep(ns);
                    if (ns < 256) ns *= 2;
                }
            }
        }
        if (!ok) {
            latch_status(sc, GPE_ETIMEOUT);
            atomicExch(&sc->bar_abort, 1u);
        }
        *s_ok = ok;
    }
    __syncthreads();
    return *s_ok != 0;
}

// Norm, overlaps, 1/sqrt(norm) and the cavity field from the sums (Sec. 3.3
// normalisation, Eqs. 14-15), in FP64 on one thread: the quantities and the
// status latching of finalize_fields, with one reciprocal per denominator
// instead of a division per quantity (every CTA runs this between two passes
// while its other threads wait).
__device__ void coop_finalize(const double *S, const RedArgs &r, DevScalars *sc)
{
    const double inv0 = 1.0 / S[0];
    const double norm = S[0] * r.dxdy, O = S[1] * inv0, B = S[2] * inv0;
    sc->norm = norm;
    sc->O = O;
    sc->B = B;
    sc->c = rsqrt(norm);
    if (!isfinite(norm) || !(norm > 0.0) || !isfinite(O) || !isfinite(B)) {
        latch_status(sc, GPE_ENONFINITE);
        return;
    }
    if (r.cavity) {
        const double dr = r.dc - r.U0 * B, di = r.kappa;
        const double den = dr * dr + di * di;
        if (!(den > 1e-24)) {
            latch_status(sc, GPE_EILLCOND);
            sc->alpha_re = 0.0;
            sc->alpha_im = 0.0;
            return;
        }
        const double iden = 1.0 / den;
        double ps = 0.0, pc = 0.0;               // probe Omega_c exp(i (Delta_p t + phi)) (Sec. 5.4)
        if (r.probe_omega != 0.0) sincos(r.probe_delta * r.t + r.probe_phi, &ps, &pc);
        const double fa = r.N * r.eta * O + r.probe_omega * pc, fb = r.probe_omega * ps;
        sc->alpha_re = (fa * dr + fb * di) * iden;
        sc->alpha_im = (fb * dr - fa * di) * iden;
    } else {
        sc->alpha_re = 0.0;
        sc->alpha_im = 0.0;
    }
}

// Sum of the first `count` rows of part[][NQ] (K of them), by warp 0 alone in
// a fixed order (lane-strided, then a shuffle tree): the same in every CTA.
// Valid in lane 0.
__device__ void coop_sum_partials(const double *part, int count, double (&S)[3])
{
    const int lane = threadIdx.x & 31;
    double acc[3] = {0.0, 0.0, 0.0};
    for (int b = lane; b < count; b += 32)
#pragma unroll
        for (int i = 0; i < 3; ++i) acc[i] += __ldcg(&part[(size_t)b * NQ + i]);
    for (int off = 16; off > 0; off >>= 1)
#pragma unroll
        for (int i = 0; i < 3; ++i) acc[i] += __shfl_down_sync(0xffffffffu, acc[i], off);
#pragma unroll
    for (int i = 0; i < 3; ++i) S[i] = acc[i];
}

// Finish a reducing pass: the CTA's FP64 partials (norm, O and B sums) into
// part[blockIdx.x], the grid barrier, then warp 0 of every CTA sums all
// partials in block order and thread 0 finalises norm, c and alpha into the
// CTA's own copy `loc`; CTA 0 also writes them to the context's scalars.
__device__ bool coop_reduce(const CoopArgs &a, const float (&q)[3], const RedArgs &rd, double *part, DevScalars *loc,
                            double *red, int *s_ok, unsigned int *k)
{
    block_sum<3>(q, part + (size_t)blockIdx.x * NQ, red);
    if (!coop_sync(a, s_ok, k)) return false;
    double S[3];
    if (threadIdx.x < 32) coop_sum_partials(part, (int)gridDim.x, S);
    if (threadIdx.x == 0) {
        coop_finalize(S, rd, loc);
        if (blockIdx.x == 0) {
            DevScalars *sc = a.T.sc;
            sc->norm = loc->norm;
            sc->O = loc->O;
            sc->B = loc->B;
            sc->c = loc->c;
            sc->alpha_re = loc->alpha_re;
            sc->alpha_im = loc->alpha_im;
            if (loc->status) latch_status(sc, loc->status);
        }
    }
    __syncthreads();
    return true;
}

// ------------------------------------------------------------------ passes
// The pass functions are not inlined into the kernel: compiled as one
// function, the kernel's five transforming passes kept enough values live
// across the step loop to spill 1-3 KB at 128 and 255 registers per thread;
// out of line each pass gets its own allocation and spills at most 20 bytes.
//
// Units (pencil pairs) are dealt to groups CTA-first: unit u goes to CTA
// u mod gridDim.x, so a pass narrower than the grid's groups spreads over
// every SM.  All threads of a group share its units, and the named barrier
// inside the transform is the group's own, so a group without a unit skips
// the pass and waits at the CTA barrier that ends it.
// The thread's and the CTA's index are read with volatile moves at every
// pass, so that the index and address arithmetic derived from them (the
// exchange-slot offsets of every stage, the elements' offsets) is pass-local
// for the compiler rather than hoisted out of the step loop and kept live
// across all passes.
__device__ __forceinline__ int tid_fresh()
{
    int t;
    asm volatile("mov.u32 %0, %%tid.x;" : "=r"(t));
    return t;
}
__device__ __forceinline__ int cta_fresh()
{
    int b;
    asm volatile("mov.u32 %0, %%ctaid.x;" : "=r"(b));
    return b;
}

// A pass's view of the CTA: its CT threads start at thread `base` (0, or CT
// for the second role of coop_adjrec_kernel); g is the thread's group among
// them, j its thread in the group, gg its first unit, G the units' stride,
// bid the group's named barrier (unique in the CTA: 1 + the group's index
// among all the CTA's groups).
template <int N, int CT, int E> struct CoopUnits {
    int g, j, gg, G, bid;
    __device__ explicit CoopUnits(int base = 0)
    {
        using A = CoopAxis<N, CT, E>;
        const int t = tid_fresh();
        g = (t - base) / A::TP;
        j = (t - base) % A::TP;
        gg = cta_fresh() + gridDim.x * g;
        G = gridDim.x * A::GPB;
        bid = 1 + t / A::TP;
    }
};

// Row pass ROW_PT on the row pairs (2u, 2u + 1): [scale c] potential phase,
// T_x, as row_pair_kernel computes it, from src into dst (the same buffer
// when the step is in place).
template <int N, int CT, int EE>
__device__ __noinline__ void coop_rows_pt(const CoopArgs &a, const CoopPtrs &P, const PhaseArgs &ph, int use_c,
                             const DevScalars &loc, float4 *slots, const float2 *src, float2 *dst,
                             int base = 0)
{
    const Tables &T = P.T;
    using A = CoopAxis<N, CT, EE>;
    constexpr int E = A::E, TP = A::TP;
    const int units = a.ny / 2;
    const CoopUnits<N, CT, EE> U(base);
    float4 *sb = slots + U.g * A::SLOTS;
    const GroupSync gs{U.bid, TP};
    const float cs = use_c ? (float)loc.c : 1.f;
    float acx2, acxcy;
    alpha_amps(ph, loc.alpha_re, loc.alpha_im, acx2, acxcy);
    for (int u = U.gg; u < units; u += U.G) {
        const bool act = check_index((long long)2 * u + 1, a.ny, T.sc);
        const int y0 = act ? 2 * u : 0;
        const float2 *ia = src + (size_t)y0 * N, *ib = ia + N;
        float2 *ra = dst + (size_t)y0 * N, *rb = ra + N;
        float2 X[E], Y[E], V[E];
#pragma unroll
        for (int r = 0; r < E; ++r) {
            const int xi = U.j + r * TP;
            const float2 p = act ? __ldcg(ia + xi) : make_float2(0.f, 0.f);
            const float2 q = act ? __ldcg(ib + xi) : make_float2(0.f, 0.f);
            X[r] = make_float2(p.x * cs, q.x * cs);
            Y[r] = make_float2(p.y * cs, q.y * cs);
        }
        const PotCoefs pa = row_coefs_from(ph, acx2, acxcy, __ldg(&T.ytab[y0]));
        const PotCoefs pb = row_coefs_from(ph, acx2, acxcy, __ldg(&T.ytab[y0 + 1]));
        const float *Va = P.V ? P.V + (size_t)y0 * N : nullptr;
#pragma unroll
        for (int r = 0; r < E; ++r) {
            const int xi = U.j + r * TP;
            V[r] = pot_at2(pa, pb, __ldg(&T.xtab[xi]));
            if (Va) V[r] = fma2(bc2(a.V_scale), make_float2(__ldg(&Va[xi]), __ldg(&Va[N + xi])), V[r]);
        }
        phase_all2<E>(X, Y, V, a.g, ph.h, a.imag);
        transform_pair<N, E, TP>(X, Y, sb, U.j, E == 8 ? T.tw8x : T.twx, T.kinx, a.sx, a.imag, gs);
        if (act) {
#pragma unroll
            for (int r = 0; r < E; ++r) {
                const int xi = U.j + r * TP;
                __stcg(ra + xi, make_float2(X[r].x, Y[r].x));
                __stcg(rb + xi, make_float2(X[r].y, Y[r].y));
            }
        }
    }
}

// Column pass on the column pairs (2u, 2u + 1) of columns of N points in a
// grid NX wide, as col_pair_kernel computes it: T_y, then (COL_T_P,
// COL_T_PR) the closing half phase, then (COL_T_R, COL_T_PR) the norm and
// overlap sums added to q, in place on psi.  With the width a constant, a
// thread's strided elements are immediate offsets from one address.
template <int N, int NX, int MODE, int CT, int EE>
__device__ __noinline__ void coop_cols(const CoopArgs &a, const CoopPtrs &P, const PhaseArgs &ph, const DevScalars &loc,
                          float4 *slots, float (&q)[3], float2 *psi, int base = 0)
{
    const Tables &T = P.T;
    using A = CoopAxis<N, CT, EE>;
    constexpr int E = A::E, TP = A::TP;
    constexpr bool PHASE = (MODE == COL_T_P || MODE == COL_T_PR);
    constexpr bool REDUCE = (MODE == COL_T_R || MODE == COL_T_PR);
    constexpr int units = NX / 2, w4 = NX / 2;                 // float4 per grid row
    const CoopUnits<N, CT, EE> U(base);
    float4 *sb = slots + U.g * A::SLOTS;
    const GroupSync gs{U.bid, TP};
    float acx2, acxcy;
    alpha_amps(ph, loc.alpha_re, loc.alpha_im, acx2, acxcy);
    for (int u = U.gg; u < units; u += U.G) {
        const bool act = check_index((long long)2 * u + 1, NX, T.sc);
        const int x0 = act ? 2 * u : 0;
        // {re, im} of columns x0, x0 + 1 at row j + r TP: cb[r TP w4]
        float4 *cb = reinterpret_cast<float4 *>(psi + x0) + (size_t)U.j * w4;
        float2 X[E], Y[E];
#pragma unroll
        for (int r = 0; r < E; ++r) {
            const float4 t = act ? __ldcg(cb + r * TP * w4) : make_float4(0.f, 0.f, 0.f, 0.f);
            X[r] = make_float2(t.x, t.z);
            Y[r] = make_float2(t.y, t.w);
        }
        transform_pair<N, E, TP>(X, Y, sb, U.j, E == 8 ? T.tw8y : T.twy, T.kiny, a.sy, a.imag, gs);
        const float4 xa = __ldg(&T.xtab[x0]), xb = __ldg(&T.xtab[x0 + 1]);
        if constexpr (PHASE) {
            const PotCoefs pa = col_coefs_from(ph, acx2, acxcy, xa), pb = col_coefs_from(ph, acx2, acxcy, xb);
            float2 V[E];
#pragma unroll
            for (int r = 0; r < E; ++r) {
                const int y = U.j + r * TP;
                V[r] = pot_at2(pa, pb, __ldg(&T.ytab[y]));
                if (P.V) {
                    const float2 va = make_float2(__ldg(&P.V[(size_t)y * NX + x0]), __ldg(&P.V[(size_t)y * NX + x0 + 1]));
                    V[r] = fma2(bc2(a.V_scale), va, V[r]);
                }
            }
            phase_all2<E>(X, Y, V, a.g, ph.h, a.imag);
        }
        if constexpr (REDUCE) {
            float2 n0 = make_float2(0.f, 0.f), n1 = n0;
#pragma unroll
            for (int r = 0; r < E; ++r) {
                const float2 nn = fma2(X[r], X[r], mul2(Y[r], Y[r]));
                n0 = add2(n0, nn);
                n1 = fma2(bc2(__ldg(&T.ytab[U.j + r * TP]).z), nn, n1);
            }
            if (act) {
                q[0] += n0.x + n0.y;
                q[1] += xa.z * n1.x + xb.z * n1.y;
                q[2] += xa.z * xa.z * n0.x + xb.z * xb.z * n0.y;
            }
        }
        if (act) {
#pragma unroll
            for (int r = 0; r < E; ++r) __stcg(cb + r * TP * w4, make_float4(X[r].x, Y[r].x, X[r].y, Y[r].y));
        }
    }
}

// Pointwise row passes over the whole grid (grid-stride): ROW_PHASE (the
// closing half phase), ROW_PHASE_R (the same, then the sums), ROW_REDUCE_R
// (the sums only, nothing stored), ROW_SCALE (multiply by c).  Point
// arithmetic as in row_kernel.
template <int NX, int MODE>
__device__ __noinline__ void coop_points(const CoopArgs &a, const CoopPtrs &P, const PhaseArgs &ph, const DevScalars &loc,
                            float (&q)[3])
{
    const Tables &T = P.T;
    constexpr bool PHASE = (MODE == ROW_PHASE || MODE == ROW_PHASE_R);
    constexpr bool REDUCE = (MODE == ROW_PHASE_R || MODE == ROW_REDUCE_R);
    const int total = NX * a.ny;
    float acx2, acxcy;
    alpha_amps(ph, loc.alpha_re, loc.alpha_im, acx2, acxcy);
    const float cs = (float)loc.c;
    for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < total; idx += gridDim.x * blockDim.x) {
        const int x = idx & (NX - 1), y = idx / NX;
        float2 v = __ldcg(a.psi + idx);
        const float4 xt = __ldg(&T.xtab[x]);
        if constexpr (MODE == ROW_SCALE) v = make_float2(v.x * cs, v.y * cs);
        if constexpr (PHASE) {
            const PotCoefs pc = row_coefs_from(ph, acx2, acxcy, __ldg(&T.ytab[y]));
            float V = pot_at(pc, xt);
            if (P.V) V += a.V_scale * __ldg(&P.V[idx]);
            v = phase_mul(v, V, a.g, ph.h, a.imag);
        }
        if constexpr (REDUCE) {
            const float n = v.x * v.x + v.y * v.y, cy = __ldg(&T.ytab[y]).z;
            q[0] += n;
            q[1] += xt.z * cy * n;
            q[2] += xt.z * xt.z * n;
        }
        if constexpr (MODE != ROW_REDUCE_R) __stcg(a.psi + idx, v);
    }
}

// ------------------------------------------------------------------ kernel
// The program of step_prologue (alpha of the initial density), n x step_part
// and step_epilogue, with the same pass times, phase lengths and modes.
template <int NX, int NY>
__global__ void __launch_bounds__(CoopCfg<NX, NY>::CT, CoopCfg<NX, NY>::CPS) coop_kernel(const __grid_constant__ CoopArgs a)
{
    extern __shared__ unsigned char smraw[];
    __shared__ double red[32 * NQ];
    __shared__ DevScalars loc;                     // c and alpha of the last reduction, the same in every CTA
    __shared__ PhaseArgs s_ph;
    __shared__ RedArgs s_rd;
    __shared__ CoopPtrs s_P;
    __shared__ int s_ok;
    __shared__ unsigned int s_k;                   // grid barriers this CTA has passed

    const uint32_t s0 = smem_u32(smraw);
    float4 *slots = reinterpret_cast<float4 *>(smraw + ((128u - (s0 & 127u)) & 127u));
    if (threadIdx.x == 0) {
        memset(&loc, 0, sizeof(loc));
        loc.c = __ldcg(&a.T.sc->c);
        loc.alpha_re = __ldcg(&a.T.sc->alpha_re);
        loc.alpha_im = __ldcg(&a.T.sc->alpha_im);
        memset(&s_ph, 0, sizeof(s_ph));
        s_k = 0;
        s_P.T = a.T;
        s_P.V = a.V;
        s_ok = check_index((long long)((unsigned char *)slots + CoopCfg<NX, NY>::SLOT_BYTES - smraw) - 1, dyn_smem_bytes(),
                           a.T.sc);
        if (!s_ok) atomicExch(&a.T.sc->bar_abort, 1u);
    }
    __syncthreads();
    if (!s_ok) return;                             // the others stop at their first barrier

    const double t0 = a.t0, dt = a.dt, hh = __dmul_rn(0.5, dt);
    const int n = a.n, imag = a.imag, cav = a.cavity;
    float q[3];
    bool ok = true;
    if (cav) {                                     // alpha of the initial density (Eq. 14)
        if (threadIdx.x == 0) s_rd = red_dev(a, t0);
        __syncthreads();
        q[0] = q[1] = q[2] = 0.f;
        coop_points<NX, ROW_REDUCE_R>(a, s_P, s_ph, loc, q);
        ok = coop_reduce(a, q, s_rd, a.T.part_row, &loc, red, &s_ok, &s_k);
    }
    for (int s = 0; ok && s < n; ++s) {
        const double ts = __dadd_rn(t0, __dmul_rn((double)s, dt));
        const double te = __dadd_rn(t0, __dmul_rn((double)(s + 1), dt));
        if (threadIdx.x == 0) s_ph = phase_dev(a, ts, (imag || s == 0) ? hh : dt);
        __syncthreads();
        coop_rows_pt<NX, CoopCfg<NX, NY>::CT, CoopCfg<NX, NY>::E>(a, s_P, s_ph, imag && s > 0, loc, slots, a.psi,
                                                                   a.psi);
        if (!coop_sync(a, &s_ok, &s_k)) {
            ok = false;
            break;
        }
        q[0] = q[1] = q[2] = 0.f;
        if (!imag && !cav) {
            if (s == n - 1) {
                if (threadIdx.x == 0) s_ph = phase_dev(a, te, hh);
                __syncthreads();
                coop_cols<NY, NX, COL_T_P, CoopCfg<NX, NY>::CT, CoopCfg<NX, NY>::E>(a, s_P, s_ph, loc, slots, q, a.psi);
            } else {
                coop_cols<NY, NX, COL_T, CoopCfg<NX, NY>::CT, CoopCfg<NX, NY>::E>(a, s_P, s_ph, loc, slots, q, a.psi);
                ok = coop_sync(a, &s_ok, &s_k);
            }
        } else if (!imag) {
            if (threadIdx.x == 0) s_rd = red_dev(a, te);
            __syncthreads();
            coop_cols<NY, NX, COL_T_R, CoopCfg<NX, NY>::CT, CoopCfg<NX, NY>::E>(a, s_P, s_ph, loc, slots, q, a.psi);
            ok = coop_reduce(a, q, s_rd, a.T.part_col, &loc, red, &s_ok, &s_k);
        } else if (!cav) {
            if (threadIdx.x == 0) {
                s_ph = phase_dev(a, te, hh);
                s_rd = red_dev(a, te);
            }
            __syncthreads();
            coop_cols<NY, NX, COL_T_PR, CoopCfg<NX, NY>::CT, CoopCfg<NX, NY>::E>(a, s_P, s_ph, loc, slots, q, a.psi);
            ok = coop_reduce(a, q, s_rd, a.T.part_col, &loc, red, &s_ok, &s_k);
        } else {                                   // imaginary time with a cavity: a third, pointwise pass
            if (threadIdx.x == 0) s_rd = red_dev(a, te);
            __syncthreads();
            coop_cols<NY, NX, COL_T_R, CoopCfg<NX, NY>::CT, CoopCfg<NX, NY>::E>(a, s_P, s_ph, loc, slots, q, a.psi);
            ok = coop_reduce(a, q, s_rd, a.T.part_col, &loc, red, &s_ok, &s_k);
            if (!ok) break;
            if (threadIdx.x == 0) s_ph = phase_dev(a, te, hh);
            __syncthreads();
            q[0] = q[1] = q[2] = 0.f;
            coop_points<NX, ROW_PHASE_R>(a, s_P, s_ph, loc, q);
            ok = coop_reduce(a, q, s_rd, a.T.part_row, &loc, red, &s_ok, &s_k);
        }
    }
    if (!ok) return;
    const double tn = __dadd_rn(t0, __dmul_rn((double)n, dt));
    if (!imag && cav) {                            // the closing half phase with alpha of the final density
        if (threadIdx.x == 0) s_ph = phase_dev(a, tn, hh);
        __syncthreads();
        coop_points<NX, ROW_PHASE>(a, s_P, s_ph, loc, q);
    } else if (imag) {                             // the pending normalisation
        coop_points<NX, ROW_SCALE>(a, s_P, s_ph, loc, q);
    }
}

// ------------------------------------------------------------------ states of a segment
// Real-time steps s0 .. s1 - 1 of a context without a cavity, each a whole
// V/2 - T - V/2 step (Eq. 3) as one gpe_step call of one step runs it, with
// every state kept: the row pass reads psi_s from st[s - s0] and writes into
// st[s - s0 + 1], where the column pass finishes psi_{s+1} in place (T_y and
// the closing half phase).  A fused run of several steps never holds
// psi_{s+1}: its closing half phase is merged into the next opening one.
// Step s opens at t0 + s dt and closes at that time plus dt, the times the
// adjoint passes of the same step take.  The checkpointed adjoint runs its
// forward sweep and each segment's recomputation through this kernel, so
// the states it recomputes are bit for bit the ones of the forward sweep.
template <int NX, int NY>
__global__ void __launch_bounds__(CoopCfg<NX, NY>::CT, CoopCfg<NX, NY>::CPS)
    coop_states_kernel(const __grid_constant__ CoopArgs a)
{
    using C = CoopCfg<NX, NY>;
    extern __shared__ unsigned char smraw[];
    __shared__ DevScalars loc;                     // c = 1, alpha = 0: no reduction on this path
    __shared__ PhaseArgs s_ph;
    __shared__ CoopPtrs s_P;
    __shared__ int s_ok;
    __shared__ unsigned int s_k;

    const uint32_t s0 = smem_u32(smraw);
    float4 *slots = reinterpret_cast<float4 *>(smraw + ((128u - (s0 & 127u)) & 127u));
    if (threadIdx.x == 0) {
        memset(&loc, 0, sizeof(loc));
        loc.c = 1.0;
        s_k = 0;
        s_P.T = a.T;
        s_P.V = a.V;
        s_ok = check_index((long long)((unsigned char *)slots + C::SLOT_BYTES - smraw) - 1, dyn_smem_bytes(), a.T.sc);
        if (!s_ok) atomicExch(&a.T.sc->bar_abort, 1u);
    }
    __syncthreads();
    if (!s_ok) return;
    const double hh = __dmul_rn(0.5, a.dt);
    float q[3] = {0.f, 0.f, 0.f};
    for (int s = a.s0; s < a.s1; ++s) {
        const double ts = __dadd_rn(a.t0, __dmul_rn((double)s, a.dt));
        const double te = __dadd_rn(ts, a.dt);
        const float2 *from = a.st + (size_t)(s - a.s0) * a.P;
        float2 *to = a.st + (size_t)(s + 1 - a.s0) * a.P;
        if (threadIdx.x == 0) s_ph = phase_dev(a, ts, hh);
        __syncthreads();
        coop_rows_pt<NX, C::CT, C::E>(a, s_P, s_ph, 0, loc, slots, from, to);
        if (!coop_sync(a, &s_ok, &s_k)) return;
        if (threadIdx.x == 0) s_ph = phase_dev(a, te, hh);
        __syncthreads();
        coop_cols<NY, NX, COL_T_P, C::CT, C::E>(a, s_P, s_ph, loc, slots, q, to);
        if (s + 1 < a.s1 && !coop_sync(a, &s_ok, &s_k)) return;
    }
}

// ------------------------------------------------------------------ adjoint segment
// The reverse sweep of one segment of the checkpointed adjoint (the
// discrete adjoint of the real-time step, Sec. 3.1, for a lattice-depth
// control, Eq. 9): for s = s1 - 1 down to s0, the adjoint row pass with the
// step's end state and the adjoint column pass with its start state, as
// row_kernel<ROW_ADJ> and col_kernel<COL_ADJ> compute them, on pencil pairs,
// separated by grid barriers.  Each pass's CTAs store their FP64 partials
// of its dJ/dv; the sums are taken in CTA order after a grid barrier every
// few hundred steps and at the end of the segment, off the passes' critical
// path (the per-pass kernels finish each sum in the CTA that ends last).  No
// cavity on this path.

// Row pass of step s on the row pairs of lambda: the adjoint of the closing
// half phase (its output psi2 = psi_{s+1} has the phase's density; its input
// is exp(+i theta) psi2), then T_x^H.  gq: sum of Im(conj(mu) in) L(r).
template <int N, int CT, int EE>
__device__ __noinline__ void coop_adj_rows(const CoopArgs &a, const CoopPtrs &P, const PhaseArgs &ph,
                                           const float2 *psi2, float4 *slots, float &gq, int base = 0)
{
    const Tables &T = P.T;
    using A = CoopAxis<N, CT, EE>;
    constexpr int E = A::E, TP = A::TP;
    const int units = a.ny / 2;
    const CoopUnits<N, CT, EE> U(base);
    float4 *sb = slots + U.g * A::SLOTS;
    const GroupSync gs{U.bid, TP};
    float acx2, acxcy;
    alpha_amps(ph, 0.0, 0.0, acx2, acxcy);
    for (int u = U.gg; u < units; u += U.G) {
        const bool act = check_index((long long)2 * u + 1, a.ny, T.sc);
        const int y0 = act ? 2 * u : 0;
        float2 *ra = a.lam + (size_t)y0 * N, *rb = ra + N;
        const float2 *oa = psi2 + (size_t)y0 * N, *ob = oa + N;
        const float4 ya = __ldg(&T.ytab[y0]), yb = __ldg(&T.ytab[y0 + 1]);
        const PotCoefs pa = row_coefs_from(ph, acx2, acxcy, ya), pb = row_coefs_from(ph, acx2, acxcy, yb);
        const float *Va = P.V ? P.V + (size_t)y0 * N : nullptr;
        // 8 elements per thread: the pointwise adjoint on the packed pair; 16
        // (1024-point rows): per row, which keeps the pass within 255 registers
        float2 X[E], Y[E];
        if constexpr (E == 8) {
            // lambda and psi_{s+1} of the two rows packed (row a, row b); V, then theta
            float2 OX[E], OY[E], V[E];
            bool small = true;
#pragma unroll
            for (int r = 0; r < E; ++r) {
                const int xi = U.j + r * TP;
                const float2 la = act ? __ldcg(ra + xi) : make_float2(0.f, 0.f);
                const float2 lb = act ? __ldcg(rb + xi) : make_float2(0.f, 0.f);
                const float2 o_a = act ? __ldcg(oa + xi) : make_float2(0.f, 0.f);
                const float2 o_b = act ? __ldcg(ob + xi) : make_float2(0.f, 0.f);
                X[r] = make_float2(la.x, lb.x);
                Y[r] = make_float2(la.y, lb.y);
                OX[r] = make_float2(o_a.x, o_b.x);
                OY[r] = make_float2(o_a.y, o_b.y);
                V[r] = pot_at2(pa, pb, __ldg(&T.xtab[xi]));
                if (Va) V[r] = fma2(bc2(a.V_scale), make_float2(__ldg(&Va[xi]), __ldg(&Va[N + xi])), V[r]);
                const float2 th = mul2(fma2(bc2(a.g), fma2(OX[r], OX[r], mul2(OY[r], OY[r])), V[r]), bc2(ph.h));
                small = small && fabsf(th.x) <= 1.f && fabsf(th.y) <= 1.f;
            }
            float2 g2 = make_float2(0.f, 0.f);
            if (small) {
                // the phase's input exp(+i theta) psi_{s+1}, then the adjoint of the
                // phase on it, both rotations in the packed Taylor form
#pragma unroll
                for (int r = 0; r < E; ++r) {
                    const int xi = U.j + r * TP;
                    const float2 th = mul2(fma2(bc2(a.g), fma2(OX[r], OX[r], mul2(OY[r], OY[r])), V[r]), bc2(ph.h));
                    float2 IX = OX[r], IY = OY[r];
                    rot2_taylor(IX, IY, make_float2(-th.x, -th.y));
                    const float2 thi = mul2(fma2(bc2(a.g), fma2(IX, IX, mul2(IY, IY)), V[r]), bc2(ph.h));
                    const float2 q = adjoint2_taylor(X[r], Y[r], IX, IY, thi, a.g, ph.h);
                    const float lx = a.L0x * __ldg(&T.xtab[xi]).y;
                    g2 = fma2(q, fma2(bc2(a.L0y), make_float2(ya.y, yb.y), bc2(lx)), g2);
                }
            } else {
#pragma unroll
                for (int r = 0; r < E; ++r) {
                    const int xi = U.j + r * TP;
                    const float4 xt = __ldg(&T.xtab[xi]);
                    float2 la = make_float2(X[r].x, Y[r].x), lb = make_float2(X[r].y, Y[r].y);
                    const float2 o_a = make_float2(OX[r].x, OY[r].x), o_b = make_float2(OX[r].y, OY[r].y);
                    const float tha = (V[r].x + a.g * (o_a.x * o_a.x + o_a.y * o_a.y)) * ph.h;
                    const float thb = (V[r].y + a.g * (o_b.x * o_b.x + o_b.y * o_b.y)) * ph.h;
                    g2.x += phase_adjoint(la, phase_rot(o_a, -tha), V[r].x, a.g, ph.h) * (a.L0x * xt.y + a.L0y * ya.y);
                    g2.y += phase_adjoint(lb, phase_rot(o_b, -thb), V[r].y, a.g, ph.h) * (a.L0x * xt.y + a.L0y * yb.y);
                    X[r] = make_float2(la.x, lb.x);
                    Y[r] = make_float2(la.y, lb.y);
                }
            }
            gq += g2.x + g2.y;
        } else {
#pragma unroll
            for (int r = 0; r < E; ++r) {
                const int xi = U.j + r * TP;
                const float4 xt = __ldg(&T.xtab[xi]);
                float2 la = act ? __ldcg(ra + xi) : make_float2(0.f, 0.f);
                float2 lb = act ? __ldcg(rb + xi) : make_float2(0.f, 0.f);
                const float2 o_a = act ? __ldcg(oa + xi) : make_float2(0.f, 0.f);
                const float2 o_b = act ? __ldcg(ob + xi) : make_float2(0.f, 0.f);
                float Vxa = pot_at(pa, xt), Vxb = pot_at(pb, xt);
                if (Va) {
                    Vxa += a.V_scale * __ldg(&Va[xi]);
                    Vxb += a.V_scale * __ldg(&Va[N + xi]);
                }
                const float tha = (Vxa + a.g * (o_a.x * o_a.x + o_a.y * o_a.y)) * ph.h;
                const float thb = (Vxb + a.g * (o_b.x * o_b.x + o_b.y * o_b.y)) * ph.h;
                gq += phase_adjoint(la, phase_rot(o_a, -tha), Vxa, a.g, ph.h) * (a.L0x * xt.y + a.L0y * ya.y);
                gq += phase_adjoint(lb, phase_rot(o_b, -thb), Vxb, a.g, ph.h) * (a.L0x * xt.y + a.L0y * yb.y);
                X[r] = make_float2(la.x, lb.x);
                Y[r] = make_float2(la.y, lb.y);
            }
        }
        transform_pair<N, E, TP, GroupSync, true>(X, Y, sb, U.j, E == 8 ? T.tw8x : T.twx, T.kinx, a.sx, 0, gs);
        if (act) {
#pragma unroll
            for (int r = 0; r < E; ++r) {
                const int xi = U.j + r * TP;
                __stcg(ra + xi, make_float2(X[r].x, Y[r].x));
                __stcg(rb + xi, make_float2(X[r].y, Y[r].y));
            }
        }
    }
}

// Column pass of step s on the column pairs of lambda: T_y^H, then the
// adjoint of the opening half phase, whose input psi2 = psi_s is the step's
// start state.  gq as in the row pass.
template <int N, int NX, int CT, int EE>
__device__ __noinline__ void coop_adj_cols(const CoopArgs &a, const CoopPtrs &P, const PhaseArgs &ph,
                                           const float2 *psi2, float4 *slots, float &gq, int base = 0)
{
    const Tables &T = P.T;
    using A = CoopAxis<N, CT, EE>;
    constexpr int E = A::E, TP = A::TP;
    constexpr int units = NX / 2, w4 = NX / 2;
    const CoopUnits<N, CT, EE> U(base);
    float4 *sb = slots + U.g * A::SLOTS;
    const GroupSync gs{U.bid, TP};
    float acx2, acxcy;
    alpha_amps(ph, 0.0, 0.0, acx2, acxcy);
    for (int u = U.gg; u < units; u += U.G) {
        const bool act = check_index((long long)2 * u + 1, NX, T.sc);
        const int x0 = act ? 2 * u : 0;
        float4 *cb = reinterpret_cast<float4 *>(a.lam + x0) + (size_t)U.j * w4;
        const float4 *ib = reinterpret_cast<const float4 *>(psi2 + x0) + (size_t)U.j * w4;
        float2 X[E], Y[E];
        // psi_s loaded before the transform rather than after it, where the
        // registers allow (8 elements per thread; 16 would spill)
        constexpr bool EARLY = E == 8;
        float4 in[EARLY ? E : 1];
#pragma unroll
        for (int r = 0; r < E; ++r) {
            const float4 t = act ? __ldcg(cb + r * TP * w4) : make_float4(0.f, 0.f, 0.f, 0.f);
            if constexpr (EARLY) in[r] = act ? __ldcg(ib + r * TP * w4) : make_float4(0.f, 0.f, 0.f, 0.f);
            X[r] = make_float2(t.x, t.z);
            Y[r] = make_float2(t.y, t.w);
        }
        transform_pair<N, E, TP, GroupSync, true>(X, Y, sb, U.j, E == 8 ? T.tw8y : T.twy, T.kiny, a.sy, 0, gs);
        const float4 xa = __ldg(&T.xtab[x0]), xb = __ldg(&T.xtab[x0 + 1]);
        const PotCoefs pa = col_coefs_from(ph, acx2, acxcy, xa), pb = col_coefs_from(ph, acx2, acxcy, xb);
        if constexpr (E == 8) {
            // psi_s of the two columns packed (column a, column b); V, then theta
            float2 PX[E], PY[E], V[E];
            bool small = true;
#pragma unroll
            for (int r = 0; r < E; ++r) {
                const int y = U.j + r * TP;
                const float4 pin = in[r];
                PX[r] = make_float2(pin.x, pin.z);
                PY[r] = make_float2(pin.y, pin.w);
                V[r] = pot_at2(pa, pb, __ldg(&T.ytab[y]));
                if (P.V)
                    V[r] = fma2(bc2(a.V_scale),
                                make_float2(__ldg(&P.V[(size_t)y * NX + x0]), __ldg(&P.V[(size_t)y * NX + x0 + 1])),
                                V[r]);
                const float2 th = mul2(fma2(bc2(a.g), fma2(PX[r], PX[r], mul2(PY[r], PY[r])), V[r]), bc2(ph.h));
                small = small && fabsf(th.x) <= 1.f && fabsf(th.y) <= 1.f;
            }
            float2 g2 = make_float2(0.f, 0.f);
            if (small) {
#pragma unroll
                for (int r = 0; r < E; ++r) {
                    const float2 th = mul2(fma2(bc2(a.g), fma2(PX[r], PX[r], mul2(PY[r], PY[r])), V[r]), bc2(ph.h));
                    const float2 q = adjoint2_taylor(X[r], Y[r], PX[r], PY[r], th, a.g, ph.h);
                    const float ly = a.L0y * __ldg(&T.ytab[U.j + r * TP]).y;
                    g2 = fma2(q, fma2(bc2(a.L0x), make_float2(xa.y, xb.y), bc2(ly)), g2);
                }
            } else {
#pragma unroll
                for (int r = 0; r < E; ++r) {
                    const float4 yt = __ldg(&T.ytab[U.j + r * TP]);
                    float2 la = make_float2(X[r].x, Y[r].x), lb = make_float2(X[r].y, Y[r].y);
                    g2.x += phase_adjoint(la, make_float2(PX[r].x, PY[r].x), V[r].x, a.g, ph.h) *
                            (a.L0x * xa.y + a.L0y * yt.y);
                    g2.y += phase_adjoint(lb, make_float2(PX[r].y, PY[r].y), V[r].y, a.g, ph.h) *
                            (a.L0x * xb.y + a.L0y * yt.y);
                    X[r] = make_float2(la.x, lb.x);
                    Y[r] = make_float2(la.y, lb.y);
                }
            }
            gq += g2.x + g2.y;
        } else {
#pragma unroll
            for (int r = 0; r < E; ++r) {
                const int y = U.j + r * TP;
                const float4 yt = __ldg(&T.ytab[y]);
                float Vya = pot_at(pa, yt), Vyb = pot_at(pb, yt);
                if (P.V) {
                    Vya += a.V_scale * __ldg(&P.V[(size_t)y * NX + x0]);
                    Vyb += a.V_scale * __ldg(&P.V[(size_t)y * NX + x0 + 1]);
                }
                const float4 pin = act ? __ldcg(ib + r * TP * w4) : make_float4(0.f, 0.f, 0.f, 0.f);
                float2 la = make_float2(X[r].x, Y[r].x), lb = make_float2(X[r].y, Y[r].y);
                gq += phase_adjoint(la, make_float2(pin.x, pin.y), Vya, a.g, ph.h) * (a.L0x * xa.y + a.L0y * yt.y);
                gq += phase_adjoint(lb, make_float2(pin.z, pin.w), Vyb, a.g, ph.h) * (a.L0x * xb.y + a.L0y * yt.y);
                X[r] = make_float2(la.x, lb.x);
                Y[r] = make_float2(la.y, lb.y);
            }
        }
        if (act) {
#pragma unroll
            for (int r = 0; r < E; ++r) __stcg(cb + r * TP * w4, make_float4(X[r].x, Y[r].x, X[r].y, Y[r].y));
        }
    }
}

// The dJ/dv partials of an adjoint sweep (coop_adj_kernel, coop_rev_kernel):
// step s's row-pass partial of CTA b sits at part_row[(hi - s) G + b] and its
// column-pass partial at part_col[(hi - s) G + b], hi the latest step since
// the last flush.  Called by every thread after a grid barrier: sums the m =
// hi - lo + 1 steps' partials, one warp per sum, in CTA order (the same in
// every run), into gout[2 s + 1] (row) and gout[2 s] (column).
__device__ void coop_flush_grad(const CoopArgs &a, int hi, int lo)
{
    const int G = (int)gridDim.x, m = hi - lo + 1, W = (int)(blockDim.x >> 5), lane = threadIdx.x & 31;
    for (int i = blockIdx.x * W + (int)(threadIdx.x >> 5); i < 2 * m; i += G * W) {
        const double *src = ((i & 1) ? a.T.part_row : a.T.part_col) + (size_t)(i >> 1) * G;
        double acc = 0.0;
        for (int b = lane; b < G; b += 32) acc += __ldcg(&src[b]);
        for (int off = 16; off > 0; off >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, off);
        if (lane == 0) a.gout[2 * (hi - (i >> 1)) + (i & 1)] = acc;
    }
}

template <int NX, int NY>
__global__ void __launch_bounds__(CoopCfg<NX, NY>::CT, CoopCfg<NX, NY>::CPS)
    coop_adj_kernel(const __grid_constant__ CoopArgs a)
{
    using C = CoopCfg<NX, NY>;
    extern __shared__ unsigned char smraw[];
    __shared__ double red[32 * NQ];
    __shared__ PhaseArgs s_ph;
    __shared__ CoopPtrs s_P;
    __shared__ int s_ok;
    __shared__ unsigned int s_k;

    const uint32_t s0 = smem_u32(smraw);
    float4 *slots = reinterpret_cast<float4 *>(smraw + ((128u - (s0 & 127u)) & 127u));
    if (threadIdx.x == 0) {
        s_k = 0;
        s_P.T = a.T;
        s_P.V = a.V;
        s_ok = check_index((long long)((unsigned char *)slots + C::SLOT_BYTES - smraw) - 1, dyn_smem_bytes(), a.T.sc);
        if (!s_ok) atomicExch(&a.T.sc->bar_abort, 1u);
    }
    __syncthreads();
    if (!s_ok) return;
    const double hh = __dmul_rn(0.5, a.dt);
    // dJ/dv partials: step s's row-pass partial of CTA b at part_row[j G + b]
    // and its column-pass partial at part_col[j G + b], j = hi - s counting
    // the steps since the last flush (hi); every R steps, and at the end, the
    // 2 R sums are taken after a grid barrier, so no pass waits on them
    const int G = (int)gridDim.x, R = NQ * MAX_BLOCKS / G;
    int hi = a.s1 - 1;
    for (int s = a.s1 - 1; s >= a.s0; --s) {
        // the times of the step's closing and opening half phases, as the
        // host computes them (t0 + s dt + dt, t0 + s dt)
        const double ts = __dadd_rn(a.t0, __dmul_rn((double)s, a.dt));
        const double te = __dadd_rn(ts, a.dt);
        const size_t slot = (size_t)(hi - s) * G + blockIdx.x;
        // psi_s, which the column pass reads, into L2 during the row pass:
        // the segment's states outgrow L2 (65 x 2 MB at 512^2), and the
        // column pass would otherwise wait on DRAM after its transform
        prefetch_l2_share(a.st + (size_t)(s - a.s0) * a.P, sizeof(float2) * (size_t)NX * NY);
        if (threadIdx.x == 0) s_ph = phase_dev(a, te, hh);
        __syncthreads();
        float gq = 0.f;
        coop_adj_rows<NX, C::CT, C::E>(a, s_P, s_ph, a.st + (size_t)(s + 1 - a.s0) * a.P, slots, gq);
        float q1[1] = {2.f * s_ph.h * gq};
        block_sum<1>(q1, a.T.part_row + slot, red);
        if (!coop_sync(a, &s_ok, &s_k)) return;
        if (threadIdx.x == 0) s_ph = phase_dev(a, ts, hh);
        __syncthreads();
        gq = 0.f;
        coop_adj_cols<NY, NX, C::CT, C::E>(a, s_P, s_ph, a.st + (size_t)(s - a.s0) * a.P, slots, gq);
        q1[0] = 2.f * s_ph.h * gq;
        block_sum<1>(q1, a.T.part_col + slot, red);
        if (!coop_sync(a, &s_ok, &s_k)) return;
        if (hi - s + 1 == R || s == a.s0) {         // a barrier before the slots are written again
            coop_flush_grad(a, hi, s);
            hi = s - 1;
            if (s > a.s0 && !coop_sync(a, &s_ok, &s_k)) return;
        }
    }
}

// ------------------------------------------------------------------ adjoint and recomputation side by side
// One epoch per step: the adjoint passes of segment k (steps s1 - 1 down to
// s0, on st) on threads [0, CT) of each CTA, and the recomputation of segment
// k - 1 (steps r0 .. r1 - 1, into st2) on threads [CT, 2 CT), with the pass
// functions of coop_adj_kernel and coop_states_kernel, each role with its own
// groups, exchange slots and named barriers.  Both programs take two grid
// barriers per step, so they share them: epoch i runs adjoint step s1 - 1 - i
// and recomputation step r0 + i (either only while it has steps left).  The
// two roles touch different buffers (lambda and st; st2).  Every pass on
// one CTA runs as one warp per scheduler and waits on its own latency, so two
// roles per SM take little longer than one.  The recomputation role adds
// exact zeros to the CTA's dJ/dv partial, so the gradient is bit for bit that
// of coop_adj_kernel; the recomputed states are bit for bit coop_states_kernel's.
template <int NX, int NY>
__global__ void __launch_bounds__(2 * CoopCfg<NX, NY>::CT, 1) coop_adjrec_kernel(const __grid_constant__ CoopArgs a)
{
    using C = CoopCfg<NX, NY>;
    static_assert(C::CPS == 1, "one CTA of both roles per SM");
    extern __shared__ unsigned char smraw[];
    __shared__ double red[32 * NQ];
    __shared__ DevScalars loc;                     // c = 1, alpha = 0 for the recomputation
    __shared__ PhaseArgs s_ph, s_phr;
    __shared__ CoopPtrs s_P;
    __shared__ int s_ok;
    __shared__ unsigned int s_k;

    const uint32_t s0 = smem_u32(smraw);
    float4 *slots = reinterpret_cast<float4 *>(smraw + ((128u - (s0 & 127u)) & 127u));
    if (threadIdx.x == 0) {
        memset(&loc, 0, sizeof(loc));
        loc.c = 1.0;
        s_k = 0;
        s_P.T = a.T;
        s_P.V = a.V;
        s_ok = check_index((long long)((unsigned char *)slots + 2 * C::SLOT_BYTES - smraw) - 1, dyn_smem_bytes(),
                           a.T.sc);
        if (!s_ok) atomicExch(&a.T.sc->bar_abort, 1u);
    }
    __syncthreads();
    if (!s_ok) return;
    const bool rec = threadIdx.x >= C::CT;         // whole warps: CT is a multiple of 32
    float4 *my = slots + (rec ? C::SLOT_BYTES / sizeof(float4) : 0);
    const double hh = __dmul_rn(0.5, a.dt);
    const int G = (int)gridDim.x, R = NQ * MAX_BLOCKS / G;
    const int m = a.s1 - a.s0, mr = a.r1 - a.r0, epochs = m > mr ? m : mr;
    float q[3] = {0.f, 0.f, 0.f};
    int hi = a.s1 - 1;
    for (int i = 0; i < epochs; ++i) {
        const bool adj = i < m, rc = i < mr;
        const int s = a.s1 - 1 - i, sr = a.r0 + i;
        const double ts = __dadd_rn(a.t0, __dmul_rn((double)s, a.dt)), te = __dadd_rn(ts, a.dt);
        const double tr = __dadd_rn(a.t0, __dmul_rn((double)sr, a.dt)), tre = __dadd_rn(tr, a.dt);
        const size_t slot = (size_t)(hi - s) * G + blockIdx.x;
        if (adj) prefetch_l2_share(a.st + (size_t)(s - a.s0) * a.P, sizeof(float2) * (size_t)NX * NY);
        if (threadIdx.x == 0) {
            if (adj) s_ph = phase_dev(a, te, hh);
            if (rc) s_phr = phase_dev(a, tr, hh);
        }
        __syncthreads();
        float gq = 0.f;
        if (!rec) {
            if (adj) coop_adj_rows<NX, C::CT, C::E>(a, s_P, s_ph, a.st + (size_t)(s + 1 - a.s0) * a.P, my, gq, 0);
        } else if (rc) {
            coop_rows_pt<NX, C::CT, C::E>(a, s_P, s_phr, 0, loc, my, a.st2 + (size_t)(sr - a.r0) * a.P,
                                          a.st2 + (size_t)(sr + 1 - a.r0) * a.P, C::CT);
        }
        float q1[1] = {adj ? 2.f * s_ph.h * gq : 0.f};
        if (adj) block_sum<1>(q1, a.T.part_row + slot, red);
        if (!coop_sync(a, &s_ok, &s_k)) return;
        if (threadIdx.x == 0) {
            if (adj) s_ph = phase_dev(a, ts, hh);
            if (rc) s_phr = phase_dev(a, tre, hh);
        }
        __syncthreads();
        gq = 0.f;
        if (!rec) {
            if (adj) coop_adj_cols<NY, NX, C::CT, C::E>(a, s_P, s_ph, a.st + (size_t)(s - a.s0) * a.P, my, gq, 0);
        } else if (rc) {
            coop_cols<NY, NX, COL_T_P, C::CT, C::E>(a, s_P, s_phr, loc, my, q, a.st2 + (size_t)(sr + 1 - a.r0) * a.P,
                                                    C::CT);
        }
        q1[0] = adj ? 2.f * s_ph.h * gq : 0.f;
        if (adj) block_sum<1>(q1, a.T.part_col + slot, red);
        if (i + 1 < epochs || adj) {
            if (!coop_sync(a, &s_ok, &s_k)) return;
        }
        if (adj && (hi - s + 1 == R || s == a.s0)) {
            coop_flush_grad(a, hi, s);
            hi = s - 1;
            if (s > a.s0 && !coop_sync(a, &s_ok, &s_k)) return;
        }
    }
}

// ------------------------------------------------------------------ reverse sweep by time reversal
// The reverse sweep without checkpoints (GPE_ADJ_REVERSE) in one launch: for
// s = s1 - 1 down to s0, the adjoint row pass on psi_{s+1} (the context's
// psi), one real-time step of -dt from t_{s+1} that turns psi into psi_s (the
// conjugate opening half phase at t_{s+1}, T(-dt) from the kinetic tables
// kxb / kyb, the conjugate closing half phase at t_s), then the adjoint
// column pass on psi_s.  Two phases and two grid barriers per step: the
// adjoint row pass and the step back's row pass run on the same row pairs
// one after the other, as do the step back's column pass and the adjoint
// column pass on the same column pairs.  Within a pair every thread reads and
// writes its own elements only (the same ones in every pass), so each
// element of psi is read by the adjoint row pass before the step back
// overwrites it, and the adjoint column pass reads psi_s that the same
// thread has just stored; consecutive transforms of a group are ordered by
// the barriers inside each exchange.  The dJ/dv partials as in
// coop_adj_kernel.
template <int NX, int NY>
__global__ void __launch_bounds__(CoopCfg<NX, NY>::CT, CoopCfg<NX, NY>::CPS)
    coop_rev_kernel(const __grid_constant__ CoopArgs a)
{
    using C = CoopCfg<NX, NY>;
    extern __shared__ unsigned char smraw[];
    __shared__ double red[32 * NQ];
    __shared__ DevScalars loc;                     // c = 1, alpha = 0 for the step back
    __shared__ PhaseArgs s_ph, s_ph2;
    __shared__ CoopPtrs s_P, s_Pb;                 // kinetic tables of +dt (adjoint) and -dt (step back)
    __shared__ int s_ok;
    __shared__ unsigned int s_k;

    const uint32_t s0 = smem_u32(smraw);
    float4 *slots = reinterpret_cast<float4 *>(smraw + ((128u - (s0 & 127u)) & 127u));
    if (threadIdx.x == 0) {
        memset(&loc, 0, sizeof(loc));
        loc.c = 1.0;
        s_k = 0;
        s_P.T = a.T;
        s_P.V = a.V;
        s_Pb = s_P;
        s_Pb.T.kinx = const_cast<float2 *>(a.kxb);
        s_Pb.T.kiny = const_cast<float2 *>(a.kyb);
        s_ok = check_index((long long)((unsigned char *)slots + C::SLOT_BYTES - smraw) - 1, dyn_smem_bytes(), a.T.sc);
        if (!s_ok) atomicExch(&a.T.sc->bar_abort, 1u);
    }
    __syncthreads();
    if (!s_ok) return;
    const double hh = __dmul_rn(0.5, a.dt), mh = -hh;
    const int G = (int)gridDim.x, R = NQ * MAX_BLOCKS / G;
    float q[3] = {0.f, 0.f, 0.f};
    int hi = a.s1 - 1;
    for (int s = a.s1 - 1; s >= a.s0; --s) {
        const double ts = __dadd_rn(a.t0, __dmul_rn((double)s, a.dt));
        const double te = __dadd_rn(ts, a.dt);
        const size_t slot = (size_t)(hi - s) * G + blockIdx.x;
        // rows: the adjoint row pass with psi_{s+1}, then psi's opening phase
        // and T_x of the step of -dt
        if (threadIdx.x == 0) {
            s_ph = phase_dev(a, te, hh);
            s_ph2 = phase_dev(a, te, mh);
        }
        __syncthreads();
        float gq = 0.f;
        coop_adj_rows<NX, C::CT, C::E>(a, s_P, s_ph, a.psi, slots, gq);
        coop_rows_pt<NX, C::CT, C::E>(a, s_Pb, s_ph2, 0, loc, slots, a.psi, a.psi);
        float q1[1] = {2.f * s_ph.h * gq};
        block_sum<1>(q1, a.T.part_row + slot, red);
        if (!coop_sync(a, &s_ok, &s_k)) return;
        // columns: T_y and the closing phase of the step of -dt (psi <- psi_s),
        // then the adjoint column pass with psi_s
        if (threadIdx.x == 0) {
            s_ph = phase_dev(a, ts, mh);
            s_ph2 = phase_dev(a, ts, hh);
        }
        __syncthreads();
        coop_cols<NY, NX, COL_T_P, C::CT, C::E>(a, s_Pb, s_ph, loc, slots, q, a.psi);
        gq = 0.f;
        coop_adj_cols<NY, NX, C::CT, C::E>(a, s_P, s_ph2, a.psi, slots, gq);
        q1[0] = 2.f * s_ph2.h * gq;
        block_sum<1>(q1, a.T.part_col + slot, red);
        if (!coop_sync(a, &s_ok, &s_k)) return;
        if (hi - s + 1 == R || s == a.s0) {
            coop_flush_grad(a, hi, s);
            hi = s - 1;
            if (s > a.s0 && !coop_sync(a, &s_ok, &s_k)) return;
        }
    }
}

// ------------------------------------------------------------------ reverse sweep, two roles
// The reverse sweep by time reversal on 512^2 in 256-thread CTAs: threads
// [0, CT) run the adjoint passes of step s (row pass with psi_{s+1}, column
// pass with psi_s) while threads [CT, 2 CT) run the step of -dt one step
// ahead, psi_s -> psi_{s-1} (row pass from psi_s into the next buffer, column
// pass there in place), with the pass functions and times of
// coop_rev_kernel.  psi_k lives in buffer (s1 - k) mod 3 of {psi, st, st2}:
// in each epoch the step back writes only psi_{s-1}'s buffer, which the
// adjoint role does not read before the next step.  A prologue takes the
// step back of step s1 - 1 alone.  Both roles share the two grid barriers of
// each step; the step-back role adds exact zeros to the dJ/dv partials, so
// gradient and states are coop_rev_kernel's bit for bit.  On return psi_{s0}
// is in buffer (s1 - s0) mod 3.
template <int NX, int NY>
__global__ void __launch_bounds__(2 * CoopCfg<NX, NY>::CT, 1) coop_rev2_kernel(const __grid_constant__ CoopArgs a)
{
    using C = CoopCfg<NX, NY>;
    static_assert(C::CPS == 1, "one CTA of both roles per SM");
    extern __shared__ unsigned char smraw[];
    __shared__ double red[32 * NQ];
    __shared__ DevScalars loc;                     // c = 1, alpha = 0 for the step back
    __shared__ PhaseArgs s_ph, s_phb;
    __shared__ CoopPtrs s_P, s_Pb;                 // kinetic tables of +dt (adjoint) and -dt (step back)
    __shared__ int s_ok;
    __shared__ unsigned int s_k;

    const uint32_t s0 = smem_u32(smraw);
    float4 *slots = reinterpret_cast<float4 *>(smraw + ((128u - (s0 & 127u)) & 127u));
    if (threadIdx.x == 0) {
        memset(&loc, 0, sizeof(loc));
        loc.c = 1.0;
        s_k = 0;
        s_P.T = a.T;
        s_P.V = a.V;
        s_Pb = s_P;
        s_Pb.T.kinx = const_cast<float2 *>(a.kxb);
        s_Pb.T.kiny = const_cast<float2 *>(a.kyb);
        s_ok = check_index((long long)((unsigned char *)slots + 2 * C::SLOT_BYTES - smraw) - 1, dyn_smem_bytes(),
                           a.T.sc);
        if (!s_ok) atomicExch(&a.T.sc->bar_abort, 1u);
    }
    __syncthreads();
    if (!s_ok) return;
    const bool back = threadIdx.x >= C::CT;        // whole warps: CT is a multiple of 32
    float4 *my = slots + (back ? C::SLOT_BYTES / sizeof(float4) : 0);
    float2 *const buf[3] = {a.psi, a.st, a.st2};
    auto state = [&](int k) { return buf[(a.s1 - k) % 3]; };
    const double hh = __dmul_rn(0.5, a.dt), mh = -hh;
    const int G = (int)gridDim.x, R = NQ * MAX_BLOCKS / G;
    float q[3] = {0.f, 0.f, 0.f};
    // the step back of step r: the conjugate opening phase at t_{r+1}, T(-dt),
    // the conjugate closing phase at t_r, psi_{r+1} -> psi_r; row half
    // (phase 0) or column half (phase 1), run by the step-back role
    auto step_back = [&](int r, int half) {
        if (!back) return;
        if (half == 0)
            coop_rows_pt<NX, C::CT, C::E>(a, s_Pb, s_phb, 0, loc, my, state(r + 1), state(r), C::CT);
        else
            coop_cols<NY, NX, COL_T_P, C::CT, C::E>(a, s_Pb, s_phb, loc, my, q, state(r), C::CT);
    };
    auto back_phase = [&](int r, int half) {
        const double tr = __dadd_rn(a.t0, __dmul_rn((double)r, a.dt));
        return half == 0 ? phase_dev(a, __dadd_rn(tr, a.dt), mh) : phase_dev(a, tr, mh);
    };
    // prologue: psi_{s1 - 1}
    for (int half = 0; half < 2; ++half) {
        if (threadIdx.x == 0) s_phb = back_phase(a.s1 - 1, half);
        __syncthreads();
        step_back(a.s1 - 1, half);
        if (!coop_sync(a, &s_ok, &s_k)) return;
    }
    int hi = a.s1 - 1;
    for (int s = a.s1 - 1; s >= a.s0; --s) {
        const bool ahead = s - 1 >= a.s0;          // the step back of step s - 1 runs beside this step
        const double ts = __dadd_rn(a.t0, __dmul_rn((double)s, a.dt));
        const double te = __dadd_rn(ts, a.dt);
        const size_t slot = (size_t)(hi - s) * G + blockIdx.x;
        if (threadIdx.x == 0) {
            s_ph = phase_dev(a, te, hh);
            if (ahead) s_phb = back_phase(s - 1, 0);
        }
        __syncthreads();
        float gq = 0.f;
        if (!back) coop_adj_rows<NX, C::CT, C::E>(a, s_P, s_ph, state(s + 1), my, gq, 0);
        else if (ahead) step_back(s - 1, 0);
        float q1[1] = {back ? 0.f : 2.f * s_ph.h * gq};
        block_sum<1>(q1, a.T.part_row + slot, red);
        if (!coop_sync(a, &s_ok, &s_k)) return;
        if (threadIdx.x == 0) {
            s_ph = phase_dev(a, ts, hh);
            if (ahead) s_phb = back_phase(s - 1, 1);
        }
        __syncthreads();
        gq = 0.f;
        if (!back) coop_adj_cols<NY, NX, C::CT, C::E>(a, s_P, s_ph, state(s), my, gq, 0);
        else if (ahead) step_back(s - 1, 1);
        q1[0] = back ? 0.f : 2.f * s_ph.h * gq;
        block_sum<1>(q1, a.T.part_col + slot, red);
        if (!coop_sync(a, &s_ok, &s_k)) return;
        if (hi - s + 1 == R || s == a.s0) {
            coop_flush_grad(a, hi, s);
            hi = s - 1;
            if (s > a.s0 && !coop_sync(a, &s_ok, &s_k)) return;
        }
    }
}

// ------------------------------------------------------------------ launch
bool coop_ok(int nx, int ny) { return (nx == 512 || nx == 1024) && (ny == 512 || ny == 1024); }

// One cooperative launch of kernel K<NX, NY>: every CTA resident (CPS per
// SM), or cudaErrorCooperativeLaunchTooLarge without launching.  `attr`
// remembers the devices whose shared-memory limit was raised for K.
template <int NX, int NY>
static cudaError_t coop_go(void (*K)(CoopArgs), std::atomic<unsigned long long> &attr, const CoopArgs &a,
                           cudaStream_t s, int roles = 1)
{
    using C = CoopCfg<NX, NY>;
    const int threads = roles * C::CT;
    const size_t smem = roles * C::SLOT_BYTES + 128;
    const cudaError_t e = smem_opt_in(K, (int)smem, attr);
    if (e != cudaSuccess) return e;
    int per = 0;
    const cudaError_t r = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, K, threads, smem);
    if (r != cudaSuccess) return r;
    if (per < C::CPS) return cudaErrorCooperativeLaunchTooLarge;
    const int grid = C::CPS * sm_count();          // all resident
    if (grid < 1) return cudaErrorInvalidValue;
    void *args[] = {const_cast<CoopArgs *>(&a)};
    return cudaLaunchCooperativeKernel((const void *)K, dim3(grid), dim3(threads), args, smem, s);
}

enum { COOP_STEPS, COOP_STATES, COOP_ADJ, COOP_REV };

template <int NX, int NY> static cudaError_t coop_launch(int which, const CoopArgs &a, cudaStream_t s)
{
    static std::atomic<unsigned long long> attr[4];
    if (which == COOP_STATES) return coop_go<NX, NY>(coop_states_kernel<NX, NY>, attr[1], a, s);
    if (which == COOP_ADJ) return coop_go<NX, NY>(coop_adj_kernel<NX, NY>, attr[2], a, s);
    if (which == COOP_REV) return coop_go<NX, NY>(coop_rev_kernel<NX, NY>, attr[3], a, s);
    return coop_go<NX, NY>(coop_kernel<NX, NY>, attr[0], a, s);
}

static cudaError_t coop_dispatch(int which, const CoopArgs &a, cudaStream_t s)
{
    if (a.nx == 512) return a.ny == 512 ? coop_launch<512, 512>(which, a, s) : coop_launch<512, 1024>(which, a, s);
    return a.ny == 512 ? coop_launch<1024, 512>(which, a, s) : coop_launch<1024, 1024>(which, a, s);
}

cudaError_t launch_coop_adj(const CoopArgs &a, cudaStream_t s)
{
    if (!coop_ok(a.nx, a.ny) || a.cavity || a.nctrl < 0 || a.nctrl > COOP_MAX_CTRL || a.s1 <= a.s0)
        return cudaErrorInvalidValue;
    return coop_dispatch(COOP_ADJ, a, s);
}

bool coop_adjrec_ok(int nx, int ny) { return nx == 512 && ny == 512; }

cudaError_t launch_coop_adjrec(const CoopArgs &a, cudaStream_t s)
{
    if (!coop_adjrec_ok(a.nx, a.ny) || a.cavity || a.imag || a.nctrl < 0 || a.nctrl > COOP_MAX_CTRL ||
        a.s1 <= a.s0 || a.r1 < a.r0 || !a.st2)
        return cudaErrorInvalidValue;
    static std::atomic<unsigned long long> attr{0};
    return coop_go<512, 512>(coop_adjrec_kernel<512, 512>, attr, a, s, 2);
}

cudaError_t launch_coop_rev2(const CoopArgs &a, cudaStream_t s)
{
    if (!coop_adjrec_ok(a.nx, a.ny) || a.cavity || a.imag || a.nctrl < 0 || a.nctrl > COOP_MAX_CTRL ||
        a.s1 <= a.s0 || !a.kxb || !a.kyb || !a.st || !a.st2)
        return cudaErrorInvalidValue;
    static std::atomic<unsigned long long> attr{0};
    return coop_go<512, 512>(coop_rev2_kernel<512, 512>, attr, a, s, 2);
}

cudaError_t launch_coop_rev(const CoopArgs &a, cudaStream_t s)
{
    if (!coop_ok(a.nx, a.ny) || a.cavity || a.imag || a.nctrl < 0 || a.nctrl > COOP_MAX_CTRL || a.s1 <= a.s0 ||
        !a.kxb || !a.kyb)
        return cudaErrorInvalidValue;
    return coop_dispatch(COOP_REV, a, s);
}

cudaError_t launch_coop_states(const CoopArgs &a, cudaStream_t s)
{
    if (!coop_ok(a.nx, a.ny) || a.cavity || a.imag || a.nctrl < 0 || a.nctrl > COOP_MAX_CTRL || a.s1 <= a.s0)
        return cudaErrorInvalidValue;
    return coop_dispatch(COOP_STATES, a, s);
}

cudaError_t launch_coop(const CoopArgs &a, cudaStream_t s)
{
    if (!coop_ok(a.nx, a.ny) || a.nctrl < 0 || a.nctrl > COOP_MAX_CTRL) return cudaErrorInvalidValue;
    return coop_dispatch(COOP_STEPS, a, s);
}

}  // namespace gpe
