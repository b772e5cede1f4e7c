// gpe_kernels.cu -- sm_103a kernels of the split-step GPE propagator.
//
// A step of Sec. 3.1 (Eqs. 3-4), V/2 - T - V/2, is executed as passes over
// psi[ny][nx] in HBM, each pass one kernel reading and writing psi in place.
// The kinetic propagator F^-1 exp(-i (kx^2 + ky^2) dt / 2m) F factorises
// exactly into T_x T_y with T_a = F_a^-1 exp(-i ka^2 dt / 2m) F_a along one
// axis, so psi is in real space between passes:
//   row pass    (x, rows contiguous): potential phase (V(x,y,t) + g|psi|^2 and
//               the cavity terms of Eqs. 10-13, in registers), then T_x;
//   column pass (y, TMA-loaded tiles of W columns): T_y, then optionally the
//               closing half phase, with the norm and cavity overlaps
//               (Eqs. 14-15) reduced in FP64 from the result.
#include <cuda.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <atomic>

#include "../../include/gpe.h"
#include "gpe_device.cuh"
#include "gpe_fft.cuh"
#include "gpe_internal.h"

// GPE_PART selects which launchers (and so which kernel instantiations) this
// compilation emits, so that the build can compile the file in parts side by
// side: 0 tables and readout kernels, shared host helpers and the pass
// dispatchers; 1 row passes of 8..256 points; 2 row passes of 512..8192
// points (one-shot, grouped, streaming); 3 column passes of 8..256 points;
// 4 column passes of 512..8192 points (one-shot, streaming).  Undefined:
// everything.
#ifndef GPE_PART
#define GPE_PART -1
#endif
#define GPE_IN_PART(k) (GPE_PART < 0 || GPE_PART == (k))

namespace gpe {

// ------------------------------------------------------------------ row pass
template <int N> struct RowCfg {
    static constexpr int E = N >= 16 ? 16 : N;
    static constexpr int TP = N / E;
    static constexpr int PS = N + N / 16;          // padded pencil stride (float2)
    static constexpr int TWN = fft_tw_count(N);    // twiddle entries staged in shared memory
};

template <int N, int MODE>
__global__ void __launch_bounds__(N >= 8192 ? 512 : 256) row_kernel(const PassArgs a)
{
    using C = RowCfg<N>;
    constexpr int E = C::E, TP = C::TP;
    extern __shared__ float4 smem4[];
    __shared__ double red[32 * NQ];
    float4 *stw = smem4;                                     // twiddles (C::TWN entries)
    float2 *smem = reinterpret_cast<float2 *>(smem4 + C::TWN);

    const int lr = threadIdx.x / TP, j = threadIdx.x % TP;
    const int rpc = blockDim.x / TP;
    const Tables &T = a.T;
    // this thread's row of the grid, and its pencil's exchange buffer within
    // the launch's shared memory (checked in the bounds-check build)
    const bool inb = check_index((long long)blockIdx.x * rpc + lr, a.ny, T.sc) &&
                     check_index((long long)C::TWN * 16 + (long long)(lr + 1) * C::PS * 8 - 1, dyn_smem_bytes(), T.sc);
    const int y = inb ? blockIdx.x * rpc + lr : 0;
    float2 *row = a.psi + (size_t)y * N;
    float2 *sb = smem + (inb ? lr : 0) * C::PS;
    constexpr bool FFT = (MODE == ROW_PT || MODE == ROW_FFT_F || MODE == ROW_FFT_I || MODE == ROW_OBS ||
                          MODE == ROW_ADJ);
    __shared__ __align__(8) uint64_t twbar;
    if constexpr (FFT && C::TWN > 0) {
        if (threadIdx.x == 0) mbar_init(&twbar, 1);
        __syncthreads();
        if (threadIdx.x == 0 && check_index((long long)C::TWN * 16 - 1, dyn_smem_bytes(), T.sc)) {
            mbar_expect_tx(&twbar, twiddle_bytes<N>());
            stage_twiddles_async<N>(stw, T.twx, &twbar);
        }
    }

    float2 v[E];
#pragma unroll
    for (int r = 0; r < E; ++r) v[r] = inb ? __ldcs(&row[j + r * TP]) : make_float2(0.f, 0.f);   // streamed
    // live: the twiddle table arrived in time.  A CTA whose wait ran out lets
    // the copy land, then runs on without storing anything and adds zero
    // partial sums, so that every reduction still counts all of its CTAs.
    bool live = true;
    if constexpr (FFT && C::TWN > 0) {
        if (!__syncthreads_and(mbar_wait_bounded(&twbar, 0, a.spins))) {
            if (threadIdx.x == 0) latch_status(T.sc, GPE_ETIMEOUT);
            mbar_drain(&twbar, 0);
            live = false;
        }
    }
    const bool keep = live && inb;              // this thread's results may be stored
    if constexpr (MODE == ROW_SCALE) {
        const float c = (float)T.sc->c;
#pragma unroll
        for (int r = 0; r < E; ++r) v[r] = make_float2(v[r].x * c, v[r].y * c);
    }
    if constexpr (MODE == ROW_FFT_F) fft_pencil<N, E, false>(v, sb, j, 1, stw);
    if constexpr (MODE == ROW_FFT_I) {
        fft_pencil<N, E, true>(v, sb, j, 1, stw);
#pragma unroll
        for (int r = 0; r < E; ++r) v[r] = make_float2(v[r].x * a.sx, v[r].y * a.sx);
    }

    const float4 yt = T.ytab[y];
    constexpr bool PHASE = (MODE == ROW_PT || MODE == ROW_PHASE || MODE == ROW_PHASE_R);
    if constexpr (PHASE) {
        const PotCoefs pc = row_coefs(a, yt);
        float cs = 1.f;
        if (MODE == ROW_PT && a.use_c) cs = (float)T.sc->c;
        const float *Vr = a.V ? a.V + (size_t)y * N : nullptr;
#pragma unroll
        for (int r = 0; r < E; ++r) {
            const int xi = j + r * TP;
            float V = pot_at(pc, __ldg(&T.xtab[xi]));
            if (Vr) V += a.V_scale * __ldg(&Vr[xi]);
            v[r] = phase_mul(make_float2(v[r].x * cs, v[r].y * cs), V, a.g, a.ph.h, a.imag);
        }
    }

    constexpr bool REDUCE = (MODE == ROW_PHASE_R || MODE == ROW_REDUCE_R);
    if constexpr (REDUCE) {
        float q[3] = {0.f, 0.f, 0.f};
#pragma unroll
        for (int r = 0; r < E; ++r) {
            const float cx = __ldg(&T.xtab[j + r * TP]).z;
            const float n = v[r].x * v[r].x + v[r].y * v[r].y;
            q[0] += n;
            q[1] += cx * n;
            q[2] += cx * cx * n;
        }
        q[1] *= yt.z;
        if (!inb) q[0] = q[1] = q[2] = 0.f;
        block_sum<3>(q, T.part_row + (size_t)blockIdx.x * NQ, red);
        double S[3];
        if (last_block_total<3>(T.part_row, &T.sc->ticket[0], S, red) && threadIdx.x == 0)
            finalize_fields(S, a.red, T.sc);
    }

    if constexpr (MODE == ROW_OBS) {
        // observable sums of the real-space state: S0 |psi|^2, S1 V_static |psi|^2,
        // S2 |psi|^4, S3 cos cos |psi|^2, S4 cos^2(kc x)|psi|^2, S5 cos^2(kc y)|psi|^2,
        // then S6 = sum kx^2 |F_x psi|^2 (kinetic energy along x by Parseval)
        const PhaseArgs &p = a.ph;
        const float vrow = yt.x + p.a_laty * yt.y + p.a_pump * yt.z * yt.z;
        const float *Vr = a.V ? a.V + (size_t)y * N : nullptr;
        float q[7] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int r = 0; r < E; ++r) {
            const int xi = j + r * TP;
            const float4 xt = __ldg(&T.xtab[xi]);
            float V = vrow + xt.x + p.a_latx * xt.y;
            if (Vr) V += a.V_scale * __ldg(&Vr[xi]);
            const float n = v[r].x * v[r].x + v[r].y * v[r].y;
            q[0] += n;
            q[1] += V * n;
            q[2] += n * n;
            q[3] += xt.z * n;
            q[4] += xt.z * xt.z * n;
        }
        q[3] *= yt.z;
        q[5] = yt.z * yt.z * q[0];
        fft_pencil<N, E, false>(v, sb, j, 1, stw);
#pragma unroll
        for (int r = 0; r < E; ++r) {
            const int e = j + r * TP;
            const float kx = (float)(e < N / 2 ? e : e - N);   // in units of 2 pi / Lx
            q[6] += kx * kx * (v[r].x * v[r].x + v[r].y * v[r].y);
        }
        if (!keep)
#pragma unroll
            for (int i = 0; i < 7; ++i) q[i] = 0.f;
        block_sum<7>(q, T.part_row + (size_t)blockIdx.x * NQ, red);
        double S[7];
        if (last_block_total<7>(T.part_row, &T.sc->ticket[0], S, red) && threadIdx.x == 0)
#pragma unroll
            for (int i = 0; i < 7; ++i) T.sc->sums[0][i] = S[i];
        return;
    }

    if constexpr (MODE == ROW_PT) {
        fft_pencil<N, E, false>(v, sb, j, 1, stw);
        kinetic_axis<E, TP>(v, T.kinx, j, a.sx, a.imag);
        fft_pencil<N, E, true>(v, sb, j, 1, stw);
    }

    if constexpr (MODE == ROW_ADJ) {
        // v = lambda after the step; psi2 = the step's output, whose density
        // is the closing phase's (a phase keeps |psi|), so the phase input is
        // exp(+i theta) psi2 and Im(conj(mu) input) = Im(conj(lambda) psi2)
        const PotCoefs pc = row_coefs(a, yt);
        const float2 *p2 = a.psi2 + (size_t)y * N;
        float gq = 0.f;
#pragma unroll
        for (int r = 0; r < E; ++r) {
            const int xi = j + r * TP;
            const float4 xt = __ldg(&T.xtab[xi]);
            float V = pot_at(pc, xt);
            if (a.V) V += a.V_scale * __ldg(&a.V[(size_t)y * N + xi]);
            const float2 o = __ldg(&p2[xi]);
            const float th = (V + a.g * (o.x * o.x + o.y * o.y)) * a.ph.h;
            const float2 in = phase_rot(o, -th);               // the phase's input
            float2 lam = v[r];
            gq += phase_adjoint(lam, in, V, a.g, a.ph.h) * (a.L0x * xt.y + a.L0y * yt.y);
            v[r] = lam;
        }
        fft_pencil<N, E, false>(v, sb, j, 1, stw);
        kinetic_axis<E, TP, true>(v, T.kinx, j, a.sx, 0);
        fft_pencil<N, E, true>(v, sb, j, 1, stw);
        if (keep)
#pragma unroll
            for (int r = 0; r < E; ++r) __stcs(&row[j + r * TP], v[r]);
        float q1[1] = {keep ? 2.f * a.ph.h * gq : 0.f};
        block_sum<1>(q1, T.part_row + (size_t)blockIdx.x * NQ, red);
        double S[1];
        if (last_block_total<1>(T.part_row, &T.sc->ticket[0], S, red) && threadIdx.x == 0) *a.gout = S[0];
        return;
    }

    constexpr bool STORE = !(MODE == ROW_REDUCE_R || MODE == ROW_OBS);
    if constexpr (STORE) {
        if (keep)
#pragma unroll
            for (int r = 0; r < E; ++r) __stcs(&row[j + r * TP], v[r]);
    }
}

// ------------------------------------------------------------------ grouped row pass
// ROW_PT for 512..2048-point rows with one CTA per SM: NG = 4 groups of 128
// threads (RG = 128 / TP rows, 16 KB, per work item).  The CTA copies the
// twiddle, coordinate and kinetic tables into shared memory once, so the
// pointwise steps read them there instead of through L1/L2.  Each group
// streams its items through two buffers: while it transforms one, TMA is
// already copying the next one in, and the finished item goes back to HBM by
// a TMA store from the buffer it was transformed in.  A group synchronises
// only its own warps (a named barrier), so the groups drift apart as
// separate CTAs would while sharing one copy of the tables.
template <int N> struct RowGroupCfg {
    static constexpr int E = 16, TP = N / 16, GT = 128, NG = 4, THREADS = GT * NG;
    static constexpr int RG = GT / TP;                       // rows per item
    static constexpr int PS = N + N / 16;                    // padded pencil stride (float2)
    static constexpr int BUF = RG * PS;                      // float2 per buffer
    static constexpr uint32_t ITEM_BYTES = RG * N * 8;
    static constexpr int TWN = fft_tw_count(N);
    static constexpr uint32_t TAB_BYTES = TWN * 16 + N * 16 + N * 8;
    // dynamic shared memory: twiddles | x coordinate table | x kinetic factors | NG x 2 buffers
    static constexpr size_t OFF_X = (size_t)TWN * 16;
    static constexpr size_t OFF_K = OFF_X + (size_t)N * 16;
    static constexpr size_t OFF_B = OFF_K + (size_t)N * 8;
    static constexpr size_t SMEM = OFF_B + (size_t)NG * 2 * BUF * 8;
    static_assert(TP <= GT && GT % TP == 0, "a group holds whole rows");
    static_assert(OFF_B % 16 == 0 && (BUF * 8) % 16 == 0 && ITEM_BYTES % 16 == 0, "bulk copies need 16 B");
    static_assert(SMEM <= 232448, "shared memory of one CTA");
};

// AND of p over the threads of a named barrier (all of them must arrive)
__device__ __forceinline__ bool group_all(bool p, int id, int n)
{
    uint32_t r;
    asm volatile(
        "{\n\t.reg .pred pi, po;\n\t"
        "setp.ne.u32 pi, %1, 0;\n\t"
        "bar.red.and.pred po, %2, %3, pi;\n\t"
        "selp.u32 %0, 1, 0, po;\n\t}"
        : "=r"(r)
        : "r"((uint32_t)p), "r"(id), "r"(n)
        : "memory");
    return r != 0;
}

// (launch bounds without a minimum CTA count: one 512-thread CTA per SM
// either way, and ptxas then fits the kernel in 128 registers without the
// 40 bytes of spill it made when asked for at least one CTA per SM)
template <int N>
__global__ void __launch_bounds__(RowGroupCfg<N>::THREADS) row_group_kernel(const PassArgs a, int nitems)
{
    using C = RowGroupCfg<N>;
    constexpr int E = C::E, TP = C::TP, RG = C::RG;
    extern __shared__ __align__(128) unsigned char smraw[];
    __shared__ __align__(8) uint64_t tbar;
    __shared__ __align__(8) uint64_t full[C::NG][2];
    float4 *stw = reinterpret_cast<float4 *>(smraw);
    const float4 *sx = reinterpret_cast<const float4 *>(smraw + C::OFF_X);
    const float2 *sk = reinterpret_cast<const float2 *>(smraw + C::OFF_K);
    const Tables &T = a.T;
    const int g = threadIdx.x / C::GT, t = threadIdx.x % C::GT;
    const int lr = t / TP, j = t % TP;
    float2 *buf0 = reinterpret_cast<float2 *>(smraw + C::OFF_B) + (size_t)g * 2 * C::BUF;
    const GroupSync gs{1 + g, C::GT};
    const bool leader = (t == 0);
    const int gstride = gridDim.x * C::NG;
    const int first = blockIdx.x * C::NG + g;

    if (threadIdx.x == 0) {
        mbar_init(&tbar, 1);
        for (int i = 0; i < C::NG; ++i) {
            mbar_init(&full[i][0], 1);
            mbar_init(&full[i][1], 1);
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        mbar_expect_tx(&tbar, C::TAB_BYTES);
        bulk_load_1d(stw, T.twx, C::TWN * 16, &tbar);
        bulk_load_1d(smraw + C::OFF_X, T.xtab, N * 16, &tbar);
        bulk_load_1d(smraw + C::OFF_K, T.kinx, N * 8, &tbar);
    }
    // an item's rows lie in the grid and its buffers in the launch's shared
    // memory (bounds-check build; a failed check issues no copy, so the
    // group's bounded wait runs out and the group stops)
    const bool bufs_ok = check_index((long long)C::OFF_B + (long long)(g + 1) * 2 * C::BUF * 8 - 1, dyn_smem_bytes(),
                                     T.sc);
    if (leader && first < nitems && bufs_ok && check_index((long long)(first + 1) * RG - 1, a.ny, T.sc)) {
        mbar_expect_tx(&full[g][0], C::ITEM_BYTES);
        bulk_load_1d(buf0, a.psi + (size_t)first * RG * N, C::ITEM_BYTES, &full[g][0]);
    }
    const float cs = a.use_c ? (float)T.sc->c : 1.f;
    if (!__syncthreads_and(mbar_wait_bounded(&tbar, 0, a.spins))) {
        // let the table copies and each group's first item land before the
        // CTA exits; nothing is stored
        if (threadIdx.x == 0) {
            latch_status(T.sc, GPE_ETIMEOUT);
            mbar_drain(&tbar, 0);
        }
        if (leader && first < nitems) mbar_drain(&full[g][0], 0);
        return;
    }

    uint32_t parity = 0;      // bit b: phase of full[g][b]
    int it = 0;
    for (int item = first; item < nitems; item += gstride, ++it) {
        const int b = it & 1;
        float2 *buf = buf0 + b * C::BUF;
        const int next = item + gstride;
        if (!group_all(mbar_wait_bounded(&full[g][b], (parity >> b) & 1u, a.spins), 1 + g, C::GT)) {
            // only this buffer's load is in flight (the next one is issued
            // after this wait); let it land, then stop this group
            if (leader) {
                latch_status(T.sc, GPE_ETIMEOUT);
                mbar_drain(&full[g][b], (parity >> b) & 1u);
            }
            break;
        }
        parity ^= 1u << b;
        const int y = item * RG + lr;
        float2 v[E];
#pragma unroll
        for (int r = 0; r < E; ++r) v[r] = buf[lr * N + j + r * TP];
        if (leader && next < nitems && check_index((long long)(next + 1) * RG - 1, a.ny, T.sc)) {
            bulk_wait_read_all();                    // the store of the other buffer has read it
            mbar_expect_tx(&full[g][b ^ 1], C::ITEM_BYTES);
            bulk_load_1d(buf0 + (b ^ 1) * C::BUF, a.psi + (size_t)next * RG * N, C::ITEM_BYTES, &full[g][b ^ 1]);
        }
        gs();                                        // dense reads done before the exchange writes
        float2 *sb = buf + lr * C::PS;

        const PotCoefs pc = row_coefs(a, __ldg(&T.ytab[y]));
        const float *Vr = a.V ? a.V + (size_t)y * N : nullptr;
#pragma unroll
        for (int r = 0; r < E; ++r) {
            const int xi = j + r * TP;
            float V = pot_at(pc, sx[xi]);
            if (Vr) V += a.V_scale * __ldg(&Vr[xi]);
            v[r] = phase_mul(make_float2(v[r].x * cs, v[r].y * cs), V, a.g, a.ph.h, a.imag);
        }
        fft_pencil<N, E, false>(v, sb, j, 1, stw, gs);
        if (a.imag) {
#pragma unroll
            for (int r = 0; r < E; ++r) {
                const float f = sk[j + r * TP].x * a.sx;
                v[r] = make_float2(v[r].x * f, v[r].y * f);
            }
        } else {
#pragma unroll
            for (int r = 0; r < E; ++r) {
                const float2 d = sk[j + r * TP];
                const float2 p = v[r];
                const float2 pd = cmul(p, d);
                v[r] = make_float2((p.x + pd.x) * a.sx, (p.y + pd.y) * a.sx);
            }
        }
        fft_pencil<N, E, true>(v, sb, j, 1, stw, gs);
#pragma unroll
        for (int r = 0; r < E; ++r) buf[lr * N + j + r * TP] = v[r];
        fence_proxy_async();                         // generic-proxy writes visible to the TMA store
        gs();
        if (leader) {
            bulk_store_1d(a.psi + (size_t)item * RG * N, buf, C::ITEM_BYTES);
            bulk_commit();
        }
    }
    if (leader) bulk_wait_read_all();
}

// ------------------------------------------------------------------ column pass
template <int N> struct ColCfg {
    static constexpr int E = N >= 16 ? 16 : N;
    static constexpr int TP = N / E;
    static constexpr int BR = N < 256 ? N : 256;    // rows per TMA box
    static constexpr int PS = N + N / 16;          // padded pencil stride (float2)
    // twiddles staged in shared memory except for 8192 rows (no room left)
    static constexpr int TWN = N >= 8192 ? 0 : fft_tw_count(N);
};

// Tile width for columns of length N: the narrowest tile whose CTA is at
// least one warp (W N/16 >= 32 threads), so that small grids spread over
// many CTAs; 2 columns (a 16-byte TMA box row) from N = 256 on, at most 8
// (a grid is at least 8 wide, so the width is a function of N only).
// Measured on a single 512^2 grid: 10.5 us per column pass against 12.4 us
// with 8-column tiles.
__host__ __device__ constexpr int col_w(int n) { return n >= 64 ? (512 / n > 2 ? 512 / n : 2) : 8; }
// Columns transformed at once: up to 256 threads (512 for N >= 4096); the
// 8192-row tile does its second column in a second round.
__host__ __device__ constexpr int col_g(int n)
{
    const int tp = n >= 16 ? n / 16 : 1;
    const int t = n >= 4096 ? 512 : 256;
    const int g = t / tp < 1 ? 1 : t / tp;
    return g > col_w(n) ? col_w(n) : g;
}

// Twiddle entries a column pass of mode MODE stages in shared memory: the
// whole table in every mode.  Reading it through L1 instead in the modes
// that also read the y-table at every point (so that L1 keeps room for the
// y-table) measured slower at 2048^2: closing phase + norm 76.7 against 67.0
// us, cavity overlaps 61.8 against 55.8 us.
template <int N, int MODE> __host__ __device__ constexpr int col_twn()
{
    (void)MODE;
    return ColCfg<N>::TWN;
}

// Column pass over a tile of W columns: TMA load of the dense [N][W] tile,
// per-column FFT through padded per-column exchange buffers, the kinetic
// factor, inverse FFT, optional closing phase and reductions, results written
// back into the dense tile and stored with TMA.
template <int N, int MODE>
__global__ void __launch_bounds__(col_g(N) * ColCfg<N>::TP, N >= 4096 ? 1 : 3)
    col_kernel(const PassArgs a, const __grid_constant__ CUtensorMap map)
{
    using C = ColCfg<N>;
    constexpr int E = C::E, TP = C::TP, W = col_w(N), G = col_g(N), TWN = col_twn<N, MODE>();
    constexpr bool INPLACE = (G == W);   // exchange buffers may overlay the dense tile
    extern __shared__ unsigned char smraw[];
    __shared__ __align__(8) uint64_t bar;
    __shared__ double red[32 * NQ];

    const uint32_t s0 = smem_u32(smraw);
    float2 *tile = reinterpret_cast<float2 *>(smraw + ((128u - (s0 & 127u)) & 127u));
    float2 *pen = INPLACE ? tile : tile + N * W;
    float4 *stw = reinterpret_cast<float4 *>(tile + (INPLACE ? W * C::PS : N * W + G * C::PS));

    const Tables &T = a.T;
    // the tile's columns lie in the grid and its buffers in the launch's
    // shared memory (checked in the bounds-check build; TMA itself clips)
    const bool inb = check_index((long long)blockIdx.x * W + W - 1, a.nx, T.sc) &&
                     check_index((long long)((unsigned char *)(stw + TWN) - smraw) - 1, dyn_smem_bytes(), T.sc);
    const int c0 = inb ? blockIdx.x * W : 0;
    const float4 *tw = TWN ? stw : T.twy;

    if (threadIdx.x == 0) mbar_init(&bar, 1);
    __syncthreads();
    if (threadIdx.x == 0) {
        // one arrival per phase: the tile and the twiddle table share it
        mbar_expect_tx(&bar, (uint32_t)(N * W * 8) + (TWN > 0 ? twiddle_bytes<N>() : 0u));
        if constexpr (TWN > 0) stage_twiddles_async<N>(stw, T.twy, &bar);
        for (int r0 = 0; r0 < N; r0 += C::BR) tma_load_2d(tile + (size_t)r0 * W, &map, &bar, 2 * c0, r0);
    }
    // ok: the tile (and twiddles) arrived in time.  Otherwise the copies are
    // given time to land, the CTA runs on without storing and adds zero
    // partial sums, so that every reduction still counts all of its CTAs.
    const bool ok = __syncthreads_and(mbar_wait_bounded(&bar, 0, a.spins));
    if (!ok) {
        if (threadIdx.x == 0) latch_status(T.sc, GPE_ETIMEOUT);
        mbar_drain(&bar, 0);
    }

    constexpr bool REDUCE = (MODE == COL_T_R || MODE == COL_T_PR);
    const int j = threadIdx.x % TP, cg = threadIdx.x / TP;
    float2 *sb = pen + cg * C::PS;
    float q[3] = {0.f, 0.f, 0.f};
#pragma unroll 1
    for (int g0 = 0; g0 < W; g0 += G) {
        const int c = g0 + cg;
        float2 v[E];
#pragma unroll
        for (int r = 0; r < E; ++r) v[r] = tile[(j + r * TP) * W + c];
        if constexpr (INPLACE) __syncthreads();      // dense reads done before exchange writes

        if constexpr (MODE == COL_FFT_I) {
            fft_pencil<N, E, true>(v, sb, j, 1, tw);
#pragma unroll
            for (int r = 0; r < E; ++r) v[r] = make_float2(v[r].x * a.sy, v[r].y * a.sy);
        } else {
            fft_pencil<N, E, false>(v, sb, j, 1, tw);
        }

        if constexpr (MODE == COL_T || MODE == COL_T_R || MODE == COL_T_PR || MODE == COL_T_P) {
            kinetic_axis<E, TP>(v, T.kiny, j, a.sy, a.imag);
            fft_pencil<N, E, true>(v, sb, j, 1, tw);
        }

        if constexpr (MODE == COL_ADJ) {
            // v = lambda; T_y^H, then the adjoint of the opening half phase
            // whose input psi2 is the step's initial state
            kinetic_axis<E, TP, true>(v, T.kiny, j, a.sy, 0);
            fft_pencil<N, E, true>(v, sb, j, 1, tw);
            const float4 xt = __ldg(&T.xtab[c0 + c]);
            const PotCoefs pc = col_coefs(a, xt);
            float gq = 0.f;
#pragma unroll
            for (int r = 0; r < E; ++r) {
                const int yi = j + r * TP;
                const float4 yt = __ldg(&T.ytab[yi]);
                float V = pot_at(pc, yt);
                if (a.V) V += a.V_scale * __ldg(&a.V[(size_t)yi * a.nx + c0 + c]);
                const float2 in = __ldg(&a.psi2[(size_t)yi * a.nx + c0 + c]);
                gq += phase_adjoint(v[r], in, V, a.g, a.ph.h) * (a.L0x * xt.y + a.L0y * yt.y);
            }
            q[0] += 2.f * a.ph.h * gq;
        }

        if constexpr (MODE == COL_T_PR || MODE == COL_T_P) {
            // closing half phase [and the reduction of its result] in one
            // loop: each y-table entry is read once
            const float4 xt = __ldg(&T.xtab[c0 + c]);
            const PotCoefs pc = col_coefs(a, xt);
            float n0 = 0.f, n1 = 0.f;
#pragma unroll
            for (int r = 0; r < E; ++r) {
                const int yi = j + r * TP;
                const float4 yt = __ldg(&T.ytab[yi]);
                float V = pot_at(pc, yt);
                if (a.V) V += a.V_scale * __ldg(&a.V[(size_t)yi * a.nx + c0 + c]);
                v[r] = phase_mul(v[r], V, a.g, a.ph.h, a.imag);
                if constexpr (REDUCE) {
                    const float n = v[r].x * v[r].x + v[r].y * v[r].y;
                    n0 += n;
                    n1 += yt.z * n;
                }
            }
            q[0] += n0;
            q[1] += xt.z * n1;
            q[2] += xt.z * xt.z * n0;
        } else if constexpr (REDUCE) {
            const float cx = __ldg(&T.xtab[c0 + c]).z;
            float n0 = 0.f, n1 = 0.f;
#pragma unroll
            for (int r = 0; r < E; ++r) {
                const float n = v[r].x * v[r].x + v[r].y * v[r].y;
                n0 += n;
                n1 += __ldg(&T.ytab[j + r * TP]).z * n;
            }
            q[0] += n0;
            q[1] += cx * n1;
            q[2] += cx * cx * n0;
        }

        if constexpr (MODE == COL_OBS) {
#pragma unroll
            for (int r = 0; r < E; ++r) {
                const int e = j + r * TP;
                const float ky = (float)(e < N / 2 ? e : e - N);    // in units of 2 pi / Ly
                q[0] += ky * ky * (v[r].x * v[r].x + v[r].y * v[r].y);
            }
        } else {
            // every exchange read of this round finished at the last stage's barrier
#pragma unroll
            for (int r = 0; r < E; ++r) tile[(j + r * TP) * W + c] = v[r];
        }
        if constexpr (!INPLACE) __syncthreads();
    }

    if (!ok || !inb) q[0] = q[1] = q[2] = 0.f;
    if constexpr (MODE == COL_OBS) {
        float q1[1] = {q[0]};
        block_sum<1>(q1, T.part_col + (size_t)blockIdx.x * NQ, red);
        double S[1];
        if (last_block_total<1>(T.part_col, &T.sc->ticket[1], S, red) && threadIdx.x == 0)
            T.sc->sums[1][0] = S[0];
        return;
    }

    // make the generic-proxy tile writes visible to the TMA engine, then store
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (threadIdx.x == 0 && ok && inb) {
        for (int r0 = 0; r0 < N; r0 += C::BR) tma_store_2d(&map, tile + (size_t)r0 * W, 2 * c0, r0);
        asm volatile("cp.async.bulk.commit_group;" ::: "memory");
    }
    if constexpr (REDUCE) {
        block_sum<3>(q, T.part_col + (size_t)blockIdx.x * NQ, red);
        double S[3];
        if (last_block_total<3>(T.part_col, &T.sc->ticket[1], S, red) && threadIdx.x == 0)
            finalize_fields(S, a.red, T.sc);
    }
    if constexpr (MODE == COL_ADJ) {
        float q1[1] = {q[0]};
        block_sum<1>(q1, T.part_col + (size_t)blockIdx.x * NQ, red);
        double S[1];
        if (last_block_total<1>(T.part_col, &T.sc->ticket[1], S, red) && threadIdx.x == 0) *a.gout = S[0];
    }
    if (threadIdx.x == 0) asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");   // tile read before exit
}

// ------------------------------------------------------------------ streaming passes
// Persistent versions of the two hot passes (row: phase + T_x; column: T_y
// [+ phase] [+ reductions]), used for 4096-point axes where they measured
// faster than the one-shot passes (at 2048 and below the one-shot passes, with
// three CTAs per SM, are faster).  Each CTA walks work items (a group of whole
// rows, or a tile of W columns) with stride gridDim.x, double-buffered in
// shared memory: while item i is transformed in one buffer, the TMA engine
// loads item i + gridDim.x into the other; results are written back into the
// buffer and stored with TMA.  The twiddle table is staged once per CTA.
template <int N> struct RowStreamCfg {
    static constexpr int E = 16, TP = N / 16, THREADS = 256, RPC = THREADS / TP;
    static constexpr int PS = N + N / 16;
    static constexpr int BUF = RPC * PS;                       // float2 per buffer (padded layout)
    static constexpr bool STW = fft_tw_count(N) * 16 <= 40960; // twiddles in shared memory
    static constexpr int TWN = STW ? fft_tw_count(N) : 0;
    static constexpr int CTAS_PER_SM = 2;
    static constexpr size_t SMEM = (size_t)2 * BUF * 8 + (size_t)TWN * 16 + 128;
};

template <int N>
__global__ void __launch_bounds__(256, 2) row_stream_kernel(const PassArgs a, int nitems)
{
    using C = RowStreamCfg<N>;
    constexpr int E = C::E, TP = C::TP, RPC = C::RPC;
    constexpr uint32_t BYTES = RPC * N * 8;
    extern __shared__ unsigned char smraw[];
    __shared__ __align__(8) uint64_t bar[2];
    const uint32_t s0 = smem_u32(smraw);
    float2 *buf0 = reinterpret_cast<float2 *>(smraw + ((128u - (s0 & 127u)) & 127u));
    float4 *stw = reinterpret_cast<float4 *>(buf0 + 2 * C::BUF);
    const Tables &T = a.T;
    const float4 *tw = C::STW ? stw : T.twx;
    if constexpr (C::STW) stage_twiddles<N>(stw, T.twx);

    if (threadIdx.x == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
    }
    __syncthreads();
    if (threadIdx.x == 0 && (int)blockIdx.x < nitems &&
        check_index((long long)(blockIdx.x + 1) * RPC - 1, a.ny, T.sc) &&
        check_index((long long)((unsigned char *)(buf0 + 2 * C::BUF) - smraw) - 1, dyn_smem_bytes(), T.sc)) {
        mbar_expect_tx(&bar[0], BYTES);
        bulk_load_1d(buf0, a.psi + (size_t)blockIdx.x * RPC * N, BYTES, &bar[0]);
    }
    const int lr = threadIdx.x / TP, j = threadIdx.x % TP;
    uint32_t parity = 0;      // bit b: phase of bar[b]
    int it = 0;
    for (int item = blockIdx.x; item < nitems; item += gridDim.x, ++it) {
        const int b = it & 1;
        float2 *buf = buf0 + b * C::BUF;
        const int next = item + gridDim.x;
        if (threadIdx.x == 0 && next < nitems && check_index((long long)(next + 1) * RPC - 1, a.ny, T.sc)) {
            bulk_wait_read_all();                     // the other buffer's last store has read it
            mbar_expect_tx(&bar[b ^ 1], BYTES);
            bulk_load_1d(buf0 + (b ^ 1) * C::BUF, a.psi + (size_t)next * RPC * N, BYTES, &bar[b ^ 1]);
        }
        const uint32_t pb = (parity >> b) & 1u;
        const bool ok = __syncthreads_and(mbar_wait_bounded(&bar[b], pb, a.spins));
        parity ^= 1u << b;
        if (!ok) {
            // both loads may be in flight (this item's and the next one's,
            // issued above): let them land before the CTA stops
            if (threadIdx.x == 0) {
                latch_status(T.sc, GPE_ETIMEOUT);
                mbar_drain(&bar[b], pb);
                if (next < nitems) mbar_drain(&bar[b ^ 1], (parity >> (b ^ 1)) & 1u);
            }
            break;
        }
        const int y = item * RPC + lr;
        float2 v[E];
#pragma unroll
        for (int r = 0; r < E; ++r) v[r] = buf[lr * N + j + r * TP];
        __syncthreads();                              // dense reads done before exchange writes
        float2 *sb = buf + lr * C::PS;

        const float4 yt = T.ytab[y];
        const PotCoefs pc = row_coefs(a, yt);
        float cs = 1.f;
        if (a.use_c) cs = (float)T.sc->c;
        const float *Vr = a.V ? a.V + (size_t)y * N : nullptr;
#pragma unroll
        for (int r = 0; r < E; ++r) {
            const int xi = j + r * TP;
            float V = pot_at(pc, __ldg(&T.xtab[xi]));
            if (Vr) V += a.V_scale * __ldg(&Vr[xi]);
            v[r] = phase_mul(make_float2(v[r].x * cs, v[r].y * cs), V, a.g, a.ph.h, a.imag);
        }
        fft_pencil<N, E, false>(v, sb, j, 1, tw);
        kinetic_axis<E, TP>(v, T.kinx, j, a.sx, a.imag);
        fft_pencil<N, E, true>(v, sb, j, 1, tw);
#pragma unroll
        for (int r = 0; r < E; ++r) buf[lr * N + j + r * TP] = v[r];
        fence_proxy_async();
        __syncthreads();
        if (threadIdx.x == 0) {
            bulk_store_1d(a.psi + (size_t)item * RPC * N, buf, BYTES);
            bulk_commit();
        }
    }
    if (threadIdx.x == 0) bulk_wait_read_all();
}

template <int N> struct ColStreamCfg {
    static constexpr int E = 16, TP = N / 16, W = col_w(N), G = col_g(N), THREADS = G * TP;
    static constexpr int BR = N < 256 ? N : 256;
    static constexpr int PS = N + N / 16;
    static constexpr int BUF = W * PS;                           // float2 per buffer (padded layout)
    static constexpr bool STW = fft_tw_count(N) * 16 <= 40960;
    static constexpr int TWN = STW ? fft_tw_count(N) : 0;
    static constexpr int CTAS_PER_SM = N >= 4096 ? 1 : 2;
    static constexpr size_t SMEM = (size_t)2 * BUF * 8 + (size_t)TWN * 16 + 128;
};

template <int N, int MODE>
__global__ void __launch_bounds__(ColStreamCfg<N>::THREADS, ColStreamCfg<N>::CTAS_PER_SM)
    col_stream_kernel(const PassArgs a, const __grid_constant__ CUtensorMap map, int nitems)
{
    using C = ColStreamCfg<N>;
    constexpr int E = C::E, TP = C::TP, W = C::W;
    static_assert(C::G == W, "one round per tile");
    extern __shared__ unsigned char smraw[];
    __shared__ __align__(8) uint64_t bar[2];
    __shared__ double red[32 * NQ];
    const uint32_t s0 = smem_u32(smraw);
    float2 *buf0 = reinterpret_cast<float2 *>(smraw + ((128u - (s0 & 127u)) & 127u));
    float4 *stw = reinterpret_cast<float4 *>(buf0 + 2 * C::BUF);
    const Tables &T = a.T;
    const float4 *tw = C::STW ? stw : T.twy;
    if constexpr (C::STW) stage_twiddles<N>(stw, T.twy);

    if (threadIdx.x == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
    }
    __syncthreads();
    if (threadIdx.x == 0 && (int)blockIdx.x < nitems &&
        check_index((long long)(blockIdx.x + 1) * W - 1, a.nx, T.sc) &&
        check_index((long long)((unsigned char *)(buf0 + 2 * C::BUF) - smraw) - 1, dyn_smem_bytes(), T.sc)) {
        mbar_expect_tx(&bar[0], (uint32_t)(N * W * 8));
        for (int r0 = 0; r0 < N; r0 += C::BR) tma_load_2d(buf0 + r0 * W, &map, &bar[0], 2 * blockIdx.x * W, r0);
    }
    constexpr bool REDUCE = (MODE == COL_T_R || MODE == COL_T_PR);
    const int j = threadIdx.x % TP, c = threadIdx.x / TP;
    float q[3] = {0.f, 0.f, 0.f};
    uint32_t parity = 0;
    int it = 0;
    for (int item = blockIdx.x; item < nitems; item += gridDim.x, ++it) {
        const int b = it & 1;
        float2 *buf = buf0 + b * C::BUF;
        const int next = item + gridDim.x;
        if (threadIdx.x == 0 && next < nitems && check_index((long long)(next + 1) * W - 1, a.nx, T.sc)) {
            bulk_wait_read_all();
            float2 *nb = buf0 + (b ^ 1) * C::BUF;
            mbar_expect_tx(&bar[b ^ 1], (uint32_t)(N * W * 8));
            for (int r0 = 0; r0 < N; r0 += C::BR) tma_load_2d(nb + r0 * W, &map, &bar[b ^ 1], 2 * next * W, r0);
        }
        const uint32_t pb = (parity >> b) & 1u;
        const bool ok = __syncthreads_and(mbar_wait_bounded(&bar[b], pb, a.spins));
        parity ^= 1u << b;
        if (!ok) {
            // both loads may be in flight (this item's and the next one's,
            // issued above): let them land before the CTA stops
            if (threadIdx.x == 0) {
                latch_status(T.sc, GPE_ETIMEOUT);
                mbar_drain(&bar[b], pb);
                if (next < nitems) mbar_drain(&bar[b ^ 1], (parity >> (b ^ 1)) & 1u);
            }
            break;
        }
        const int c0 = item * W;
        float2 v[E];
#pragma unroll
        for (int r = 0; r < E; ++r) v[r] = buf[(j + r * TP) * W + c];
        __syncthreads();
        float2 *sb = buf + c * C::PS;
        fft_pencil<N, E, false>(v, sb, j, 1, tw);
        kinetic_axis<E, TP>(v, T.kiny, j, a.sy, a.imag);
        fft_pencil<N, E, true>(v, sb, j, 1, tw);
        if constexpr (MODE == COL_T_PR || MODE == COL_T_P) {
            // closing half phase [and its reduction] in one loop (one y-table read per point)
            const float4 xt = __ldg(&T.xtab[c0 + c]);
            const PotCoefs pc = col_coefs(a, xt);
            float n0 = 0.f, n1 = 0.f;
#pragma unroll
            for (int r = 0; r < E; ++r) {
                const int yi = j + r * TP;
                const float4 yt = __ldg(&T.ytab[yi]);
                float V = pot_at(pc, yt);
                if (a.V) V += a.V_scale * __ldg(&a.V[(size_t)yi * a.nx + c0 + c]);
                v[r] = phase_mul(v[r], V, a.g, a.ph.h, a.imag);
                if constexpr (REDUCE) {
                    const float n = v[r].x * v[r].x + v[r].y * v[r].y;
                    n0 += n;
                    n1 += yt.z * n;
                }
            }
            q[0] += n0;
            q[1] += xt.z * n1;
            q[2] += xt.z * xt.z * n0;
        } else if constexpr (REDUCE) {
            const float cx = __ldg(&T.xtab[c0 + c]).z;
            float n0 = 0.f, n1 = 0.f;
#pragma unroll
            for (int r = 0; r < E; ++r) {
                const float n = v[r].x * v[r].x + v[r].y * v[r].y;
                n0 += n;
                n1 += __ldg(&T.ytab[j + r * TP]).z * n;
            }
            q[0] += n0;
            q[1] += cx * n1;
            q[2] += cx * cx * n0;
        }
#pragma unroll
        for (int r = 0; r < E; ++r) buf[(j + r * TP) * W + c] = v[r];
        fence_proxy_async();
        __syncthreads();
        if (threadIdx.x == 0) {
            for (int r0 = 0; r0 < N; r0 += C::BR) tma_store_2d(&map, buf + r0 * W, 2 * c0, r0);
            bulk_commit();
        }
    }
    if constexpr (REDUCE) {
        block_sum<3>(q, T.part_col + (size_t)blockIdx.x * NQ, red);
        double S[3];
        if (last_block_total<3>(T.part_col, &T.sc->ticket[1], S, red) && threadIdx.x == 0)
            finalize_fields(S, a.red, T.sc);
    }
    if (threadIdx.x == 0) bulk_wait_read_all();
}

#if GPE_IN_PART(0)
// ------------------------------------------------------------------ tables
// Entry i of the per-stage twiddle table of an n-point axis in the schedule
// of main radix 2^LR (fftg_tw_offset layout): W_{NS R}^{r k} = exp(-2 pi i r
// k / (NS R)) as {re_hi, im_hi, re_lo, im_lo}, hi = float(x), lo = float(x -
// hi).  Entries past the table are 1.
template <int LR> static __device__ float4 twiddle_entry(int i, int n)
{
    long long num = 0, den = 1;
    for (int s = 1; s < fftg_stages<LR>(n); ++s) {
        const int ns = fftg_ns<LR>(n, s), R = fftg_radix<LR>(n, s), off = fftg_tw_offset<LR>(n, s);
        if (i >= off && i < off + (R - 1) * ns) {
            const int r = (i - off) / ns + 1, k = (i - off) % ns;
            num = (long long)r * k;
            den = (long long)ns * R;
        }
    }
    double s, c;
    sincospi(2.0 * (double)(num % den) / (double)den, &s, &c);
    const float ch = (float)c, sh = (float)-s;
    return make_float4(ch, sh, (float)(c - (double)ch), (float)(-s - (double)sh));
}

// Coordinates, trap and lattice profiles and twiddles in FP64, rounded once.
// The radix-8 tables are written only where the caller's Tables has them
// (the allocation-free reduction's scratch holds the coordinate and radix-16
// tables alone).
__global__ void tables_kernel(Tables T, int nx, int ny, double Lx, double Ly, double m, double wx,
                              double wy, double lkx, double lky, double kc)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < nx) {
        const double x = -0.5 * Lx + (double)i * (Lx / nx);
        const double cl = cos(lkx * x), cc = cos(kc * x);
        T.xtab[i] = make_float4((float)(0.5 * m * wx * wx * x * x), (float)(cl * cl), (float)cc, (float)x);
        T.twx[i] = twiddle_entry<4>(i, nx);
        if (T.tw8x) T.tw8x[i] = twiddle_entry<3>(i, nx);
    }
    if (i < ny) {
        const double y = -0.5 * Ly + (double)i * (Ly / ny);
        const double cl = cos(lky * y), cc = cos(kc * y);
        T.ytab[i] = make_float4((float)(0.5 * m * wy * wy * y * y), (float)(cl * cl), (float)cc, (float)y);
        T.twy[i] = twiddle_entry<4>(i, ny);
        if (T.tw8y) T.tw8y[i] = twiddle_entry<3>(i, ny);
    }
}

// Kinetic factors per axis (FP64, rounded once).  Real time: D = e^{-i k^2 dt/2m} - 1
// written as (-2 sin^2(a/2), -sin a); imaginary time: (e^{-k^2 dt/2m}, 0).
__global__ void kinetic_tables_kernel(Tables T, int nx, int ny, double Lx, double Ly, double m, double dt,
                                      int imag)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    for (int axis = 0; axis < 2; ++axis) {
        const int n = axis ? ny : nx;
        if (i >= n) continue;
        const double L = axis ? Ly : Lx;
        const double k = 2.0 * M_PI / L * (double)(i < n / 2 ? i : i - n);
        const double ang = k * k / (2.0 * m) * dt;
        float2 out;
        if (imag) {
            out = make_float2((float)exp(-ang), 0.f);
        } else {
            double s, c;
            sincos(0.5 * ang, &s, &c);
            out = make_float2((float)(-2.0 * s * s), (float)(-2.0 * s * c));
        }
        (axis ? T.kiny : T.kinx)[i] = out;
    }
}

// ------------------------------------------------------------------ adjoint: terminal pieces
// Spectrum times the kinetic energy density: f_k <- f_k (kx^2 + ky^2) / 2m
// (k in FFT order), for H psi = F^-1[(k^2/2m) F psi] + ... in the terminal
// adjoint dJ/dconj(psi_T) of the final energy.
__global__ void kin_energy_mul_kernel(float2 *f, int nx, int ny, double Lx, double Ly, double m)
{
    const size_t n = (size_t)nx * ny;
    const double ax = 2.0 * M_PI / Lx, ay = 2.0 * M_PI / Ly;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const int x = (int)(i % nx), y = (int)(i / nx);
        const double kx = ax * (x < nx / 2 ? x : x - nx), ky = ay * (y < ny / 2 ? y : y - ny);
        const float e = (float)((kx * kx + ky * ky) / (2.0 * m));
        f[i] = make_float2(f[i].x * e, f[i].y * e);
    }
}

// S0 + i S1 = sum conj(phi) psi, S2 = sum |psi|^2 L (L = dV/dv of the
// lattice control), without the cell area; the last CTA stores them in sums[0].
__global__ void __launch_bounds__(256) adj_overlap_kernel(const float2 *__restrict__ psi,
                                                          const float2 *__restrict__ phi, Tables T, int nx,
                                                          int ny, float L0x, float L0y)
{
    __shared__ double red[32 * NQ];
    const size_t n = (size_t)nx * ny;
    float q[3] = {0.f, 0.f, 0.f};
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const int x = (int)(i % nx), y = (int)(i / nx);
        const float2 v = psi[i], f = phi[i];
        q[0] += f.x * v.x + f.y * v.y;
        q[1] += f.x * v.y - f.y * v.x;
        q[2] += (v.x * v.x + v.y * v.y) * (L0x * __ldg(&T.xtab[x]).y + L0y * __ldg(&T.ytab[y]).y);
    }
    block_sum<3>(q, T.part_row + (size_t)blockIdx.x * NQ, red);
    double S[3];
    if (last_block_total<3>(T.part_row, &T.sc->ticket[0], S, red) && threadIdx.x == 0)
        for (int k = 0; k < 3; ++k) T.sc->sums[0][k] = S[k];
}

// lam <- dxdy (lam + (V(T) + g |psi|^2) psi + c phi), lam holding the
// kinetic part F^-1[(k^2/2m) F psi] on entry: the terminal adjoint of
// J = E(psi_T) + |<phi|psi_T>|^2 with c = <phi|psi_T>.
__global__ void adj_terminal_kernel(float2 *__restrict__ lam, const float2 *__restrict__ psi,
                                    const float2 *__restrict__ phi, const PassArgs a, float c_re, float c_im,
                                    float dxdy)
{
    const size_t n = (size_t)a.nx * a.ny;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const int x = (int)(i % a.nx), y = (int)(i / a.nx);
        const PotCoefs pc = row_coefs(a, __ldg(&a.T.ytab[y]));
        float V = pot_at(pc, __ldg(&a.T.xtab[x]));
        if (a.V) V += a.V_scale * __ldg(&a.V[i]);
        const float2 v = psi[i], f = phi[i], k = lam[i];
        const float w = V + a.g * (v.x * v.x + v.y * v.y);
        lam[i] = make_float2(dxdy * (k.x + w * v.x + c_re * f.x - c_im * f.y),
                             dxdy * (k.y + w * v.y + c_re * f.y + c_im * f.x));
    }
}

// ------------------------------------------------------------------ momentum populations
// Kapitza-Dirac readout (Sec. 5.2) on a spectrum f = F psi: the weight
// |f|^2 of every mode whose momentum along `axis` is within k0 of 2 n k0
// (n = -nmax..nmax, nmax <= 3; a momentum exactly between two windows goes
// to the smaller |n|), summed over the other axis; q[7] is the total.  The
// last CTA stores the 8 sums in sums[0].
__global__ void __launch_bounds__(256) kbin_kernel(const float2 *__restrict__ f, Tables T, int nx, int ny, double Lx,
                                                   double Ly, int axis, double k0, int nmax)
{
    __shared__ double red[32 * NQ];
    const size_t n = (size_t)nx * ny;
    float q[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const int x = (int)(i % nx), y = (int)(i / nx);
        const float2 v = f[i];
        const float w = v.x * v.x + v.y * v.y;
        q[7] += w;
        const int m = axis == 0 ? (x < nx / 2 ? x : x - nx) : (y < ny / 2 ? y : y - ny);
        const double r = 2.0 * M_PI / (axis == 0 ? Lx : Ly) * m / (2.0 * k0);
        int b = (int)floor(fabs(r) + 0.5);
        if (b > 0 && fabs(fabs(r) - (b - 0.5)) < 1e-12) b -= 1;
        if (b <= nmax) {
            const int idx = (r < 0 ? -b : b) + nmax;
#pragma unroll
            for (int k = 0; k < 7; ++k)
                if (k == idx) q[k] += w;                 // register-resident bins
        }
    }
    block_sum<8>(q, T.part_row + (size_t)blockIdx.x * NQ, red);
    double S[8];
    if (last_block_total<8>(T.part_row, &T.sc->ticket[0], S, red) && threadIdx.x == 0)
        for (int k = 0; k < 8; ++k) T.sc->sums[0][k] = S[k];
}

__global__ void timeout_probe_kernel(DevScalars *sc, int spins)
{
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) mbar_init(&bar, 1);
    __syncthreads();
    // nothing ever arrives on this barrier: the bounded wait must give up
    const bool ok = mbar_wait_bounded(&bar, 0, spins);
    if (!ok && threadIdx.x == 0) latch_status(sc, GPE_ETIMEOUT);
}

#endif  // GPE_IN_PART(0)

// ------------------------------------------------------------------ launchers

#if GPE_IN_PART(0)
// Rows per CTA of the one-shot row pass: 256 threads' worth, divided by
// 2^tile_shift for rows of 256 points and more (the tuner's smaller tiles
// spread a small grid over more SMs), never below one warp's worth nor above
// the grid.
int row_rows_per_cta(int nx, int ny, int tile_shift)
{
    const int E = nx >= 16 ? 16 : nx;
    const int tp = nx / E;
    int rpc = (256 / tp) >> (nx >= 256 ? tile_shift : 0);
    if (rpc * tp < 32) rpc = (32 + tp - 1) / tp;
    if (rpc < 1) rpc = 1;
    if (rpc > ny) rpc = ny;
    return rpc;
}

int col_tile_width(int nx, int ny)
{
    (void)nx;
    return col_w(ny);
}

bool row_group_ok(int nx, int ny) { return (nx == 512 || nx == 1024 || nx == 2048) && ny % (2048 / nx) == 0; }

// Streaming row pass for ROW_PT when the grid has enough rows; false = not applicable.
bool row_stream_ok(int nx, int ny) { return nx == 4096 && ny >= 8; }

// Streaming column pass: 4096-point columns (the default there) and 2048 (a
// variant the autotuner may pick: the twiddles staged once per CTA instead
// of once per 2-column tile, at 2 CTAs per SM instead of 3)
bool col_stream_ok(int nx, int ny) { return (ny == 2048 || ny == 4096) && nx >= 8 * col_w(ny); }

cudaError_t launch_row(int mode, const PassArgs &a, cudaStream_t s, int tile_shift)
{
    return a.nx <= 256 ? launch_row_lo(mode, a, s, tile_shift) : launch_row_hi(mode, a, s, tile_shift);
}

cudaError_t launch_col(int mode, const PassArgs &a, const CUtensorMap &map, cudaStream_t s)
{
    return a.ny <= 256 ? launch_col_lo(mode, a, map, s) : launch_col_hi(mode, a, map, s);
}
#endif  // GPE_IN_PART(0)

template <int N, int MODE> static cudaError_t row_launch(const PassArgs &a, cudaStream_t s, int tile_shift)
{
    using C = RowCfg<N>;
    const int rpc = row_rows_per_cta(N, a.ny, tile_shift);
    const int threads = rpc * C::TP;
    const size_t smem = (size_t)rpc * C::PS * sizeof(float2) + (size_t)C::TWN * sizeof(float4);
    constexpr int rpc_max = 256 / C::TP > 1 ? 256 / C::TP : 1;
    constexpr int smem_max = rpc_max * C::PS * (int)sizeof(float2) + C::TWN * (int)sizeof(float4);
    if constexpr (smem_max > 48 * 1024) {
        static std::atomic<unsigned long long> attr{0};
        const cudaError_t e = smem_opt_in(row_kernel<N, MODE>, smem_max, attr);
        if (e != cudaSuccess) return e;
    }
    row_kernel<N, MODE><<<a.ny / rpc, threads, smem, s>>>(a);
    return cudaGetLastError();
}

template <int N> static cudaError_t row_dispatch_mode(int mode, const PassArgs &a, cudaStream_t s, int ts)
{
    switch (mode) {
    case ROW_PT: return row_launch<N, ROW_PT>(a, s, ts);
    case ROW_PHASE: return row_launch<N, ROW_PHASE>(a, s, ts);
    case ROW_PHASE_R: return row_launch<N, ROW_PHASE_R>(a, s, ts);
    case ROW_REDUCE_R: return row_launch<N, ROW_REDUCE_R>(a, s, ts);
    case ROW_SCALE: return row_launch<N, ROW_SCALE>(a, s, ts);
    case ROW_FFT_F: return row_launch<N, ROW_FFT_F>(a, s, ts);
    case ROW_FFT_I: return row_launch<N, ROW_FFT_I>(a, s, ts);
    case ROW_OBS: return row_launch<N, ROW_OBS>(a, s, ts);
    case ROW_ADJ: return row_launch<N, ROW_ADJ>(a, s, ts);
    default: return cudaErrorInvalidValue;
    }
}

#if GPE_IN_PART(1)
cudaError_t launch_row_lo(int mode, const PassArgs &a, cudaStream_t s, int tile_shift)
{
    switch (a.nx) {
    case 8: return row_dispatch_mode<8>(mode, a, s, tile_shift);
    case 16: return row_dispatch_mode<16>(mode, a, s, tile_shift);
    case 32: return row_dispatch_mode<32>(mode, a, s, tile_shift);
    case 64: return row_dispatch_mode<64>(mode, a, s, tile_shift);
    case 128: return row_dispatch_mode<128>(mode, a, s, tile_shift);
    case 256: return row_dispatch_mode<256>(mode, a, s, tile_shift);
    default: return cudaErrorInvalidValue;
    }
}
#endif

#if GPE_IN_PART(2)
cudaError_t launch_row_hi(int mode, const PassArgs &a, cudaStream_t s, int tile_shift)
{
    switch (a.nx) {
    case 512: return row_dispatch_mode<512>(mode, a, s, tile_shift);
    case 1024: return row_dispatch_mode<1024>(mode, a, s, tile_shift);
    case 2048: return row_dispatch_mode<2048>(mode, a, s, tile_shift);
    case 4096: return row_dispatch_mode<4096>(mode, a, s, tile_shift);
    case 8192: return row_dispatch_mode<8192>(mode, a, s, tile_shift);
    default: return cudaErrorInvalidValue;
    }
}
#endif

template <int N, int MODE>
static cudaError_t col_launch(const PassArgs &a, const CUtensorMap &map, cudaStream_t s)
{
    using C = ColCfg<N>;
    constexpr int W = col_w(N), G = col_g(N);
    constexpr size_t smem = (G == W ? (size_t)W * C::PS : (size_t)N * W + (size_t)G * C::PS) * sizeof(float2) +
                            (size_t)col_twn<N, MODE>() * sizeof(float4) + 128;
    if constexpr (smem > 48 * 1024) {
        static std::atomic<unsigned long long> attr{0};
        const cudaError_t e = smem_opt_in(col_kernel<N, MODE>, (int)smem, attr);
        if (e != cudaSuccess) return e;
    }
    col_kernel<N, MODE><<<a.nx / W, G * C::TP, smem, s>>>(a, map);
    return cudaGetLastError();
}

template <int N> static cudaError_t col_dispatch_mode(int mode, const PassArgs &a, const CUtensorMap &map,
                                                      cudaStream_t s)
{
    switch (mode) {
    case COL_T: return col_launch<N, COL_T>(a, map, s);
    case COL_T_R: return col_launch<N, COL_T_R>(a, map, s);
    case COL_T_PR: return col_launch<N, COL_T_PR>(a, map, s);
    case COL_T_P: return col_launch<N, COL_T_P>(a, map, s);
    case COL_FFT_F: return col_launch<N, COL_FFT_F>(a, map, s);
    case COL_FFT_I: return col_launch<N, COL_FFT_I>(a, map, s);
    case COL_OBS: return col_launch<N, COL_OBS>(a, map, s);
    case COL_ADJ: return col_launch<N, COL_ADJ>(a, map, s);
    default: return cudaErrorInvalidValue;
    }
}

#if GPE_IN_PART(3)
cudaError_t launch_col_lo(int mode, const PassArgs &a, const CUtensorMap &map, cudaStream_t s)
{
    switch (a.ny) {
    case 8: return col_dispatch_mode<8>(mode, a, map, s);
    case 16: return col_dispatch_mode<16>(mode, a, map, s);
    case 32: return col_dispatch_mode<32>(mode, a, map, s);
    case 64: return col_dispatch_mode<64>(mode, a, map, s);
    case 128: return col_dispatch_mode<128>(mode, a, map, s);
    case 256: return col_dispatch_mode<256>(mode, a, map, s);
    default: return cudaErrorInvalidValue;
    }
}
#endif

#if GPE_IN_PART(4)
cudaError_t launch_col_hi(int mode, const PassArgs &a, const CUtensorMap &map, cudaStream_t s)
{
    switch (a.ny) {
    case 512: return col_dispatch_mode<512>(mode, a, map, s);
    case 1024: return col_dispatch_mode<1024>(mode, a, map, s);
    case 2048: return col_dispatch_mode<2048>(mode, a, map, s);
    case 4096: return col_dispatch_mode<4096>(mode, a, map, s);
    case 8192: return col_dispatch_mode<8192>(mode, a, map, s);
    default: return cudaErrorInvalidValue;
    }
}
#endif


#if GPE_IN_PART(2)
template <int N> static cudaError_t row_group_launch(const PassArgs &a, cudaStream_t s)
{
    using C = RowGroupCfg<N>;
    static std::atomic<unsigned long long> attr{0};
    const cudaError_t e = smem_opt_in(row_group_kernel<N>, (int)C::SMEM, attr);
    if (e != cudaSuccess) return e;
    // as few CTAs as finish the items in the fewest rounds (items per group):
    // 2048 rows on 148 SMs take 4 rounds either way, and 128 CTAs of 4 full
    // rounds leave 20 SMs to other grids' passes instead of idle groups in a
    // partial last round (8 x 2048^2 under gpe_step_many: 74.4 against 74.1
    // G pt*steps/s; no difference with 2 lanes and no graphs)
    const int items = a.ny / C::RG;
    const int slots = sm_count() * C::NG;
    const int rounds = (items + slots - 1) / slots;
    const int grid = (items + rounds * C::NG - 1) / (rounds * C::NG);
    row_group_kernel<N><<<grid, C::THREADS, C::SMEM, s>>>(a, items);
    return cudaGetLastError();
}

cudaError_t launch_row_group(const PassArgs &a, cudaStream_t s)
{
    switch (a.nx) {
    case 512: return row_group_launch<512>(a, s);
    case 1024: return row_group_launch<1024>(a, s);
    case 2048: return row_group_launch<2048>(a, s);
    default: return cudaErrorInvalidValue;
    }
}

template <int N> static cudaError_t row_stream_launch(const PassArgs &a, cudaStream_t s)
{
    using C = RowStreamCfg<N>;
    static std::atomic<unsigned long long> attr{0};
    const cudaError_t e = smem_opt_in(row_stream_kernel<N>, (int)C::SMEM, attr);
    if (e != cudaSuccess) return e;
    const int items = a.ny / C::RPC;
    int grid = C::CTAS_PER_SM * sm_count();
    if (grid > items) grid = items;
    row_stream_kernel<N><<<grid, C::THREADS, C::SMEM, s>>>(a, items);
    return cudaGetLastError();
}

cudaError_t launch_row_stream(const PassArgs &a, cudaStream_t s)
{
    switch (a.nx) {
    case 4096: return row_stream_launch<4096>(a, s);
    default: return cudaErrorInvalidValue;
    }
}
#endif  // GPE_IN_PART(2)

#if GPE_IN_PART(4)
template <int N, int MODE> static cudaError_t col_stream_launch(const PassArgs &a, const CUtensorMap &map, cudaStream_t s)
{
    using C = ColStreamCfg<N>;
    static std::atomic<unsigned long long> attr{0};
    const cudaError_t e = smem_opt_in(col_stream_kernel<N, MODE>, (int)C::SMEM, attr);
    if (e != cudaSuccess) return e;
    const int items = a.nx / C::W;
    int grid = C::CTAS_PER_SM * sm_count();
    if (grid > items) grid = items;
    col_stream_kernel<N, MODE><<<grid, C::THREADS, C::SMEM, s>>>(a, map, items);
    return cudaGetLastError();
}

template <int N> static cudaError_t col_stream_mode(int mode, const PassArgs &a, const CUtensorMap &map, cudaStream_t s)
{
    switch (mode) {
    case COL_T: return col_stream_launch<N, COL_T>(a, map, s);
    case COL_T_R: return col_stream_launch<N, COL_T_R>(a, map, s);
    case COL_T_PR: return col_stream_launch<N, COL_T_PR>(a, map, s);
    case COL_T_P: return col_stream_launch<N, COL_T_P>(a, map, s);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_col_stream(int mode, const PassArgs &a, const CUtensorMap &map, cudaStream_t s)
{
    switch (a.ny) {
    case 2048: return col_stream_mode<2048>(mode, a, map, s);
    case 4096: return col_stream_mode<4096>(mode, a, map, s);
    default: return cudaErrorInvalidValue;
    }
}
#endif  // GPE_IN_PART(4)

#if GPE_IN_PART(0)
cudaError_t launch_tables(const Tables &T, int nx, int ny, double Lx, double Ly, double m, double wx,
                          double wy, double lkx, double lky, double kc, cudaStream_t s)
{
    const int n = nx > ny ? nx : ny;
    tables_kernel<<<(n + 255) / 256, 256, 0, s>>>(T, nx, ny, Lx, Ly, m, wx, wy, lkx, lky, kc);
    return cudaGetLastError();
}

cudaError_t launch_kinetic_tables(const Tables &T, int nx, int ny, double Lx, double Ly, double m, double dt,
                                  int imag, cudaStream_t s)
{
    const int n = nx > ny ? nx : ny;
    kinetic_tables_kernel<<<(n + 255) / 256, 256, 0, s>>>(T, nx, ny, Lx, Ly, m, dt, imag);
    return cudaGetLastError();
}

static int grid_for(size_t n, int cap)
{
    const size_t b = (n + 255) / 256;
    return (int)(b < (size_t)cap ? b : (size_t)cap);
}

cudaError_t launch_kin_energy_mul(float2 *f, int nx, int ny, double Lx, double Ly, double m, cudaStream_t s)
{
    kin_energy_mul_kernel<<<grid_for((size_t)nx * ny, 4 * 148), 256, 0, s>>>(f, nx, ny, Lx, Ly, m);
    return cudaGetLastError();
}

cudaError_t launch_adj_overlap(const float2 *psi, const float2 *phi, const Tables &T, int nx, int ny, float L0x,
                               float L0y, cudaStream_t s)
{
    adj_overlap_kernel<<<grid_for((size_t)nx * ny, 1024), 256, 0, s>>>(psi, phi, T, nx, ny, L0x, L0y);
    return cudaGetLastError();
}

cudaError_t launch_adj_terminal(float2 *lam, const float2 *psi, const float2 *phi, const PassArgs &a, float c_re,
                                float c_im, float dxdy, cudaStream_t s)
{
    adj_terminal_kernel<<<grid_for((size_t)a.nx * a.ny, 4 * 148), 256, 0, s>>>(lam, psi, phi, a, c_re, c_im, dxdy);
    return cudaGetLastError();
}

cudaError_t launch_kbin(const float2 *f, const Tables &T, int nx, int ny, double Lx, double Ly, int axis, double k0,
                        int nmax, cudaStream_t s)
{
    kbin_kernel<<<grid_for((size_t)nx * ny, 1024), 256, 0, s>>>(f, T, nx, ny, Lx, Ly, axis, k0, nmax);
    return cudaGetLastError();
}

cudaError_t launch_timeout_probe(DevScalars *sc, int spins, cudaStream_t s)
{
    timeout_probe_kernel<<<1, 32, 0, s>>>(sc, spins);
    return cudaGetLastError();
}
#endif  // GPE_IN_PART(0)

}  // namespace gpe
