// gpe_pair.cu -- pencil-pair variants of the column and row passes (sm_103a).
//
// The column pass of Sec. 3.1's split step (T_y = F_y^-1 K_y F_y on every
// column, Eq. 3, optionally followed by the closing half phase and the FP64
// reductions of Eqs. 14-15) on a TMA tile of two columns, transformed as one
// pencil pair by the packed f32x2 FFT of gpe_fft2.cuh: each thread holds the
// same 16 elements of both columns, so every add and multiply of the
// transform, the kinetic factor and the phase is one f32x2 instruction for
// the two columns, and each twiddle, kinetic-factor and y-table entry is
// loaded once for both.  Against the one-pencil pass (gpe_kernels.cu) that
// halves the twiddle and table reads, and removes the stride-2 dense tile
// accesses; the CTA has half the threads (N/16 for a 2-column tile), each
// with twice the registers.
#include <cuda.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <atomic>

#include "../../include/gpe.h"
#include "gpe_device.cuh"
#include "gpe_fft2.cuh"
#include "gpe_internal.h"
#include "gpe_pair.cuh"

namespace gpe {

// Shared memory holds the exchange slots alone: the twiddle table is read
// through L1 at every length.  Staged per CTA (32.6 KB at 2048 points) it
// held an SM to 3 CTAs of 4 warps; from L1 the registers set the limit, 4
// CTAs at 2048 points.  Each pass alone ran a little slower (2048: row 34.0
// -> 34.6 us, column 33.0 -> 34.7 us), but the lockstep step of 8 grids,
// whose passes share the SMs, ran 95.5 -> 98.1 G pt*steps/s (1024^2: 89.4 ->
// 93.7).
template <int N> struct PairOccupancy {
    static constexpr int E = 16, TP = N / E;       // threads per pencil pair
    static constexpr int SLOTS = pad8_len(N);      // 16-byte exchange slots, overlaying the dense pair
    static constexpr size_t SMEM = (size_t)SLOTS * 16 + 128;
    // CTAs per SM the registers are sized for: as many as the shared memory
    // holds, but no fewer than 128 registers per thread (4 CTAs at 2048
    // points, 2 at 4096, 1 at 8192), at most 16
    static constexpr int BY_SMEM = (int)((224u * 1024u) / (SMEM + 1024));
    static constexpr int BY_REGS = 65536 / (TP * 128);
    static constexpr int CAP = BY_REGS < 16 ? BY_REGS : 16;
    static constexpr int MIN_CTAS = BY_SMEM < CAP ? BY_SMEM : CAP;
};

template <int N> struct ColPairCfg : PairOccupancy<N> {
    static constexpr int BR = N < 256 ? N : 256;   // rows per TMA box (the context's tensor map)
};

// Column pass over a 2-column tile as one pencil pair.  MODE: COL_T (T_y),
// COL_T_R (T_y, then the norm and cavity overlaps of the result reduced in
// FP64, Eqs. 14-15), COL_T_PR (T_y, the closing half phase, the reductions),
// COL_T_P (T_y, the closing half phase).
template <int N, int MODE>
__global__ void __launch_bounds__(ColPairCfg<N>::TP, ColPairCfg<N>::MIN_CTAS)
    col_pair_kernel(const PassArgs a, const __grid_constant__ CUtensorMap map)
{
    using C = ColPairCfg<N>;
    constexpr int E = C::E, TP = C::TP;
    constexpr bool REDUCE = (MODE == COL_T_R || MODE == COL_T_PR);
    extern __shared__ unsigned char smraw[];
    __shared__ __align__(8) uint64_t bar;
    __shared__ double red[32 * NQ];

    const uint32_t s0 = smem_u32(smraw);
    float4 *tile = reinterpret_cast<float4 *>(smraw + ((128u - (s0 & 127u)) & 127u));   // [N] {A, B} rows
    const Tables &T = a.T;
    const bool inb = check_index((long long)blockIdx.x * 2 + 1, a.nx, T.sc) &&
                     check_index((long long)((unsigned char *)(tile + C::SLOTS) - smraw) - 1, dyn_smem_bytes(), T.sc);
    const int c0 = inb ? blockIdx.x * 2 : 0;

    if (threadIdx.x == 0) mbar_init(&bar, 1);
    __syncthreads();
    if (threadIdx.x == 0) {
        mbar_expect_tx(&bar, (uint32_t)N * 16u);
        for (int r0 = 0; r0 < N; r0 += C::BR) tma_load_2d(tile + r0, &map, &bar, 2 * c0, r0);
    }
    // the tile arrived in time.  Otherwise the copies are
    // given time to land, the CTA stores nothing and adds zero partial sums,
    // so that every reduction still counts all of its CTAs.
    const bool ok = __syncthreads_and(mbar_wait_bounded(&bar, 0, a.spins));
    if (!ok) {
        if (threadIdx.x == 0) {
            latch_status(T.sc, GPE_ETIMEOUT);
            mbar_drain(&bar, 0);
        }
        if constexpr (!REDUCE) return;
    }

    const int j = threadIdx.x;
    float2 X[E], Y[E];
#pragma unroll
    for (int r = 0; r < E; ++r) {
        const float4 t = tile[j + r * TP];          // {re_A, im_A, re_B, im_B}
        X[r] = make_float2(t.x, t.z);
        Y[r] = make_float2(t.y, t.w);
    }
    __syncthreads();                                // dense reads done before the exchange writes

    transform_pair<N, E, TP>(X, Y, tile, j, T.twy, T.kiny, a.sy, a.imag);

    float q[3] = {0.f, 0.f, 0.f};
    if constexpr (MODE == COL_T_P) {
        // the closing half phase alone (each y-table entry read once for both columns)
        const PotCoefs pa = col_coefs(a, __ldg(&T.xtab[c0])), pb = col_coefs(a, __ldg(&T.xtab[c0 + 1]));
        float2 V[E];
#pragma unroll
        for (int r = 0; r < E; ++r) {
            const int yi = j + r * TP;
            V[r] = pot_at2(pa, pb, __ldg(&T.ytab[yi]));
            if (a.V) {
                const float2 va = make_float2(__ldg(&a.V[(size_t)yi * a.nx + c0]), __ldg(&a.V[(size_t)yi * a.nx + c0 + 1]));
                V[r] = fma2(bc2(a.V_scale), va, V[r]);
            }
        }
        phase_all2<E>(X, Y, V, a.g, a.ph.h, a.imag);
    }
    if constexpr (REDUCE) {
        // per column: n0 = sum |psi|^2, n1 = sum cos(kc y) |psi|^2 (after the
        // closing phase in COL_T_PR; each y-table entry read once for both)
        const float4 xa = __ldg(&T.xtab[c0]), xb = __ldg(&T.xtab[c0 + 1]);
        PotCoefs pa{}, pb{};
        if constexpr (MODE == COL_T_PR) {
            pa = col_coefs(a, xa);
            pb = col_coefs(a, xb);
        }
        float2 n0 = make_float2(0.f, 0.f), n1 = n0;
        float cz[E];                                // cos(kc y) of each element
        if constexpr (MODE == COL_T_PR) {
            float2 V[E];
#pragma unroll
            for (int r = 0; r < E; ++r) {
                const int yi = j + r * TP;
                const float4 yt = __ldg(&T.ytab[yi]);
                cz[r] = yt.z;
                V[r] = pot_at2(pa, pb, yt);
                if (a.V) {
                    const float2 va = make_float2(__ldg(&a.V[(size_t)yi * a.nx + c0]), __ldg(&a.V[(size_t)yi * a.nx + c0 + 1]));
                    V[r] = fma2(bc2(a.V_scale), va, V[r]);
                }
            }
            phase_all2<E>(X, Y, V, a.g, a.ph.h, a.imag);
        } else {
#pragma unroll
            for (int r = 0; r < E; ++r) cz[r] = __ldg(&T.ytab[j + r * TP]).z;
        }
#pragma unroll
        for (int r = 0; r < E; ++r) {
            const float2 n = fma2(X[r], X[r], mul2(Y[r], Y[r]));
            n0 = add2(n0, n);
            n1 = fma2(bc2(cz[r]), n, n1);
        }
        q[0] = n0.x + n0.y;
        q[1] = xa.z * n1.x + xb.z * n1.y;
        q[2] = xa.z * xa.z * n0.x + xb.z * xb.z * n0.y;
    }

    // every exchange read finished at the last stage's barrier
#pragma unroll
    for (int r = 0; r < E; ++r) tile[j + r * TP] = make_float4(X[r].x, Y[r].x, X[r].y, Y[r].y);
    fence_proxy_async();                            // generic-proxy writes visible to the TMA store
    __syncthreads();
    if (threadIdx.x == 0 && ok && inb) {
        for (int r0 = 0; r0 < N; r0 += C::BR) tma_store_2d(&map, tile + r0, 2 * c0, r0);
        bulk_commit();
    }
    if constexpr (REDUCE) {
        if (!ok || !inb) q[0] = q[1] = q[2] = 0.f;
        block_sum<3>(q, T.part_col + (size_t)blockIdx.x * NQ, red);
        double S[3];
        if (last_block_total<3>(T.part_col, &T.sc->ticket[1], S, red) && threadIdx.x == 0)
            finalize_fields(S, a.red, T.sc);
    }
    if (threadIdx.x == 0) bulk_wait_read_all();     // the tile is read before the CTA exits
}

// ------------------------------------------------------------------ row pass
// Row pass ROW_PT ([scale c] potential phase, T_x = F_x^-1 K_x F_x) on two
// consecutive rows as one pencil pair: one CTA of N/16 threads per row pair,
// the two rows (contiguous in psi) brought in with one bulk copy and written
// back with one; the coordinate table and kinetic factors of each x are read
// once for both rows.  Twiddles through L1 as in the column pass.
template <int N> struct RowPairCfg : PairOccupancy<N> {
    static constexpr uint32_t ROW_BYTES = 2u * N * 8u;
};

template <int N>
__global__ void __launch_bounds__(RowPairCfg<N>::TP, RowPairCfg<N>::MIN_CTAS) row_pair_kernel(const PassArgs a)
{
    using C = RowPairCfg<N>;
    constexpr int E = C::E, TP = C::TP;
    extern __shared__ unsigned char smraw[];
    __shared__ __align__(8) uint64_t bar;

    const uint32_t s0 = smem_u32(smraw);
    float4 *tile = reinterpret_cast<float4 *>(smraw + ((128u - (s0 & 127u)) & 127u));
    float2 *rows = reinterpret_cast<float2 *>(tile);                  // row A [0, N), row B [N, 2N)
    const Tables &T = a.T;
    const bool inb = check_index((long long)blockIdx.x * 2 + 1, a.ny, T.sc) &&
                     check_index((long long)((unsigned char *)(tile + C::SLOTS) - smraw) - 1, dyn_smem_bytes(), T.sc);
    const int y0 = inb ? blockIdx.x * 2 : 0;
    float2 *src = a.psi + (size_t)y0 * N;

    if (threadIdx.x == 0) mbar_init(&bar, 1);
    __syncthreads();
    if (threadIdx.x == 0) {
        mbar_expect_tx(&bar, C::ROW_BYTES);
        bulk_load_1d(rows, src, C::ROW_BYTES, &bar);
    }
    // the rows arrived in time; otherwise the copy is
    // given time to land and the CTA stores nothing
    if (!__syncthreads_and(mbar_wait_bounded(&bar, 0, a.spins))) {
        if (threadIdx.x == 0) {
            latch_status(T.sc, GPE_ETIMEOUT);
            mbar_drain(&bar, 0);
        }
        return;
    }

    const int j = threadIdx.x;
    const float cs = a.use_c ? (float)T.sc->c : 1.f;
    float2 X[E], Y[E];
#pragma unroll
    for (int r = 0; r < E; ++r) {
        const float2 p = rows[j + r * TP], q = rows[N + j + r * TP];
        X[r] = make_float2(p.x * cs, q.x * cs);
        Y[r] = make_float2(p.y * cs, q.y * cs);
    }
    __syncthreads();                                // dense reads done before the exchange writes

    const PotCoefs pa = row_coefs(a, __ldg(&T.ytab[y0])), pb = row_coefs(a, __ldg(&T.ytab[y0 + 1]));
    const float *Va = a.V ? a.V + (size_t)y0 * N : nullptr;
    float2 V[E];
#pragma unroll
    for (int r = 0; r < E; ++r) {
        const int xi = j + r * TP;
        V[r] = pot_at2(pa, pb, __ldg(&T.xtab[xi]));
        if (Va) V[r] = fma2(bc2(a.V_scale), make_float2(__ldg(&Va[xi]), __ldg(&Va[N + xi])), V[r]);
    }
    phase_all2<E>(X, Y, V, a.g, a.ph.h, a.imag);
    transform_pair<N, E, TP>(X, Y, tile, j, T.twx, T.kinx, a.sx, a.imag);

    // every exchange read finished at the last stage's barrier
#pragma unroll
    for (int r = 0; r < E; ++r) {
        rows[j + r * TP] = make_float2(X[r].x, Y[r].x);
        rows[N + j + r * TP] = make_float2(X[r].y, Y[r].y);
    }
    fence_proxy_async();                            // generic-proxy writes visible to the bulk store
    __syncthreads();
    if (threadIdx.x == 0) {
        if (inb) {
            bulk_store_1d(src, rows, C::ROW_BYTES);
            bulk_commit();
        }
        bulk_wait_read_all();                       // the rows are read before the CTA exits
    }
}

template <int N> static cudaError_t row_pair_launch(const PassArgs &a, cudaStream_t s)
{
    using C = RowPairCfg<N>;
    static std::atomic<unsigned long long> attr{0};
    const cudaError_t e = smem_opt_in(row_pair_kernel<N>, (int)C::SMEM, attr);
    if (e != cudaSuccess) return e;
    row_pair_kernel<N><<<a.ny / 2, C::TP, C::SMEM, s>>>(a);
    return cudaGetLastError();
}

// Rows of 512..8192 points (the grid has at least 8 rows, an even number).
bool row_pair_ok(int nx, int ny) { return nx >= 512 && nx <= 8192 && (nx & (nx - 1)) == 0 && ny >= 2; }

cudaError_t launch_row_pair(const PassArgs &a, cudaStream_t s)
{
    if (!row_pair_ok(a.nx, a.ny)) return cudaErrorInvalidValue;
    switch (a.nx) {
    case 512: return row_pair_launch<512>(a, s);
    case 1024: return row_pair_launch<1024>(a, s);
    case 2048: return row_pair_launch<2048>(a, s);
    case 4096: return row_pair_launch<4096>(a, s);
    case 8192: return row_pair_launch<8192>(a, s);
    default: return cudaErrorInvalidValue;
    }
}

// ------------------------------------------------------------------ column launchers
template <int N, int MODE>
static cudaError_t col_pair_launch(const PassArgs &a, const CUtensorMap &map, cudaStream_t s)
{
    using C = ColPairCfg<N>;
    static std::atomic<unsigned long long> attr{0};
    const cudaError_t e = smem_opt_in(col_pair_kernel<N, MODE>, (int)C::SMEM, attr);
    if (e != cudaSuccess) return e;
    col_pair_kernel<N, MODE><<<a.nx / 2, C::TP, C::SMEM, s>>>(a, map);
    return cudaGetLastError();
}

template <int N> static cudaError_t col_pair_mode(int mode, const PassArgs &a, const CUtensorMap &map, cudaStream_t s)
{
    switch (mode) {
    case COL_T: return col_pair_launch<N, COL_T>(a, map, s);
    case COL_T_R: return col_pair_launch<N, COL_T_R>(a, map, s);
    case COL_T_PR: return col_pair_launch<N, COL_T_PR>(a, map, s);
    case COL_T_P: return col_pair_launch<N, COL_T_P>(a, map, s);
    default: return cudaErrorInvalidValue;
    }
}

// Columns of 512..8192 points in tiles of 2 (the context's tensor map box).
bool col_pair_ok(int nx, int ny)
{
    return (ny == 512 || ny == 1024 || ny == 2048 || ny == 4096 || ny == 8192) && nx >= 2;
}

cudaError_t launch_col_pair(int mode, const PassArgs &a, const CUtensorMap &map, cudaStream_t s)
{
    if (!col_pair_ok(a.nx, a.ny)) return cudaErrorInvalidValue;
    switch (a.ny) {
    case 512: return col_pair_mode<512>(mode, a, map, s);
    case 1024: return col_pair_mode<1024>(mode, a, map, s);
    case 2048: return col_pair_mode<2048>(mode, a, map, s);
    case 4096: return col_pair_mode<4096>(mode, a, map, s);
    case 8192: return col_pair_mode<8192>(mode, a, map, s);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace gpe
