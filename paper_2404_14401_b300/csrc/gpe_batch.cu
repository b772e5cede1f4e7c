// gpe_batch.cu -- the persistent batch kernel: n lockstep split steps
// (Sec. 3.1, Eqs. 3-4; imaginary time Sec. 3.3; cavity Sec. 5.3, Eqs. 10-15)
// of many contexts, of any mix of supported sizes, in one launch.
//
// The passes are those of the host scheduler (gpe_api.cu): row pass = the
// potential phase then T_x = F_x^-1 K_x F_x; column pass = T_y, optionally the
// closing half phase, with the FP64 norm / overlap reductions that set the
// renormalisation and the cavity field.  Here every pass of every context is
// cut into items of 256 threads' work: a row item is 256/(N/16) whole rows
// (plain coalesced loads, registers, stores), a column item a tile of
// 256/(N/16) whole columns loaded with TMA into shared memory and stored back
// with coalesced stores.  All items of all passes form one queue, ordered by
// pass (lockstep: pass q of every context before pass q + 1 of any), which
// the CTAs take in order from one global counter.  An item of pass q of
// context i first waits until pass q - 1 of context i is complete: a
// per-context counter that the item finishing a pass raises, after it has
// summed the pass's per-item partial sums in item order and updated the
// context's scalars (1/sqrt(norm), alpha).  Every item before it in the queue
// is held by a running CTA, so every wait ends; each wait is still bounded,
// and one that runs out sets an abort flag that ends the launch with
// GPE_ETIMEOUT latched.
//
// Coherence between CTAs of the one launch: psi, the partial sums and the
// scalars are read through L2 (ld.global.cg) and written with st.global.cg,
// never through the non-coherent L1; a pass's completion is published with a
// release store after a fence by every thread of the finishing item, and
// acquired before an item starts; before a TMA load of data that other CTAs
// wrote through the generic proxy the loading thread issues a proxy fence.
#include <cuda.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <atomic>

#include "../../include/gpe.h"
#include "gpe_ctrl.cuh"
#include "gpe_device.cuh"
#include "gpe_fft.cuh"
#include "gpe_internal.h"

namespace gpe {

constexpr int kE = 16;                                        // elements per thread
// padded pencils of one tile of BT threads (float2)
template <int BT> __host__ __device__ constexpr int buf_f2() { return BT * kE + BT; }

int batch_rows_per_item(int n, int bt) { return n >= 16 && bt >= n / kE ? bt / (n / kE) : 0; }

int batch_supported(int nx, int ny, int bt)
{
    auto ok = [](int n) { return n >= 64 && n <= 2048 && (n & (n - 1)) == 0; };
    const int rpi = batch_rows_per_item(nx, bt), cpi = batch_rows_per_item(ny, bt);
    // a row tile holds whole rows; a column tile at least 2 whole columns (a
    // TMA box row of 16 bytes) and at most the grid's width
    return ok(nx) && ok(ny) && rpi >= 1 && rpi <= ny && cpi >= 2 && cpi <= nx;
}

// ------------------------------------------------------------------ the queue
// One queue entry: pass q (its mode, a row or a column pass) of context i,
// item k of that pass; the phase time and length and the reduction time of
// the pass.  The program of a launch (prologue, n steps, epilogue) is the
// host scheduler's: see step_prologue / step_part / step_epilogue.
struct Item {
    int q, mode, col, i, k, use_c, reduce;
    double tp, h, tr;                      // phase at tp over h; reduction at tr (h = 0: no phase)
};

__device__ int per_step_passes(const BatchArgs &b) { return b.imag && b.cavity ? 3 : 2; }

// mode and kind of pass position `pos` of step s
__device__ void step_pass(const BatchArgs &b, int s, int pos, Item &it)
{
    const double ts = __dadd_rn(b.t0, __dmul_rn((double)s, b.dt));
    const double te = __dadd_rn(b.t0, __dmul_rn((double)(s + 1), b.dt));
    it.use_c = 0;
    it.h = 0.0;
    if (pos == 0) {                        // row pass: phase, T_x
        it.mode = ROW_PT;
        it.col = 0;
        it.tp = it.tr = ts;
        it.h = b.imag ? 0.5 * b.dt : (s == 0 ? 0.5 * b.dt : b.dt);
        it.use_c = b.imag && s > 0;
        it.reduce = 0;
    } else if (pos == 1) {                 // column pass: T_y [+ closing phase] [+ reductions]
        it.col = 1;
        it.tr = it.tp = te;
        if (b.cavity) {
            it.mode = COL_T_R;
            it.reduce = 1;
        } else if (b.imag || s == b.n - 1) {
            it.mode = COL_T_PR;
            it.h = 0.5 * b.dt;
            it.reduce = 1;
        } else {
            it.mode = COL_T;
            it.reduce = 0;
        }
    } else {                               // imaginary time with a cavity: closing phase with alpha of the new density
        it.mode = ROW_PHASE_R;
        it.col = 0;
        it.tp = it.tr = te;
        it.h = 0.5 * b.dt;
        it.reduce = 1;
    }
}

__device__ int items_of(const BatchArgs &b, int col) { return col ? b.col_prefix[b.count] : b.row_prefix[b.count]; }

__device__ Item locate(const BatchArgs &b, unsigned int idx)
{
    Item it;
    const int R = items_of(b, 0);
    const int Pp = b.cavity ? 1 : 0, Ps = per_step_passes(b);
    int ST = 0;
    for (int pos = 0; pos < Ps; ++pos) ST += (pos == 1) ? items_of(b, 1) : R;
    long long r = idx;
    if (r < (long long)Pp * R) {           // prologue: alpha of the initial density
        it.q = 0;
        it.mode = ROW_REDUCE_R;
        it.col = 0;
        it.tp = it.tr = b.t0;
        it.h = 0.0;
        it.use_c = 0;
        it.reduce = 1;
    } else {
        r -= (long long)Pp * R;
        const long long s = r / ST;
        if (s < b.n) {
            r -= s * ST;
            int pos = 0;
            for (; pos < Ps; ++pos) {
                const int cnt = (pos == 1) ? items_of(b, 1) : R;
                if (r < cnt) break;
                r -= cnt;
            }
            step_pass(b, (int)s, pos, it);
            it.q = Pp + (int)s * Ps + pos;
        } else {                           // epilogue
            r -= (long long)b.n * ST;
            const double tn = __dadd_rn(b.t0, __dmul_rn((double)b.n, b.dt));
            it.q = Pp + b.n * Ps;
            it.col = 0;
            it.tp = it.tr = tn;
            it.use_c = 0;
            it.reduce = 0;
            if (b.imag) {
                it.mode = ROW_SCALE;
                it.h = 0.0;
            } else {
                it.mode = ROW_PHASE;
                it.h = 0.5 * b.dt;
            }
        }
    }
    const int *pre = it.col ? b.col_prefix : b.row_prefix;
    int lo = 0, hi = b.count;              // pre[lo] <= r < pre[hi]
    while (hi - lo > 1) {
        const int mid = (lo + hi) / 2;
        if (pre[mid] <= r) lo = mid; else hi = mid;
    }
    it.i = lo;
    it.k = (int)(r - pre[lo]);
    return it;
}

// total queue length for the program of a launch (host and device)
__host__ __device__ inline long long batch_total(int n, int imag, int cavity, int R, int C)
{
    const int Pp = cavity ? 1 : 0;
    const long long ST = (long long)R + C + (imag && cavity ? R : 0);
    const int Pe = (imag || cavity) ? 1 : 0;
    return (long long)Pp * R + (long long)n * ST + (long long)Pe * R;
}

// ------------------------------------------------------------------ items
// One row tile: RPI whole rows, plain coalesced loads through L2, the pass's
// pointwise work and T_x in registers and shared memory, stores through L2;
// the tile's norm / overlap sums are added to q.
template <int N, int BT>
__device__ void row_tile(const BatchCtx &c, int tile, const Item &it, const PhaseArgs &ph, int imag, float2 *buf,
                         float (&q)[3])
{
    constexpr int E = kE, TP = N / E, RPI = BT / TP, PS = N + N / 16;
    const int lr = threadIdx.x / TP, j = threadIdx.x % TP;
    const Tables &T = c.T;
    const bool inb = check_index((long long)tile * RPI + lr, c.ny, T.sc);   // bounds-check build
    const int y = inb ? tile * RPI + lr : 0;
    float2 *row = c.psi + (size_t)y * N;
    float2 *sb = buf + lr * PS;
    float2 v[E];
#pragma unroll
    for (int r = 0; r < E; ++r) v[r] = inb ? __ldcg(&row[j + r * TP]) : make_float2(0.f, 0.f);
    const float4 yt = __ldg(&T.ytab[y]);
    const int mode = it.mode;
    if (mode == ROW_PT || mode == ROW_PHASE || mode == ROW_PHASE_R) {
        float acx2, acxcy;
        if (ph.use_alpha) alpha_amps(ph, __ldcg(&T.sc->alpha_re), __ldcg(&T.sc->alpha_im), acx2, acxcy);
        else alpha_amps(ph, 0.0, 0.0, acx2, acxcy);
        const PotCoefs pc = row_coefs_from(ph, acx2, acxcy, yt);
        const float cs = (mode == ROW_PT && it.use_c) ? (float)__ldcg(&T.sc->c) : 1.f;
        const float *Vr = c.V ? c.V + (size_t)y * N : nullptr;
#pragma unroll
        for (int r = 0; r < E; ++r) {
            const int xi = j + r * TP;
            float V = pot_at(pc, __ldg(&T.xtab[xi]));
            if (Vr) V += c.V_scale * __ldg(&Vr[xi]);
            v[r] = phase_mul(make_float2(v[r].x * cs, v[r].y * cs), V, c.g, ph.h, imag);
        }
    }
    if (mode == ROW_SCALE) {
        const float cs = (float)__ldcg(&T.sc->c);
#pragma unroll
        for (int r = 0; r < E; ++r) v[r] = make_float2(v[r].x * cs, v[r].y * cs);
    }
    if (mode == ROW_PT) {
        fft_pencil<N, E, false>(v, sb, j, 1, T.twx);
        kinetic_axis<E, TP>(v, T.kinx, j, c.sx, imag);
        fft_pencil<N, E, true>(v, sb, j, 1, T.twx);
    }
    if (it.reduce && inb) {
        float q0 = 0.f, q1 = 0.f, q2 = 0.f;
#pragma unroll
        for (int r = 0; r < E; ++r) {
            const float cx = __ldg(&T.xtab[j + r * TP]).z;
            const float n = v[r].x * v[r].x + v[r].y * v[r].y;
            q0 += n;
            q1 += cx * n;
            q2 += cx * cx * n;
        }
        q[0] += q0;
        q[1] += q1 * yt.z;
        q[2] += q2;
    }
    if (mode != ROW_REDUCE_R && inb)
#pragma unroll
        for (int r = 0; r < E; ++r) __stcg(&row[j + r * TP], v[r]);
}

// A row item: tiles k tpi .. min((k + 1) tpi, row_tiles) - 1, then one
// FP64 partial sum of the item.  The exchange buffers are free again when a
// tile ends (its last exchange ends with a barrier after the reads).
template <int N, int BT>
__device__ void row_item(const BatchCtx &c, const Item &it, const PhaseArgs &ph, int imag, int tpi, float2 *buf,
                         double *red)
{
    float q[3] = {0.f, 0.f, 0.f};
    const int t0 = it.k * tpi, t1 = min(t0 + tpi, c.row_tiles);
    for (int t = t0; t < t1; ++t) row_tile<N, BT>(c, t, it, ph, imag, buf, q);
    if (it.reduce) block_sum<3>(q, c.T.part_row + (size_t)it.k * NQ, red);
}

// One column tile: TMA load of the dense [N][G] tile, T_y [+ closing phase]
// [+ the tile's sums into q], results back into the tile and out with
// coalesced stores through L2.  False if the tile's bounded wait ran out (the
// copy has then been given its time to land; nothing is stored).
template <int N, int BT>
__device__ bool col_tile(const BatchCtx &c, int tile, const Item &it, const PhaseArgs &ph, int imag, float2 *buf,
                         uint64_t *bar, uint32_t &parity, int spins, float (&q)[3])
{
    constexpr int E = kE, TP = N / E, G = BT / TP, BR = N < 256 ? N : 256, PS = N + N / 16;
    static_assert(G >= 2 && G * PS <= buf_f2<BT>(), "a tile is 2 or more columns and fits the item buffer");
    const Tables &T = c.T;
    const bool inb = check_index((long long)tile * G + G - 1, c.nx, T.sc);  // bounds-check build
    const int c0 = inb ? tile * G : 0;
    float2 *tile_buf = buf;
    if (threadIdx.x == 0) {
        // psi was written by other CTAs through the generic proxy (acquired
        // above): order those writes before this thread's async-proxy loads.
        // The tensor map itself lives in global memory (written by the host
        // before the launch): acquire it for the tensormap proxy.
        asm volatile("fence.proxy.async.global;" ::: "memory");
        asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(&c.map) : "memory");
        mbar_expect_tx(bar, (uint32_t)(N * G * 8));
        for (int r0 = 0; r0 < N; r0 += BR) tma_load_2d(tile_buf + (size_t)r0 * G, &c.map, bar, 2 * c0, r0);
    }
    const bool ok = __syncthreads_and(mbar_wait_bounded(bar, parity, spins));
    if (!ok) mbar_drain(bar, parity);
    parity ^= 1u;
    if (!ok) return false;

    const int j = threadIdx.x % TP, cg = threadIdx.x / TP;
    float2 v[E];
#pragma unroll
    for (int r = 0; r < E; ++r) v[r] = tile_buf[(j + r * TP) * G + cg];
    __syncthreads();                                   // dense reads done before the exchange writes
    float2 *sb = tile_buf + cg * PS;
    fft_pencil<N, E, false>(v, sb, j, 1, T.twy);
    kinetic_axis<E, TP>(v, T.kiny, j, c.sy, imag);
    fft_pencil<N, E, true>(v, sb, j, 1, T.twy);
    const int mode = it.mode, x = c0 + cg;
    if (mode == COL_T_PR) {
        // closing half phase and its reduction in one loop (one y-table read per point)
        float acx2, acxcy;
        if (ph.use_alpha) alpha_amps(ph, __ldcg(&T.sc->alpha_re), __ldcg(&T.sc->alpha_im), acx2, acxcy);
        else alpha_amps(ph, 0.0, 0.0, acx2, acxcy);
        const float4 xt = __ldg(&T.xtab[x]);
        const PotCoefs pc = col_coefs_from(ph, acx2, acxcy, xt);
        float n0 = 0.f, n1 = 0.f;
#pragma unroll
        for (int r = 0; r < E; ++r) {
            const int yi = j + r * TP;
            const float4 yt = __ldg(&T.ytab[yi]);
            float V = pot_at(pc, yt);
            if (c.V) V += c.V_scale * __ldg(&c.V[(size_t)yi * c.nx + x]);
            v[r] = phase_mul(v[r], V, c.g, ph.h, imag);
            const float n = v[r].x * v[r].x + v[r].y * v[r].y;
            n0 += n;
            n1 += yt.z * n;
        }
        if (inb) {
            q[0] += n0;
            q[1] += xt.z * n1;
            q[2] += xt.z * xt.z * n0;
        }
    } else if (it.reduce && inb) {
        const float cx = __ldg(&T.xtab[x]).z;
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
    // every exchange read finished at the last exchange's barrier
#pragma unroll
    for (int r = 0; r < E; ++r) tile_buf[(j + r * TP) * G + cg] = v[r];
    __syncthreads();
    for (int e = threadIdx.x; e < N * G && inb; e += BT)
        __stcg(&c.psi[(size_t)(e / G) * c.nx + c0 + e % G], tile_buf[e]);
    __syncthreads();                                   // the tile is read out before the next load reuses it
    return true;
}

template <int N, int BT>
__device__ bool col_item(const BatchCtx &c, const Item &it, const PhaseArgs &ph, int imag, int tpi, float2 *buf,
                         double *red, uint64_t *bar, uint32_t &parity, int spins)
{
    float q[3] = {0.f, 0.f, 0.f};
    const int t0 = it.k * tpi, t1 = min(t0 + tpi, c.col_tiles);
    for (int t = t0; t < t1; ++t)
        if (!col_tile<N, BT>(c, t, it, ph, imag, buf, bar, parity, spins, q)) return false;
    if (it.reduce) block_sum<3>(q, c.T.part_col + (size_t)it.k * NQ, red);
    return true;
}

// N: the pencil length of the item's pass (nx for a row pass, ny for a
// column pass).  The 64-thread variant holds rows of at most 1024 points and
// columns of at most 512 (a column tile is at least 2 columns); sizes outside
// a variant are never queued (batch_supported), the branches only keep the
// instantiations valid.
template <int N, int BT>
__device__ bool run_item(const BatchCtx &c, const Item &it, const PhaseArgs &ph, int imag, int tpi, float2 *buf,
                         double *red, uint64_t *bar, uint32_t &parity, int spins)
{
    if (it.col) {
        if constexpr (BT / (N / kE) >= 2) return col_item<N, BT>(c, it, ph, imag, tpi, buf, red, bar, parity, spins);
        else return false;
    }
    if constexpr (BT / (N / kE) >= 1) row_item<N, BT>(c, it, ph, imag, tpi, buf, red);
    else return false;
    return true;
}

template <int BT>
__device__ bool dispatch(int n, const BatchCtx &c, const Item &it, const PhaseArgs &ph, int imag, int tpi,
                         float2 *buf, double *red, uint64_t *bar, uint32_t &parity, int spins)
{
    switch (n) {
    case 64: return run_item<64, BT>(c, it, ph, imag, tpi, buf, red, bar, parity, spins);
    case 128: return run_item<128, BT>(c, it, ph, imag, tpi, buf, red, bar, parity, spins);
    case 256: return run_item<256, BT>(c, it, ph, imag, tpi, buf, red, bar, parity, spins);
    case 512: return run_item<512, BT>(c, it, ph, imag, tpi, buf, red, bar, parity, spins);
    case 1024: return run_item<1024, BT>(c, it, ph, imag, tpi, buf, red, bar, parity, spins);
    default: return run_item<2048, BT>(c, it, ph, imag, tpi, buf, red, bar, parity, spins);
    }
}

// ------------------------------------------------------------------ kernel
// BT: threads per CTA and per tile (256 for batches that fill the GPU with
// such tiles, 64 for narrow ones); CPS: CTAs per SM the launch bounds ask for
// (256 threads: 3 per SM at 80 registers; with 2 per SM, 128 registers and no
// spill, the sweep ran 12% slower)
template <int BT, int CPS>
__global__ void __launch_bounds__(BT, CPS) batch_kernel(const BatchArgs b)
{
    __shared__ __align__(128) float2 buf[buf_f2<BT>()];
    __shared__ double red[32 * NQ];
    __shared__ __align__(8) uint64_t bar;
    __shared__ unsigned int s_idx, s_next;
    __shared__ int s_flag;
    __shared__ PhaseArgs s_ph;
    __shared__ RedArgs s_rd;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        s_next = atomicAdd(&b.head[0], 1u);
    }
    __syncthreads();
    uint32_t parity = 0;
    for (;;) {
        // the queue entry taken one item ahead: the CTA holds at most two
        // entries and starts the later only after finishing the earlier, so
        // the smallest unfinished entry is always being worked on
        if (threadIdx.x == 0) {
            s_idx = ld_acquire(&b.head[1]) ? b.total : s_next;
            if (s_idx < b.total) s_next = atomicAdd(&b.head[0], 1u);
        }
        __syncthreads();
        const unsigned int idx = s_idx;
        if (idx >= b.total) break;
        const Item it = locate(b, idx);
        const BatchCtx &c = b.ctx[it.i];
        // pass q - 1 of this context must be complete (bounded wait: at most
        // min(spins, 2^22) polls of about 64 ns plus an L2 round trip each;
        // a pass of the largest batches takes milliseconds)
        if (threadIdx.x == 0) {
            // the pass's arguments do not depend on the previous pass: work
            // them out while it may still be running
            if (it.h != 0.0) s_ph = phase_dev(c, it.tp, it.h);
            else memset(&s_ph, 0, sizeof(s_ph));
            s_rd = red_dev(c, it.tr);
            int ok = 1, polls = 0;
            unsigned int ns = 32;                      // back off: many CTAs may wait on one counter
            const int limit = b.spins < (1 << 22) ? b.spins : (1 << 22);
            while (ld_acquire(&b.epoch[it.i]) < (unsigned int)it.q) {
                if (polls++ >= limit || ld_acquire(&b.head[1])) {
                    ok = 0;
                    break;
                }
                __nanosleep(ns);
                if (ns < 256) ns *= 2;
            }
            if (!ok) {
                latch_status(c.T.sc, GPE_ETIMEOUT);
                atomicExch(&b.head[1], 1u);
            }
            __threadfence();
            s_flag = ok;
        }
        __syncthreads();
        if (!s_flag) break;
        const PhaseArgs ph = s_ph;
        const int n = it.col ? c.ny : c.nx;
        if (!dispatch<BT>(n, c, it, ph, b.imag, b.tpi, buf, red, &bar, parity, b.spins)) {
            if (threadIdx.x == 0) {
                latch_status(c.T.sc, GPE_ETIMEOUT);
                atomicExch(&b.head[1], 1u);
            }
            break;
        }
        // item complete: count it (the barrier orders every thread's stores
        // before thread 0's fence, which is cumulative); the item that
        // finishes the pass sums the partials, updates the scalars and opens
        // the next pass
        __syncthreads();
        const int items = it.col ? c.col_items : c.row_items;
        if (threadIdx.x == 0) {
            __threadfence();
            s_flag = (atomicAdd(&b.done[it.i], 1u) + 1u == (unsigned int)items);
        }
        __syncthreads();
        if (s_flag) {
            if (it.reduce) {
                double S[3];
                sum_partials<3>(it.col ? c.T.part_col : c.T.part_row, items, S, red);
                if (threadIdx.x == 0) finalize_fields(S, s_rd, c.T.sc);
            }
            if (threadIdx.x == 0) {
                b.done[it.i] = 0u;
                __threadfence();
                st_release(&b.epoch[it.i], (unsigned int)it.q + 1u);
            }
        }
        __syncthreads();
    }
}

// resident CTAs of one variant on the current device (cached per device)
template <int BT, int CPS> static int batch_grid()
{
    static std::atomic<int> cache[64];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    std::atomic<int> &g = cache[dev & 63];
    int v = g.load(std::memory_order_relaxed);
    if (v <= 0) {
        int sms = 0, per = 0;
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, batch_kernel<BT, CPS>, BT, 0) != cudaSuccess)
            return 0;
        v = sms * (per > 0 ? per : 1);
        g.store(v, std::memory_order_relaxed);
    }
    return v;
}

constexpr int kSmallCps = 8;                       // 64-thread CTAs per SM (128 registers at most)

int batch_resident_ctas(int bt) { return bt == 64 ? batch_grid<64, kSmallCps>() : batch_grid<256, 3>(); }

cudaError_t launch_batch(const BatchArgs &b, cudaStream_t s, int grid)
{
    if (grid <= 0) return cudaErrorInvalidConfiguration;
    if ((unsigned int)grid > b.total) grid = (int)b.total;
    if (b.bt == 64) batch_kernel<64, kSmallCps><<<grid, 64, 0, s>>>(b);
    else batch_kernel<256, 3><<<grid, 256, 0, s>>>(b);
    return cudaGetLastError();
}

long long batch_queue_length(int n, int imag, int cavity, int R, int C) { return batch_total(n, imag, cavity, R, C); }

}  // namespace gpe
