// gpe_device.cuh -- device building blocks shared by the pass kernels
// (gpe_kernels.cu) and the persistent batch kernel (gpe_batch.cu): TMA and
// mbarrier wrappers with bounded waits, FP64 block reductions with a
// deterministic last-CTA total, the cavity-field finalisation (Eqs. 14-15),
// and the pointwise pieces of the split step (potential phase, Sec. 3.1;
// kinetic factor, Eq. 3; the adjoint phase).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <atomic>

#include "../../include/gpe.h"
#include "gpe_fft.cuh"
#include "gpe_internal.h"

namespace gpe {

// ------------------------------------------------------------------ TMA / mbarrier
__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// Poll the barrier at most `spins` times; false if it never completed.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity, int spins)
{
    for (int i = 0; i < spins; ++i)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}
// After a wait has run out: give a bulk copy already issued towards this CTA's
// shared memory a fixed number of polls to land, whatever the caller's wait
// limit, so that the CTA does not reuse or release shared memory that the copy
// may still write.  If even this runs out the CTA goes on (nothing better is
// possible without waiting forever).
constexpr int kDrainSpins = 1 << 22;
__device__ __forceinline__ bool mbar_drain(uint64_t *bar, uint32_t parity)
{
    return mbar_wait_bounded(bar, parity, kDrainSpins);
}
__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *map, uint64_t *bar, int x, int y)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%3, %4}], [%2];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_u32(bar)), "r"(x), "r"(y)
        : "memory");
}

__device__ __forceinline__ void tma_store_2d(const CUtensorMap *map, const void *src, int x, int y)
{
    asm volatile("cp.async.bulk.tensor.2d.global.shared::cta.bulk_group [%0, {%2, %3}], [%1];" ::"l"(
                     reinterpret_cast<uint64_t>(map)),
                 "r"(smem_u32(src)), "r"(x), "r"(y)
                 : "memory");
}

__device__ __forceinline__ void bulk_load_1d(void *dst, const void *src, uint32_t bytes, uint64_t *bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}
__device__ __forceinline__ void bulk_store_1d(void *dst, const void *src, uint32_t bytes)
{
    asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(dst), "r"(smem_u32(src)),
                 "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void bulk_wait_read_all() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ void latch_status(DevScalars *sc, int code) { atomicCAS(&sc->status, 0, code); }

// acquire load / release store of a flag or counter that other CTAs of the
// same launch write (GPU scope)
__device__ __forceinline__ unsigned int ld_acquire(const unsigned int *p)
{
    unsigned int v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release(unsigned int *p, unsigned int v)
{
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// ------------------------------------------------------------------ debug bounds checks
// The bounds-check build (GPE_DEBUG_BOUNDS=1) checks, in every pass kernel,
// the global row / column index of each thread's accesses and the extent of
// each CTA's shared-memory regions against their buffers.  A failed check
// latches GPE_EBOUNDS and the access is skipped (loads give zero, stores are
// dropped): nothing traps and the context stays usable.  In the normal build
// every check is true at compile time and costs nothing.
#ifndef GPE_DEBUG_BOUNDS
#define GPE_DEBUG_BOUNDS 0
#endif

// bytes of dynamic shared memory this launch was given
__device__ __forceinline__ uint32_t dyn_smem_bytes()
{
    uint32_t r;
    asm("mov.u32 %0, %%dynamic_smem_size;" : "=r"(r));
    return r;
}

// true if 0 <= i < n; otherwise (bounds-check build) latch GPE_EBOUNDS
__device__ __forceinline__ bool check_index(long long i, long long n, DevScalars *sc)
{
#if GPE_DEBUG_BOUNDS
    if (i >= 0 && i < n) return true;
    latch_status(sc, GPE_EBOUNDS);
    return false;
#else
    (void)i;
    (void)n;
    (void)sc;
    return true;
#endif
}

// ------------------------------------------------------------------ reductions
// Sum K per-thread FP32 partials over the CTA in FP64 with a fixed shuffle
// tree and a fixed warp order; thread 0 writes them to dst[0..K).
template <int K>
__device__ __forceinline__ void block_sum(const float (&q)[K], double *__restrict__ dst, double *red)
{
    double d[K];
#pragma unroll
    for (int i = 0; i < K; ++i) d[i] = (double)q[i];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int width = blockDim.x < 32 ? blockDim.x : 32;
    const unsigned mask = width == 32 ? 0xffffffffu : ((1u << width) - 1u);
    for (int off = width >> 1; off > 0; off >>= 1)
#pragma unroll
        for (int i = 0; i < K; ++i) d[i] += __shfl_down_sync(mask, d[i], off);
    if (lane == 0)
#pragma unroll
        for (int i = 0; i < K; ++i) red[warp * NQ + i] = d[i];
    __syncthreads();
    if (threadIdx.x == 0) {
        const int nw = (blockDim.x + 31) >> 5;
#pragma unroll
        for (int i = 0; i < K; ++i) {
            double s = 0.0;
            for (int w = 0; w < nw; ++w) s += red[w * NQ + i];
            dst[i] = s;
        }
    }
}

// Sum `count` FP64 partial rows part[b][0..K) in a fixed order (a strided
// pass over b per thread, a fixed shuffle tree, warps in order), whatever
// produced them; every thread of the CTA must call it; out[0..K) is valid in
// thread 0.
template <int K>
__device__ __forceinline__ void sum_partials(const double *part, int count, double *out, double *red)
{
    double acc[K];
#pragma unroll
    for (int i = 0; i < K; ++i) acc[i] = 0.0;
    for (int b = threadIdx.x; b < count; b += blockDim.x)
#pragma unroll
        for (int i = 0; i < K; ++i) acc[i] += __ldcg(&part[(size_t)b * NQ + i]);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int width = blockDim.x < 32 ? blockDim.x : 32;
    const unsigned mask = width == 32 ? 0xffffffffu : ((1u << width) - 1u);
    for (int off = width >> 1; off > 0; off >>= 1)
#pragma unroll
        for (int i = 0; i < K; ++i) acc[i] += __shfl_down_sync(mask, acc[i], off);
    __syncthreads();
    if (lane == 0)
#pragma unroll
        for (int i = 0; i < K; ++i) red[warp * NQ + i] = acc[i];
    __syncthreads();
    if (threadIdx.x == 0) {
        const int nw = (blockDim.x + 31) >> 5;
#pragma unroll
        for (int i = 0; i < K; ++i) {
            double s = 0.0;
            for (int w = 0; w < nw; ++w) s += red[w * NQ + i];
            out[i] = s;
        }
    }
}

// After every CTA has stored its partials: the CTA that arrives last sums
// them in block order (deterministic whatever CTA is last) into out[0..K).
// Returns true in the last CTA (all threads), with out valid in thread 0.
template <int K>
__device__ __forceinline__ bool last_block_total(const double *part, unsigned int *ticket, double *out,
                                                 double *red)
{
    __shared__ int s_last;
    if (threadIdx.x == 0) {
        __threadfence();
        const unsigned t = atomicAdd(ticket, 1u);
        s_last = (t == gridDim.x - 1);
    }
    __syncthreads();
    if (!s_last) return false;
    __threadfence();
    sum_partials<K>(part, (int)gridDim.x, out, red);
    if (threadIdx.x == 0) *ticket = 0u;
    return true;
}

// Norm, overlaps, renormalisation scale and cavity field from the sums
// S0 = sum |psi|^2, S1 = sum cos(kc x)cos(kc y)|psi|^2, S2 = sum cos^2(kc x)|psi|^2
// (Sec. 3.3 normalisation; Eqs. 14-15).  One thread, FP64.
[[maybe_unused]] static __device__ void finalize_fields(const double *S, const RedArgs &r, DevScalars *sc)
{
    const double norm = S[0] * r.dxdy;
    const double O = S[1] / S[0], B = S[2] / S[0];
    sc->norm = norm;
    sc->O = O;
    sc->B = B;
    sc->c = 1.0 / sqrt(norm);
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
        // alpha = (num + probe) / (dr + i di), probe = Omega_c exp(i (Delta_p t + phi))
        double ps = 0.0, pc = 0.0;
        if (r.probe_omega != 0.0) sincos(r.probe_delta * r.t + r.probe_phi, &ps, &pc);
        const double a = r.N * r.eta * O + r.probe_omega * pc, b = r.probe_omega * ps;
        sc->alpha_re = (a * dr + b * di) / den;
        sc->alpha_im = (b * dr - a * di) / den;
    } else {
        sc->alpha_re = 0.0;
        sc->alpha_im = 0.0;
    }
}

// ------------------------------------------------------------------ pointwise pieces
// Per-CTA potential coefficients.  V at a point is
//   F + t.x + A t.y + (B t.z + C) t.z
// where t is the coordinate-table entry {trap, cos^2(k_lat .), cos(kc .), .}
// of the axis that varies along the pencil and F, A, B, C fold in the fixed
// axis: row pencils vary x (A = lattice x depth, B = U0|alpha|^2, C = 2 eta
// Re(alpha) cos(kc y)); column pencils vary y (A = lattice y depth, B = pump
// depth eta^2/U0, C = 2 eta Re(alpha) cos(kc x)).  Eqs. (9)-(13).
struct PotCoefs {
    float F, A, B, C;
};

// V_c and V_i amplitudes for a cavity field alpha = ar + i ai (Eqs. 12-13)
__device__ __forceinline__ void alpha_amps(const PhaseArgs &ph, double ar, double ai, float &acx2, float &acxcy)
{
    acx2 = 0.f;
    acxcy = 0.f;
    if (ph.use_alpha) {
        acx2 = (float)((double)ph.U0 * (ar * ar + ai * ai));       // V_c amplitude, Eq. (12)
        acxcy = (float)((double)ph.two_eta * ar);                   // V_i amplitude, Eq. (13)
    }
}

__device__ __forceinline__ void alpha_terms(const PassArgs &a, float &acx2, float &acxcy)
{
    if (a.ph.use_alpha) alpha_amps(a.ph, a.T.sc->alpha_re, a.T.sc->alpha_im, acx2, acxcy);
    else alpha_amps(a.ph, 0.0, 0.0, acx2, acxcy);
}

// row pencil at fixed y (yt = ytab[y]) for V_c, V_i amplitudes acx2, acxcy
__device__ __forceinline__ PotCoefs row_coefs_from(const PhaseArgs &ph, float acx2, float acxcy, float4 yt)
{
    return PotCoefs{yt.x + ph.a_laty * yt.y + ph.a_pump * yt.z * yt.z, ph.a_latx, acx2, acxcy * yt.z};
}

// column pencil at fixed x (xt = xtab[x])
__device__ __forceinline__ PotCoefs col_coefs_from(const PhaseArgs &ph, float acx2, float acxcy, float4 xt)
{
    return PotCoefs{xt.x + ph.a_latx * xt.y + acx2 * xt.z * xt.z, ph.a_laty, ph.a_pump, acxcy * xt.z};
}

__device__ __forceinline__ PotCoefs row_coefs(const PassArgs &a, float4 yt)
{
    float acx2, acxcy;
    alpha_terms(a, acx2, acxcy);
    return row_coefs_from(a.ph, acx2, acxcy, yt);
}

__device__ __forceinline__ PotCoefs col_coefs(const PassArgs &a, float4 xt)
{
    float acx2, acxcy;
    alpha_terms(a, acx2, acxcy);
    return col_coefs_from(a.ph, acx2, acxcy, xt);
}

__device__ __forceinline__ float pot_at(const PotCoefs &p, float4 t)
{
    return p.F + t.x + p.A * t.y + (p.B * t.z + p.C) * t.z;
}

// psi <- exp(-i theta) psi (real time) or exp(-theta) psi (imaginary time),
// theta = (V + g |psi|^2) h (Sec. 3.1, Sec. 3.3).  Real time multiplies by
// 1 + d with d = exp(-i theta) - 1 = -2 sin^2(theta/2) - 2 i sin(theta/2)
// cos(theta/2): small phases keep their relative precision and |1 + d| = 1
// up to unbiased rounding.  For |theta| <= 1, sin and cos of w = theta/2 come
// from their Taylor series in w^2 (remainders w^11/11! and w^10/10! below
// 3e-10); larger phases use sincosf.
__device__ __forceinline__ float2 phase_mul(float2 q, float V, float g, float h, int imag)
{
    const float n = q.x * q.x + q.y * q.y;
    const float th = (V + g * n) * h;
    if (imag) {
        const float f = expf(-th);
        return make_float2(q.x * f, q.y * f);
    }
    const float w = 0.5f * th;
    float s, c;
    if (fabsf(th) <= 1.f) {
        const float v = w * w;
        float ps = fmaf(v, 1.f / 362880.f, -1.f / 5040.f);     // sin w = w (1 - v/3! + v^2/5! - ...)
        ps = fmaf(v, ps, 1.f / 120.f);
        ps = fmaf(v, ps, -1.f / 6.f);
        s = fmaf(w * v, ps, w);
        float pc = fmaf(v, 1.f / 40320.f, -1.f / 720.f);       // cos w = 1 - v/2! + v^2/4! - ...
        pc = fmaf(v, pc, 1.f / 24.f);
        pc = fmaf(v, pc, -0.5f);
        c = fmaf(v, pc, 1.f);
    } else {
        sincosf(w, &s, &c);
    }
    const float dr = -2.f * s * s, di = -2.f * s * c;
    return make_float2(q.x + (q.x * dr - q.y * di), q.y + (q.x * di + q.y * dr));
}

// psi <- exp(-i theta) psi for a given theta (real time), in the same 1 + d
// form as phase_mul; used by the adjoint passes, whose theta comes from the
// forward state rather than from the value being rotated.
__device__ __forceinline__ float2 phase_rot(float2 q, float th)
{
    const float w = 0.5f * th;
    float s, c;
    if (fabsf(th) <= 1.f) {
        const float v = w * w;
        float ps = fmaf(v, 1.f / 362880.f, -1.f / 5040.f);
        ps = fmaf(v, ps, 1.f / 120.f);
        ps = fmaf(v, ps, -1.f / 6.f);
        s = fmaf(w * v, ps, w);
        float pc = fmaf(v, 1.f / 40320.f, -1.f / 720.f);
        pc = fmaf(v, pc, 1.f / 24.f);
        pc = fmaf(v, pc, -0.5f);
        c = fmaf(v, pc, 1.f);
    } else {
        sincosf(w, &s, &c);
    }
    const float dr = -2.f * s * s, di = -2.f * s * c;
    return make_float2(q.x + (q.x * dr - q.y * di), q.y + (q.x * di + q.y * dr));
}

// Adjoint of one real-time half phase at one point (discrete adjoint of
// psi' = exp(-i theta) psi, theta = h (V + g |psi|^2)): lam = mu + 2 h g
// Im(conj(mu) psi) psi with mu = exp(+i theta) lam'; returns Im(conj(mu) psi),
// whose 2 h L(r) multiple is dJ/dv at this point.  `psi` is the phase's input.
__device__ __forceinline__ float phase_adjoint(float2 &lam, float2 psi, float V, float g, float h)
{
    const float th = (V + g * (psi.x * psi.x + psi.y * psi.y)) * h;
    const float2 mu = phase_rot(lam, -th);
    const float q = mu.x * psi.y - mu.y * psi.x;
    const float f = 2.f * h * g * q;
    lam = make_float2(fmaf(f, psi.x, mu.x), fmaf(f, psi.y, mu.y));
    return q;
}

// one axis of the kinetic propagator in k-space: real time psi <- s (psi + psi D)
// with D = exp(-i k^2 dt / 2m) - 1, imaginary time psi <- s K psi with
// K = exp(-k^2 dtau / 2m); s = 1/n exact (the inverse FFT's normalisation).
// CONJ: the adjoint (conjugate) propagator, D -> conj(D).
template <int E, int TP, bool CONJ = false>
__device__ __forceinline__ void kinetic_axis(float2 (&v)[E], const float2 *__restrict__ D, int j, float s, int imag)
{
    if (imag) {
#pragma unroll
        for (int r = 0; r < E; ++r) {
            const float f = __ldg(&D[j + r * TP]).x * s;
            v[r] = make_float2(v[r].x * f, v[r].y * f);
        }
    } else {
#pragma unroll
        for (int r = 0; r < E; ++r) {
            float2 d = __ldg(&D[j + r * TP]);
            if constexpr (CONJ) d.y = -d.y;
            const float2 p = v[r];
            const float2 pd = cmul(p, d);
            v[r] = make_float2((p.x + pd.x) * s, (p.y + pd.y) * s);
        }
    }
}

// Copy an axis' twiddle table into shared memory (every thread of the CTA;
// visible to the first twiddled stage through the barrier of the stage-0
// exchange that precedes it).
template <int N>
__device__ __forceinline__ void stage_twiddles(float4 *__restrict__ dst, const float4 *__restrict__ src)
{
    for (int i = threadIdx.x; i < fft_tw_count(N); i += blockDim.x) dst[i] = __ldg(&src[i]);
}

// Asynchronous variant: one bulk copy of the table into shared memory whose
// bytes complete on `bar`.  The caller (thread 0) has already armed `bar` with
// a single arrive.expect_tx covering these bytes (a barrier of count 1 takes
// exactly one arrival per phase).
template <int N> __host__ __device__ constexpr uint32_t twiddle_bytes() { return (uint32_t)(fft_tw_count(N) * 16); }
template <int N>
__device__ __forceinline__ void stage_twiddles_async(float4 *__restrict__ dst, const float4 *__restrict__ src,
                                                     uint64_t *bar)
{
    bulk_load_1d(dst, src, twiddle_bytes<N>(), bar);
}

// Ask L2 to fetch this CTA's share of a `bytes`-long buffer (bytes and the
// buffer's address multiples of 16): CTA b of G takes the b-th 16-byte-aligned
// slice, in 4 KB bulk prefetches issued by the lanes of warp 0.  A hint
// only: nothing waits for it, and it never reads outside the buffer.
__device__ __forceinline__ void prefetch_l2_share(const void *buf, size_t bytes)
{
    if (threadIdx.x >= 32) return;
    const size_t G = gridDim.x, chunk = ((bytes + G - 1) / G + 15) & ~(size_t)15;
    const size_t lo = (size_t)blockIdx.x * chunk, hi = lo + chunk < bytes ? lo + chunk : bytes;
    for (size_t o = lo + (size_t)threadIdx.x * 4096; o < hi; o += 32 * 4096) {
        const unsigned n = (unsigned)(hi - o < 4096 ? hi - o : 4096);
        asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"((const char *)buf + o), "r"(n) : "memory");
    }
}

// Opt func in to `bytes` of dynamic shared memory once per device (function
// attributes belong to the device's context), safe from several host threads.
template <class F> [[maybe_unused]] static cudaError_t smem_opt_in(F *func, int bytes,
                                                                   std::atomic<unsigned long long> &done)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const unsigned long long bit = 1ull << (dev & 63);
    if (done.load(std::memory_order_acquire) & bit) return cudaSuccess;
    e = cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess) done.fetch_or(bit, std::memory_order_acq_rel);
    return e;
}

// SM count of the current device (cached per device; 148 if it cannot be read)
[[maybe_unused]] static int sm_count()
{
    static std::atomic<int> cache[64];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 148;
    std::atomic<int> &c = cache[dev & 63];
    int n = c.load(std::memory_order_relaxed);
    if (n <= 0) {
        if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) n = 148;
        c.store(n, std::memory_order_relaxed);
    }
    return n;
}

}  // namespace gpe
