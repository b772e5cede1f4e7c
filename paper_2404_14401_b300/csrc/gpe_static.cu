// gpe_static.cu -- gpe_overlaps_static: the density reduction of the row pass
// (norm and the two cavity overlaps) for callers that cannot allocate device
// memory.  Its scratch (per-CTA partial sums, the last-CTA counter, the
// coordinate and twiddle tables and the result scalars) lives in one fixed array of this
// library instead of a caller-provided workspace.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <mutex>

#include "../../include/gpe.h"
#include "gpe_internal.h"

using namespace gpe;

namespace {

constexpr size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// Row-pass CTAs for nx, ny <= GPE_STATIC_MAX_N: rows per CTA is 256/(nx/16)
// (at least 1, at most ny), so at most GPE_STATIC_MAX_N / 2 CTAs reduce.
constexpr int kMaxBlocks = GPE_STATIC_MAX_N / 2;
constexpr size_t kOffSc = 0;
constexpr size_t kOffPart = align256(sizeof(DevScalars));
constexpr size_t kOffX = align256(kOffPart + sizeof(double) * NQ * kMaxBlocks);
constexpr size_t kOffY = align256(kOffX + sizeof(float4) * GPE_STATIC_MAX_N);
constexpr size_t kOffTwx = align256(kOffY + sizeof(float4) * GPE_STATIC_MAX_N);   // written by the
constexpr size_t kOffTwy = align256(kOffTwx + sizeof(float4) * GPE_STATIC_MAX_N); // tables kernel
constexpr size_t kBytes = align256(kOffTwy + sizeof(float4) * GPE_STATIC_MAX_N);

}  // namespace

// The scratch itself: one copy per GPU that loads this library, kept until
// the process exits.  Host code must not pass its name to a kernel (on the
// host the name is only a stand-in); it uses the address from
// cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_static_scratch[kBytes];

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_mu;
unsigned char *g_dev_ptr[kMaxDevices];

// Device address of the scratch on the current device, looked up once per
// device (the first call on a device does this; it must come before any
// stream capture that includes the call).
gpe_status scratch_on_current_device(unsigned char **out)
{
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return GPE_ECUDA;
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_dev_ptr[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_static_scratch) != cudaSuccess || !p) return GPE_ECUDA;
        g_dev_ptr[dev] = static_cast<unsigned char *>(p);
    }
    *out = g_dev_ptr[dev];
    return GPE_OK;
}

bool pow2_between(int n, int lo, int hi) { return n >= lo && n <= hi && (n & (n - 1)) == 0; }

}  // namespace

extern "C" gpe_status gpe_overlaps_static(const void *psi_dev, int nx, int ny, double Lx, double Ly,
                                          double kc, void *stream, double *out)
{
    if (!psi_dev || !out || ((uintptr_t)psi_dev & 15u)) return GPE_EINVAL;
    if (!pow2_between(nx, 8, 8192) || !pow2_between(ny, 8, 8192)) return GPE_EINVAL;
    if (nx > GPE_STATIC_MAX_N || ny > GPE_STATIC_MAX_N) return GPE_ENOMEM;   // beyond the fixed scratch
    // one partial-sum slot per CTA of the reducing row pass: refuse a launch
    // with more CTAs than the scratch has slots (the bound above keeps it at
    // most GPE_STATIC_MAX_N / 2 with today's row tiling; this check keeps the
    // call safe if that tiling changes)
    if (ny / row_rows_per_cta(nx, ny, 0) > kMaxBlocks) return GPE_ENOMEM;
    if (!(Lx > 0.0) || !(Ly > 0.0)) return GPE_EINVAL;
    unsigned char *base = nullptr;
    if (scratch_on_current_device(&base) != GPE_OK) return GPE_ECUDA;
    const cudaStream_t s = static_cast<cudaStream_t>(stream);

    Tables T;
    memset(&T, 0, sizeof(T));
    T.sc = reinterpret_cast<DevScalars *>(base + kOffSc);
    T.part_row = reinterpret_cast<double *>(base + kOffPart);
    T.xtab = reinterpret_cast<float4 *>(base + kOffX);
    T.ytab = reinterpret_cast<float4 *>(base + kOffY);
    T.twx = reinterpret_cast<float4 *>(base + kOffTwx);   // the tables kernel fills these too
    T.twy = reinterpret_cast<float4 *>(base + kOffTwy);
    // tw8x / tw8y stay null: no pass here transforms, and the tables kernel
    // skips the radix-8 tables of a Tables that has none

    // the scratch keeps whatever the previous call left: the counter and the
    // status word must start at zero, the tables are rewritten for this grid
    if (cudaMemsetAsync(T.sc, 0, sizeof(DevScalars), s) != cudaSuccess) return GPE_ECUDA;
    if (launch_tables(T, nx, ny, Lx, Ly, 1.0, 0.0, 0.0, 0.0, 0.0, kc, s) != cudaSuccess) return GPE_ECUDA;

    PassArgs a;
    memset(&a, 0, sizeof(a));
    a.psi = const_cast<float2 *>(static_cast<const float2 *>(psi_dev));   // read only in this mode
    a.nx = nx;
    a.ny = ny;
    a.T = T;
    a.red.dxdy = (Lx / nx) * (Ly / ny);
    a.red.N = 1.0;
    if (launch_row(ROW_REDUCE_R, a, s) != cudaSuccess) return GPE_ECUDA;

    DevScalars h;
    if (cudaMemcpyAsync(&h, T.sc, sizeof(h), cudaMemcpyDeviceToHost, s) != cudaSuccess) return GPE_ECUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return GPE_ECUDA;
    out[0] = h.norm;
    out[1] = h.O;
    out[2] = h.B;
    return h.status ? static_cast<gpe_status>(h.status) : GPE_OK;
}
