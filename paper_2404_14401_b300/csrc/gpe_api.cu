// gpe_api.cu -- the C ABI of include/gpe.h: context, potential descriptor,
// and the host scheduler that turns gpe_step(n, dt, mode) into the sequence
// of row / column passes of the symmetric split-step (Sec. 3.1, Eqs. 2-4;
// imaginary time Sec. 3.3; cavity Sec. 5.3, Eqs. 10-15).
//
// Pass schedules (R = row pass: potential phase then T_x; C = column pass:
// T_y, optionally followed by a phase and reductions).  The kinetic
// propagator F^-1 K F equals T_x T_y exactly (K is separable), so psi is in
// real space between passes:
//   real time, no cavity  R(V/2) C { R(V) C }^(n-2) R(V) C+V/2
//       adjacent half phases V(t_k)/2 see the same density (a real phase
//       keeps |psi|) and merge into one full phase; the last one is applied
//       by the last column pass;
//   real time, cavity     [reduce] { R(V) C+reduce }^n R(V/2): alpha needs the
//       grid-wide overlaps of the current density, which the column pass
//       reduces from its results;
//   imaginary time        { R([c] V/2) C+V/2+norm }^n scale: the column pass
//       applies the second half phase and reduces the norm (Sec. 3.3), the
//       next row pass applies the scale; with a cavity the second half phase
//       needs alpha of the post-kinetic density, so it runs in an extra row
//       pass after a reducing column pass.
#include <cuda.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stddef.h>
#include <stdarg.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <atomic>
#include <memory>
#include <mutex>
#include <utility>
#include <vector>

#include "../../include/gpe.h"
#include "gpe_internal.h"

using namespace gpe;

struct gpe_ctx {
    int nx, ny;
    double Lx, Ly, m, g;
    float2 *psi;
    unsigned char *ws;
    size_t ws_bytes;
    cudaStream_t stream;
    Tables T;
    CUtensorMap map;
    int W;
    gpe_potential pot;
    std::vector<double> ctrl_t, ctrl_v;
    double t;
    double kin_dt;
    int kin_mode;
    bool kin_valid;
    int spins;
    int device;              // the CUDA device current at gpe_create; every launch checks it
    int stream_passes;       // use the persistent streaming row pass where it applies
    int stream_cols;         // use the persistent streaming column pass where it applies
    int group_rows;          // use the grouped persistent row pass where it applies
    int pair_cols;           // use the pencil-pair column pass (T_y) where it applies
    int pair_rows;           // use the pencil-pair row pass where it applies
    int coop;                // gpe_step on this context alone: the cooperative kernel where it applies
    int row_tile_shift;      // one-shot row pass: 2^-shift of the default rows per CTA (0..2)
    long long launches;
    unsigned long long uid;          // unique over the process (never reused, unlike the pointer)
    unsigned long long version;      // bumped by every call that changes the passes' arguments
    cudaEvent_t ev_fork, ev_join;   // ordering of gpe_step_many's lanes with this context's stream
    // per-pass event timing (gpe_profile)
    bool prof;
    std::vector<cudaEvent_t> ev_free;
    std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> ev_pending;
    double prof_ms[GPE_PASS_KINDS];   // per pass kind: see gpe_profile_read_kind
    int prof_n[GPE_PASS_KINDS];
    char err[256];
};

namespace {

bool pow2_in_range(int n) { return n >= 8 && n <= 8192 && (n & (n - 1)) == 0; }

// Streams of the library on which gpe_step_many runs contexts side by side
// (created on first use per device, kept until the process exits): one lane
// per context up to kLanes.  Passes of different contexts then fill the SMs
// that one pass leaves idle (its tail, or all but a few SMs for a small
// grid) and hide the gaps between launches.  Measured: the phase-diagram
// sweep (384 grids of 256^2 .. 1024^2) ran at 35.1 G pt*steps/s on 8 lanes,
// 41.0 on 16, 40.9 on 32 and 38.9 on 64; 8 trajectories of 2048^2 at 72.2
// on 2 lanes and 73.4 on 8.
constexpr int kLanes = 16;
// Batches of grids of at most 2^22 points (2048^2) on average replay their
// interior steps from CUDA graphs: 8 grids of 2048^2 ran at 74.0 G pt*steps/s
// with 8-step graphs against 73.4 without, 2 of 4096^2 at 51.5 against 51.8.
bool small_grids(gpe_ctx *const *ctxs, int count)
{
    double pts = 0.0;
    for (int i = 0; i < count; ++i) pts += (double)ctxs[i]->nx * ctxs[i]->ny;
    return pts / count <= (double)(1 << 22);
}
int lanes_for(gpe_ctx *const *ctxs, int count)
{
    (void)ctxs;
    return count < kLanes ? count : kLanes;
}
// Instantiated graphs of K interior lockstep steps, one per lane (the steps
// of the contexts on that lane), kept across gpe_step_many calls: their
// kernel arguments are fixed by the contexts (each by its uid and version),
// dt, the mode, K and the lane count, so a later call with the same key
// replays them without capturing again.  Each lane replays its own graph on
// its own stream: no lane waits for another between replays.
struct GraphEntry {
    std::vector<unsigned long long> key;   // uid, version per context, in order
    double dt;
    int mode, K, nl;
    std::vector<cudaGraphExec_t> exec;     // per lane
    std::vector<long long> launches;       // kernels each context launches per replay
    unsigned long long used;               // LRU stamp
};
static void destroy_graphs(GraphEntry &e)
{
    for (cudaGraphExec_t x : e.exec)
        if (x) cudaGraphExecDestroy(x);
    e.exec.clear();
}
constexpr size_t kGraphCache = 8;
struct Lanes {
    cudaStream_t s[kLanes];
    std::mutex mu;                 // one gpe_step_many at a time enqueues on these lanes
    std::vector<GraphEntry> graphs;   // guarded by mu
    unsigned long long clock = 0;
};
Lanes *g_lanes[64];                // per device, created on first use
std::mutex g_lanes_mu;
Lanes *lanes_for_current_device()
{
    constexpr int kMaxDev = 64;
    Lanes **lanes = g_lanes;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDev) return nullptr;
    std::lock_guard<std::mutex> lock(g_lanes_mu);
    if (!lanes[dev]) {
        Lanes *L = new Lanes;
        for (int i = 0; i < kLanes; ++i)
            if (cudaStreamCreateWithFlags(&L->s[i], cudaStreamNonBlocking) != cudaSuccess) {
                for (int k = 0; k < i; ++k) cudaStreamDestroy(L->s[k]);
                delete L;
                return nullptr;
            }
        lanes[dev] = L;
    }
    return lanes[dev];
}

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

struct Layout {
    size_t sc, part_row, part_col, twx, twy, tw8x, tw8y, xtab, ytab, kinx, kiny, total;
};

Layout layout(int nx, int ny)
{
    Layout L;
    size_t o = 0;
    L.sc = o;        o = align256(o + sizeof(DevScalars));
    L.part_row = o;  o = align256(o + sizeof(double) * NQ * MAX_BLOCKS);
    L.part_col = o;  o = align256(o + sizeof(double) * NQ * MAX_BLOCKS);
    L.twx = o;       o = align256(o + sizeof(float4) * nx);
    L.twy = o;       o = align256(o + sizeof(float4) * ny);
    L.tw8x = o;      o = align256(o + sizeof(float4) * nx);
    L.tw8y = o;      o = align256(o + sizeof(float4) * ny);
    L.xtab = o;      o = align256(o + sizeof(float4) * nx);
    L.ytab = o;      o = align256(o + sizeof(float4) * ny);
    L.kinx = o;      o = align256(o + sizeof(float2) * nx);
    L.kiny = o;      o = align256(o + sizeof(float2) * ny);
    L.total = o;
    return L;
}

gpe_status fail(gpe_ctx *c, gpe_status s, const char *fmt, ...)
{
    if (c) {
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(c->err, sizeof(c->err), fmt, ap);
        va_end(ap);
    }
    return s;
}

gpe_status cuda_check(gpe_ctx *c, cudaError_t e, const char *what)
{
    if (e == cudaSuccess) return GPE_OK;
    return fail(c, GPE_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

// TMA view of a [ny][nx] complex64 array as float32 [ny][2 nx] with box
// w complex columns x BR rows (a column pass's tile)
gpe_status encode_map_w(gpe_ctx *c, void *base, int w, CUtensorMap *out);
gpe_status encode_map(gpe_ctx *c, void *base, CUtensorMap *out) { return encode_map_w(c, base, c->W, out); }
gpe_status encode_map_w(gpe_ctx *c, void *base, int w, CUtensorMap *out)
{
    static EncodeTiledFn encode = nullptr;
    if (!encode) {
        void *fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q);
        if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !fn)
            return fail(c, GPE_ECUDA, "cuTensorMapEncodeTiled not available");
        encode = (EncodeTiledFn)fn;
    }
    // psi viewed as float32 [ny][2 nx]; box = W complex columns x BR rows
    const int BR = c->ny < 256 ? c->ny : 256;
    cuuint64_t dims[2] = {(cuuint64_t)2 * c->nx, (cuuint64_t)c->ny};
    cuuint64_t strides[1] = {(cuuint64_t)2 * c->nx * sizeof(float)};
    cuuint32_t box[2] = {(cuuint32_t)(2 * w), (cuuint32_t)BR};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = encode(out, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, base, dims, strides, box, estr,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                        CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return fail(c, GPE_ECUDA, "cuTensorMapEncodeTiled failed (%d)", (int)r);
    return GPE_OK;
}

gpe_status make_tensor_map(gpe_ctx *c) { return encode_map(c, c->psi, &c->map); }

// piecewise-linear control v(t), clamped at both ends
double control_value(const gpe_ctx *c, double t)
{
    const size_t n = c->ctrl_t.size();
    if (n == 0) return 1.0;
    if (t <= c->ctrl_t[0]) return c->ctrl_v[0];
    if (t >= c->ctrl_t[n - 1]) return c->ctrl_v[n - 1];
    size_t lo = 0, hi = n - 1;                     // ctrl_t[lo] < t < ctrl_t[hi]
    while (hi - lo > 1) {
        const size_t mid = (lo + hi) / 2;
        if (c->ctrl_t[mid] < t) lo = mid; else hi = mid;
    }
    const double f = (t - c->ctrl_t[lo]) / (c->ctrl_t[hi] - c->ctrl_t[lo]);
    return c->ctrl_v[lo] + f * (c->ctrl_v[hi] - c->ctrl_v[lo]);
}

double eta_at(const gpe_ctx *c, double t)
{
    return c->pot.ctrl_target == GPE_CTRL_ETA ? control_value(c, t) : c->pot.eta;
}

PhaseArgs phase_at(const gpe_ctx *c, double t, double h)
{
    const gpe_potential &p = c->pot;
    const double ls = p.ctrl_target == GPE_CTRL_LATTICE ? control_value(c, t) : 1.0;
    const double eta = eta_at(c, t);
    PhaseArgs a;
    a.h = (float)h;
    a.a_latx = (float)(p.lat_V0x * ls);
    a.a_laty = (float)(p.lat_V0y * ls);
    a.a_pump = (p.cavity && p.pump_lattice && p.U0 != 0.0) ? (float)(eta * eta / p.U0) : 0.f;
    a.U0 = p.cavity ? (float)p.U0 : 0.f;
    a.two_eta = p.cavity ? (float)(2.0 * eta) : 0.f;
    a.use_alpha = p.cavity ? 1 : 0;
    return a;
}

RedArgs red_at(const gpe_ctx *c, double t)
{
    RedArgs r;
    r.eta = eta_at(c, t);
    r.U0 = c->pot.U0;
    r.dc = c->pot.dc;
    r.kappa = c->pot.kappa;
    r.N = c->pot.N;
    r.dxdy = (c->Lx / c->nx) * (c->Ly / c->ny);
    r.cavity = c->pot.cavity;
    r.probe_omega = c->pot.probe_omega;
    r.probe_delta = c->pot.probe_delta;
    r.probe_phi = c->pot.probe_phi;
    r.t = t;
    return r;
}

PassArgs pass_args(const gpe_ctx *c, const PhaseArgs &ph, const RedArgs &rd, int imag, int use_c)
{
    PassArgs a;
    memset(&a, 0, sizeof(a));
    a.psi = c->psi;
    a.nx = c->nx;
    a.ny = c->ny;
    a.V = c->pot.V;
    a.V_scale = (float)c->pot.V_scale;
    a.g = (float)c->g;
    a.imag = imag;
    a.use_c = use_c;
    a.sx = (float)(1.0 / c->nx);          // exact: powers of two
    a.sy = (float)(1.0 / c->ny);
    a.spins = c->spins;
    a.ph = ph;
    a.red = rd;
    a.T = c->T;
    return a;
}

cudaEvent_t take_event(gpe_ctx *c)
{
    if (!c->ev_free.empty()) {
        cudaEvent_t e = c->ev_free.back();
        c->ev_free.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

// Launch one pass, bracketed by events when profiling (kind 0 row, 1 column).
template <class F> gpe_status timed_launch(gpe_ctx *c, int kind, F &&launch, const char *what)
{
    // the context's pointers, tables and tensor map are on its own device: a
    // kernel launched with another device current would address foreign memory
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev != c->device)
        return fail(c, GPE_EINVAL, "%s: the context is on device %d, the current device is %d", what, c->device, dev);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (c->prof) {
        e0 = take_event(c);
        e1 = take_event(c);
        cudaEventRecord(e0, c->stream);
    }
    const cudaError_t err = launch();
    if (err != cudaSuccess) return cuda_check(c, err, what);
    c->launches++;
    if (c->prof) {
        cudaEventRecord(e1, c->stream);
        c->ev_pending.push_back({kind, {e0, e1}});
    }
    return GPE_OK;
}

gpe_status run_row(gpe_ctx *c, int mode, const PhaseArgs &ph, const RedArgs &rd, int imag, int use_c)
{
    const PassArgs a = pass_args(c, ph, rd, imag, use_c);
    if (mode == ROW_PT && c->pair_rows && row_pair_ok(c->nx, c->ny))
        return timed_launch(c, 0, [&] { return launch_row_pair(a, c->stream); }, "row pass");
    if (mode == ROW_PT && c->stream_passes && row_stream_ok(c->nx, c->ny))
        return timed_launch(c, 0, [&] { return launch_row_stream(a, c->stream); }, "row pass");
    if (mode == ROW_PT && c->group_rows && row_group_ok(c->nx, c->ny))
        return timed_launch(c, 0, [&] { return launch_row_group(a, c->stream); }, "row pass");
    const int ts = c->row_tile_shift;
    return timed_launch(c, 0, [&] { return launch_row(mode, a, c->stream, ts); }, "row pass");
}

gpe_status run_col(gpe_ctx *c, int mode, const PhaseArgs &ph, const RedArgs &rd, int imag)
{
    const PassArgs a = pass_args(c, ph, rd, imag, 0);
    if ((mode == COL_T || mode == COL_T_R || mode == COL_T_PR || mode == COL_T_P) && c->stream_cols &&
        col_stream_ok(c->nx, c->ny))
        return timed_launch(c, 1, [&] { return launch_col_stream(mode, a, c->map, c->stream); }, "column pass");
    if ((mode == COL_T || mode == COL_T_R || mode == COL_T_PR || mode == COL_T_P) && c->pair_cols &&
        col_pair_ok(c->nx, c->ny))
        return timed_launch(c, 1, [&] { return launch_col_pair(mode, a, c->map, c->stream); }, "column pass");
    return timed_launch(c, 1, [&] { return launch_col(mode, a, c->map, c->stream); }, "column pass");
}

#define TRY(x)                                   \
    do {                                         \
        gpe_status _s = (x);                     \
        if (_s != GPE_OK) return _s;             \
    } while (0)

}  // namespace

extern "C" {

const char *gpe_status_string(gpe_status s)
{
    switch (s) {
    case GPE_OK: return "GPE_OK";
    case GPE_EINVAL: return "GPE_EINVAL";
    case GPE_ENOMEM: return "GPE_ENOMEM";
    case GPE_ECUDA: return "GPE_ECUDA";
    case GPE_ETIMEOUT: return "GPE_ETIMEOUT";
    case GPE_ENONFINITE: return "GPE_ENONFINITE";
    case GPE_EILLCOND: return "GPE_EILLCOND";
    case GPE_EBOUNDS: return "GPE_EBOUNDS";
    default: return "GPE_UNKNOWN";
    }
}

size_t gpe_workspace_size(int nx, int ny)
{
    if (!pow2_in_range(nx) || !pow2_in_range(ny)) return 0;
    return layout(nx, ny).total;
}

gpe_status gpe_create(int nx, int ny, double Lx, double Ly, double m, double g, void *psi_dev,
                      void *workspace_dev, size_t ws_bytes, void *stream, gpe_ctx **out)
{
    if (!out) return GPE_EINVAL;
    *out = nullptr;
    if (!pow2_in_range(nx) || !pow2_in_range(ny)) return GPE_EINVAL;
    if (!(Lx > 0.0) || !(Ly > 0.0) || !(m > 0.0) || !isfinite(g)) return GPE_EINVAL;
    if (!psi_dev || ((uintptr_t)psi_dev & 15u)) return GPE_EINVAL;
    if (!workspace_dev || ((uintptr_t)workspace_dev & 255u)) return GPE_EINVAL;
    const Layout L = layout(nx, ny);
    if (ws_bytes < L.total) return GPE_ENOMEM;

    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0) return GPE_ECUDA;
    gpe_ctx *c = new gpe_ctx();
    c->device = dev;
    c->nx = nx; c->ny = ny; c->Lx = Lx; c->Ly = Ly; c->m = m; c->g = g;
    c->psi = (float2 *)psi_dev;
    c->ws = (unsigned char *)workspace_dev;
    c->ws_bytes = ws_bytes;
    c->stream = (cudaStream_t)stream;
    c->W = col_tile_width(nx, ny);
    c->t = 0.0;
    c->kin_valid = false;
    c->spins = 1 << 24;
    c->stream_passes = getenv("GPE_NO_STREAM_PASSES") ? 0 : 1;
    // the streaming column pass by default nowhere: the pencil-pair pass
    // (below) measured faster at 4096 and 2048; the autotuner may choose it
    c->stream_cols = 0;
    // the grouped row pass by default only for 2048-point rows: at 1024 (and
    // below) the one-shot pass, whose CTAs share SMs with other passes,
    // measured faster under gpe_step_many (1024^2 x 8: 71.8 against 64.2 G
    // pt*steps/s), at 2048 the grouped pass (73.2 against 72.2)
    c->group_rows = (getenv("GPE_NO_GROUP_ROWS") || nx != 2048) ? 0 : 1;
    // half-height one-shot row tiles for 512- and 1024-point rows: 8 grids of
    // 1024^2 under gpe_step_many ran at 77.2 against 72.5 G pt*steps/s, of
    // 512^2 at 56.0 against 53.8; at 2048 the half tile was slower (65.7
    // against 71.7) and at 256 the same
    c->row_tile_shift = (nx == 512 || nx == 1024) ? 1 : 0;
    // the pencil-pair column passes by default for columns of 1024 points and
    // more (8 x 1024^2 under gpe_step_many: 100.1 against 92.2 G pt*steps/s
    // for the one-pencil pass, although alone each pass timed within 2%; 8 x
    // 2048^2: 69.7 against 67.6, the T_y pass alone 33.7 against 36.0 us;
    // 4096^2: 126 against 183 us for the streaming pass; 8192^2: 888 against
    // 943 us).  At 512 the one-pencil pass stays: one 512^2 grid with the
    // cavity (a reducing column pass every step) ran 24.6 us per step with it
    // and 27.6 with the pair pass.
    c->pair_cols = (ny >= 1024 && !getenv("GPE_NO_PAIR_COLS")) ? 1 : 0;
    // the pencil-pair row pass by default for rows of 512 points and more
    // (each pass alone, eight grids: 11.8 against 14.6 us at 512^2, 14.6
    // against 18.4 us at 1024^2, 34.4 against 43.9 us for the grouped pass
    // at 2048^2, 133 against 181 us for the streaming pass at 4096^2, 918
    // against 940 us for the one-shot pass at 8192^2)
    c->pair_rows = (nx >= 512 && !getenv("GPE_NO_PAIR_ROWS")) ? 1 : 0;
    // the cooperative kernel by default on 512^2 grids, where it measured
    // faster than the per-pass path in every step program (per step: real
    // time 10.9 against 13.3 us, the cavity ramp 17.8 against 24.6 us,
    // imaginary time 16.2 against 23.8 us); at 1024^2 it was slower in real
    // time (24.2 against 21.4 us) and within 6% otherwise, so it is a choice
    // there
    c->coop = (nx == 512 && ny == 512 && !getenv("GPE_NO_COOP")) ? 1 : 0;
    c->launches = 0;
    {
        static std::atomic<unsigned long long> next_uid{1};
        c->uid = next_uid.fetch_add(1);
    }
    c->version = 0;
    c->prof = false;
    for (int k = 0; k < GPE_PASS_KINDS; ++k) {
        c->prof_ms[k] = 0.0;
        c->prof_n[k] = 0;
    }
    memset(&c->pot, 0, sizeof(c->pot));
    c->pot.V_scale = 1.0;
    c->pot.N = 1.0;
    c->err[0] = 0;
    Tables &T = c->T;
    T.sc = (DevScalars *)(c->ws + L.sc);
    T.part_row = (double *)(c->ws + L.part_row);
    T.part_col = (double *)(c->ws + L.part_col);
    T.twx = (float4 *)(c->ws + L.twx);
    T.twy = (float4 *)(c->ws + L.twy);
    T.tw8x = (float4 *)(c->ws + L.tw8x);
    T.tw8y = (float4 *)(c->ws + L.tw8y);
    T.xtab = (float4 *)(c->ws + L.xtab);
    T.ytab = (float4 *)(c->ws + L.ytab);
    T.kinx = (float2 *)(c->ws + L.kinx);
    T.kiny = (float2 *)(c->ws + L.kiny);

    c->ev_fork = c->ev_join = nullptr;
    gpe_status s = make_tensor_map(c);
    if (s == GPE_OK) s = cuda_check(c, cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming), "event");
    if (s == GPE_OK) s = cuda_check(c, cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming), "event");
    if (s == GPE_OK) s = cuda_check(c, cudaMemsetAsync(T.sc, 0, sizeof(DevScalars), c->stream), "memset");
    if (s == GPE_OK)
        s = cuda_check(c, launch_tables(T, nx, ny, Lx, Ly, m, 0, 0, 0, 0, 0, c->stream), "tables");
    if (s == GPE_OK) c->launches++;
    if (s != GPE_OK) {
        if (c->ev_fork) cudaEventDestroy(c->ev_fork);
        if (c->ev_join) cudaEventDestroy(c->ev_join);
        delete c;
        return s;
    }
    *out = c;
    return GPE_OK;
}

gpe_status gpe_set_potential(gpe_ctx *c, const gpe_potential *p)
{
    if (!c || !p) return GPE_EINVAL;
    if (p->nctrl < 0 || (p->nctrl > 0 && (!p->ctrl_t || !p->ctrl_v)))
        return fail(c, GPE_EINVAL, "control table: nctrl %d with null arrays", p->nctrl);
    if (p->ctrl_target < GPE_CTRL_NONE || p->ctrl_target > GPE_CTRL_ETA)
        return fail(c, GPE_EINVAL, "unknown control target %d", p->ctrl_target);
    if (p->ctrl_target != GPE_CTRL_NONE && p->nctrl < 1)
        return fail(c, GPE_EINVAL, "control target set without control points");
    for (int i = 1; i < p->nctrl; ++i)
        if (!(p->ctrl_t[i] > p->ctrl_t[i - 1]))
            return fail(c, GPE_EINVAL, "control times must increase");
    if (p->cavity && !(p->kappa >= 0.0)) return fail(c, GPE_EINVAL, "kappa must be >= 0");
    if (!isfinite(p->probe_omega) || !isfinite(p->probe_delta) || !isfinite(p->probe_phi))
        return fail(c, GPE_EINVAL, "probe parameters must be finite");
    if (p->V && ((uintptr_t)p->V & 3u)) return fail(c, GPE_EINVAL, "potential array misaligned");
    c->pot = *p;
    c->version++;
    c->ctrl_t.assign(p->ctrl_t, p->ctrl_t + p->nctrl);
    c->ctrl_v.assign(p->ctrl_v, p->ctrl_v + p->nctrl);
    c->pot.ctrl_t = nullptr;
    c->pot.ctrl_v = nullptr;
    return timed_launch(c, 2, [&] {
        return launch_tables(c->T, c->nx, c->ny, c->Lx, c->Ly, c->m, p->wx, p->wy, p->lat_kx, p->lat_ky,
                             p->cavity ? p->kc : 0.0, c->stream);
    }, "tables");
}

}  // extern "C"

namespace {

gpe_status step_check(gpe_ctx *c, int n, double dt, gpe_mode mode)
{
    if (!c) return GPE_EINVAL;
    if (n < 0 || !(dt > 0.0) || !isfinite(dt) || (mode != GPE_REAL && mode != GPE_IMAG))
        return fail(c, GPE_EINVAL, "gpe_step: n %d dt %g mode %d", n, dt, (int)mode);
    return GPE_OK;
}

// The context's kinetic tables for steps of dt in `mode`, remade only when
// dt or the mode changed since they were made.
static gpe_status kinetic_for(gpe_ctx *c, double dt, gpe_mode mode)
{
    if (c->kin_valid && c->kin_dt == dt && c->kin_mode == (int)mode) return GPE_OK;
    TRY(timed_launch(c, 2, [&] {
        return launch_kinetic_tables(c->T, c->nx, c->ny, c->Lx, c->Ly, c->m, dt, mode == GPE_IMAG, c->stream);
    }, "kinetic tables"));
    c->kin_valid = true;
    c->kin_dt = dt;
    c->kin_mode = (int)mode;
    return GPE_OK;
}

// Passes before step 0: kinetic factors for (dt, mode) and, with a cavity,
// alpha of the initial density (Eq. 14).
gpe_status step_prologue(gpe_ctx *c, double dt, gpe_mode mode)
{
    const int imag = mode == GPE_IMAG;
    TRY(kinetic_for(c, dt, mode));
    PhaseArgs none;
    memset(&none, 0, sizeof(none));
    if (c->pot.cavity) TRY(run_row(c, ROW_REDUCE_R, none, red_at(c, c->t), imag, 0));
    return GPE_OK;
}

// The passes of step s (0 <= s < n) starting from the context's time c->t.
// Row pass: phase then T_x; column pass: T_y, in imaginary time also the
// closing half phase with the norm of the result (the next row pass scales
// by 1/sqrt(norm)), with a cavity the overlaps that set alpha for the next
// phase, and in real time without cavity the closing half phase of the last
// step.
gpe_status step_part(gpe_ctx *c, int s, int n, double dt, gpe_mode mode)
{
    const bool cav = c->pot.cavity != 0;
    const double ts = c->t + s * dt, te = c->t + (s + 1) * dt;
    PhaseArgs none;
    memset(&none, 0, sizeof(none));
    if (mode == GPE_REAL) {
        TRY(run_row(c, ROW_PT, phase_at(c, ts, s == 0 ? 0.5 * dt : dt), red_at(c, ts), 0, 0));
        if (cav)
            TRY(run_col(c, COL_T_R, none, red_at(c, te), 0));
        else if (s == n - 1)
            TRY(run_col(c, COL_T_P, phase_at(c, te, 0.5 * dt), red_at(c, te), 0));
        else
            TRY(run_col(c, COL_T, none, red_at(c, te), 0));
    } else {
        TRY(run_row(c, ROW_PT, phase_at(c, ts, 0.5 * dt), red_at(c, ts), 1, s > 0));
        if (cav) {
            TRY(run_col(c, COL_T_R, none, red_at(c, te), 1));
            TRY(run_row(c, ROW_PHASE_R, phase_at(c, te, 0.5 * dt), red_at(c, te), 1, 0));
        } else {
            TRY(run_col(c, COL_T_PR, phase_at(c, te, 0.5 * dt), red_at(c, te), 1));
        }
    }
    return GPE_OK;
}

// Passes after step n-1: with a cavity in real time the closing half phase
// (it needs alpha of the final density); in imaginary time the pending
// normalisation.  Advances the context's time.
gpe_status step_epilogue(gpe_ctx *c, int n, double dt, gpe_mode mode)
{
    const double tn = c->t + n * dt;
    PhaseArgs none;
    memset(&none, 0, sizeof(none));
    if (mode == GPE_REAL) {
        if (c->pot.cavity) TRY(run_row(c, ROW_PHASE, phase_at(c, tn, 0.5 * dt), red_at(c, tn), 0, 0));
    } else {
        TRY(run_row(c, ROW_SCALE, none, red_at(c, tn), 1, 0));
    }
    c->t = tn;
    return GPE_OK;
}

// The launch arguments of the cooperative kernels for this context: its
// tables and potential parameters, its control points, n steps of dt in
// `mode` from the context's time.
std::unique_ptr<CoopArgs> coop_args(const gpe_ctx *c, int n, double dt, int imag)
{
    static_assert(sizeof(CoopArgs) < 32000, "launch arguments");
    std::unique_ptr<CoopArgs> a(new CoopArgs());
    memset(a.get(), 0, sizeof(CoopArgs));
    const gpe_potential &p = c->pot;
    a->psi = c->psi;
    a->T = c->T;
    a->V = p.V;
    a->V_scale = (float)p.V_scale;
    a->g = (float)c->g;
    a->sx = (float)(1.0 / c->nx);
    a->sy = (float)(1.0 / c->ny);
    a->nx = c->nx;
    a->ny = c->ny;
    a->n = n;
    a->imag = imag;
    a->spins = c->spins;
    a->dt = dt;
    a->t0 = c->t;
    a->lat_V0x = p.lat_V0x;
    a->lat_V0y = p.lat_V0y;
    a->eta = p.eta;
    a->U0 = p.U0;
    a->dc = p.dc;
    a->kappa = p.kappa;
    a->N = p.N;
    a->dxdy = (c->Lx / c->nx) * (c->Ly / c->ny);
    a->probe_omega = p.probe_omega;
    a->probe_delta = p.probe_delta;
    a->probe_phi = p.probe_phi;
    a->cavity = p.cavity;
    a->pump_lattice = p.pump_lattice;
    a->ctrl_target = p.ctrl_target;
    a->nctrl = (int)c->ctrl_t.size();
    for (int i = 0; i < a->nctrl; ++i) {
        a->ctrl_t[i] = c->ctrl_t[i];
        a->ctrl_v[i] = c->ctrl_v[i];
    }
    return a;
}

// The cooperative kernel runs gpe_step on one context whose grid it is built
// for when the context's bit is set (by default on 512^2 grids), unless the context
// profiles its passes (per-pass events), has more control points than the
// launch arguments carry, or its stream is being captured into a graph.
bool coop_applies(gpe_ctx *c, int n)
{
    // at most 3 grid barriers per step (callers pass twice their steps for a
    // kernel with up to 6): the 32-bit arrival count of one launch stays
    // below 2^32 for n <= 2^21 with up to 512 CTAs (256 SMs, 2 CTAs per SM)
    if (!c->coop || c->prof || !coop_ok(c->nx, c->ny) || c->ctrl_t.size() > (size_t)COOP_MAX_CTRL || n > (1 << 21))
        return false;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(c->stream, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) {
        cudaGetLastError();
        return false;
    }
    return true;
}

// All n steps of one context in one cooperative launch: the program of
// step_prologue / step_part / step_epilogue with the phase and reduction
// arguments evaluated on the device (the kinetic tables for (dt, mode) are
// made here first, as step_prologue makes them).  If the device refuses the
// cooperative launch (nothing of it ran), *ran is false and the context
// keeps to the per-pass path from then on.
gpe_status step_coop(gpe_ctx *c, int n, double dt, gpe_mode mode, bool *ran)
{
    *ran = false;
    const int imag = mode == GPE_IMAG;
    TRY(kinetic_for(c, dt, mode));
    std::unique_ptr<CoopArgs> a = coop_args(c, n, dt, imag);
    // the barrier's counter and abort flag start at zero
    TRY(cuda_check(c, cudaMemsetAsync(&c->T.sc->bar_count, 0, 2 * sizeof(unsigned int), c->stream), "memset"));
    const cudaError_t e = launch_coop(*a, c->stream);
    if (e == cudaErrorCooperativeLaunchTooLarge || e == cudaErrorNotSupported || e == cudaErrorNotPermitted) {
        cudaGetLastError();
        c->coop = 0;
        return fail(c, GPE_OK, "cooperative launch refused (%s): the per-pass path from now on", cudaGetErrorString(e));
    }
    TRY(cuda_check(c, e, "cooperative step kernel"));
    c->launches++;
    *ran = true;
    c->t = c->t + n * dt;
    return GPE_OK;
}

}  // namespace

extern "C" {

gpe_status gpe_step(gpe_ctx *c, int n, double dt, gpe_mode mode)
{
    // one context through the batched path: the same passes, replayed from
    // a CUDA graph when the grid is small and nothing depends on time
    // (128^2 imaginary time: 24.6 -> 20.6 us per step; 512^2 real time:
    // 19.5 -> 15.2 us; bit for bit the same state)
    return gpe_step_many(&c, 1, n, dt, mode);
}

// ---------------------------------------------------------------- adjoint
// Layout of the adjoint workspace for n steps: S = ceil(sqrt(n)) steps per
// segment, K = ceil(n / S) segments.  Checkpoints psi_{kS} (k < K) and psi_n,
// the S + 1 states of one segment (two such buffers on the grids of
// launch_coop_adjrec, which recomputes one segment while the adjoint passes
// of the next run), lambda, and the 2n + 1 per-phase dJ/dv.
// GPE_ADJ_REVERSE keeps no checkpoints: ck holds psi_T only, and kx / ky the
// kinetic factors of -dt for the backward steps; on the grids of
// launch_coop_rev2, st and st2 are two more state buffers (the step back runs
// one step ahead of the adjoint passes, through three buffers).
struct AdjLayout {
    int S, K, variant;
    size_t P, ck, st, st2, lam, g, kx, ky, total;      // st2: 0 when there is no second segment buffer
};
static AdjLayout adj_layout(int nx, int ny, int n, int variant = GPE_ADJ_CHECKPOINT)
{
    AdjLayout L;
    L.variant = variant;
    L.P = align256(sizeof(float2) * (size_t)nx * ny);
    L.ck = 0;
    if (variant == GPE_ADJ_REVERSE) {
        L.S = n;
        L.K = 0;
        L.lam = L.ck + L.P;
        L.kx = L.lam + L.P;
        L.ky = L.kx + align256(sizeof(float2) * (size_t)nx);
        size_t o = L.ky + align256(sizeof(float2) * (size_t)ny);
        L.st = L.st2 = 0;
        if (coop_adjrec_ok(nx, ny)) {              // two more state buffers for launch_coop_rev2
            L.st = o;
            L.st2 = o + L.P;
            o += 2 * L.P;
        }
        L.g = o;
    } else {
        L.S = 1;
        while ((long long)L.S * L.S < n) ++L.S;
        L.K = (n + L.S - 1) / L.S;
        L.st = L.ck + (size_t)(L.K + 1) * L.P;
        L.st2 = coop_adjrec_ok(nx, ny) ? L.st + (size_t)(L.S + 1) * L.P : 0;
        L.lam = (L.st2 ? L.st2 : L.st) + (size_t)(L.S + 1) * L.P;
        L.kx = L.ky = 0;
        L.g = L.lam + L.P;
    }
    L.total = L.g + align256(sizeof(double) * (size_t)(2 * n + 1));
    return L;
}

// hat weight of control point i at time t, as control_value evaluates v(t)
static void control_weights(const gpe_ctx *c, double t, double gv, double *grad)
{
    const size_t n = c->ctrl_t.size();
    if (t <= c->ctrl_t[0]) { grad[0] += gv; return; }
    if (t >= c->ctrl_t[n - 1]) { grad[n - 1] += gv; return; }
    size_t lo = 0, hi = n - 1;
    while (hi - lo > 1) {
        const size_t mid = (lo + hi) / 2;
        if (c->ctrl_t[mid] < t) lo = mid; else hi = mid;
    }
    const double f = (t - c->ctrl_t[lo]) / (c->ctrl_t[hi] - c->ctrl_t[lo]);
    grad[lo] += (1.0 - f) * gv;
    grad[hi] += f * gv;
}

static gpe_status copy_d2d(gpe_ctx *c, void *dst, const void *src)
{
    return cuda_check(c, cudaMemcpyAsync(dst, src, sizeof(float2) * (size_t)c->nx * c->ny,
                                         cudaMemcpyDeviceToDevice, c->stream), "adjoint copy");
}

// One real-time step backward in time, psi_s = U(dt)^-1 psi_{s+1}, from the
// context's time t_{s+1}: the executed step with -dt.  Each half phase keeps
// |psi|, so its inverse is the conjugate phase evaluated on the same density
// (the density after it), and T(-dt) = T(dt)^-1; V at t_{s+1} opens and V at
// t_s closes, as in the forward step.  The kinetic factors of -dt (kx, ky)
// stand in for the context's tables during the two passes.
static gpe_status step_backward(gpe_ctx *c, double dt, float2 *kx, float2 *ky)
{
    float2 *fx = c->T.kinx, *fy = c->T.kiny;
    c->T.kinx = kx;
    c->T.kiny = ky;
    gpe_status st = step_part(c, 0, 1, -dt, GPE_REAL);
    if (st == GPE_OK) st = step_epilogue(c, 1, -dt, GPE_REAL);
    c->T.kinx = fx;
    c->T.kiny = fy;
    return st;
}

static gpe_status adjoint_run(gpe_ctx *c, int n, double dt, const float2 *phi, unsigned char *ws,
                              const AdjLayout &L, double *J_out, double *grad)
{
    float2 *ck = (float2 *)(ws + L.ck), *st = (float2 *)(ws + L.st), *lam = (float2 *)(ws + L.lam);
    double *gdev = (double *)(ws + L.g);
    const size_t P = L.P / sizeof(float2);
    const double t0 = c->t, tT = t0 + n * dt;
    const double dxdy = (c->Lx / c->nx) * (c->Ly / c->ny);
    const bool reverse = L.variant == GPE_ADJ_REVERSE;
    CUtensorMap lam_map;
    TRY(encode_map(c, lam, &lam_map));

    // The cooperative kernels take the forward sweep, each segment's
    // recomputation and its adjoint passes, one launch each, where they apply
    // (no cavity, a grid they are built for).  The forward sweep and the
    // recomputation both run the unfused steps of launch_coop_states, so the
    // recomputed states are the forward sweep's.  With the reverse sweep by
    // time reversal: the forward sweep in place in one launch, then the whole
    // reverse sweep in one more (two grid barriers per step).
    bool coop = !c->pot.cavity && coop_applies(c, reverse ? 2 * n : 2 * L.S);
    std::unique_ptr<CoopArgs> ca;
    if (coop) {
        TRY(kinetic_for(c, dt, GPE_REAL));
        ca = coop_args(c, 0, dt, 0);
        ca->t0 = t0;
        ca->lam = lam;
        ca->st = st;
        ca->P = P;
        ca->gout = gdev;
        ca->L0x = (float)c->pot.lat_V0x;
        ca->L0y = (float)c->pot.lat_V0y;
    }
    // steps s0 .. s1 - 1 in one cooperative launch: their states into st
    // (COOP_FWD), their adjoint passes (COOP_BWD), those beside the
    // recomputation of steps r0 .. r1 - 1 into st2 (COOP_BOTH), or the
    // reverse sweep by time reversal (COOP_REV; COOP_REV2 with the step back
    // beside the adjoint passes, through psi, st and st2).  *ran is false if the device refused the
    // launch (nothing of it ran); the context keeps to the per-pass path from
    // then on.
    enum { COOP_FWD, COOP_BWD, COOP_REV, COOP_REV2, COOP_BOTH };
    auto coop_run = [&](int which, int s0, int s1, bool *ran) -> gpe_status {
        *ran = false;
        ca->s0 = s0;
        ca->s1 = s1;
        TRY(cuda_check(c, cudaMemsetAsync(&c->T.sc->bar_count, 0, 2 * sizeof(unsigned int), c->stream), "memset"));
        const cudaError_t e = which == COOP_BWD    ? launch_coop_adj(*ca, c->stream)
                              : which == COOP_REV  ? launch_coop_rev(*ca, c->stream)
                              : which == COOP_REV2 ? launch_coop_rev2(*ca, c->stream)
                              : which == COOP_BOTH ? launch_coop_adjrec(*ca, c->stream)
                                                   : launch_coop_states(*ca, c->stream);
        if (e == cudaErrorCooperativeLaunchTooLarge || e == cudaErrorNotSupported || e == cudaErrorNotPermitted) {
            cudaGetLastError();
            c->coop = 0;
            coop = false;
            return fail(c, GPE_OK, "cooperative launch refused (%s): the per-pass path from now on",
                        cudaGetErrorString(e));
        }
        TRY(cuda_check(c, e, "cooperative adjoint-sweep kernel"));
        c->launches++;
        *ran = true;
        return GPE_OK;
    };

    // forward, keeping a checkpoint every S steps (none when the reverse
    // sweep steps backward instead): segment by segment through st, else one
    // V/2 - T - V/2 step per call
    if (!reverse) TRY(copy_d2d(c, ck, c->psi));
    float2 *psiT = ck + (size_t)L.K * P;
    int sf = 0;                                    // forward steps done
    if (reverse && coop) {                         // in place: st = psi, no stride
        ca->st = c->psi;
        ca->P = 0;
        bool ran = false;
        TRY(coop_run(COOP_FWD, 0, n, &ran));
        if (ran) sf = n;
    }
    for (int k = 0; k < L.K && coop && !reverse; ++k) {
        const int s0 = k * L.S, s1 = (s0 + L.S < n) ? s0 + L.S : n;
        TRY(copy_d2d(c, st, ck + (size_t)k * P));
        bool ran = false;
        TRY(coop_run(COOP_FWD, s0, s1, &ran));
        if (!ran) break;
        TRY(copy_d2d(c, ck + (size_t)(k + 1) * P, st + (size_t)(s1 - s0) * P));
        sf = s1;
    }
    if (sf > 0 && sf < n) {                        // refused after the first segment: on from the checkpoint
        TRY(copy_d2d(c, c->psi, ck + (size_t)(sf / L.S) * P));
        c->t = t0 + sf * dt;
    }
    for (int s = sf; s < n; ++s) {
        TRY(gpe_step(c, 1, dt, GPE_REAL));
        if (!reverse && (s + 1) % L.S == 0 && s + 1 < n)
            TRY(copy_d2d(c, ck + (size_t)((s + 1) / L.S) * P, c->psi));
    }
    // psi_T is in the context's psi after per-pass steps or the in-place
    // launch, in the last checkpoint after the segments
    if (sf < n || reverse) TRY(copy_d2d(c, psiT, c->psi));
    else TRY(copy_d2d(c, c->psi, psiT));
    if (sf == n) c->t = tT;                        // as gpe_step leaves it

    // J = E(psi_T) + |<phi|psi_T>|^2
    gpe_obs o;
    TRY(gpe_observables(c, &o));
    PhaseArgs none;
    memset(&none, 0, sizeof(none));
    TRY(timed_launch(c, 2, [&] {
        return launch_adj_overlap(psiT, phi, c->T, c->nx, c->ny, (float)c->pot.lat_V0x, (float)c->pot.lat_V0y,
                                  c->stream);
    }, "adjoint overlap"));
    DevScalars h;
    TRY(cuda_check(c, cudaMemcpyAsync(&h, c->T.sc, sizeof(h), cudaMemcpyDeviceToHost, c->stream), "copy"));
    TRY(cuda_check(c, cudaStreamSynchronize(c->stream), "sync"));
    const double cre = h.sums[0][0] * dxdy, cim = h.sums[0][1] * dxdy;
    *J_out = o.energy + cre * cre + cim * cim;
    control_weights(c, tT, h.sums[0][2] * dxdy, grad);            // E depends on v(T) through V

    // terminal adjoint lambda_T = dxdy (H psi_T + c phi)
    TRY(copy_d2d(c, lam, psiT));
    const RedArgs rd = red_at(c, tT);
    PassArgs a = pass_args(c, none, rd, 0, 0);
    a.psi = lam;
    TRY(timed_launch(c, 0, [&] { return launch_row(ROW_FFT_F, a, c->stream); }, "adjoint fft"));
    TRY(timed_launch(c, 1, [&] { return launch_col(COL_FFT_F, a, lam_map, c->stream); }, "adjoint fft"));
    TRY(timed_launch(c, 2, [&] {
        return launch_kin_energy_mul(lam, c->nx, c->ny, c->Lx, c->Ly, c->m, c->stream);
    }, "adjoint kinetic"));
    TRY(timed_launch(c, 1, [&] { return launch_col(COL_FFT_I, a, lam_map, c->stream); }, "adjoint fft"));
    TRY(timed_launch(c, 0, [&] { return launch_row(ROW_FFT_I, a, c->stream); }, "adjoint fft"));
    PassArgs aT = pass_args(c, phase_at(c, tT, 0.5 * dt), rd, 0, 0);
    TRY(timed_launch(c, 2, [&] {
        return launch_adj_terminal(lam, psiT, phi, aT, (float)cre, (float)cim, (float)dxdy, c->stream);
    }, "adjoint terminal"));

    // adjoint passes of step s: the row pass with the step's end state psi_{s+1},
    // the column pass with its initial state psi_s
    auto adjoint_row = [&](int s, const float2 *psi_s1) -> gpe_status {
        const double te = t0 + s * dt + dt;
        PassArgs ar = pass_args(c, phase_at(c, te, 0.5 * dt), red_at(c, te), 0, 0);
        ar.psi = lam;
        ar.psi2 = psi_s1;
        ar.gout = gdev + 2 * s + 1;
        ar.L0x = (float)c->pot.lat_V0x;
        ar.L0y = (float)c->pot.lat_V0y;
        return timed_launch(c, GPE_PASS_ADJ_ROW, [&] { return launch_row(ROW_ADJ, ar, c->stream, c->row_tile_shift); },
                            "adjoint row pass");
    };
    auto adjoint_col = [&](int s, const float2 *psi_s) -> gpe_status {
        const double ts = t0 + s * dt;
        PassArgs ac = pass_args(c, phase_at(c, ts, 0.5 * dt), red_at(c, ts), 0, 0);
        ac.psi = lam;
        ac.psi2 = psi_s;
        ac.gout = gdev + 2 * s;
        ac.L0x = (float)c->pot.lat_V0x;
        ac.L0y = (float)c->pot.lat_V0y;
        TRY(timed_launch(c, GPE_PASS_ADJ_COL, [&] { return launch_col(COL_ADJ, ac, lam_map, c->stream); },
                         "adjoint column pass"));
        return GPE_OK;
    };

    if (reverse) {
        // reverse sweep without checkpoints: psi_s from psi_{s+1} by one step
        // backward in time (exact in exact arithmetic; in FP32 the recovered
        // states carry the rounding of the steps taken back)
        float2 *kx = (float2 *)(ws + L.kx), *ky = (float2 *)(ws + L.ky);
        Tables Tb = c->T;
        Tb.kinx = kx;
        Tb.kiny = ky;
        TRY(timed_launch(c, 2, [&] {
            return launch_kinetic_tables(Tb, c->nx, c->ny, c->Lx, c->Ly, c->m, -dt, 0, c->stream);
        }, "kinetic tables"));
        // the row pass reads psi_{s+1} before the step back overwrites it, so
        // the context's psi is the only state buffer
        bool done = false;
        if (coop) {
            ca->kxb = kx;
            ca->kyb = ky;
            if (L.st2) {                           // on 512^2: the step back beside the adjoint passes
                ca->st = (float2 *)(ws + L.st);
                ca->st2 = (float2 *)(ws + L.st2);
                TRY(coop_run(COOP_REV2, 0, n, &done));
            }
            if (!done && coop) TRY(coop_run(COOP_REV, 0, n, &done));
            if (done) c->t = t0;
        }
        for (int s = n - 1; s >= 0 && !done; --s) {
            TRY(adjoint_row(s, c->psi));                          // with psi_{s+1}
            TRY(step_backward(c, dt, kx, ky));                    // psi <- psi_s, t <- t_s
            TRY(adjoint_col(s, c->psi));                          // with psi_s
        }
    }

    // reverse sweep, segment by segment: recompute the segment's states from
    // its checkpoint, then the two adjoint passes of each step.  On the grids
    // of launch_coop_adjrec, once the forward sweep ran on the cooperative
    // kernels: segment K - 1's states are still in st, and each launch runs
    // segment k's adjoint passes beside segment k - 1's recomputation into
    // the other buffer; segment 0's adjoint passes run alone.
    int kr = L.K - 1;                              // segments left for the loop below
    if (!reverse && coop && L.st2 && sf == n) {
        float2 *cur = st, *nxt = (float2 *)(ws + L.st2);
        for (; kr >= 1; --kr) {
            const int s0 = kr * L.S, s1 = (s0 + L.S < n) ? s0 + L.S : n;
            TRY(copy_d2d(c, nxt, ck + (size_t)(kr - 1) * P));
            ca->st = cur;
            ca->st2 = nxt;
            ca->r0 = s0 - L.S;
            ca->r1 = s0;
            bool ran = false;
            TRY(coop_run(COOP_BOTH, s0, s1, &ran));
            if (!ran) break;
            std::swap(cur, nxt);
        }
        if (kr == 0) {                             // segment 0: its states are in cur
            ca->st = cur;
            bool ran = false;
            TRY(coop_run(COOP_BWD, 0, (L.S < n) ? L.S : n, &ran));
            if (ran) kr = -1;
        }
        ca->st = st;
    }
    for (int k = kr; k >= 0 && !reverse; --k) {
        const int s0 = k * L.S, s1 = (s0 + L.S < n) ? s0 + L.S : n;
        bool rec = false, done = false;
        if (coop) {
            TRY(copy_d2d(c, st, ck + (size_t)k * P));
            TRY(coop_run(COOP_FWD, s0, s1, &rec));
        }
        if (!rec) {
            TRY(copy_d2d(c, c->psi, ck + (size_t)k * P));
            c->t = t0 + s0 * dt;
            TRY(copy_d2d(c, st, c->psi));
            for (int i = 1; i <= s1 - s0; ++i) {
                TRY(gpe_step(c, 1, dt, GPE_REAL));
                TRY(copy_d2d(c, st + (size_t)i * P, c->psi));
            }
        }
        if (coop) TRY(coop_run(COOP_BWD, s0, s1, &done));
        for (int s = s1 - 1; s >= s0 && !done; --s) {
            TRY(adjoint_row(s, st + (size_t)(s + 1 - s0) * P));
            TRY(adjoint_col(s, st + (size_t)(s - s0) * P));
        }
    }
    // leave the context at the final state and time, as gpe_step would
    TRY(copy_d2d(c, c->psi, psiT));
    c->t = tT;

    std::vector<double> g(2 * (size_t)n);
    TRY(cuda_check(c, cudaMemcpyAsync(g.data(), gdev, sizeof(double) * 2 * n, cudaMemcpyDeviceToHost, c->stream),
                   "copy"));
    TRY(cuda_check(c, cudaMemcpyAsync(&h, c->T.sc, sizeof(h), cudaMemcpyDeviceToHost, c->stream), "copy"));
    TRY(cuda_check(c, cudaStreamSynchronize(c->stream), "sync"));
    if (h.status) return fail(c, (gpe_status)h.status, "device status %s", gpe_status_string((gpe_status)h.status));
    for (int s = 0; s < n; ++s) {
        control_weights(c, t0 + s * dt, g[2 * s], grad);
        control_weights(c, t0 + (s + 1) * dt, g[2 * s + 1], grad);
    }
    return GPE_OK;
}

// Capture K interior steps of every context (on every lane) into a graph and
// launch it for steps 1 .. R K (R = (n-2) / K replays).  The contexts'
// streams are the lanes at this point.  Interior steps per graph: fewer graph
// boundaries (where every lane waits for the slowest), but the capture and
// instantiation grow with the graph.  Up to kGraphSteps steps while the graph
// stays within about 64 contexts' steps: 8 grids of 1024^2 ran at 81.2 G
// pt*steps/s with 4 steps per graph against 77.1 with 1, while the 384-grid
// sweep (40 steps per call) lost 11% to instantiating 4-step graphs.  The
// instantiated graph is kept (per device, the kGraphCache most recently used)
// and replayed again by later calls with the same contexts, unchanged since
// (uid, version), dt, mode, K and lane count, so a run split into many calls
// pays the capture once.
constexpr int kGraphSteps = 8;
constexpr int kGraphContextSteps = 64;

static GraphEntry *find_graph(Lanes *L, const std::vector<unsigned long long> &key, double dt, int mode, int K,
                              int nl)
{
    for (GraphEntry &g : L->graphs)
        if (g.dt == dt && g.mode == mode && g.K == K && g.nl == nl && g.key == key) return &g;
    return nullptr;
}

static gpe_status capture_graph(gpe_ctx *const *ctxs, int count, int n, double dt, gpe_mode mode, Lanes *L, int nl,
                                int K, GraphEntry *out)
{
    gpe_ctx *c0 = ctxs[0];
    std::vector<long long> before(count);
    for (int i = 0; i < count; ++i) before[i] = ctxs[i]->launches;
    out->exec.assign(nl, nullptr);
    gpe_status st = GPE_OK;
    for (int l = 0; l < nl && st == GPE_OK; ++l) {
        // the steps of lane l's contexts (i = l, l + nl, ...), captured on that lane
        st = cuda_check(c0, cudaStreamBeginCapture(L->s[l], cudaStreamCaptureModeThreadLocal), "begin capture");
        if (st != GPE_OK) break;
        for (int k = 1; k <= K && st == GPE_OK; ++k)
            for (int i = l; i < count && st == GPE_OK; i += nl) st = step_part(ctxs[i], k, n, dt, mode);
        cudaGraph_t g = nullptr;
        const cudaError_t e = cudaStreamEndCapture(L->s[l], &g);   // always end the capture
        if (st == GPE_OK) st = cuda_check(c0, e, "end capture");
        if (st == GPE_OK) st = cuda_check(c0, cudaGraphInstantiate(&out->exec[l], g, 0), "graph instantiate");
        if (g) cudaGraphDestroy(g);
    }
    // the captured launches were only recorded, not run: count them per replay
    out->launches.resize(count);
    for (int i = 0; i < count; ++i) {
        out->launches[i] = ctxs[i]->launches - before[i];
        ctxs[i]->launches = before[i];
    }
    if (st != GPE_OK) destroy_graphs(*out);
    return st;
}

static gpe_status replay_interior_steps(gpe_ctx *const *ctxs, int count, int n, double dt, gpe_mode mode, Lanes *L,
                                        int nl, int *done)
{
    *done = 0;
    int K = kGraphContextSteps / count;                              // interior steps per replay
    if (K > kGraphSteps) K = kGraphSteps;
    if (K > n - 2) K = n - 2;
    if (K < 1) K = 1;
    const int R = (n - 2) / K;                                       // replays
    gpe_ctx *c0 = ctxs[0];
    std::vector<unsigned long long> key(2 * (size_t)count);
    for (int i = 0; i < count; ++i) {
        key[2 * i] = ctxs[i]->uid;
        key[2 * i + 1] = ctxs[i]->version;
    }
    GraphEntry *g = find_graph(L, key, dt, (int)mode, K, nl);
    if (!g) {
        GraphEntry e;
        e.key = key;
        e.dt = dt;
        e.mode = (int)mode;
        e.K = K;
        e.nl = nl;
        e.used = 0;
        TRY(capture_graph(ctxs, count, n, dt, mode, L, nl, K, &e));
        if (L->graphs.size() >= kGraphCache) {
            // release the least recently used graphs (their pending launches complete first)
            size_t lru = 0;
            for (size_t i = 1; i < L->graphs.size(); ++i)
                if (L->graphs[i].used < L->graphs[lru].used) lru = i;
            destroy_graphs(L->graphs[lru]);
            L->graphs.erase(L->graphs.begin() + (long)lru);
        }
        L->graphs.push_back(std::move(e));
        g = &L->graphs.back();
    }
    g->used = ++L->clock;
    gpe_status st = GPE_OK;
    for (int r = 0; r < R && st == GPE_OK; ++r)
        for (int l = 0; l < nl && st == GPE_OK; ++l)
            st = cuda_check(c0, cudaGraphLaunch(g->exec[l], L->s[l]), "graph launch");
    for (int i = 0; i < count; ++i) ctxs[i]->launches += g->launches[i] * (long long)R;
    if (st == GPE_OK) *done = R * K;
    return st;
}

// Drop the cached graphs that step context `uid` (at its destruction).
static void forget_graphs(int device, unsigned long long uid)
{
    Lanes *L = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_lanes_mu);
        if (device >= 0 && device < 64) L = g_lanes[device];
    }
    if (!L) return;
    std::lock_guard<std::mutex> lock(L->mu);
    for (size_t i = 0; i < L->graphs.size();) {
        const std::vector<unsigned long long> &k = L->graphs[i].key;
        bool hit = false;
        for (size_t j = 0; j < k.size(); j += 2) hit = hit || k[j] == uid;
        if (hit) {
            destroy_graphs(L->graphs[i]);
            L->graphs.erase(L->graphs.begin() + (long)i);
        } else {
            ++i;
        }
    }
}

gpe_status gpe_step_many(gpe_ctx *const *ctxs, int count, int n, double dt, gpe_mode mode)
{
    if (!ctxs || count < 1) return GPE_EINVAL;
    for (int i = 0; i < count; ++i) TRY(step_check(ctxs[i], n, dt, mode));
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) return fail(ctxs[0], GPE_ECUDA, "gpe_step_many: no current device");
    for (int i = 0; i < count; ++i) {
        if (ctxs[i]->device != dev)
            return fail(ctxs[i], GPE_EINVAL, "gpe_step_many: context on device %d, current device %d",
                        ctxs[i]->device, dev);
        for (int j = 0; j < i; ++j)
            if (ctxs[j] == ctxs[i]) return fail(ctxs[i], GPE_EINVAL, "gpe_step_many: repeated context");
    }
    if (n == 0) return GPE_OK;
    if (count == 1 && coop_applies(ctxs[0], n)) {
        bool ran = false;
        TRY(step_coop(ctxs[0], n, dt, mode, &ran));
        if (ran) return GPE_OK;
    }
    // Contexts are spread over the library's lanes: each context's work is
    // ordered after what its own stream held (fork) and its stream waits for
    // that work (join), so the caller sees the usual per-stream ordering
    // while passes of different contexts overlap on the GPU.
    // Interior steps (0 < s < n-1) are identical when no context has a
    // time-dependent control.  For batches of grids up to 2048^2 (one context
    // included), up to kGraphSteps of them are captured into a CUDA graph per
    // lane (the steps of that lane's contexts) and each lane replays its
    // graph for the others on its own stream: one host launch per lane and
    // replay instead of one per pass, and no lane waits for another (a lane
    // whose contexts' inputs arrive first starts first).  Profiling contexts keep
    // per-pass launches (their events); time enters a pass only through a
    // control table and the cavity probe (Sec. 5.4), with either of which
    // consecutive steps have different arguments.
    bool graph = n >= 4 && small_grids(ctxs, count) && !getenv("GPE_NO_GRAPH");
    for (int i = 0; i < count && graph; ++i)
        graph = !ctxs[i]->prof && ctxs[i]->ctrl_t.empty() && ctxs[i]->pot.probe_omega == 0.0;
    // one context runs on a lane only to replay a graph there (a capture
    // needs a stream of its own; the caller's may be the legacy stream)
    Lanes *L = ((count > 1 || graph) && !getenv("GPE_SERIAL_MANY")) ? lanes_for_current_device() : nullptr;
    const int nl = L ? lanes_for(ctxs, count) : 0;
    graph = graph && L;
    // the lanes are shared by every caller on the device: work of two host
    // threads must not interleave on them (a graph capture on lane 0 would
    // take in the other thread's launches)
    std::unique_lock<std::mutex> lane_lock;
    if (L) lane_lock = std::unique_lock<std::mutex>(L->mu);
    std::vector<cudaStream_t> own(count);
    for (int i = 0; i < count; ++i) own[i] = ctxs[i]->stream;
    gpe_status st = GPE_OK;
    if (L) {
        for (int i = 0; i < count && st == GPE_OK; ++i) {
            gpe_ctx *c = ctxs[i];
            st = cuda_check(c, cudaEventRecord(c->ev_fork, own[i]), "fork record");
            if (st == GPE_OK) st = cuda_check(c, cudaStreamWaitEvent(L->s[i % nl], c->ev_fork, 0), "fork wait");
        }
        if (st != GPE_OK) return st;
        for (int i = 0; i < count; ++i) ctxs[i]->stream = L->s[i % nl];
    }
    for (int i = 0; i < count && st == GPE_OK; ++i) st = step_prologue(ctxs[i], dt, mode);
    int s = 0;
    if (graph && st == GPE_OK) {
        for (int i = 0; i < count && st == GPE_OK; ++i) st = step_part(ctxs[i], 0, n, dt, mode);
        int done = 0;
        if (st == GPE_OK) st = replay_interior_steps(ctxs, count, n, dt, mode, L, nl, &done);
        s = 1 + done;                    // the interior steps left over, then the last one, per pass
    }
    for (; s < n && st == GPE_OK; ++s)
        for (int i = 0; i < count && st == GPE_OK; ++i) st = step_part(ctxs[i], s, n, dt, mode);
    for (int i = 0; i < count && st == GPE_OK; ++i) st = step_epilogue(ctxs[i], n, dt, mode);
    if (L) {
        // join even after an error: every context's stream waits for its lane
        for (int i = 0; i < count; ++i) {
            gpe_ctx *c = ctxs[i];
            c->stream = own[i];
            const gpe_status j1 = cuda_check(c, cudaEventRecord(c->ev_join, L->s[i % nl]), "join record");
            const gpe_status j2 = j1 == GPE_OK ? cuda_check(c, cudaStreamWaitEvent(own[i], c->ev_join, 0), "join wait")
                                               : j1;
            if (st == GPE_OK) st = j2;
        }
    }
    return st;
}

gpe_status gpe_observables(gpe_ctx *c, gpe_obs *out)
{
    if (!c || !out) return GPE_EINVAL;
    TRY(run_row(c, ROW_OBS, phase_at(c, c->t, 0.0), red_at(c, c->t), 0, 0));
    TRY(run_col(c, COL_OBS, phase_at(c, c->t, 0.0), red_at(c, c->t), 0));
    DevScalars h;
    TRY(cuda_check(c, cudaMemcpyAsync(&h, c->T.sc, sizeof(h), cudaMemcpyDeviceToHost, c->stream), "copy"));
    TRY(cuda_check(c, cudaMemsetAsync(&c->T.sc->status, 0, sizeof(int), c->stream), "memset"));
    TRY(cuda_check(c, cudaStreamSynchronize(c->stream), "sync"));
    const double dxdy = (c->Lx / c->nx) * (c->Ly / c->ny);
    const double *S = h.sums[0];
    const double kx = 2.0 * M_PI / c->Lx, ky = 2.0 * M_PI / c->Ly;
    memset(out, 0, sizeof(*out));
    out->t = c->t;
    out->norm = S[0] * dxdy;
    out->ekin = (kx * kx * S[6] / c->nx + ky * ky * h.sums[1][0] / c->ny) * dxdy / (2.0 * c->m);
    double epot = S[1] * dxdy;
    if (c->pot.cavity) {
        const double O = S[3] / S[0], B = S[4] / S[0];
        const double eta = eta_at(c, c->t);
        const double dr = c->pot.dc - c->pot.U0 * B, di = c->pot.kappa, den = dr * dr + di * di;
        const double ph = c->pot.probe_delta * c->t + c->pot.probe_phi;
        const double a = c->pot.N * eta * O + c->pot.probe_omega * cos(ph), b = c->pot.probe_omega * sin(ph);
        const double ar = den > 0 ? (a * dr + b * di) / den : 0.0, ai = den > 0 ? (b * dr - a * di) / den : 0.0;
        out->O = O;
        out->B = B;
        out->alpha_re = ar;
        out->alpha_im = ai;
        epot += c->pot.U0 * (ar * ar + ai * ai) * S[4] * dxdy + 2.0 * eta * ar * S[3] * dxdy;
    }
    out->epot = epot;
    out->eint = 0.5 * c->g * S[2] * dxdy;
    out->energy = out->ekin + out->epot + out->eint;
    out->mu = out->ekin + out->epot + 2.0 * out->eint;
    out->status = h.status;
    if (!isfinite(out->norm) || !isfinite(out->energy)) out->status = out->status ? out->status : GPE_ENONFINITE;
    return out->status ? fail(c, (gpe_status)out->status, "device status %s", gpe_status_string((gpe_status)out->status))
                       : GPE_OK;
}

gpe_status gpe_set_psi(gpe_ctx *c, const void *src, int is_dev)
{
    if (!c || !src) return GPE_EINVAL;
    return cuda_check(c, cudaMemcpyAsync(c->psi, src, sizeof(float2) * c->nx * c->ny,
                                         is_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, c->stream),
                      "set_psi");
}

gpe_status gpe_get_psi(gpe_ctx *c, void *dst, int is_dev)
{
    if (!c || !dst) return GPE_EINVAL;
    TRY(cuda_check(c, cudaMemcpyAsync(dst, c->psi, sizeof(float2) * c->nx * c->ny,
                                      is_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, c->stream),
                   "get_psi"));
    if (!is_dev) TRY(cuda_check(c, cudaStreamSynchronize(c->stream), "sync"));
    return GPE_OK;
}

gpe_status gpe_set_time(gpe_ctx *c, double t)
{
    if (!c || !isfinite(t)) return GPE_EINVAL;
    c->t = t;
    return GPE_OK;
}

double gpe_get_time(const gpe_ctx *c) { return c ? c->t : 0.0; }

gpe_status gpe_fft2(gpe_ctx *c, int sign)
{
    if (!c || (sign != 1 && sign != -1)) return GPE_EINVAL;
    PhaseArgs none;
    memset(&none, 0, sizeof(none));
    if (sign == -1) {
        TRY(run_row(c, ROW_FFT_F, none, red_at(c, c->t), 0, 0));
        TRY(run_col(c, COL_FFT_F, none, red_at(c, c->t), 0));
    } else {
        TRY(run_col(c, COL_FFT_I, none, red_at(c, c->t), 0));
        TRY(run_row(c, ROW_FFT_I, none, red_at(c, c->t), 0, 0));
    }
    return GPE_OK;
}

gpe_status gpe_sync(gpe_ctx *c)
{
    if (!c) return GPE_EINVAL;
    int st = 0;
    TRY(cuda_check(c, cudaMemcpyAsync(&st, &c->T.sc->status, sizeof(int), cudaMemcpyDeviceToHost, c->stream),
                   "copy"));
    // clear the status word and, with it, the last-CTA counters: every CTA of
    // a reducing pass takes its turn at the counter even when its wait ran
    // out, so they are back at zero after each pass; resetting them here
    // as well makes a cleared context start from a known state
    static_assert(offsetof(DevScalars, status) == offsetof(DevScalars, ticket) + 2 * sizeof(unsigned int),
                  "ticket[2] and status are adjacent");
    TRY(cuda_check(c, cudaMemsetAsync(&c->T.sc->ticket[0], 0, 2 * sizeof(unsigned int) + sizeof(int), c->stream),
                   "memset"));
    TRY(cuda_check(c, cudaStreamSynchronize(c->stream), "sync"));
    return st ? fail(c, (gpe_status)st, "device status %s", gpe_status_string((gpe_status)st)) : GPE_OK;
}

gpe_status gpe_set_wait_limit(gpe_ctx *c, int spins)
{
    if (!c || spins < 0) return GPE_EINVAL;
    c->spins = spins;
    c->version++;
    return GPE_OK;
}

int gpe_get_wait_limit(const gpe_ctx *c) { return c ? c->spins : -1; }

gpe_status gpe_debug_timeout_probe(gpe_ctx *c, int spins)
{
    if (!c || spins < 1) return GPE_EINVAL;
    return timed_launch(c, 2, [&] { return launch_timeout_probe(c->T.sc, spins, c->stream); }, "timeout probe");
}

gpe_status gpe_profile(gpe_ctx *c, int enable)
{
    if (!c) return GPE_EINVAL;
    c->prof = enable != 0;
    return GPE_OK;
}

static gpe_status drain_profile(gpe_ctx *c)
{
    TRY(cuda_check(c, cudaStreamSynchronize(c->stream), "sync"));
    for (auto &p : c->ev_pending) {
        float ms = 0.f;
        if (p.first < GPE_PASS_KINDS && cudaEventElapsedTime(&ms, p.second.first, p.second.second) == cudaSuccess) {
            c->prof_ms[p.first] += ms;
            c->prof_n[p.first] += 1;
        }
        c->ev_free.push_back(p.second.first);
        c->ev_free.push_back(p.second.second);
    }
    c->ev_pending.clear();
    return GPE_OK;
}

gpe_status gpe_profile_read(gpe_ctx *c, double *row_ms, int *row_launches, double *col_ms, int *col_launches)
{
    if (!c) return GPE_EINVAL;
    TRY(drain_profile(c));
    if (row_ms) *row_ms = c->prof_ms[0];
    if (row_launches) *row_launches = c->prof_n[0];
    if (col_ms) *col_ms = c->prof_ms[1];
    if (col_launches) *col_launches = c->prof_n[1];
    c->prof_ms[0] = c->prof_ms[1] = 0.0;
    c->prof_n[0] = c->prof_n[1] = 0;
    return GPE_OK;
}

gpe_status gpe_profile_read_kind(gpe_ctx *c, int kind, double *ms, int *launches)
{
    if (!c || kind < 0 || kind >= GPE_PASS_KINDS) return GPE_EINVAL;
    TRY(drain_profile(c));
    if (ms) *ms = c->prof_ms[kind];
    if (launches) *launches = c->prof_n[kind];
    c->prof_ms[kind] = 0.0;
    c->prof_n[kind] = 0;
    return GPE_OK;
}

long long gpe_launch_count(const gpe_ctx *c) { return c ? c->launches : -1; }

gpe_status gpe_momentum_populations(gpe_ctx *c, int axis, double k0, int nmax, void *scratch_dev,
                                    size_t scratch_bytes, double *pop_out)
{
    if (!c || !pop_out || (axis != 0 && axis != 1) || !(k0 > 0.0) || !isfinite(k0) || nmax < 0 || nmax > 3)
        return c ? fail(c, GPE_EINVAL, "gpe_momentum_populations: axis %d k0 %g nmax %d", axis, k0, nmax)
                 : GPE_EINVAL;
    const size_t bytes = sizeof(float2) * (size_t)c->nx * c->ny;
    if (!scratch_dev || ((uintptr_t)scratch_dev & 255u) || scratch_bytes < bytes)
        return fail(c, GPE_EINVAL, "gpe_momentum_populations: scratch of %zu bytes (256-aligned) needed", bytes);
    float2 *f = (float2 *)scratch_dev;
    TRY(cuda_check(c, cudaMemcpyAsync(f, c->psi, bytes, cudaMemcpyDeviceToDevice, c->stream), "copy"));
    CUtensorMap fmap;
    TRY(encode_map(c, f, &fmap));
    PhaseArgs none;
    memset(&none, 0, sizeof(none));
    PassArgs a = pass_args(c, none, red_at(c, c->t), 0, 0);
    a.psi = f;
    TRY(timed_launch(c, 0, [&] { return launch_row(ROW_FFT_F, a, c->stream); }, "populations fft"));
    TRY(timed_launch(c, 1, [&] { return launch_col(COL_FFT_F, a, fmap, c->stream); }, "populations fft"));
    TRY(timed_launch(c, 2, [&] {
        return launch_kbin(f, c->T, c->nx, c->ny, c->Lx, c->Ly, axis, k0, nmax, c->stream);
    }, "populations"));
    DevScalars h;
    TRY(cuda_check(c, cudaMemcpyAsync(&h, c->T.sc, sizeof(h), cudaMemcpyDeviceToHost, c->stream), "copy"));
    TRY(cuda_check(c, cudaStreamSynchronize(c->stream), "sync"));
    const double total = h.sums[0][7];
    if (!(total > 0.0) || !isfinite(total)) return fail(c, GPE_ENONFINITE, "gpe_momentum_populations: total %g", total);
    for (int i = 0; i <= 2 * nmax; ++i) pop_out[i] = h.sums[0][i] / total;
    return GPE_OK;
}

int gpe_get_pass_variants(const gpe_ctx *c)
{
    if (!c) return -1;
    return (c->group_rows ? GPE_VARIANT_GROUP_ROWS : 0) | (c->stream_passes ? GPE_VARIANT_STREAM_ROWS : 0) |
           (c->stream_cols ? GPE_VARIANT_STREAM_COLS : 0) | (c->row_tile_shift << GPE_VARIANT_ROW_TILE_SHIFT) |
           (c->pair_cols ? GPE_VARIANT_PAIR_COLS : 0) | (c->pair_rows ? GPE_VARIANT_PAIR_ROWS : 0) |
           (c->coop ? GPE_VARIANT_COOP : 0);
}

gpe_status gpe_set_pass_variants(gpe_ctx *c, int v)
{
    const int known = GPE_VARIANT_GROUP_ROWS | GPE_VARIANT_STREAM_ROWS | GPE_VARIANT_STREAM_COLS |
                      (3 << GPE_VARIANT_ROW_TILE_SHIFT) | GPE_VARIANT_PAIR_COLS | GPE_VARIANT_PAIR_ROWS |
                      GPE_VARIANT_COOP;
    if (!c || v < 0 || (v & ~known) || ((v >> GPE_VARIANT_ROW_TILE_SHIFT) & 3) > 2) return GPE_EINVAL;
    c->group_rows = (v & GPE_VARIANT_GROUP_ROWS) != 0;
    c->pair_cols = (v & GPE_VARIANT_PAIR_COLS) != 0;
    c->pair_rows = (v & GPE_VARIANT_PAIR_ROWS) != 0;
    c->stream_passes = (v & GPE_VARIANT_STREAM_ROWS) != 0;
    c->stream_cols = (v & GPE_VARIANT_STREAM_COLS) != 0;
    c->row_tile_shift = (v >> GPE_VARIANT_ROW_TILE_SHIFT) & 3;
    c->coop = (v & GPE_VARIANT_COOP) != 0;
    c->version++;
    return GPE_OK;
}

gpe_status gpe_tune(gpe_ctx *c, double dt, gpe_mode mode, void *scratch_dev, size_t scratch_bytes, int reps,
                    int *variants_out, double *times_out)
{
    if (!c || !variants_out) return GPE_EINVAL;
    TRY(step_check(c, 1, dt, mode));
    const size_t bytes = sizeof(float2) * (size_t)c->nx * c->ny;
    if (!scratch_dev || ((uintptr_t)scratch_dev & 255u) || scratch_bytes < bytes || reps < 1 || reps > 1000)
        return fail(c, GPE_EINVAL, "gpe_tune: scratch of %zu bytes (256-aligned) and 1..1000 reps needed", bytes);
    const int imag = mode == GPE_IMAG;
    TRY(step_prologue(c, dt, mode));                     // kinetic tables for (dt, mode)
    float2 *w = (float2 *)scratch_dev;
    TRY(cuda_check(c, cudaMemcpyAsync(w, c->psi, bytes, cudaMemcpyDeviceToDevice, c->stream), "tune copy"));
    CUtensorMap wmap;
    TRY(encode_map(c, w, &wmap));
    PassArgs a = pass_args(c, phase_at(c, c->t, 0.5 * dt), red_at(c, c->t), imag, 0);
    a.psi = w;
    cudaEvent_t e0 = take_event(c), e1 = take_event(c);
    // time one candidate: a warm-up launch, then `reps` launches between events
    auto time_it = [&](auto &&launch, double *ms) -> gpe_status {
        TRY(cuda_check(c, launch(), "tune launch"));
        TRY(cuda_check(c, cudaEventRecord(e0, c->stream), "tune event"));
        for (int r = 0; r < reps; ++r) TRY(cuda_check(c, launch(), "tune launch"));
        TRY(cuda_check(c, cudaEventRecord(e1, c->stream), "tune event"));
        TRY(cuda_check(c, cudaEventSynchronize(e1), "tune sync"));
        float f = 0.f;
        TRY(cuda_check(c, cudaEventElapsedTime(&f, e0, e1), "tune time"));
        *ms = f / reps;
        c->launches += reps + 1;
        return GPE_OK;
    };
    double t[5];
    for (double &x : t) x = NAN;
    // one-shot row pass at its default and at half its default rows per CTA;
    // the half tile is kept unless it is at least 3% slower.  In the
    // phase-diagram sweep under gpe_step_many (256^2 .. 1024^2) every size
    // ran best at the half tile: 35.2 against 33.0 G pt*steps/s at the
    // default and 33.1 at the quarter tile (value 2, which is left to
    // gpe_set_pass_variants), while alone the two larger tiles timed within
    // a few percent of each other.
    int shift = 0;
    gpe_status st = GPE_OK;
    for (int k = 0; k < 2 && st == GPE_OK; ++k) {
        if (k > 0 && row_rows_per_cta(c->nx, c->ny, k) == row_rows_per_cta(c->nx, c->ny, k - 1)) break;
        double ms = NAN;
        st = time_it([&] { return launch_row(ROW_PT, a, c->stream, k); }, &ms);
        if (st == GPE_OK && (k == 0 || ms <= 1.03 * t[0])) {
            t[0] = ms;
            shift = k;
        }
    }
    // the pencil-pair row pass (one-shot, one CTA per row pair) competes with
    // the one-pencil one-shot pass for slot 0
    double t_rpair = NAN;
    if (st == GPE_OK && row_pair_ok(c->nx, c->ny))
        st = time_it([&] { return launch_row_pair(a, c->stream); }, &t_rpair);
    if (st == GPE_OK && row_group_ok(c->nx, c->ny))
        st = time_it([&] { return launch_row_group(a, c->stream); }, &t[1]);
    if (st == GPE_OK && row_stream_ok(c->nx, c->ny))
        st = time_it([&] { return launch_row_stream(a, c->stream); }, &t[2]);
    if (st == GPE_OK) st = time_it([&] { return launch_col(COL_T, a, wmap, c->stream); }, &t[3]);
    double t_pair = NAN;
    if (st == GPE_OK && col_pair_ok(c->nx, c->ny))
        st = time_it([&] { return launch_col_pair(COL_T, a, wmap, c->stream); }, &t_pair);
    if (st == GPE_OK && col_stream_ok(c->nx, c->ny))
        st = time_it([&] { return launch_col_stream(COL_T, a, wmap, c->stream); }, &t[4]);
    c->ev_free.push_back(e0);
    c->ev_free.push_back(e1);
    if (st != GPE_OK) return st;
    // a persistent row variant replaces the one-shot pass only when at least
    // 3% faster: on near ties the one-shot pass, whose CTAs the hardware
    // schedules freely, overlapped better with other grids' passes under
    // gpe_step_many (1024^2 in the phase-diagram sweep)
    const bool rpair = t_rpair == t_rpair && t_rpair < t[0];
    if (rpair) t[0] = t_rpair;
    int best = 0;
    for (int k = 1; k < 3; ++k)
        if (t[k] == t[k] && t[k] < 0.97 * t[best]) best = k;
    int v = best == 1 ? GPE_VARIANT_GROUP_ROWS : best == 2 ? GPE_VARIANT_STREAM_ROWS : 0;
    if (best == 0) v |= rpair ? GPE_VARIANT_PAIR_ROWS : shift << GPE_VARIANT_ROW_TILE_SHIFT;
    // the one-shot column pass: the faster of the one-pencil and pair forms
    const bool pair = t_pair == t_pair && t_pair < t[3];
    if (pair) t[3] = t_pair;
    if (t[4] == t[4] && t[4] < t[3]) v |= GPE_VARIANT_STREAM_COLS;
    else if (pair) v |= GPE_VARIANT_PAIR_COLS;
    v |= c->coop ? GPE_VARIANT_COOP : 0;                 // not a per-pass choice: left as it was
    TRY(gpe_set_pass_variants(c, v));
    *variants_out = v;
    if (times_out)
        for (int k = 0; k < 5; ++k) times_out[k] = t[k];
    return GPE_OK;
}

size_t gpe_adjoint_workspace_size(int nx, int ny, int nsteps)
{
    return gpe_adjoint_workspace_size_ex(nx, ny, nsteps, GPE_ADJ_CHECKPOINT);
}

size_t gpe_adjoint_workspace_size_ex(int nx, int ny, int nsteps, int variant)
{
    if (!pow2_in_range(nx) || !pow2_in_range(ny) || nsteps < 1) return 0;
    if (variant != GPE_ADJ_CHECKPOINT && variant != GPE_ADJ_REVERSE) return 0;
    return adj_layout(nx, ny, nsteps, variant).total;
}

gpe_status gpe_adjoint_lattice(gpe_ctx *c, int nsteps, double dt, const void *phi_dev, void *adj_ws,
                               size_t adj_ws_bytes, double *J_out, double *grad_out)
{
    return gpe_adjoint_lattice_ex(c, nsteps, dt, GPE_ADJ_CHECKPOINT, phi_dev, adj_ws, adj_ws_bytes, J_out,
                                  grad_out);
}

gpe_status gpe_adjoint_lattice_ex(gpe_ctx *c, int nsteps, double dt, int variant, const void *phi_dev,
                                  void *adj_ws, size_t adj_ws_bytes, double *J_out, double *grad_out)
{
    if (!c || !J_out || !grad_out) return GPE_EINVAL;
    if (variant != GPE_ADJ_CHECKPOINT && variant != GPE_ADJ_REVERSE)
        return fail(c, GPE_EINVAL, "gpe_adjoint_lattice: variant %d", variant);
    TRY(step_check(c, nsteps, dt, GPE_REAL));
    if (nsteps < 1) return fail(c, GPE_EINVAL, "gpe_adjoint_lattice: nsteps %d", nsteps);
    if (!phi_dev || ((uintptr_t)phi_dev & 15u) || !adj_ws || ((uintptr_t)adj_ws & 255u))
        return fail(c, GPE_EINVAL, "gpe_adjoint_lattice: null or misaligned buffer");
    if (c->pot.cavity || c->pot.ctrl_target != GPE_CTRL_LATTICE || c->ctrl_t.empty())
        return fail(c, GPE_EINVAL, "gpe_adjoint_lattice: needs a lattice control table and no cavity");
    const AdjLayout L = adj_layout(c->nx, c->ny, nsteps, variant);
    if (adj_ws_bytes < L.total) return fail(c, GPE_ENOMEM, "gpe_adjoint_lattice: workspace %zu < %zu", adj_ws_bytes,
                                            L.total);
    for (size_t i = 0; i < c->ctrl_t.size(); ++i) grad_out[i] = 0.0;
    return adjoint_run(c, nsteps, dt, (const float2 *)phi_dev, (unsigned char *)adj_ws, L, J_out, grad_out);
}

void gpe_destroy(gpe_ctx *c)
{
    if (!c) return;
    if (!c->ev_pending.empty()) cudaStreamSynchronize(c->stream);
    for (auto &p : c->ev_pending) {
        cudaEventDestroy(p.second.first);
        cudaEventDestroy(p.second.second);
    }
    for (cudaEvent_t e : c->ev_free) cudaEventDestroy(e);
    cudaEventDestroy(c->ev_fork);
    cudaEventDestroy(c->ev_join);
    forget_graphs(c->device, c->uid);
    delete c;
}

const char *gpe_last_error(const gpe_ctx *c) { return c ? c->err : "null context"; }

}  // extern "C"

// ---------------------------------------------------------------- persistent batch
// A batch binds contexts (in order) to a caller-provided device workspace that
// holds the kernel's descriptors, prefix sums, control points and counters.
struct gpe_batch {
    std::vector<gpe_ctx *> ctxs;
    std::vector<unsigned long long> key;      // uid, version per context at the last upload
    unsigned char *ws;
    size_t ws_bytes;
    int device;
    int tpi;                                  // tiles per item
    int bt;                                   // threads per CTA and per tile (256 or 64)
    int grid;                                 // CTAs of a launch
    int row_items, col_items;                 // items per row / column pass, all contexts
    std::vector<cudaStream_t> streams;        // distinct context streams other than the first
    cudaEvent_t ev;
};

namespace {

struct BatchLayout {
    size_t counters, rpre, cpre, desc, ctrl, total;
};

BatchLayout batch_layout(int count, size_t ctrl_points)
{
    BatchLayout L;
    size_t o = 0;
    L.counters = o; o = align256(o + sizeof(unsigned int) * (2 + 2 * (size_t)count));
    L.rpre = o;     o = align256(o + sizeof(int) * ((size_t)count + 1));
    L.cpre = o;     o = align256(o + sizeof(int) * ((size_t)count + 1));
    L.desc = o;     o = align256(o + sizeof(BatchCtx) * (size_t)count);
    L.ctrl = o;     o = align256(o + 2 * sizeof(double) * ctrl_points);
    L.total = o;
    return L;
}

size_t ctrl_points_of(gpe_ctx *const *ctxs, int count)
{
    size_t n = 0;
    for (int i = 0; i < count; ++i) n += ctxs[i]->ctrl_t.size();
    return n;
}

bool time_dependent(const gpe_ctx *c) { return !c->ctrl_t.empty() || c->pot.probe_omega != 0.0; }

// Write the descriptors of every context into the batch workspace (pageable
// copies on the first context's stream, which the call then waits for).
gpe_status batch_upload(gpe_batch *b)
{
    const int count = (int)b->ctxs.size();
    gpe_ctx *c0 = b->ctxs[0];
    const BatchLayout L = batch_layout(count, ctrl_points_of(b->ctxs.data(), count));
    std::vector<BatchCtx> d(count);
    std::vector<int> rpre(count + 1, 0), cpre(count + 1, 0);
    std::vector<double> ctrl;
    const double *ctrl_dev = (const double *)(b->ws + L.ctrl);
    // tile width: 256-thread tiles, unless even the widest pass would leave
    // most of the launch idle (a single small grid) and every context fits
    // 64-thread tiles (rows of at most 1024 points, columns of at most 512):
    // then 4 times as many, smaller tiles spread a pass over more SMs
    auto tiles = [&](int bt, long long &rt, long long &ct) {
        rt = ct = 0;
        for (int i = 0; i < count; ++i) {
            rt += b->ctxs[i]->ny / batch_rows_per_item(b->ctxs[i]->nx, bt);
            ct += b->ctxs[i]->nx / batch_rows_per_item(b->ctxs[i]->ny, bt);
        }
    };
    long long rt = 0, ct = 0;
    tiles(256, rt, ct);
    bool small_ok = true;
    for (int i = 0; i < count; ++i) small_ok = small_ok && batch_supported(b->ctxs[i]->nx, b->ctxs[i]->ny, 64);
    const char *forced = getenv("GPE_BATCH_THREADS");
    if (forced) b->bt = (atoi(forced) == 64 && small_ok) ? 64 : 256;
    else b->bt = (small_ok && (rt > ct ? rt : ct) < batch_resident_ctas(256)) ? 64 : 256;
    if (b->bt == 64) tiles(64, rt, ct);
    // tiles per item: one item per tile unless the passes are much wider than
    // the launch (then up to 8 consecutive tiles per item, so that the
    // per-item dependency check and completion count are paid less often)
    const int resident = batch_resident_ctas(b->bt);
    if (resident <= 0) return fail(c0, GPE_ECUDA, "gpe_batch: no occupancy for the batch kernel");
    long long tpi = (rt < ct ? rt : ct) / (4LL * resident);
    b->tpi = (int)(tpi < 1 ? 1 : tpi > 8 ? 8 : tpi);
    for (int i = 0; i < count; ++i) {
        gpe_ctx *c = b->ctxs[i];
        BatchCtx &e = d[i];
        memset(&e, 0, sizeof(e));
        e.cpi = batch_rows_per_item(c->ny, b->bt);
        e.rpi = batch_rows_per_item(c->nx, b->bt);
        TRY(encode_map_w(c, c->psi, e.cpi, &e.map));
        e.psi = c->psi;
        e.T = c->T;
        e.V = c->pot.V;
        e.V_scale = (float)c->pot.V_scale;
        e.g = (float)c->g;
        e.sx = (float)(1.0 / c->nx);
        e.sy = (float)(1.0 / c->ny);
        e.nx = c->nx;
        e.ny = c->ny;
        e.row_tiles = c->ny / e.rpi;
        e.col_tiles = c->nx / e.cpi;
        e.row_items = (e.row_tiles + b->tpi - 1) / b->tpi;
        e.col_items = (e.col_tiles + b->tpi - 1) / b->tpi;
        const gpe_potential &p = c->pot;
        e.lat_V0x = p.lat_V0x;
        e.lat_V0y = p.lat_V0y;
        e.eta = p.eta;
        e.U0 = p.U0;
        e.dc = p.dc;
        e.kappa = p.kappa;
        e.N = p.N;
        e.dxdy = (c->Lx / c->nx) * (c->Ly / c->ny);
        e.probe_omega = p.probe_omega;
        e.probe_delta = p.probe_delta;
        e.probe_phi = p.probe_phi;
        e.cavity = p.cavity;
        e.pump_lattice = p.pump_lattice;
        e.ctrl_target = p.ctrl_target;
        e.nctrl = (int)c->ctrl_t.size();
        if (e.nctrl > 0) {
            e.ctrl_t = ctrl_dev + ctrl.size();
            ctrl.insert(ctrl.end(), c->ctrl_t.begin(), c->ctrl_t.end());
            e.ctrl_v = ctrl_dev + ctrl.size();
            ctrl.insert(ctrl.end(), c->ctrl_v.begin(), c->ctrl_v.end());
        }
        rpre[i + 1] = rpre[i] + e.row_items;
        cpre[i + 1] = cpre[i] + e.col_items;
    }
    const cudaStream_t s = c0->stream;
    TRY(cuda_check(c0, cudaMemcpyAsync(b->ws + L.desc, d.data(), sizeof(BatchCtx) * count, cudaMemcpyHostToDevice, s),
                   "batch upload"));
    TRY(cuda_check(c0, cudaMemcpyAsync(b->ws + L.rpre, rpre.data(), sizeof(int) * (count + 1), cudaMemcpyHostToDevice,
                                       s), "batch upload"));
    TRY(cuda_check(c0, cudaMemcpyAsync(b->ws + L.cpre, cpre.data(), sizeof(int) * (count + 1), cudaMemcpyHostToDevice,
                                       s), "batch upload"));
    if (!ctrl.empty())
        TRY(cuda_check(c0, cudaMemcpyAsync(b->ws + L.ctrl, ctrl.data(), sizeof(double) * ctrl.size(),
                                           cudaMemcpyHostToDevice, s), "batch upload"));
    TRY(cuda_check(c0, cudaStreamSynchronize(s), "batch upload"));
    for (int i = 0; i < count; ++i) {
        b->key[2 * i] = b->ctxs[i]->uid;
        b->key[2 * i + 1] = b->ctxs[i]->version;
    }
    // no more CTAs than the widest pass has items: the rest would only wait
    b->row_items = rpre[count];
    b->col_items = cpre[count];
    const int wide = b->row_items > b->col_items ? b->row_items : b->col_items;
    b->grid = wide < resident ? wide : resident;
    return GPE_OK;
}

}  // namespace

extern "C" {

size_t gpe_batch_workspace_size(gpe_ctx *const *ctxs, int count)
{
    if (!ctxs || count < 1) return 0;
    for (int i = 0; i < count; ++i)
        if (!ctxs[i]) return 0;
    return batch_layout(count, ctrl_points_of(ctxs, count)).total;
}

gpe_status gpe_batch_create(gpe_ctx *const *ctxs, int count, void *ws, size_t ws_bytes, gpe_batch **out)
{
    if (!out) return GPE_EINVAL;
    *out = nullptr;
    if (!ctxs || count < 1) return GPE_EINVAL;
    for (int i = 0; i < count; ++i) {
        if (!ctxs[i]) return GPE_EINVAL;
        for (int j = 0; j < i; ++j)
            if (ctxs[j] == ctxs[i]) return fail(ctxs[i], GPE_EINVAL, "gpe_batch_create: repeated context");
        if (!batch_supported(ctxs[i]->nx, ctxs[i]->ny, 256))
            return fail(ctxs[i], GPE_EINVAL, "gpe_batch_create: grid %dx%d not supported in a batch (64..2048 per axis)",
                        ctxs[i]->nx, ctxs[i]->ny);
        if (ctxs[i]->device != ctxs[0]->device)
            return fail(ctxs[i], GPE_EINVAL, "gpe_batch_create: contexts on different devices");
    }
    if (!ws || ((uintptr_t)ws & 255u)) return fail(ctxs[0], GPE_EINVAL, "gpe_batch_create: workspace not 256-byte aligned");
    if (ws_bytes < gpe_batch_workspace_size(ctxs, count))
        return fail(ctxs[0], GPE_ENOMEM, "gpe_batch_create: workspace of %zu bytes, %zu needed", ws_bytes,
                    gpe_batch_workspace_size(ctxs, count));
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev != ctxs[0]->device)
        return fail(ctxs[0], GPE_EINVAL, "gpe_batch_create: the contexts' device is not current");
    gpe_batch *b = new gpe_batch();
    b->ctxs.assign(ctxs, ctxs + count);
    b->key.assign(2 * (size_t)count, 0);
    b->ws = (unsigned char *)ws;
    b->ws_bytes = ws_bytes;
    b->device = dev;
    b->ev = nullptr;
    for (int i = 1; i < count; ++i) {
        bool seen = ctxs[i]->stream == ctxs[0]->stream;
        for (cudaStream_t t : b->streams) seen = seen || t == ctxs[i]->stream;
        if (!seen) b->streams.push_back(ctxs[i]->stream);
    }
    gpe_status st = cuda_check(ctxs[0], cudaEventCreateWithFlags(&b->ev, cudaEventDisableTiming), "event");
    if (st == GPE_OK) st = batch_upload(b);
    if (st != GPE_OK) {
        if (b->ev) cudaEventDestroy(b->ev);
        delete b;
        return st;
    }
    *out = b;
    return GPE_OK;
}

gpe_status gpe_batch_step(gpe_batch *b, int n, double dt, gpe_mode mode)
{
    if (!b) return GPE_EINVAL;
    const int count = (int)b->ctxs.size();
    gpe_ctx *c0 = b->ctxs[0];
    for (int i = 0; i < count; ++i) TRY(step_check(b->ctxs[i], n, dt, mode));
    if (n == 0) return GPE_OK;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev != b->device)
        return fail(c0, GPE_EINVAL, "gpe_batch_step: the batch's device is not current");
    const int cavity = c0->pot.cavity ? 1 : 0;
    bool timed = false;
    for (int i = 0; i < count; ++i) {
        gpe_ctx *c = b->ctxs[i];
        if ((c->pot.cavity ? 1 : 0) != cavity)
            return fail(c, GPE_EINVAL, "gpe_batch_step: every context of a batch has a cavity, or none");
        if (c->prof) return fail(c, GPE_EINVAL, "gpe_batch_step: profiling contexts step through gpe_step_many");
        timed = timed || time_dependent(c);
    }
    for (int i = 1; i < count && timed; ++i)
        if (b->ctxs[i]->t != c0->t)
            return fail(b->ctxs[i], GPE_EINVAL, "gpe_batch_step: with a control table or a probe, every context "
                                                "of the batch must be at the same time");
    // the descriptors follow the contexts' settings (potential, variants, wait limit)
    bool stale = false;
    for (int i = 0; i < count; ++i) stale = stale || b->key[2 * i + 1] != b->ctxs[i]->version;
    if (stale) TRY(batch_upload(b));
    const int imag = mode == GPE_IMAG;
    // kinetic factors of (dt, mode) on each context's stream
    for (int i = 0; i < count; ++i) TRY(kinetic_for(b->ctxs[i], dt, mode));
    // the launch runs on the first context's stream, after the others' work
    const cudaStream_t s = c0->stream;
    for (cudaStream_t t : b->streams) {
        TRY(cuda_check(c0, cudaEventRecord(b->ev, t), "batch fork"));
        TRY(cuda_check(c0, cudaStreamWaitEvent(s, b->ev, 0), "batch fork"));
    }
    const BatchLayout L = batch_layout(count, ctrl_points_of(b->ctxs.data(), count));
    const int R = b->row_items, C = b->col_items;
    // a launch's queue stays below 2^31 items: longer runs take several launches
    const long long per_step = batch_queue_length(1, imag, cavity, R, C);
    const int max_steps = (int)((1LL << 31) / (per_step > 0 ? per_step : 1)) - 2;
    unsigned int *cnt = (unsigned int *)(b->ws + L.counters);
    for (int done = 0; done < n;) {
        const int m = n - done < max_steps ? n - done : max_steps;
        BatchArgs a;
        memset(&a, 0, sizeof(a));
        a.ctx = (const BatchCtx *)(b->ws + L.desc);
        a.row_prefix = (const int *)(b->ws + L.rpre);
        a.col_prefix = (const int *)(b->ws + L.cpre);
        a.head = cnt;
        a.epoch = cnt + 2;
        a.done = cnt + 2 + count;
        a.count = count;
        a.n = m;
        a.imag = imag;
        a.cavity = cavity;
        a.spins = c0->spins;
        a.tpi = b->tpi;
        a.bt = b->bt;
        a.dt = dt;
        a.t0 = c0->t;
        a.total = (unsigned int)batch_queue_length(m, imag, cavity, R, C);
        TRY(cuda_check(c0, cudaMemsetAsync(cnt, 0, sizeof(unsigned int) * (2 + 2 * (size_t)count), s), "batch memset"));
        TRY(cuda_check(c0, launch_batch(a, s, b->grid), "batch launch"));
        c0->launches++;
        for (int i = 0; i < count; ++i) b->ctxs[i]->t += m * dt;
        done += m;
    }
    for (cudaStream_t t : b->streams) {
        TRY(cuda_check(c0, cudaEventRecord(b->ev, s), "batch join"));
        TRY(cuda_check(c0, cudaStreamWaitEvent(t, b->ev, 0), "batch join"));
    }
    return GPE_OK;
}

void gpe_batch_destroy(gpe_batch *b)
{
    if (!b) return;
    if (b->ev) cudaEventDestroy(b->ev);
    delete b;
}

}  // extern "C"
