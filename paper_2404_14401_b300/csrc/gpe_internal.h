// gpe_internal.h -- types shared by the host scheduler (gpe_api.cu) and the
// kernels (gpe_kernels.cu).  Not part of the public C ABI.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace gpe {

constexpr int NQ = 8;              // quantities per reduction partial
constexpr int MAX_BLOCKS = 8192;   // upper bound on CTAs of one reducing pass

// Scalars living in the workspace.  Written by the last CTA of a reducing
// pass, read by the passes that follow on the same stream.
struct DevScalars {
    double alpha_re, alpha_im;     // cavity field for the next potential phase (Eq. 14)
    double c;                      // pending normalisation 1/sqrt(norm) (Sec. 3.3)
    double norm;                   // last reduced norm  int |psi|^2
    double O, B;                   // last normalised overlaps (Eqs. 14-15)
    double sums[2][NQ];            // finalised sums: [0] row passes, [1] column passes
    unsigned int ticket[2];        // last-CTA counters (row / column kernels)
    int status;                    // first device error (gpe_status), 0 = none
    int pad;
    // grid barrier of the cooperative kernel (gpe_coop.cu): arrivals so far
    // in the launch and the abort flag, zeroed before each launch
    unsigned int bar_count, bar_abort;
};

// Device pointers into the caller's workspace.
struct Tables {
    DevScalars *sc;
    double *part_row;              // [MAX_BLOCKS][NQ] per-CTA partial sums
    double *part_col;              // [MAX_BLOCKS][NQ]
    float4 *twx, *twy;             // per-stage twiddles of the radix-16 schedule: {re_hi, im_hi, re_lo, im_lo}
    float4 *tw8x, *tw8y;           // the same for the radix-8 schedule (8 elements per thread)
    float4 *xtab, *ytab;           // {(m/2) w^2 x^2, cos^2(k_lat x), cos(kc x), x}
    float2 *kinx, *kiny;           // kinetic factors (see kinetic_tables_kernel)
};

// One potential phase, evaluated on the host at the phase's time.
struct PhaseArgs {
    float h;                       // theta = (V + g |psi|^2) h
    float a_latx, a_laty;          // lattice depths at this time (Eq. 9)
    float a_pump;                  // eta^2 / U0 (pump lattice, Eq. 11) or 0
    float U0;                      // cavity U0 (Eq. 12)
    float two_eta;                 // 2 eta (Eq. 13)
    int use_alpha;                 // read alpha from DevScalars for V_c, V_i
};

// Cavity reduction / finalisation parameters (Eqs. 14-15).
struct RedArgs {
    double eta, U0, dc, kappa, N, dxdy;
    int cavity;
    // on-axis cavity probe at the time t of the reduction (Sec. 5.4):
    // alpha' = alpha + Omega_c exp(i (Delta_p t + phi)) / (Delta_c - U0 B + i kappa)
    double probe_omega, probe_delta, probe_phi, t;
};

// Row passes (x axis).  T_x = F_x^-1 K_x F_x is the x part of the kinetic
// propagator; F^-1 K F = T_x T_y exactly because K = K_x K_y is separable.
enum RowMode {
    ROW_PT = 0,         // [scale c] potential phase, T_x, store
    ROW_PHASE = 1,      // potential phase, store
    ROW_PHASE_R = 2,    // potential phase, reduce (norm, O, B -> c, alpha), store
    ROW_REDUCE_R = 3,   // reduce (-> c, alpha), no store
    ROW_SCALE = 4,      // multiply by c, store
    ROW_FFT_F = 5,      // F_x only
    ROW_FFT_I = 6,      // F_x^-1 (with 1/nx)
    ROW_OBS = 7,        // observable sums + F_x kinetic sum, no store
    ROW_ADJ = 8         // adjoint of a closing half phase (psi2 = its output), then T_x^H; reduce dJ/dv
};

// Column passes (y axis), on TMA-loaded tiles of W columns.
enum ColMode {
    COL_T = 0,          // T_y, store
    COL_T_R = 1,        // T_y, reduce (-> c, alpha), store
    COL_T_PR = 2,       // T_y, potential phase, reduce, store
    COL_FFT_F = 3,      // F_y only
    COL_FFT_I = 4,      // F_y^-1 (with 1/ny)
    COL_OBS = 5,        // F_y, sum ky^2 |.|^2, no store
    COL_ADJ = 6,        // T_y^H, then the adjoint of an opening half phase (psi2 = its input); reduce dJ/dv
    COL_T_P = 7         // T_y, potential phase, store (no reductions: the last real-time step without cavity)
};

struct PassArgs {
    float2 *psi;
    int nx, ny;
    const float *V;
    float V_scale, g;
    int imag, use_c;
    float sx, sy;                  // exact 1/nx, 1/ny
    int spins;                     // bound on the TMA barrier wait
    PhaseArgs ph;
    RedArgs red;
    Tables T;
    // adjoint passes: the forward state the phase adjoint needs ([ny][nx]),
    // where the last CTA writes the reduced dJ/dv, and the base lattice
    // depths L = L0x cos^2(k x) + L0y cos^2(k y) = dV/dv (Eq. 9)
    const float2 *psi2;
    double *gout;
    float L0x, L0y;
};

// ---- Persistent batch (gpe_batch.cu): one launch steps many contexts.
// Every pass of every context is cut into tiles of one CTA's work (256 or 64
// threads: a group of whole rows, or of whole columns); the items (runs of
// consecutive tiles) of all passes of all
// contexts form one queue in lockstep order (pass q of every context before
// pass q + 1 of any), which the CTAs of one launch take in order from a
// global counter.  An item of pass q of context i waits until pass q - 1 of
// context i is complete (a per-context counter), so the queue order makes
// every wait end: all earlier items are held by running CTAs.
struct BatchCtx {                 // 128-byte aligned by its tensor map
    CUtensorMap map;               // TMA view of psi as float32 [ny][2 nx], box 2 cpi x min(ny, 256)
    float2 *psi;
    Tables T;
    const float *V;
    float V_scale, g, sx, sy;
    int nx, ny;
    int rpi, row_tiles;            // rows per row tile (one CTA's worth), tiles per row pass
    int cpi, col_tiles;            // columns per column tile, tiles per column pass
    int row_items, col_items;      // items (runs of tpi consecutive tiles) per row / column pass
    // potential parameters for the per-pass phase and reduction arguments,
    // evaluated on the device as the host scheduler does (phase_at, red_at)
    double lat_V0x, lat_V0y, eta, U0, dc, kappa, N, dxdy, probe_omega, probe_delta, probe_phi;
    int cavity, pump_lattice, ctrl_target, nctrl;
    const double *ctrl_t, *ctrl_v; // the context's control points, copied into the batch workspace
};
struct BatchArgs {
    const BatchCtx *ctx;           // count descriptors
    const int *row_prefix;         // count + 1 prefix sums of row items
    const int *col_prefix;         // count + 1 prefix sums of column items
    unsigned int *head;            // [0] next queue index, [1] abort flag (cleared before the launch)
    unsigned int *epoch;           // per context: passes of this launch completed
    unsigned int *done;            // per context: items of the current pass completed
    int count, n, imag, cavity, spins;
    int tpi;                       // tiles per item (the last item of a pass may have fewer)
    int bt;                        // threads per CTA and per tile: 256 or 64
    double dt, t0;
    unsigned int total;            // items in the queue
};
cudaError_t launch_batch(const BatchArgs &b, cudaStream_t s, int grid);
int batch_resident_ctas(int bt);          // CTAs of a batch-kernel variant that fit the current device at once
int batch_supported(int nx, int ny, int bt);   // 1 if a context of this size can join a batch of bt-thread tiles
int batch_rows_per_item(int n, int bt);   // rows (of n points) in a row tile; columns of length n in a column tile
long long batch_queue_length(int n, int imag, int cavity, int row_items, int col_items);

// ---- Cooperative single-grid kernel (gpe_coop.cu): all n steps of one
// context whose grid fits on chip in one cooperative launch, one CTA per SM;
// the passes of the host scheduler's program (step_prologue / step_part /
// step_epilogue, minus the kinetic tables) separated by a grid barrier with
// bounded waits, the FP64 reductions finished by every CTA from the per-CTA
// partials in the same fixed order.
constexpr int COOP_MAX_CTRL = 256; // control points carried in the launch arguments
struct CoopArgs {
    float2 *psi;
    Tables T;
    const float *V;
    float V_scale, g, sx, sy;
    int nx, ny;
    int n, imag, spins;
    double dt, t0;
    // potential parameters for the per-pass phase and reduction arguments,
    // evaluated on the device as the host scheduler does (phase_at, red_at)
    double lat_V0x, lat_V0y, eta, U0, dc, kappa, N, dxdy, probe_omega, probe_delta, probe_phi;
    int cavity, pump_lattice, ctrl_target, nctrl;
    double ctrl_t[COOP_MAX_CTRL], ctrl_v[COOP_MAX_CTRL];
    // one checkpointed-adjoint segment, steps s0 .. s1 - 1: the segment's
    // states psi_{s0} .. psi_{s1}, P elements apart (written by
    // launch_coop_states from psi_{s0}, read by launch_coop_adj); lambda,
    // updated in place; dJ/dv of each half phase (gout[2 s], gout[2 s + 1]);
    // the base lattice depths L0x, L0y (Eq. 9).  t0 is the time of step 0.
    float2 *lam;
    float2 *st;
    size_t P;
    double *gout;
    float L0x, L0y;
    int s0, s1;
    // the reverse sweep by time reversal (launch_coop_rev): kinetic factors
    // of -dt for the steps back, nx and ny entries
    const float2 *kxb, *kyb;
    // launch_coop_adjrec: the previous segment's steps r0 .. r1 - 1,
    // recomputed from st2[0] = psi_{r0} into st2 (P elements apart) while
    // the adjoint passes of steps s1 - 1 .. s0 run on st
    float2 *st2;
    int r0, r1;
};
bool coop_ok(int nx, int ny);              // grid sizes the cooperative kernels are built for
cudaError_t launch_coop(const CoopArgs &a, cudaStream_t s);
// the adjoint passes of steps s1 - 1 down to s0 (ROW_ADJ, COL_ADJ of each) in
// one cooperative launch, for a context without a cavity
cudaError_t launch_coop_adj(const CoopArgs &a, cudaStream_t s);
// real-time steps s0 .. s1 - 1 of a context without a cavity, unfused, from
// st[0] = psi_{s0}, every state kept in st (one cooperative launch)
cudaError_t launch_coop_states(const CoopArgs &a, cudaStream_t s);
// the reverse sweep of GPE_ADJ_REVERSE over steps s1 - 1 down to s0 in one
// cooperative launch: psi holds psi_{s1} on entry and psi_{s0} on return
cudaError_t launch_coop_rev(const CoopArgs &a, cudaStream_t s);
// the same on the grids of launch_coop_adjrec, with the step back one step
// ahead beside the adjoint passes; psi_k in buffer (s1 - k) mod 3 of
// {psi, st, st2}
cudaError_t launch_coop_rev2(const CoopArgs &a, cudaStream_t s);
// grids launch_coop_adjrec is built for (512^2)
bool coop_adjrec_ok(int nx, int ny);
// the adjoint passes of one checkpointed segment (as launch_coop_adj) and
// the recomputation of the segment before it (as launch_coop_states, into
// st2) side by side in one cooperative launch
cudaError_t launch_coop_adjrec(const CoopArgs &a, cudaStream_t s);

// Launchers (gpe_kernels.cu).  Return cudaGetLastError() of the launch.
// tile_shift: the one-shot row pass takes 2^-tile_shift of its default rows
// per CTA (0, 1 or 2; see row_rows_per_cta)
cudaError_t launch_row(int mode, const PassArgs &a, cudaStream_t s, int tile_shift = 0);
cudaError_t launch_col(int mode, const PassArgs &a, const CUtensorMap &map, cudaStream_t s);
// the same for rows / columns of at most 256 points (lo) and more (hi)
cudaError_t launch_row_lo(int mode, const PassArgs &a, cudaStream_t s, int tile_shift);
cudaError_t launch_row_hi(int mode, const PassArgs &a, cudaStream_t s, int tile_shift);
cudaError_t launch_col_lo(int mode, const PassArgs &a, const CUtensorMap &map, cudaStream_t s);
cudaError_t launch_col_hi(int mode, const PassArgs &a, const CUtensorMap &map, cudaStream_t s);
cudaError_t launch_row_stream(const PassArgs &a, cudaStream_t s);
cudaError_t launch_col_stream(int mode, const PassArgs &a, const CUtensorMap &map, cudaStream_t s);
bool row_stream_ok(int nx, int ny);
bool row_group_ok(int nx, int ny);
cudaError_t launch_row_group(const PassArgs &a, cudaStream_t s);
bool col_stream_ok(int nx, int ny);
// pencil-pair column pass (gpe_pair.cu): COL_T, COL_T_R, COL_T_PR on 2-column
// tiles of 512..2048-point columns
bool col_pair_ok(int nx, int ny);
cudaError_t launch_col_pair(int mode, const PassArgs &a, const CUtensorMap &map, cudaStream_t s);
// pencil-pair row pass (gpe_pair.cu): ROW_PT on pairs of 2048..8192-point rows
bool row_pair_ok(int nx, int ny);
cudaError_t launch_row_pair(const PassArgs &a, cudaStream_t s);
cudaError_t launch_tables(const Tables &T, int nx, int ny, double Lx, double Ly, double m,
                          double wx, double wy, double lkx, double lky, double kc, cudaStream_t s);
cudaError_t launch_kinetic_tables(const Tables &T, int nx, int ny, double Lx, double Ly,
                                  double m, double dt, int imag, cudaStream_t s);
cudaError_t launch_timeout_probe(DevScalars *sc, int spins, cudaStream_t s);
cudaError_t launch_kbin(const float2 *f, const Tables &T, int nx, int ny, double Lx, double Ly, int axis, double k0,
                        int nmax, cudaStream_t s);
cudaError_t launch_kin_energy_mul(float2 *f, int nx, int ny, double Lx, double Ly, double m, cudaStream_t s);
cudaError_t launch_adj_overlap(const float2 *psi, const float2 *phi, const Tables &T, int nx, int ny, float L0x,
                               float L0y, cudaStream_t s);
cudaError_t launch_adj_terminal(float2 *lam, const float2 *psi, const float2 *phi, const PassArgs &a, float c_re,
                                float c_im, float dxdy, cudaStream_t s);
int col_tile_width(int nx, int ny);
int row_rows_per_cta(int nx, int ny, int tile_shift = 0);

}  // namespace gpe
