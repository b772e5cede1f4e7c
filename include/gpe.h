/*
 * gpe.h -- C ABI of the B300 (sm_103a) split-step Fourier propagator for the
 * 2D Gross-Pitaevskii equation (TorchGPE, arXiv 2404.14401).
 *
 * The problem (Eq. 1, Sec. 2), in oscillator units (Sec. 3.2, hbar = 1):
 *     i dpsi/dt = [ -lap/(2m) + V(x, y, t, psi) + g |psi|^2 ] psi
 * on a periodic Nx x Ny grid (Sec. 3.1: the FFT imposes periodicity),
 * x_j = -Lx/2 + j Lx/Nx, y_i = -Ly/2 + i Ly/Ny.
 *
 * One step of length dt is the symmetric (Strang) splitting of Sec. 3.1,
 * Eqs. (2)-(4), taken in the order  V/2 - T - V/2:
 *     psi <- exp(-i (V(t) + g|psi|^2) dt/2) psi
 *     psi <- F^-1 exp(-i k^2 dt / 2m) F psi
 *     psi <- exp(-i (V(t+dt) + g|psi|^2) dt/2) psi
 * where each half-step uses the density at its start and, with a cavity,
 * the field alpha recomputed from that density (Sec. 3.1 last paragraph,
 * Sec. 5.3).  GPE_IMAG replaces dt by -i dtau and renormalises psi to
 * unit norm after every step (Sec. 3.3).
 *
 * Data layout: psi is complex64 (interleaved float re, im), row-major
 * [Ny][Nx], x contiguous, in device memory owned by the caller.  All
 * device memory (psi, workspace, optional potential array) is borrowed:
 * the library never allocates or frees device memory.  Calls on one
 * context are not thread-safe; distinct contexts are independent.  Work
 * is enqueued on the caller's CUDA stream; only gpe_observables,
 * gpe_get_psi (to host) and gpe_sync wait for it.
 *
 * Every call returns a gpe_status; on error, gpe_last_error() gives a
 * message.  Device-side conditions (non-finite values, an ill-conditioned
 * cavity denominator, a bounded wait that ran out) are latched in a
 * device status word and reported by gpe_sync / gpe_observables.
 */
#ifndef GPE_H
#define GPE_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct gpe_ctx gpe_ctx;

typedef enum {
    GPE_OK = 0,
    GPE_EINVAL = 1,      /* bad argument (sizes, pointers, alignment, dt)        */
    GPE_ENOMEM = 2,      /* workspace smaller than gpe_workspace_size()          */
    GPE_ECUDA = 3,       /* a CUDA runtime/driver call failed; see gpe_last_error */
    GPE_ETIMEOUT = 4,    /* a bounded device wait (TMA barrier) ran out          */
    GPE_ENONFINITE = 5,  /* NaN/Inf found in a norm or cavity reduction          */
    GPE_EILLCOND = 6,    /* |Delta_c - U0 B + i kappa| below 1e-12 (Eq. 14)      */
    GPE_EBOUNDS = 7      /* debug bounds-check build only: an index check failed
                            (the access was skipped, nothing trapped)           */
} gpe_status;

typedef enum { GPE_REAL = 0, GPE_IMAG = 1 } gpe_mode;

/* Targets of the optional piecewise-linear control v(t). */
typedef enum {
    GPE_CTRL_NONE = 0,
    GPE_CTRL_LATTICE = 1,   /* lattice depths become lat_V0x v(t), lat_V0y v(t) (Eq. 9) */
    GPE_CTRL_ETA = 2        /* cavity pump eta(t) = v(t) (Sec. 5.3 ramp)               */
} gpe_ctrl_target;

/*
 * Potential descriptor (plain data).  V(x, y, t; alpha) is the sum of
 *   trap     (m/2)(wx^2 x^2 + wy^2 y^2)                        Sec. 5.1
 *   lattice  s(t) [lat_V0x cos^2(lat_kx x) + lat_V0y cos^2(lat_ky y)]  Eq. (9)
 *   array    V_scale * V[y][x]   (device float32 [Ny][Nx], borrowed; NULL = none)
 *   cavity   (Eqs. 10-13, cavity axis x, pump axis y, wavenumber kc)
 *            V_p = (eta^2/U0) cos^2(kc y)        (if pump_lattice and U0 != 0)
 *            V_c = U0 |alpha|^2 cos^2(kc x)
 *            V_i = 2 eta Re(alpha) cos(kc x) cos(kc y)
 *            alpha = N eta O / (Delta_c - U0 B + i kappa)      Eqs. (14)-(15)
 *            O = <cos(kc x) cos(kc y)>, B = <cos^2(kc x)> over |psi|^2/norm
 * where eta = sqrt(V0 U0).  ctrl_t/ctrl_v (host, nctrl points, increasing
 * times; copied) define v(t), clamped outside [ctrl_t[0], ctrl_t[n-1]].
 */
typedef struct {
    double wx, wy;
    double lat_V0x, lat_V0y, lat_kx, lat_ky;
    const float *V;
    double V_scale;
    int cavity;
    double eta, U0, dc, kappa, kc, N;
    int pump_lattice;
    int ctrl_target;
    int nctrl;
    const double *ctrl_t, *ctrl_v;
    /* on-axis cavity probe (Sec. 5.4, Bragg spectroscopy of the soft mode):
     * alpha' = alpha + probe_omega exp(i (probe_delta t + probe_phi))
     *                  / (Delta_c - U0 B + i kappa), used for V_c, V_i and the
     * observables; 0 = no probe */
    double probe_omega, probe_delta, probe_phi;
} gpe_potential;

/* Observables of the current state at the context's time t (host struct).
 *   norm   = int |psi|^2                 ekin = <-lap/2m> (spectral, per axis Parseval)
 *   epot   = int V |psi|^2 (alpha from this density)
 *   eint   = (g/2) int |psi|^4           energy = ekin + epot + eint
 *   mu     = ekin + epot + 2 eint        O, B, alpha as in gpe_potential
 *   status = latched device status (gpe_status), cleared by this call.     */
typedef struct {
    double norm, ekin, epot, eint, energy, mu, O, B, alpha_re, alpha_im, t;
    int status;
} gpe_obs;

/* Bytes of device workspace a context of this size needs (0 for bad sizes).
 * Nx, Ny must be powers of two in [8, 8192] (Sec. 4.1 uses N = 2^n). */
size_t gpe_workspace_size(int nx, int ny);

/* Create a context.  psi_dev: complex64 [ny][nx], 16-byte aligned, borrowed
 * for the context's life.  workspace_dev: >= gpe_workspace_size bytes,
 * 256-byte aligned, borrowed.  stream: a cudaStream_t (NULL = legacy default).
 * m > 0, Lx, Ly > 0.  The context starts at t = 0 with no potential.  The
 * device current at this call is the context's device: every later call that
 * launches work on the context must be made with that device current (the
 * call returns GPE_EINVAL otherwise, before launching anything).
 * Errors: GPE_EINVAL (sizes/pointers/alignment), GPE_ENOMEM (workspace too
 * small), GPE_ECUDA. *out is NULL on failure. */
gpe_status gpe_create(int nx, int ny, double Lx, double Ly, double m, double g,
                      void *psi_dev, void *workspace_dev, size_t ws_bytes,
                      void *stream, gpe_ctx **out);

/* Set the potential (copied, except the borrowed V array).  Enqueues the
 * FP64-computed coordinate tables on the stream.  Errors: GPE_EINVAL. */
gpe_status gpe_set_potential(gpe_ctx *ctx, const gpe_potential *p);

/* Enqueue n >= 0 split steps of length dt > 0 (Sec. 3.1; GPE_IMAG: Sec. 3.3),
 * advancing the context's time by n dt.  psi is in real space before and
 * after.  Asynchronous.  The same as gpe_step_many over this one context:
 * on a 512 x 512 grid (GPE_VARIANT_COOP, below) all n steps are one
 * cooperative launch; otherwise small grids with nothing time-dependent
 * replay their interior steps from a CUDA graph on a library lane, ordered
 * with the context's stream.  Errors: GPE_EINVAL, GPE_ECUDA. */
gpe_status gpe_step(gpe_ctx *ctx, int n, double dt, gpe_mode mode);

/* Enqueue n steps on each of `count` contexts in lockstep: step s of every
 * context is enqueued before step s+1 of any, so the grids share one pass
 * schedule -- e.g. a batch of trajectories of a parameter sweep (Sec. 5.3
 * phase diagram), possibly of different sizes.  With count > 1 the passes
 * run on streams owned by the library ("lanes", created on first use per
 * device: one per context, at most 16), so that passes of different contexts
 * overlap on the GPU; each context's steps are ordered after the work
 * already on its own stream, and its stream waits for them, so callers see
 * the same ordering as with gpe_step.  For batches of grids of at most 2^22
 * points on average with no time-dependent control or probe and no profiling, the
 * interior steps 1 .. n-2 are captured into CUDA graphs of up to 8 steps
 * (fewer for large batches), one per lane, and replayed (same results bit
 * for bit, one host launch per lane and graph; each lane replays on its own
 * stream, so a context whose earlier work on its stream -- an upload, say
 * -- finishes first also starts its steps first).  The instantiated graphs
 * are kept (those of the 8 most recently used batches per device) and
 * replayed again by later calls on the same contexts,
 * in the same order, with the same dt, mode and step count per graph, as
 * long as none of the contexts has changed its potential, pass variants or
 * wait limit since; gpe_destroy releases the graphs of its context.  Calls from several
 * host threads on one device take turns on the lanes.  Contexts must be on
 * the current device.  Same argument rules and errors as gpe_step; contexts
 * must be distinct.  Environment: GPE_SERIAL_MANY (no lanes: the contexts'
 * own streams, one pass at a time) and GPE_NO_GRAPH (no graph replay).
 * Read when a context is created, GPE_NO_PAIR_ROWS, GPE_NO_PAIR_COLS,
 * GPE_NO_GROUP_ROWS, GPE_NO_STREAM_PASSES and GPE_NO_COOP clear the
 * corresponding default pass variants (below). */
gpe_status gpe_step_many(gpe_ctx *const *ctxs, int count, int n, double dt, gpe_mode mode);

/* ---- Persistent batch: n lockstep steps of many contexts in one launch ----
 * The same steps as gpe_step_many (Sec. 3.1, Eqs. 3-4; imaginary time Sec.
 * 3.3; cavity Sec. 5.3) -- e.g. the instances of a phase-diagram sweep (Sec.
 * 5.3, Fig. 5(b)), of uneven sizes -- run as ONE kernel launch per call
 * instead of one launch per pass and context.  Every pass of every context is
 * cut into items of 256 threads' work (whole rows; TMA-loaded tiles of whole
 * columns), all items form one queue in lockstep order, and the CTAs of one
 * persistent launch take them in order; an item waits (bounded) until the
 * previous pass of its context is complete, whose last item sums the pass's
 * FP64 partial sums in a fixed order and updates 1/sqrt(norm) and alpha.  The
 * results equal those of gpe_step_many within the propagator's tolerances
 * (not bit for bit: the items group the reductions differently).
 *
 * gpe_batch_workspace_size: device bytes a batch of these contexts needs
 * (descriptors, counters, copies of the control points); 0 for bad input.
 * gpe_batch_create: binds `count` distinct contexts, in order, to ws (>= that
 * size, 256-byte aligned, borrowed for the batch's life; the caller must not
 * write it meanwhile) and writes the descriptors there; waits for the first
 * context's stream.  Every context must be on the current device, with nx, ny
 * powers of two in 64..2048 (and each axis at least 256 / (other axis / 16)
 * points: a row or column item is never cut).  The contexts must outlive the
 * batch; a context's later gpe_set_potential / gpe_set_pass_variants /
 * gpe_set_wait_limit is picked up by the next gpe_batch_step.
 * gpe_batch_step: enqueues n >= 0 steps of dt in `mode` for every context on
 * the first context's stream (ordered after the work on every context's
 * stream, which all wait for the launch), advancing each context's time by
 * n dt.  Every context must have a cavity or none; with a control table or a
 * probe, all must be at the same time.  A bounded wait that runs out ends the
 * launch and latches GPE_ETIMEOUT in that context's status (gpe_sync).  The
 * launch is counted in the first context's gpe_launch_count.
 * Errors: GPE_EINVAL, GPE_ENOMEM (workspace too small), GPE_ECUDA. */
typedef struct gpe_batch gpe_batch;
size_t gpe_batch_workspace_size(gpe_ctx *const *ctxs, int count);
gpe_status gpe_batch_create(gpe_ctx *const *ctxs, int count, void *ws, size_t ws_bytes, gpe_batch **out);
gpe_status gpe_batch_step(gpe_batch *batch, int n, double dt, gpe_mode mode);
void gpe_batch_destroy(gpe_batch *batch);

/* Compute the observables of psi at the current time; waits for the stream.
 * Returns the latched device status if it is not GPE_OK (out is filled). */
gpe_status gpe_observables(gpe_ctx *ctx, gpe_obs *out);

/* Copy psi from src (complex64 [ny][nx]) -- host memory if is_dev == 0,
 * device memory otherwise.  Stream-ordered (host source must stay valid
 * until the stream reaches the copy; pinned memory makes it asynchronous). */
gpe_status gpe_set_psi(gpe_ctx *ctx, const void *src, int is_dev);

/* Copy psi to dst; a host destination waits for the stream. */
gpe_status gpe_get_psi(gpe_ctx *ctx, void *dst, int is_dev);

/* Set / read the context's time t (used by V(t) and the controls). */
gpe_status gpe_set_time(gpe_ctx *ctx, double t);
double gpe_get_time(const gpe_ctx *ctx);

/* In-place 2D DFT of psi with the propagator's own FFT passes (diagnostic):
 * sign = -1 forward (unnormalised), +1 inverse (divides by nx ny).  The
 * same row/column kernels as gpe_step with the phases switched off. */
gpe_status gpe_fft2(gpe_ctx *ctx, int sign);

/* Wait for the stream; return and clear the latched device status (and the
 * counters the reducing passes use to find their last CTA). */
gpe_status gpe_sync(gpe_ctx *ctx);

/* Bound on every device wait of this context's kernels: the number of polls
 * of a TMA barrier before the kernel gives up, latches GPE_ETIMEOUT and goes
 * on without storing its results (default 2^24, far longer than any copy
 * takes).  A CTA whose wait ran out still lets the copies it issued land (a
 * fixed number of further polls) and still adds zero partial sums to the
 * pass's reductions, so the context stays usable: after gpe_sync has
 * returned and cleared the status, later calls compute correctly from the
 * state psi then holds (rows or tiles of the failed pass keep their old
 * values).  0 makes every wait give up at once, to test that path.
 * Errors: GPE_EINVAL for a null context or a negative limit. */
gpe_status gpe_set_wait_limit(gpe_ctx *ctx, int spins);
int gpe_get_wait_limit(const gpe_ctx *ctx);              /* -1 for a null context */

/* Run one kernel whose bounded barrier wait is given nothing to wait for,
 * so it must run out after about `spins` polls and latch GPE_ETIMEOUT
 * (failure-path check of the timeout mechanism; touches no psi data).  */
gpe_status gpe_debug_timeout_probe(gpe_ctx *ctx, int spins);

/* Diagnostics: with enable = 1 every pass this context launches is bracketed
 * by CUDA events on its stream; gpe_profile_read waits for the stream and
 * returns the summed device milliseconds and launch counts of row passes and
 * column passes since profiling was enabled (then resets them).  Events cost
 * a few microseconds per pass; leave profiling off for throughput runs. */
gpe_status gpe_profile(gpe_ctx *ctx, int enable);
gpe_status gpe_profile_read(gpe_ctx *ctx, double *row_ms, int *row_launches, double *col_ms,
                            int *col_launches);

/* Per-kind variant of gpe_profile_read: milliseconds and launch count of the
 * timed launches of one kind since the last read of that kind (then reset).
 * Kinds: GPE_PASS_ROW, GPE_PASS_COL (forward passes), GPE_PASS_OTHER (tables,
 * pointwise kernels), GPE_PASS_ADJ_ROW, GPE_PASS_ADJ_COL (adjoint passes).
 * Errors: GPE_EINVAL for an unknown kind, GPE_ECUDA. */
enum { GPE_PASS_ROW = 0, GPE_PASS_COL = 1, GPE_PASS_OTHER = 2, GPE_PASS_ADJ_ROW = 3, GPE_PASS_ADJ_COL = 4,
       GPE_PASS_KINDS = 5 };
gpe_status gpe_profile_read_kind(gpe_ctx *ctx, int kind, double *ms, int *launches);

/* Number of kernels this context has launched since it was created. */
long long gpe_launch_count(const gpe_ctx *ctx);

/* Allocation-free variant for callers that may not allocate device memory
 * (the paper has no counterpart; this is a library convenience).  Some
 * callers only hold pointers handed to them: a plug-in whose host
 * application owns every device allocation through its own pool, or a hook
 * that must not call cudaMalloc/cudaFree because those can synchronise the
 * whole device.  They cannot supply the workspace gpe_create borrows, so
 * this call runs the row-pass density reduction with its scratch in a fixed
 * array inside the library (about 200 KB, held on every GPU that loads the
 * library until the process exits) and returns
 *     out[0] = int |psi|^2 dx dy,
 *     out[1] = O = <cos(kc x) cos(kc y)>,  out[2] = B = <cos^2(kc x)>
 * (averages over |psi|^2 / norm, the overlaps of Eqs. 14-15) for psi
 * complex64 [ny][nx] on the device (16-byte aligned), box Lx x Ly.  It waits
 * for `stream` and writes out on the host.  nx, ny: powers of two from 8 to
 * GPE_STATIC_MAX_N; larger grids return GPE_ENOMEM, malformed ones
 * GPE_EINVAL.  The first call on a device looks up the array's device
 * address (make that first call before any stream capture that includes
 * it).  Every call uses the same array: calls that overlap on the GPU (other
 * streams or threads) race and give wrong results.  Nothing is allocated. */
#define GPE_STATIC_MAX_N 2048
gpe_status gpe_overlaps_static(const void *psi_dev, int nx, int ny, double Lx, double Ly, double kc,
                               void *stream, double *out);

/* Momentum-state populations (Kapitza-Dirac readout, Sec. 5.2): the
 * fractions of sum_k |F psi|^2 whose momentum along `axis` (0: x, 1: y) lies
 * within k0 of 2 n k0, summed over the other axis, for n = -nmax..nmax
 * (0 <= nmax <= 3); a momentum exactly between two windows counts for the
 * smaller |n|.  pop_out: 2 nmax + 1 doubles, n = -nmax first.  The transform
 * runs on a copy of psi in scratch_dev (>= nx*ny*8 bytes, 256-byte aligned,
 * borrowed); psi is not changed.  FP64 accumulation.  Synchronises the
 * stream.  Errors: GPE_EINVAL, GPE_ENONFINITE (empty or non-finite state),
 * GPE_ECUDA. */
gpe_status gpe_momentum_populations(gpe_ctx *ctx, int axis, double k0, int nmax, void *scratch_dev,
                                    size_t scratch_bytes, double *pop_out);

/* ---- Pass variants and the autotuner ----------------------------------
 * Each pass has more than one kernel design for some grids: the row pass
 * of 512..2048-point rows has a grouped persistent variant (one CTA per SM,
 * tables in shared memory, TMA double buffering), rows and columns of 4096
 * points a streaming persistent variant; every grid has the one-shot
 * variant (a CTA per group of rows or per TMA tile of columns), and the
 * row and column passes of 512..8192 points a pencil-pair form (bits 5 and
 * 6).  A context starts with the streaming row pass on where it applies,
 * the grouped row pass on for 2048-point rows only, the half row tile
 * (below) for 512- and 1024-point rows, the pencil-pair row pass for rows
 * of 512 points and more and the pencil-pair column pass for columns of
 * 1024 points and more (the streaming column pass off): with those the
 * passes of other grids overlapped best under gpe_step_many.  The bits
 * select them: */
enum { GPE_VARIANT_GROUP_ROWS = 1, GPE_VARIANT_STREAM_ROWS = 2, GPE_VARIANT_STREAM_COLS = 4 };
/* Bits 3-4 (value << GPE_VARIANT_ROW_TILE_SHIFT, value 0..2): on rows of
 * 256 points and more the one-shot row passes of the context's steps,
 * observables and adjoint run 2^-value of their default rows per CTA (256
 * threads' worth, at least one warp), so that a small grid spreads over more
 * SMs; shorter rows ignore it. */
enum { GPE_VARIANT_ROW_TILE_SHIFT = 3 };
/* Bit 5: the column passes (T_y [+ closing phase] [+ reductions]) of
 * 512..8192-point columns as pencil pairs: both columns of a 2-column tile
 * in one packed f32x2 transform, each table entry read once for both (equal
 * to the one-pencil passes to FP32 rounding).  On by default for columns
 * of 1024 points and more, where it measured faster. */
enum { GPE_VARIANT_PAIR_COLS = 32 };
/* Bit 6: the row pass (potential phase + T_x) of 512..8192-point rows as
 * pencil pairs of consecutive rows, one CTA per pair (equal to the
 * one-pencil passes to FP32 rounding).  On by default for rows of 512
 * points and more, where it measured faster; it takes precedence over bits
 * 0 and 1. */
enum { GPE_VARIANT_PAIR_ROWS = 64 };
/* Bit 7: gpe_step (or gpe_step_many of one context) on a grid of 512 or
 * 1024 points per axis runs all n steps as ONE cooperative launch of a
 * persistent kernel, one CTA per SM: the same passes (pencil-pair row and
 * column transforms, the pointwise prologue and epilogue passes) separated
 * by a grid barrier, the phase and reduction arguments evaluated on the
 * device, psi kept in L2 between passes.  Equal to the per-pass path to
 * FP32 rounding.  On by default for 512 x 512 grids, where it measured
 * faster than the per-pass path (per step on a B300: real time 10.9 against
 * 13.3 us, the cavity ramp 17.8 against 24.6 us, imaginary time 16.2 against
 * 23.8 us); at 1024 points it was slower in real time and is off unless set.  It takes
 * one host launch per call instead of two or three per step.  It does not apply while the context
 * profiles its passes (gpe_profile), when it has more than 256 control
 * points, for more than 2^22 steps in one call, or while its stream is being
 * captured; a device that refuses the cooperative launch makes the context
 * fall back to the per-pass path (gpe_last_error says so).  The barrier's
 * waits are bounded by the wait limit (gpe_set_wait_limit): one that runs
 * out latches GPE_ETIMEOUT and ends the launch.  gpe_tune leaves this bit
 * as it was. */
enum { GPE_VARIANT_COOP = 128 };
int gpe_get_pass_variants(const gpe_ctx *ctx);                /* -1 for a null context */
/* GPE_EINVAL for bits other than those above or a row-tile value above 2 */
gpe_status gpe_set_pass_variants(gpe_ctx *ctx, int variants);
/* Autotuner: times every applicable variant of the interior row pass
 * (potential phase + T_x; the one-shot pass at row-tile values 0 and 1, the
 * half tile kept unless at least 3% slower; a persistent variant replaces
 * the one-shot pass only when at least 3% faster) and column pass (T_y)
 * of a step of dt in `mode` on a copy of psi in scratch_dev (>= nx*ny*8
 * bytes, 256-byte aligned, borrowed; psi itself is not changed), `reps`
 * launches each after one warm-up, with CUDA events on the context's
 * stream, and selects the fastest row and column variants for this context.
 * variants_out receives the bits; times_out (5 doubles or NULL) the mean
 * milliseconds of the row pass one-shot (the faster of the one-pencil pass
 * at its kept tile and the pencil-pair pass; bit 6 is set when it is the
 * pair) / grouped / streaming and the column pass one-shot (the faster of
 * the one-pencil and pencil-pair forms; bit 5 is set when it is the pair) /
 * streaming, NaN where a variant
 * does not apply.  Synchronises the stream.  Errors:
 * GPE_EINVAL, GPE_ECUDA. */
gpe_status gpe_tune(gpe_ctx *ctx, double dt, gpe_mode mode, void *scratch_dev, size_t scratch_bytes, int reps,
                    int *variants_out, double *times_out);

/* ---- Adjoint of the real-time split step (lattice-depth control) ------
 * For the control of the lattice depth v(t) (ctrl_target GPE_CTRL_LATTICE:
 * V = trap + v(t) (lat_V0x cos^2(kx x) + lat_V0y cos^2(ky y)), Sec. 5.2 Eq. 9)
 * and the objective J = E(psi_T) + |<phi|psi_T>|^2 (E: the GP energy of the
 * state after nsteps real-time steps of dt, <phi|psi> = sum conj(phi) psi
 * dx dy), gpe_adjoint_lattice returns J and dJ/dv_i for every control value
 * v_i of the context's control table.  It is the discrete adjoint of the
 * V/2 - T - V/2 steps gpe_step takes: the steps are run forward keeping a
 * checkpoint every S = ceil(sqrt(nsteps)) steps, then swept in reverse one
 * segment at a time (each segment's states recomputed from its checkpoint),
 * with per point lambda <- mu + 2 h g Im(conj(mu) psi) psi, mu = exp(i theta)
 * lambda for each half phase and the conjugate kinetic propagator in between,
 * starting from lambda_T = dx dy (H psi_T + <phi|psi_T> phi).  On grids the
 * cooperative kernels are built for (512 and 1024 points per axis; by default
 * those whose context has GPE_VARIANT_COOP, i.e. 512^2), unless the context
 * profiles its passes, each segment takes cooperative launches: the
 * forward sweep and the recomputation run the steps unfused with every state
 * kept, so the recomputed states are the forward sweep's bit for bit, and
 * the segment's adjoint passes follow in one launch.  Elsewhere the passes
 * are launched one by one.  On 512^2 one segment's adjoint passes run beside
 * the previous segment's recomputation in one launch.  (512^2, 4000 steps:
 * 0.157 s against 0.350 s.)
 * GPE_ADJ_REVERSE on those grids: the forward sweep in place in one launch
 * (the same unfused steps, so J is the checkpointed call's bit for bit) and
 * the whole reverse sweep in one more, on 512^2 with the step back one
 * step ahead beside the adjoint passes (0.152 s against 0.305 s).
 *
 * phi_dev: target state, complex64 [ny][nx] on the device (borrowed, 16-byte
 * aligned).  adj_ws: device scratch of at least
 * gpe_adjoint_workspace_size(nx, ny, nsteps) bytes (256-byte aligned,
 * borrowed): (ceil(nsteps/S) + S + 3) copies of psi (S + 1 more on 512^2
 * grids, where one segment is recomputed while the adjoint passes of the
 * next run) plus 2 nsteps + 1 doubles.  grad_out: host array of nctrl
 * doubles.  The call synchronises the
 * context's stream.  On return psi is the final state and the context's time
 * has advanced by nsteps dt, as after gpe_step.  Errors: GPE_EINVAL (no
 * lattice control table, a cavity, bad sizes or pointers), GPE_ENOMEM
 * (workspace too small), GPE_ECUDA, device statuses as gpe_step. */
size_t gpe_adjoint_workspace_size(int nx, int ny, int nsteps);
gpe_status gpe_adjoint_lattice(gpe_ctx *ctx, int nsteps, double dt, const void *phi_dev, void *adj_ws,
                               size_t adj_ws_bytes, double *J_out, double *grad_out);

/* The same adjoint with a choice of how the reverse sweep gets the forward
 * states (GPE_ADJ_CHECKPOINT: the calls above).  GPE_ADJ_REVERSE keeps no
 * checkpoints: since each real-time half phase keeps |psi| and the kinetic
 * step is unitary, psi_s = U(dt)^-1 psi_{s+1} is one step of -dt from
 * t_{s+1} (conjugate phases on the same densities, T(-dt)), taken before the
 * adjoint passes of step s.  Exact in exact arithmetic; in FP32 the
 * recovered states carry the rounding of the steps taken back, so the
 * gradient differs from the checkpointed one by about that much (the
 * reverse sweep costs the same passes as the recomputation it replaces).
 * Workspace (gpe_adjoint_workspace_size_ex): 2 copies of psi (psi_T and
 * lambda; 2 more on 512^2 grids, where the step back runs one step ahead of
 * the adjoint passes through three state buffers), the kinetic factors of
 * -dt and 2 nsteps + 1 doubles, independent of the number of steps apart
 * from those doubles; elsewhere the step back overwrites the context's psi
 * after the row adjoint pass of that step has read it.  Returns 0 /
 * GPE_EINVAL for an unknown
 * variant; otherwise as gpe_adjoint_workspace_size / gpe_adjoint_lattice. */
typedef enum { GPE_ADJ_CHECKPOINT = 0, GPE_ADJ_REVERSE = 1 } gpe_adjoint_variant;
size_t gpe_adjoint_workspace_size_ex(int nx, int ny, int nsteps, int variant);
gpe_status gpe_adjoint_lattice_ex(gpe_ctx *ctx, int nsteps, double dt, int variant, const void *phi_dev,
                                  void *adj_ws, size_t adj_ws_bytes, double *J_out, double *grad_out);

/* Release the context (host memory only; borrowed memory is untouched).
 * It does not wait for work already enqueued on the context's stream: keep
 * psi, the workspace and any borrowed V array valid until that work is done
 * (gpe_sync, or a synchronisation of the stream). */
void gpe_destroy(gpe_ctx *ctx);

/* Message for the last error on ctx (never NULL). */
const char *gpe_last_error(const gpe_ctx *ctx);

/* Name of a status code. */
const char *gpe_status_string(gpe_status s);

#ifdef __cplusplus
}
#endif
#endif /* GPE_H */
