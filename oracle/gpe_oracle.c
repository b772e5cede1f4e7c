/*
 * gpe_oracle.c -- plain FP64 CPU oracle for the symmetric split-step
 * Fourier propagator of the 2D Gross-Pitaevskii equation.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links,
 * includes or calls this file; only the tests, the smoke check and the
 * CPU-baseline leg of the benchmark do.  It shares no code with the CUDA
 * path (no headers, tables or helpers): it has its own radix-2 FFT, its
 * own grid and potential evaluation and its own reductions, all in double
 * precision, written for readability rather than speed.
 *
 * What it follows (paper: "TorchGPE", arXiv 2404.14401):
 *   Eq. (1), Sec. 2       i dpsi/dt = [-(1/2m) lap + V(r,t,psi) + g|psi|^2] psi
 *                         (hbar = 1, oscillator units of Sec. 3.2)
 *   Eqs. (2)-(4), Sec. 3.1  one step = product of exponentials of the
 *                         kinetic part (diagonal in k-space) and of the
 *                         potential part (diagonal in real space); FFTs
 *                         move between the two and impose periodic
 *                         boundaries; the potential is re-evaluated from
 *                         the most recent wave function.
 *   Sec. 3.3              imaginary time: dt -> -i dtau, then normalise the
 *                         wave function after every iteration.
 *   Eqs. (10)-(15), Sec. 5.3  cavity potential V_t+V_p+V_c+V_i with the
 *                         field alpha and the shifted detuning recomputed
 *                         from the current density at every step.
 *   Eq. (9), Sec. 5.2     time-dependent lattice depth V0(t) cos^2(k y).
 *
 * Readings where the paper is silent or ambiguous:
 *   - default operator order is V/2 - T - V/2; the printed order
 *     T/2 - V - T/2 (Eq. 4) is available with paper_order = 1;
 *   - the density used by a half-step phase is the one at the start of
 *     that half-step (frozen during the half-step);
 *   - the first half-step uses V(t_n), the second V(t_n + dt); the
 *     T/2-V-T/2 order uses V(t_n + dt/2);
 *   - alpha is recomputed before every potential phase from the density
 *     at that moment, with the overlaps divided by the norm (so N is the
 *     atom number multiplying eta, default 1), eta = sqrt(V0 U0) and the
 *     pump depth V0 = eta^2 / U0;
 *   - grid x_j = -L/2 + j L/N (periodic box, right end excluded), k-grid
 *     in FFT order, forward FFT unnormalised, inverse FFT carries 1/N.
 *
 * Build: gcc -O2 -fopenmp -shared -fPIC gpe_oracle.c -o liboracle.so -lm
 * OpenMP only splits independent rows/columns; every reduction is a plain
 * serial loop in index order, so results do not depend on the thread count.
 */
#include <complex.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef double complex cplx;

/* Problem description.  Field order must match oracle/__init__.py. */
typedef struct {
    int nx, ny;          /* grid points (powers of two)                     */
    double Lx, Ly;       /* box lengths; x in [-Lx/2, Lx/2)                   */
    double m, g;         /* particle mass, contact coupling (Eq. 1)           */
    /* harmonic trap V_t = (m/2)(wx^2 x^2 + wy^2 y^2)  (Sec. 5.1)             */
    double wx, wy;
    /* optical lattice V0x cos^2(kx x) + V0y cos^2(ky y)  (Eq. 9)             */
    double lat_V0x, lat_V0y, lat_kx, lat_ky;
    /* optional static potential array [ny][nx] times V_scale                 */
    const double *Varr;
    double V_scale;
    /* cavity (Eqs. 10-15): on/off, eta = sqrt(V0 U0), U0, Delta_c, kappa,
     * mode wavenumber kc (cavity along x, pump along y), atom number N,
     * include the pump lattice V_p = (eta^2/U0) cos^2(kc y)                  */
    int cavity;
    double eta, U0, dc, kappa, kc, Nat;
    int pump_lattice;
    /* piecewise-linear control v(t): target 0 none, 1 lattice depth scale
     * (V0x v(t), V0y v(t)), 2 eta(t) = v(t)                                   */
    int ctrl_target, nctrl;
    const double *ctrl_t, *ctrl_v;
    /* 0: V/2 - T - V/2 (default), 1: T/2 - V - T/2 as printed in Eq. (4)      */
    int paper_order;
    /* on-axis cavity probe (Sec. 5.4): alpha' = alpha + delta_alpha(t) with
     * delta_alpha = Omega_c exp(i (Delta_p t + phi)) / (Delta_c - U0 B + i kappa) */
    double probe_omega, probe_delta, probe_phi;
} orc_params;

enum { CTRL_NONE = 0, CTRL_LATTICE = 1, CTRL_ETA = 2 };

/* ------------------------------------------------------------------ */
/* FFT: iterative radix-2 Cooley-Tukey, decimation in time.            */
/* sign = -1: forward sum_j a_j e^{-2 pi i jk/n}; sign = +1: backward. */
/* No normalisation here.                                              */
/* ------------------------------------------------------------------ */
static int is_pow2(int n) { return n >= 1 && (n & (n - 1)) == 0; }

static void fft1d_inplace(cplx *a, int n, const cplx *w)
{
    /* w[k] = exp(sign * 2 pi i k / n), k < n/2, each computed directly */
    for (int i = 1, j = 0; i < n; i++) {             /* bit reversal */
        int bit = n >> 1;
        for (; j & bit; bit >>= 1) j ^= bit;
        j ^= bit;
        if (i < j) { cplx t = a[i]; a[i] = a[j]; a[j] = t; }
    }
    for (int len = 2; len <= n; len <<= 1) {
        int half = len / 2, step = n / len;
        for (int i = 0; i < n; i += len)
            for (int k = 0; k < half; k++) {
                cplx u = a[i + k];
                cplx v = a[i + k + half] * w[k * step];
                a[i + k] = u + v;
                a[i + k + half] = u - v;
            }
    }
}

static cplx *twiddles(int n, int sign)
{
    cplx *w = malloc(sizeof(cplx) * (size_t)(n / 2 > 0 ? n / 2 : 1));
    for (int k = 0; k < n / 2; k++) {
        double th = 2.0 * M_PI * (double)k / (double)n;
        w[k] = cos(th) + I * (sign * sin(th));
    }
    return w;
}

int orc_fft1(double *data, int n, int sign)
{
    if (!is_pow2(n) || (sign != 1 && sign != -1)) return -1;
    cplx *w = twiddles(n, sign);
    fft1d_inplace((cplx *)data, n, w);
    free(w);
    return 0;
}

/* 2D transform of psi[ny][nx]: rows (x) then columns (y).  The inverse
 * (sign = +1) divides by nx*ny (forward unnormalised, numpy style).    */
int orc_fft2(double *data, int nx, int ny, int sign)
{
    if (!is_pow2(nx) || !is_pow2(ny) || (sign != 1 && sign != -1)) return -1;
    cplx *psi = (cplx *)data;
    cplx *wx = twiddles(nx, sign), *wy = twiddles(ny, sign);
    #pragma omp parallel for schedule(static)
    for (int y = 0; y < ny; y++) fft1d_inplace(psi + (size_t)y * nx, nx, wx);
    #pragma omp parallel
    {
        cplx *col = malloc(sizeof(cplx) * (size_t)ny);
        #pragma omp for schedule(static)
        for (int x = 0; x < nx; x++) {
            for (int y = 0; y < ny; y++) col[y] = psi[(size_t)y * nx + x];
            fft1d_inplace(col, ny, wy);
            for (int y = 0; y < ny; y++) psi[(size_t)y * nx + x] = col[y];
        }
        free(col);
    }
    if (sign == 1) {
        double s = 1.0 / ((double)nx * (double)ny);
        size_t n = (size_t)nx * ny;
        #pragma omp parallel for schedule(static)
        for (size_t i = 0; i < n; i++) psi[i] *= s;
    }
    free(wx); free(wy);
    return 0;
}

/* ------------------------------------------------------------------ */
/* Grid                                                                 */
/* ------------------------------------------------------------------ */
static double xcoord(int j, int n, double L) { return -0.5 * L + (double)j * L / (double)n; }
static double kcoord(int j, int n, double L)
{
    int s = (j < n / 2) ? j : j - n;
    return 2.0 * M_PI * (double)s / L;
}

/* ------------------------------------------------------------------ */
/* Time-dependent scalar controls (piecewise-linear, clamped ends)      */
/* ------------------------------------------------------------------ */
static double ctrl_eval(const orc_params *p, double t)
{
    int n = p->nctrl;
    if (n <= 0) return 1.0;
    if (t <= p->ctrl_t[0]) return p->ctrl_v[0];
    if (t >= p->ctrl_t[n - 1]) return p->ctrl_v[n - 1];
    int i = 0;
    while (i + 1 < n && p->ctrl_t[i + 1] < t) i++;
    double t0 = p->ctrl_t[i], t1 = p->ctrl_t[i + 1];
    double f = (t - t0) / (t1 - t0);
    return p->ctrl_v[i] + f * (p->ctrl_v[i + 1] - p->ctrl_v[i]);
}

static double lattice_scale(const orc_params *p, double t)
{ return p->ctrl_target == CTRL_LATTICE ? ctrl_eval(p, t) : 1.0; }

static double eta_at(const orc_params *p, double t)
{ return p->ctrl_target == CTRL_ETA ? ctrl_eval(p, t) : p->eta; }

/* ------------------------------------------------------------------ */
/* Cavity field, Eqs. (14)-(15).                                        */
/* O = int cos(kc x) cos(kc y) |psi|^2 / int |psi|^2                     */
/* B = int cos^2(kc x) |psi|^2 / int |psi|^2                             */
/* alpha = N eta O / (Delta_c - U0 B + i kappa)                          */
/* ------------------------------------------------------------------ */
typedef struct { double norm, O, B; } overlaps;

static overlaps density_overlaps(const orc_params *p, const cplx *psi)
{
    overlaps r = {0.0, 0.0, 0.0};
    double dx = p->Lx / p->nx, dy = p->Ly / p->ny;
    for (int y = 0; y < p->ny; y++) {
        double cy = cos(p->kc * xcoord(y, p->ny, p->Ly));
        for (int x = 0; x < p->nx; x++) {
            double cx = cos(p->kc * xcoord(x, p->nx, p->Lx));
            cplx v = psi[(size_t)y * p->nx + x];
            double n = creal(v) * creal(v) + cimag(v) * cimag(v);
            r.norm += n * dx * dy;
            r.O += cx * cy * n * dx * dy;
            r.B += cx * cx * n * dx * dy;
        }
    }
    r.O /= r.norm;
    r.B /= r.norm;
    return r;
}

static cplx cavity_alpha(const orc_params *p, const cplx *psi, double t)
{
    if (!p->cavity) return 0.0;
    overlaps ov = density_overlaps(p, psi);
    double eta = eta_at(p, t);
    cplx den = (p->dc - p->U0 * ov.B) + I * p->kappa;
    cplx probe = p->probe_omega * cexp(I * (p->probe_delta * t + p->probe_phi));
    return (p->Nat * eta * ov.O + probe) / den;
}

/* V(x, y, t) for a given cavity field alpha, Eqs. (9)-(13) plus trap.   */
static double potential_at(const orc_params *p, int xi, int yi, double t, cplx alpha)
{
    double x = xcoord(xi, p->nx, p->Lx), y = xcoord(yi, p->ny, p->Ly);
    double V = 0.5 * p->m * (p->wx * p->wx * x * x + p->wy * p->wy * y * y);
    double ls = lattice_scale(p, t);
    double cxl = cos(p->lat_kx * x), cyl = cos(p->lat_ky * y);
    V += ls * (p->lat_V0x * cxl * cxl + p->lat_V0y * cyl * cyl);
    if (p->Varr) V += p->V_scale * p->Varr[(size_t)yi * p->nx + xi];
    if (p->cavity) {
        double eta = eta_at(p, t);
        double cx = cos(p->kc * x), cy = cos(p->kc * y);
        if (p->pump_lattice && p->U0 != 0.0)
            V += (eta * eta / p->U0) * cy * cy;                    /* V_p */
        V += p->U0 * creal(alpha * conj(alpha)) * cx * cx;         /* V_c */
        V += 2.0 * eta * creal(alpha) * cx * cy;                   /* V_i */
    }
    return V;
}

int orc_potential(const orc_params *p, double t, double alpha_re, double alpha_im, double *V)
{
    cplx a = alpha_re + I * alpha_im;
    for (int y = 0; y < p->ny; y++)
        for (int x = 0; x < p->nx; x++)
            V[(size_t)y * p->nx + x] = potential_at(p, x, y, t, a);
    return 0;
}

/* ------------------------------------------------------------------ */
/* Sub-steps                                                            */
/* ------------------------------------------------------------------ */
/* Potential phase over a time h at time t (Sec. 3.1): theta = (V + g|psi|^2) h,
 * psi <- exp(-i theta) psi in real time, exp(-theta) psi in imaginary time.
 * alpha (cavity) comes from the density before the phase is applied.   */
static cplx potential_phase(const orc_params *p, cplx *psi, double t, double h, int imag)
{
    cplx alpha = cavity_alpha(p, psi, t);
    #pragma omp parallel for schedule(static)
    for (int y = 0; y < p->ny; y++)
        for (int x = 0; x < p->nx; x++) {
            size_t i = (size_t)y * p->nx + x;
            double n = creal(psi[i]) * creal(psi[i]) + cimag(psi[i]) * cimag(psi[i]);
            double theta = (potential_at(p, x, y, t, alpha) + p->g * n) * h;
            psi[i] *= imag ? exp(-theta) : cexp(-I * theta);
        }
    return alpha;
}

/* Kinetic propagator over a time h: F^-1 [ exp(-i k^2 h / 2m) F psi ]
 * (real time) or with exp(-k^2 h / 2m) (imaginary time), Eqs. (3)-(4). */
static void kinetic(const orc_params *p, cplx *psi, double h, int imag)
{
    orc_fft2((double *)psi, p->nx, p->ny, -1);
    #pragma omp parallel for schedule(static)
    for (int y = 0; y < p->ny; y++) {
        double ky = kcoord(y, p->ny, p->Ly);
        for (int x = 0; x < p->nx; x++) {
            double kx = kcoord(x, p->nx, p->Lx);
            double e = (kx * kx + ky * ky) / (2.0 * p->m) * h;
            psi[(size_t)y * p->nx + x] *= imag ? exp(-e) : cexp(-I * e);
        }
    }
    orc_fft2((double *)psi, p->nx, p->ny, +1);
}

static void normalise(const orc_params *p, cplx *psi)
{
    double dx = p->Lx / p->nx, dy = p->Ly / p->ny, s = 0.0;
    size_t n = (size_t)p->nx * p->ny;
    for (size_t i = 0; i < n; i++)
        s += (creal(psi[i]) * creal(psi[i]) + cimag(psi[i]) * cimag(psi[i])) * dx * dy;
    double c = 1.0 / sqrt(s);
    for (size_t i = 0; i < n; i++) psi[i] *= c;
}

/* Evolve psi (interleaved complex128 [ny][nx]) by nsteps steps of dt,
 * starting at time t0.  imag = 1 selects imaginary time (Sec. 3.3).
 * alpha_out (may be NULL) receives the last cavity field used.         */
int orc_evolve(const orc_params *p, double *data, int nsteps, double dt, int imag,
               double t0, double *alpha_out)
{
    if (!is_pow2(p->nx) || !is_pow2(p->ny) || nsteps < 0) return -1;
    cplx *psi = (cplx *)data;
    cplx alpha = 0.0;
    for (int s = 0; s < nsteps; s++) {
        double t = t0 + s * dt;
        if (!p->paper_order) {
            alpha = potential_phase(p, psi, t, 0.5 * dt, imag);
            kinetic(p, psi, dt, imag);
            alpha = potential_phase(p, psi, t + dt, 0.5 * dt, imag);
        } else {
            kinetic(p, psi, 0.5 * dt, imag);
            alpha = potential_phase(p, psi, t + 0.5 * dt, dt, imag);
            kinetic(p, psi, 0.5 * dt, imag);
        }
        if (imag) normalise(p, psi);
    }
    if (alpha_out) { alpha_out[0] = creal(alpha); alpha_out[1] = cimag(alpha); }
    return 0;
}

/* ------------------------------------------------------------------ */
/* Observables of the state psi at time t.                              */
/* out[0] norm      = int |psi|^2                                        */
/* out[1] E_kin     = (dx dy / nx ny) sum_k (k^2/2m) |F psi|^2 (Parseval) */
/* out[2] E_pot     = int V |psi|^2, V with alpha from this density       */
/* out[3] E_int     = (g/2) int |psi|^4                                   */
/* out[4] E         = E_kin + E_pot + E_int                               */
/* out[5] mu        = E_kin + E_pot + 2 E_int                             */
/* out[6] O, out[7] B (normalised overlaps, Eqs. 14-15)                   */
/* out[8] Re alpha, out[9] Im alpha                                      */
/* ------------------------------------------------------------------ */
int orc_observables(const orc_params *p, const double *data, double t, double *out)
{
    const cplx *psi = (const cplx *)data;
    size_t n = (size_t)p->nx * p->ny;
    double dx = p->Lx / p->nx, dy = p->Ly / p->ny;
    cplx *tmp = malloc(sizeof(cplx) * n);
    memcpy(tmp, psi, sizeof(cplx) * n);
    orc_fft2((double *)tmp, p->nx, p->ny, -1);
    double ekin = 0.0;
    for (int y = 0; y < p->ny; y++) {
        double ky = kcoord(y, p->ny, p->Ly);
        for (int x = 0; x < p->nx; x++) {
            double kx = kcoord(x, p->nx, p->Lx);
            cplx v = tmp[(size_t)y * p->nx + x];
            ekin += (kx * kx + ky * ky) / (2.0 * p->m) * (creal(v) * creal(v) + cimag(v) * cimag(v));
        }
    }
    ekin *= dx * dy / ((double)p->nx * (double)p->ny);
    free(tmp);

    cplx alpha = cavity_alpha(p, psi, t);
    double norm = 0.0, epot = 0.0, eint = 0.0;
    for (int y = 0; y < p->ny; y++)
        for (int x = 0; x < p->nx; x++) {
            cplx v = psi[(size_t)y * p->nx + x];
            double d = creal(v) * creal(v) + cimag(v) * cimag(v);
            norm += d * dx * dy;
            epot += potential_at(p, x, y, t, alpha) * d * dx * dy;
            eint += 0.5 * p->g * d * d * dx * dy;
        }
    out[0] = norm; out[1] = ekin; out[2] = epot; out[3] = eint;
    out[4] = ekin + epot + eint;
    out[5] = ekin + epot + 2.0 * eint;
    if (p->cavity) {
        overlaps ov = density_overlaps(p, psi);
        out[6] = ov.O; out[7] = ov.B;
    } else {
        out[6] = 0.0; out[7] = 0.0;
    }
    out[8] = creal(alpha); out[9] = cimag(alpha);
    return 0;
}

int orc_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ------------------------------------------------------------------ */
/* Discrete adjoint of the real-time V/2 - T - V/2 evolution (control   */
/* of the lattice depth, Sec. 5.2 Eq. (9) with a piecewise-linear V0(t)) */
/*                                                                       */
/* Objective: J = E(psi_T) + |<phi|psi_T>|^2 with E the GP energy at the */
/* final time (the observables above) and <phi|psi> = int conj(phi) psi. */
/* lambda = dJ/d conj(psi) (Wirtinger), so dJ = 2 Re sum conj(lambda)   */
/* dpsi.  For a phase sub-step psi' = exp(-i theta) psi with theta =     */
/* h (V + g |psi|^2), mu = exp(+i theta) lambda' gives                   */
/*   lambda = mu + 2 h g Im(conj(mu) psi) psi,                            */
/*   dJ/dV(r) += 2 h Im(conj(mu) psi)(r);                                 */
/* for the kinetic sub-step (unitary) lambda = F^-1 conj(K) F lambda'.   */
/* The terminal adjoint is lambda_T = dxdy (H psi_T + <phi|psi_T> phi)   */
/* with H psi = F^-1[(k^2/2m) F psi] + (V(T) + g |psi|^2) psi.           */
/* dV/dv = L(r) = V0x cos^2(kx x) + V0y cos^2(ky y) for the lattice      */
/* control v(t), and dv(t)/dv_i is the piecewise-linear hat weight of    */
/* control point i at time t (clamped at both ends, as ctrl_eval).       */
/* ------------------------------------------------------------------ */
static void ctrl_weights(const orc_params *p, double t, double *grad, double gv)
{
    int n = p->nctrl;
    if (n <= 0) return;
    if (t <= p->ctrl_t[0]) { grad[0] += gv; return; }
    if (t >= p->ctrl_t[n - 1]) { grad[n - 1] += gv; return; }
    int i = 0;
    while (i + 1 < n && p->ctrl_t[i + 1] < t) i++;
    double f = (t - p->ctrl_t[i]) / (p->ctrl_t[i + 1] - p->ctrl_t[i]);
    grad[i] += (1.0 - f) * gv;
    grad[i + 1] += f * gv;
}

static double lattice_mode(const orc_params *p, int xi, int yi)
{
    double x = xcoord(xi, p->nx, p->Lx), y = xcoord(yi, p->ny, p->Ly);
    double cx = cos(p->lat_kx * x), cy = cos(p->lat_ky * y);
    return p->lat_V0x * cx * cx + p->lat_V0y * cy * cy;
}

/* Adjoint of a real-time phase sub-step whose input was psi_in, applied
 * to lam in place; returns sum_r 2 h Im(conj(mu) psi_in) L(r) (dJ/dv at t). */
static double phase_adjoint(const orc_params *p, cplx *lam, const cplx *psi_in, double t, double h)
{
    double gv = 0.0;
    for (int y = 0; y < p->ny; y++)
        for (int x = 0; x < p->nx; x++) {
            size_t i = (size_t)y * p->nx + x;
            double n = creal(psi_in[i]) * creal(psi_in[i]) + cimag(psi_in[i]) * cimag(psi_in[i]);
            double theta = (potential_at(p, x, y, t, 0.0) + p->g * n) * h;
            cplx mu = cexp(I * theta) * lam[i];
            double q = cimag(conj(mu) * psi_in[i]);
            lam[i] = mu + 2.0 * h * p->g * q * psi_in[i];
            gv += 2.0 * h * q * lattice_mode(p, x, y);
        }
    return gv;
}

/* J and dJ/dctrl_v[i] (grad_out[nctrl]) for nsteps real-time steps of dt
 * from psi0 (interleaved complex128) at time t0.  phi: target state.
 * Requires ctrl_target = lattice and no cavity; returns -1 otherwise.    */
int orc_adjoint(const orc_params *p, const double *psi0, const double *phi_d, int nsteps, double dt,
                double t0, double *J_out, double *grad_out)
{
    if (!is_pow2(p->nx) || !is_pow2(p->ny) || nsteps < 0) return -1;
    if (p->cavity || p->ctrl_target != CTRL_LATTICE || p->paper_order) return -1;
    size_t n = (size_t)p->nx * p->ny;
    double dx = p->Lx / p->nx, dy = p->Ly / p->ny;
    const cplx *phi = (const cplx *)phi_d;
    /* forward: boundary states psi_s and the closing-phase inputs psi_b */
    cplx *st = malloc(sizeof(cplx) * n * (size_t)(nsteps + 1));
    cplx *sb = malloc(sizeof(cplx) * n * (size_t)(nsteps > 0 ? nsteps : 1));
    memcpy(st, psi0, sizeof(cplx) * n);
    for (int s = 0; s < nsteps; s++) {
        double t = t0 + s * dt;
        cplx *cur = st + n * (size_t)(s + 1);
        memcpy(cur, st + n * (size_t)s, sizeof(cplx) * n);
        potential_phase(p, cur, t, 0.5 * dt, 0);
        kinetic(p, cur, dt, 0);
        memcpy(sb + n * (size_t)s, cur, sizeof(cplx) * n);
        potential_phase(p, cur, t + dt, 0.5 * dt, 0);
    }
    const cplx *psiT = st + n * (size_t)nsteps;
    double tT = t0 + nsteps * dt;

    /* objective */
    double obs[10];
    orc_observables(p, (const double *)psiT, tT, obs);
    cplx c = 0.0;
    for (size_t i = 0; i < n; i++) c += conj(phi[i]) * psiT[i] * dx * dy;
    *J_out = obs[4] + creal(c * conj(c));

    for (int i = 0; i < p->nctrl; i++) grad_out[i] = 0.0;
    /* terminal adjoint and the explicit dependence of E on v(T) */
    cplx *lam = malloc(sizeof(cplx) * n);
    memcpy(lam, psiT, sizeof(cplx) * n);
    orc_fft2((double *)lam, p->nx, p->ny, -1);
    for (int y = 0; y < p->ny; y++) {
        double ky = kcoord(y, p->ny, p->Ly);
        for (int x = 0; x < p->nx; x++) {
            double kx = kcoord(x, p->nx, p->Lx);
            lam[(size_t)y * p->nx + x] *= (kx * kx + ky * ky) / (2.0 * p->m);
        }
    }
    orc_fft2((double *)lam, p->nx, p->ny, +1);
    double gT = 0.0;
    for (int y = 0; y < p->ny; y++)
        for (int x = 0; x < p->nx; x++) {
            size_t i = (size_t)y * p->nx + x;
            cplx v = psiT[i];
            double d = creal(v) * creal(v) + cimag(v) * cimag(v);
            lam[i] = (lam[i] + (potential_at(p, x, y, tT, 0.0) + p->g * d) * v + c * phi[i]) * dx * dy;
            gT += d * lattice_mode(p, x, y) * dx * dy;
        }
    ctrl_weights(p, tT, grad_out, gT);

    /* reverse sweep */
    for (int s = nsteps - 1; s >= 0; s--) {
        double t = t0 + s * dt;
        ctrl_weights(p, t + dt, grad_out, phase_adjoint(p, lam, sb + n * (size_t)s, t + dt, 0.5 * dt));
        kinetic(p, lam, -dt, 0);                      /* conjugate kinetic phase */
        ctrl_weights(p, t, grad_out, phase_adjoint(p, lam, st + n * (size_t)s, t, 0.5 * dt));
    }
    free(lam); free(st); free(sb);
    return 0;
}

/* ------------------------------------------------------------------ */
/* Momentum-state populations (Sec. 5.2, Kapitza-Dirac): the fraction   */
/* of sum_k |F psi|^2 whose momentum along `axis` (0: x, 1: y) lies     */
/* within k0 of 2 n k0, summed over the other axis, n = -nmax..nmax.    */
/* A momentum exactly between two windows (|k - 2 n k0| = k0) goes to   */
/* the window of smaller |n|.                                            */
/* ------------------------------------------------------------------ */
int orc_momentum_populations(const orc_params *p, const double *data, int axis, double k0, int nmax,
                             double *out)
{
    if (!is_pow2(p->nx) || !is_pow2(p->ny) || (axis != 0 && axis != 1) || !(k0 > 0.0) || nmax < 0) return -1;
    size_t n = (size_t)p->nx * p->ny;
    cplx *f = malloc(sizeof(cplx) * n);
    memcpy(f, data, sizeof(cplx) * n);
    orc_fft2((double *)f, p->nx, p->ny, -1);
    for (int i = 0; i <= 2 * nmax; i++) out[i] = 0.0;
    double total = 0.0;
    for (int y = 0; y < p->ny; y++)
        for (int x = 0; x < p->nx; x++) {
            cplx v = f[(size_t)y * p->nx + x];
            double w = creal(v) * creal(v) + cimag(v) * cimag(v);
            total += w;
            double k = axis == 0 ? kcoord(x, p->nx, p->Lx) : kcoord(y, p->ny, p->Ly);
            double r = k / (2.0 * k0);                 /* window n: |r - n| <= 1/2 */
            int b = (int)floor(fabs(r) + 0.5);
            if (fabs(fabs(r) - (b - 0.5)) < 1e-12 && b > 0) b -= 1;   /* ties to smaller |n| */
            if (b > nmax) continue;
            int idx = (r < 0 ? -b : b) + nmax;
            out[idx] += w;
        }
    for (int i = 0; i <= 2 * nmax; i++) out[i] /= total;
    free(f);
    return 0;
}
