"""Seeded synthetic inputs shared by the oracle tests, the GPU tests and the bench.

This module holds only input definitions: the counter-based random stream,
initial wave functions and the workload parameter sets.  It contains none
of the split-step arithmetic (no FFT, phase, normalisation of a step,
reduction or cavity update); both the oracle and the CUDA path receive the
same arrays from here.

Random numbers: SplitMix64 (Steele, Lea & Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014) gives 64-bit words from a
counter; the top 53 bits make a double in [0, 1); Box-Muller turns pairs
of uniforms into standard normals.

Workloads follow the paper's physical setups (Sec. 4.1 timing benchmark:
harmonic trap, imaginary time, grids N = 2^n; Sec. 5.1 trapped interacting
BEC; Sec. 5.2 lattice pulse; Sec. 5.3 cavity self-organisation) in
oscillator units (Sec. 3.2: hbar = m = omega = 1).  There is no dataset:
these synthetic states stand in for the paper's experiments.
"""
from __future__ import annotations

import numpy as np

_MASK = np.uint64(0xFFFFFFFFFFFFFFFF)


def splitmix64(seed: int, n: int, offset: int = 0) -> np.ndarray:
    """Words offset..offset+n-1 of the SplitMix64 stream for `seed`."""
    with np.errstate(over="ignore"):
        gamma = np.uint64(0x9E3779B97F4A7C15)
        idx = np.arange(offset + 1, offset + n + 1, dtype=np.uint64)
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + idx * gamma
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        z = z ^ (z >> np.uint64(31))
    return z


def uniform(seed: int, n: int, offset: int = 0) -> np.ndarray:
    """n doubles in [0, 1) from the top 53 bits of SplitMix64 words."""
    w = splitmix64(seed, n, offset)
    return (w >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def normal(seed: int, n: int) -> np.ndarray:
    """n standard normals by Box-Muller on consecutive uniform pairs (made in
    chunks of 2^21 pairs; the values depend only on the stream position)."""
    m = (n + 1) // 2
    z = np.empty(2 * m)
    chunk = 1 << 21
    for a in range(0, m, chunk):
        b = min(m, a + chunk)
        u = uniform(seed, 2 * (b - a), offset=2 * a)
        u1 = 1.0 - u[0::2]                  # (0, 1]: log is finite
        u2 = u[1::2]
        r = np.sqrt(-2.0 * np.log(u1))
        z[2 * a:2 * b:2] = r * np.cos(2.0 * np.pi * u2)
        z[2 * a + 1:2 * b:2] = r * np.sin(2.0 * np.pi * u2)
    return z[:n]


def grid_axis(n: int, L: float) -> np.ndarray:
    """x_j = -L/2 + j L/n, j = 0..n-1: the periodic box without its right end."""
    return -0.5 * L + np.arange(n) * (L / n)


def gaussian_state(nx: int, ny: int, Lx: float, Ly: float, width: float = 1.5,
                   noise: float = 1e-3, seed: int = 0, x0: float = 0.0,
                   y0: float = 0.0, kx0: float = 0.0, checker: float = 0.0,
                   kc: float = 0.0) -> np.ndarray:
    """Initial wave function, complex128 [ny][nx], unit norm on the grid.

    psi ~ exp(-((x-x0)^2 + (y-y0)^2) / (2 width^2)) e^{i kx0 x}
          (1 + checker cos(kc x) cos(kc y)),
    plus noise * max|G| * (xi_r + i xi_i) with xi ~ N(0,1) per point from the
    seeded stream, then scaled so that sum |psi|^2 dx dy = 1.  The checker
    term seeds the density modulation of the organised cavity phase (Sec. 5.3).
    """
    x = grid_axis(nx, Lx)[None, :]
    y = grid_axis(ny, Ly)[:, None]
    g = np.exp(-((x - x0) ** 2 + (y - y0) ** 2) / (2.0 * width ** 2)) * np.exp(1j * kx0 * x)
    if checker:
        g = g * (1.0 + checker * np.cos(kc * x) * np.cos(kc * y))
    if noise:
        xi = normal(seed, 2 * nx * ny).reshape(2, ny, nx)
        g = g + noise * np.abs(g).max() * (xi[0] + 1j * xi[1])
    s = np.sum(np.abs(g) ** 2) * (Lx / nx) * (Ly / ny)
    return (g / np.sqrt(s)).astype(np.complex128)


def uniform_state(nx: int, ny: int, Lx: float, Ly: float) -> np.ndarray:
    """Constant wave function of unit norm (used for lattice pins)."""
    return np.full((ny, nx), 1.0 / np.sqrt(Lx * Ly), dtype=np.complex128)


def control_points(seed: int, n: int, T: float, lo: float, hi: float):
    """n piecewise-linear control points at t_i = i T/(n-1), values uniform in [lo, hi]."""
    t = np.linspace(0.0, T, n)
    v = lo + (hi - lo) * uniform(seed, n)
    return t, v


# ---------------------------------------------------------------------------
# Workloads.  Keys are the physical parameters of both implementations.
# ---------------------------------------------------------------------------
def potential_defaults() -> dict:
    return dict(wx=0.0, wy=0.0, lat_V0x=0.0, lat_V0y=0.0, lat_kx=0.0, lat_ky=0.0,
                Varr=None, V_scale=1.0, cavity=0, eta=0.0, U0=0.0, dc=0.0,
                kappa=0.0, kc=0.0, Nat=1.0, pump_lattice=1, ctrl_target=0,
                ctrl_t=None, ctrl_v=None, probe_omega=0.0, probe_delta=0.0, probe_phi=0.0)


def harmonic_trap(n: int = 128, L: float = 20.0, g: float = 0.0, seed: int = 0) -> dict:
    """Trapped BEC, V = r^2/2, imaginary time (Secs. 4.1 and 5.1): 128^2, box 20."""
    p = potential_defaults()
    p.update(nx=n, ny=n, Lx=L, Ly=L, m=1.0, g=g, wx=1.0, wy=1.0)
    return dict(params=p, dt=1e-3, imag=True, steps=2000,
                psi0=lambda: gaussian_state(n, n, L, L, 1.5, 1e-3, seed))


def lattice_real_time(n: int = 2048, L: float = 40.0, seed: int = 1) -> dict:
    """Real-time throughput workload: trap + 2D lattice V0 = 5, k = 2 pi, g = 500, dt = 5e-4."""
    p = potential_defaults()
    k = 2.0 * np.pi / 1.0
    p.update(nx=n, ny=n, Lx=L, Ly=L, m=1.0, g=500.0, wx=1.0, wy=1.0,
             lat_V0x=5.0, lat_V0y=5.0, lat_kx=k, lat_ky=k)
    return dict(params=p, dt=5e-4, imag=False, steps=10000,
                psi0=lambda: gaussian_state(n, n, L, L, 1.5, 1e-3, seed))


def kapitza_dirac(n: int = 256, L: float = 16.0, V0: float = 100.0, tau: float = 0.01, dt: float = 1e-4,
                  g: float = 0.0, seed: int = 5) -> dict:
    """Lattice flash along y (Sec. 5.2): trap + V0 cos^2(k y) with k = 2 pi
    switched on for a duration tau (control v(t) = 1 up to tau, 0 from
    tau + dt/10 on), read out as momentum populations of |2 n k>."""
    p = potential_defaults()
    k = 2.0 * np.pi
    p.update(nx=n, ny=n, Lx=L, Ly=L, m=1.0, g=g, wx=1.0, wy=1.0, lat_V0y=V0, lat_ky=k, ctrl_target=1,
             ctrl_t=np.array([0.0, tau, tau + 0.1 * dt]), ctrl_v=np.array([1.0, 1.0, 0.0]))
    return dict(params=p, dt=dt, imag=False, steps=int(round(tau / dt)), k=k,
                psi0=lambda: gaussian_state(n, n, L, L, 1.5, 0.0, seed))


def bragg_probe(n: int = 512, L: float = 20.0, eta: float = 2.0, omega: float = 0.05, delta_p: float = 20.0,
                phi: float = 0.3, steps: int = 4000, dt: float = 2e-4, seed: int = 6) -> dict:
    """Bragg spectroscopy of the cavity soft mode (Sec. 5.4): the cavity
    setup of the self-organisation workload at a fixed pump eta, with a weak
    on-axis probe of strength omega detuned by delta_p; the response is the
    cavity field alpha(t)."""
    p = potential_defaults()
    p.update(nx=n, ny=n, Lx=L, Ly=L, m=1.0, g=100.0, wx=1.0, wy=1.0, cavity=1, eta=eta, U0=-0.5, dc=-2.0,
             kappa=1.0, kc=2.0 * np.pi, Nat=1.0, pump_lattice=1, probe_omega=omega, probe_delta=delta_p,
             probe_phi=phi)
    return dict(params=p, dt=dt, imag=False, steps=steps,
                psi0=lambda: gaussian_state(n, n, L, L, 1.5, 1e-3, seed, checker=0.2, kc=2.0 * np.pi))


def phase_diagram_sweep(seed: int = 3, L: float = 20.0, dt: float = 1e-3, g: float = 100.0,
                        counts=((256, 128), (512, 192), (1024, 64))) -> list:
    """Batched sweep of cavity instances (Sec. 5.3 phase diagram): for each
    (grid n, count) pair, `count` instances on an n x n grid, with (eta, Delta_c)
    drawn uniformly from [0, 4] x [-5, 0]; trap, U0 = -0.5, kappa = 1, pump
    lattice on, imaginary time.  Returns a list of workload dicts."""
    total = sum(c for _, c in counts)
    u = uniform(seed, 2 * total)
    out, k = [], 0
    for n, cnt in counts:
        for _ in range(cnt):
            p = potential_defaults()
            p.update(nx=n, ny=n, Lx=L, Ly=L, m=1.0, g=g, wx=1.0, wy=1.0, cavity=1,
                     eta=4.0 * u[2 * k], dc=-5.0 * u[2 * k + 1], U0=-0.5, kappa=1.0,
                     kc=2.0 * np.pi, Nat=1.0, pump_lattice=1)
            out.append(dict(params=p, dt=dt, imag=True,
                            psi0=lambda n=n, k=k: gaussian_state(n, n, L, L, 1.5, 1e-3, seed + 1000 + k,
                                                                 checker=0.1, kc=2.0 * np.pi)))
            k += 1
    return out


def target_gaussian(nx: int, ny: int, Lx: float, Ly: float) -> np.ndarray:
    """Ground state of the isotropic trap in oscillator units, exp(-r^2/2)/sqrt(pi)."""
    x, y = grid_axis(nx, Lx), grid_axis(ny, Ly)
    return np.exp(-0.5 * (x[None, :] ** 2 + y[:, None] ** 2)) / np.sqrt(np.pi)


def adjoint_control(n: int = 512, L: float = 20.0, steps: int = 4000, dt: float = 5e-4, npts: int = 200,
                    g: float = 100.0, seed: int = 4) -> dict:
    """Lattice-depth control for the adjoint: trap + lattice of wavenumber 2 pi
    whose depth is v(t) (lat_V0x = lat_V0y = 1, control target lattice), with
    npts piecewise-linear points seeded uniformly in [0, 8] over the run; the
    objective's target state is the trap ground state."""
    t, v = control_points(seed, npts, steps * dt, 0.0, 8.0)
    p = potential_defaults()
    k = 2.0 * np.pi
    p.update(nx=n, ny=n, Lx=L, Ly=L, m=1.0, g=g, wx=1.0, wy=1.0, lat_V0x=1.0, lat_V0y=1.0,
             lat_kx=k, lat_ky=k, ctrl_target=1, ctrl_t=t, ctrl_v=v)
    return dict(params=p, dt=dt, imag=False, steps=steps,
                psi0=lambda: gaussian_state(n, n, L, L, 1.5, 1e-3, seed),
                phi=lambda: target_gaussian(n, n, L, L))


def cavity_ramp(n: int = 512, L: float = 40.0, seed: int = 2, steps: int = 20000,
                dt: float = 2e-4) -> dict:
    """Self-consistent cavity (Sec. 5.3): eta ramped 0 -> 3 over the run, Delta_c = -2, U0 = -0.5, kappa = 1."""
    p = potential_defaults()
    k = 2.0 * np.pi / 1.0
    T = steps * dt
    p.update(nx=n, ny=n, Lx=L, Ly=L, m=1.0, g=100.0, wx=1.0, wy=1.0,
             cavity=1, eta=0.0, U0=-0.5, dc=-2.0, kappa=1.0, kc=k, Nat=1.0,
             pump_lattice=1, ctrl_target=2,
             ctrl_t=np.array([0.0, T]), ctrl_v=np.array([0.0, 3.0]))
    return dict(params=p, dt=dt, imag=False, steps=steps,
                psi0=lambda: gaussian_state(n, n, L, L, 1.5, 1e-3, seed))
