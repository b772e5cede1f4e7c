"""Pins for two parts of the oracle that the other pins leave open (CPU only).

1. The potential-array term V_scale * V[y][x] of the potential descriptor.
   A harmonic trap written into the array (sampled on the grid, analytic
   trap switched off) must give the same trajectory as the analytic trap
   (Sec. 5.1): on a non-square grid with an anisotropic trap, a transposed
   or shifted index into the array, or a dropped V_scale, changes V at
   almost every point and fails the comparison by many orders of magnitude.

2. The order in which the cavity field is updated in imaginary time.
   Sec. 5.3 updates alpha "at each time step" from the current density, and
   Sec. 3.1 evaluates the potential from the most recent wave function.
   The reading taken here (alpha recomputed from the density at the start of
   each half phase, then the whole half phase applied with that alpha, then
   the norm restored after the step, Sec. 3.3) is written out below a second
   time, plainly with numpy's FFT and Eqs. (10)-(15), for two imaginary-time
   steps on an 8x8 grid, and the oracle must agree with it to 1e-14.  The
   test also checks that the two nearest wrong orders (alpha kept from the
   start of the step for both half phases; alpha taken from the density
   after the phase it drives) differ from the oracle by far more than that,
   so the comparison decides between them.
"""
import numpy as np

import gpe_inputs as gi
import oracle


def grid(p):
    x = gi.grid_axis(p["nx"], p["Lx"])[None, :]
    y = gi.grid_axis(p["ny"], p["Ly"])[:, None]
    return x, y


# ---------------------------------------------------------------- potential array
def trap_params(**kw):
    p = gi.potential_defaults()
    p.update(nx=32, ny=16, Lx=12.0, Ly=8.0, m=1.3, g=30.0, wx=1.3, wy=0.7)
    p.update(kw)
    return p


def test_potential_array_reproduces_the_analytic_trap():
    pa = trap_params()
    x, y = grid(pa)
    trap = 0.5 * pa["m"] * (pa["wx"] ** 2 * x ** 2 + pa["wy"] ** 2 * y ** 2)   # Sec. 5.1 trap on the grid
    pv = trap_params(wx=0.0, wy=0.0, Varr=2.0 * trap, V_scale=0.5)
    assert np.max(np.abs(oracle.potential(pv) - trap)) < 1e-12
    psi0 = gi.gaussian_state(32, 16, 12.0, 8.0, 1.1, 1e-2, seed=41, x0=0.7, kx0=0.4)
    for imag, dt, n in ((False, 2e-3, 200), (True, 2e-3, 200)):
        a, _ = oracle.evolve(pa, psi0, n, dt, imag)
        b, _ = oracle.evolve(pv, psi0, n, dt, imag)
        assert np.max(np.abs(a - b)) < 1e-12 * np.max(np.abs(a))
    oa, ov = oracle.observables(pa, a), oracle.observables(pv, b)
    for k in ("norm", "ekin", "epot", "eint", "energy", "mu"):
        assert abs(oa[k] - ov[k]) < 1e-12 * abs(oa[k]), k


def test_potential_array_index_mistakes_are_visible():
    """The same comparison with the array transposed (as if read [x][y]) or
    shifted by one point fails by far more than the bound above."""
    pa = trap_params()
    x, y = grid(pa)
    trap = 0.5 * pa["m"] * (pa["wx"] ** 2 * x ** 2 + pa["wy"] ** 2 * y ** 2)
    psi0 = gi.gaussian_state(32, 16, 12.0, 8.0, 1.1, 1e-2, seed=41, x0=0.7, kx0=0.4)
    a, _ = oracle.evolve(pa, psi0, 200, 2e-3, False)
    wrong = [trap.T.reshape(16, 32), np.roll(trap, 1, axis=1), 0.5 * trap]
    for Varr in wrong:
        b, _ = oracle.evolve(trap_params(wx=0.0, wy=0.0, Varr=Varr), psi0, 200, 2e-3, False)
        assert np.max(np.abs(a - b)) > 1e-4 * np.max(np.abs(a))


# ---------------------------------------------------------------- cavity field update order
def cavity_params():
    p = gi.potential_defaults()
    p.update(nx=8, ny=8, Lx=4.0, Ly=4.0, m=1.0, g=20.0, wx=1.0, wy=1.0, cavity=1, eta=3.0, U0=-0.5,
             dc=-2.0, kappa=1.0, kc=np.pi, Nat=1.0, pump_lattice=1)
    return p


def field(p, psi):
    """alpha = N eta O / (Delta_c - U0 B + i kappa), O and B the overlaps of
    Eqs. (14)-(15) divided by the norm."""
    x, y = grid(p)
    d = np.abs(psi) ** 2
    O = np.sum(np.cos(p["kc"] * x) * np.cos(p["kc"] * y) * d) / np.sum(d)
    B = np.sum(np.cos(p["kc"] * x) ** 2 * d) / np.sum(d)
    return p["Nat"] * p["eta"] * O / (p["dc"] - p["U0"] * B + 1j * p["kappa"])


def potential(p, alpha):
    """Trap + pump lattice + cavity terms, Eqs. (10)-(13), cavity axis x."""
    x, y = grid(p)
    cx, cy = np.cos(p["kc"] * x), np.cos(p["kc"] * y)
    V = 0.5 * p["m"] * (p["wx"] ** 2 * x ** 2 + p["wy"] ** 2 * y ** 2)
    V = V + (p["eta"] ** 2 / p["U0"]) * cy ** 2
    V = V + p["U0"] * abs(alpha) ** 2 * cx ** 2
    return V + 2 * p["eta"] * alpha.real * cx * cy


def half_phase(p, psi, alpha, dt):
    return psi * np.exp(-(potential(p, alpha) + p["g"] * np.abs(psi) ** 2) * 0.5 * dt)


def kinetic(p, psi, dt):
    kx = 2 * np.pi * np.fft.fftfreq(p["nx"], p["Lx"] / p["nx"])[None, :]
    ky = 2 * np.pi * np.fft.fftfreq(p["ny"], p["Ly"] / p["ny"])[:, None]
    return np.fft.ifft2(np.exp(-(kx ** 2 + ky ** 2) / (2 * p["m"]) * dt) * np.fft.fft2(psi))


def normalised(p, psi):
    return psi / np.sqrt(np.sum(np.abs(psi) ** 2) * (p["Lx"] / p["nx"]) * (p["Ly"] / p["ny"]))


def imaginary_steps(p, psi, nsteps, dt, order):
    for _ in range(nsteps):
        a_start = field(p, psi)
        psi = half_phase(p, psi, a_start, dt)
        psi = kinetic(p, psi, dt)
        if order == "each half phase":
            a2 = field(p, psi)                     # density at the start of the second half phase
        elif order == "once per step":
            a2 = a_start
        else:                                      # from the density the phase itself produces
            a2 = field(p, half_phase(p, psi, field(p, psi), dt))
        psi = half_phase(p, psi, a2, dt)
        psi = normalised(p, psi)
    return psi


def test_imaginary_time_cavity_field_is_recomputed_before_each_half_phase():
    p = cavity_params()
    x, y = grid(p)
    psi0 = np.exp(-(x ** 2 + y ** 2) / 2.0) * (1.0 + 0.4 * np.cos(np.pi * x) * np.cos(np.pi * y))
    psi0 = normalised(p, psi0.astype(np.complex128))
    dt = 0.05
    want = imaginary_steps(p, psi0, 2, dt, "each half phase")
    got, alpha_last = oracle.evolve(p, psi0, 2, dt, True)
    assert abs(field(p, psi0)) > 0.1                           # the field matters at this pump
    assert np.max(np.abs(got - want)) < 1e-14 * np.max(np.abs(want))
    # the field the oracle reports is the one of its last half phase
    before_last = kinetic(p, half_phase(p, imaginary_steps(p, psi0, 1, dt, "each half phase"),
                                        field(p, imaginary_steps(p, psi0, 1, dt, "each half phase")), dt), dt)
    assert abs(alpha_last - field(p, before_last)) < 1e-14
    for order in ("once per step", "after the phase"):
        other = imaginary_steps(p, psi0, 2, dt, order)
        assert np.max(np.abs(other - want)) > 1e-6 * np.max(np.abs(want)), order
