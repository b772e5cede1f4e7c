"""Pins for the oracle's split-step propagator against closed forms (CPU only).

Each test fixes the oracle to something other than itself: an exact solution
of the GPE (free Gaussian, trapped coherent state, oscillator ground state),
an asymptotic law (Thomas-Fermi mu, Sec. 5.1), an exact invariant (norm in
real time, virial identity), an independent exact evolution (lattice in a
truncated momentum basis, Sec. 5.2 non-interacting check; Raman-Nath Bessel
populations), a convergence order (Eq. 3: Strang splitting is second order),
or a special case of the cavity model (Eqs. 10-15).
"""
import numpy as np
import pytest
import scipy.linalg
import scipy.special

import gpe_inputs as gi
import oracle


def base(n, L, **kw):
    p = gi.potential_defaults()
    p.update(nx=n, ny=n, Lx=L, Ly=L, m=1.0, g=0.0)
    p.update(kw)
    return p


def grid(p):
    x = gi.grid_axis(p["nx"], p["Lx"])[None, :]
    y = gi.grid_axis(p["ny"], p["Ly"])[:, None]
    return x, y


def rel_l2(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def phase_aligned(a, b):
    """a e^{i phi} with phi minimising |a e^{i phi} - b| (global phase freedom)."""
    z = np.vdot(a, b)
    return a * (z / abs(z))


# ---------------------------------------------------------------- free motion
@pytest.mark.parametrize("m", [1.0, 0.5])
def test_free_moving_gaussian_closed_form(m):
    """V = 0, g = 0: the split-step is exact; compare to the spreading packet."""
    p = base(128, 40.0, m=m)
    x, y = grid(p)
    s, k0, t = 1.3, 1.5, 2.0 * m                       # packet stays far from the box edge

    def packet(t):
        tau = 1.0 + 1j * t / (m * s * s)
        fx = (np.pi * s * s) ** -0.25 / np.sqrt(tau) * np.exp(
            -(x - k0 * t / m) ** 2 / (2 * s * s * tau) + 1j * k0 * x - 1j * k0 * k0 * t / (2 * m))
        fy = (np.pi * s * s) ** -0.25 / np.sqrt(tau) * np.exp(-y ** 2 / (2 * s * s * tau))
        return fx * fy

    psi0 = packet(0.0)
    out, _ = oracle.evolve(p, psi0, 50, t / 50, imag=False)
    assert rel_l2(out, packet(t)) < 1e-9


def test_free_imaginary_time_is_heat_kernel():
    """V = 0, g = 0, imaginary time: |k> decays as e^{-k^2 tau / 2m}; after
    normalisation a Gaussian of width s keeps Gaussian form with s^2 + tau/m."""
    p = base(128, 40.0)
    x, y = grid(p)
    s, tau = 1.0, 0.8
    g0 = np.exp(-(x ** 2 + y ** 2) / (2 * s * s)).astype(complex)
    g0 /= np.sqrt(np.sum(abs(g0) ** 2) * (40 / 128) ** 2)
    out, _ = oracle.evolve(p, g0, 40, tau / 40, imag=True)
    s2 = s * s + tau
    ref = np.exp(-(x ** 2 + y ** 2) / (2 * s2)).astype(complex)
    ref /= np.sqrt(np.sum(abs(ref) ** 2) * (40 / 128) ** 2)
    assert rel_l2(out, ref) < 1e-9


# ------------------------------------------------------------ harmonic trap
def test_coherent_state_density_follows_classical_orbit():
    """g = 0 trap, displaced ground state: |psi(x,t)|^2 = pi^-1 e^{-(x - x0 cos t)^2 - y^2}."""
    p = base(64, 16.0, wx=1.0, wy=1.0)
    x, y = grid(p)
    x0 = 2.0
    psi0 = (np.pi ** -0.5 * np.exp(-((x - x0) ** 2 + y ** 2) / 2)).astype(complex)
    dt, n = 2e-3, 785                                   # t = 1.57 ~ pi/2
    out, _ = oracle.evolve(p, psi0, n, dt, imag=False)
    t = n * dt
    dens = np.pi ** -1 * np.exp(-(x - x0 * np.cos(t)) ** 2 - y ** 2)
    assert np.max(np.abs(abs(out) ** 2 - dens)) < 5e-6
    obs = oracle.observables(p, out)
    assert abs(obs["norm"] - 1.0) < 1e-12


def test_oscillator_ground_state_energy_and_shape():
    """Imaginary time, g = 0: psi -> pi^-1/2 e^{-r^2/2} with E = mu = 1 (Sec. 3.3)."""
    p = base(64, 16.0, wx=1.0, wy=1.0)
    x, y = grid(p)
    psi0 = gi.gaussian_state(64, 64, 16.0, 16.0, 1.5, 1e-3, seed=0)
    out, _ = oracle.evolve(p, psi0, 10000, 1e-3, imag=True)
    obs = oracle.observables(p, out)
    assert abs(obs["norm"] - 1.0) < 1e-12
    assert abs(obs["energy"] - 1.0) < 1e-6
    assert abs(obs["mu"] - 1.0) < 1e-6
    exact = (np.pi ** -0.5 * np.exp(-(x ** 2 + y ** 2) / 2)).astype(complex)
    assert rel_l2(phase_aligned(out, exact), exact) < 1e-5


def test_harmonic_config_2000_steps_energy():
    """The 128^2, box-20 trap workload: E within 2e-4 of 1 after 2000 steps of 1e-3."""
    w = gi.harmonic_trap(g=0.0)
    out, _ = oracle.evolve(w["params"], w["psi0"](), 2000, w["dt"], imag=True)
    obs = oracle.observables(w["params"], out)
    assert abs(obs["energy"] - 1.0) < 2e-4
    assert obs["energy"] > 1.0                         # variational bound


@pytest.mark.parametrize("g", [100.0, 400.0, 1600.0])
def test_thomas_fermi_chemical_potential(g):
    """Large g: mu -> mu_TF = sqrt(g/pi) for V = r^2/2 in 2D (Sec. 5.1)."""
    w = gi.harmonic_trap(g=g)
    p = w["params"]
    out, _ = oracle.evolve(p, w["psi0"](), 5000, 2e-3, imag=True)     # tau = 10
    mu = oracle.observables(p, out)["mu"]
    ratio = mu / np.sqrt(g / np.pi)
    assert 1.0 < ratio < 1.03
    test_thomas_fermi_chemical_potential.ratios = getattr(
        test_thomas_fermi_chemical_potential, "ratios", {})
    test_thomas_fermi_chemical_potential.ratios[g] = ratio
    r = test_thomas_fermi_chemical_potential.ratios
    if len(r) == 3:                                    # kinetic correction shrinks with g
        assert r[100.0] > r[400.0] > r[1600.0]


def test_virial_identity_converges_linearly_in_dt():
    """2D trap + contact: E_kin - E_pot + E_int = 0 at the ground state; the
    split-step fixed point misses it by O(dt)."""
    w = gi.harmonic_trap(n=64, L=16.0, g=100.0)
    p = w["params"]
    res = []
    for dt in (2e-3, 1e-3):
        out, _ = oracle.evolve(p, w["psi0"](), int(8.0 / dt), dt, imag=True)
        o = oracle.observables(p, out)
        res.append(o["ekin"] - o["epot"] + o["eint"])
    assert abs(res[1]) < 1.5e-2
    assert 1.7 < res[0] / res[1] < 2.3


# ------------------------------------------------------------ real-time invariants
def test_real_time_conserves_norm_and_energy():
    w = gi.lattice_real_time(n=64, L=16.0)
    p = w["params"]
    psi0 = gi.gaussian_state(64, 64, 16.0, 16.0, 1.5, 1e-3, seed=1)
    o0 = oracle.observables(p, psi0)
    out, _ = oracle.evolve(p, psi0, 400, 5e-4, imag=False)
    o1 = oracle.observables(p, out)
    assert abs(o1["norm"] - o0["norm"]) < 1e-12
    assert abs(o1["energy"] - o0["energy"]) / abs(o0["energy"]) < 1e-3


def test_strang_is_second_order_with_time_dependent_lattice():
    """Eq. (3): local error O(dt^3) => global O(dt^2), also with V0(t) and g."""
    p = base(32, 8.0, wx=1.0, wy=1.0, g=50.0, lat_V0x=3.0, lat_V0y=2.0,
             lat_kx=2 * np.pi / 2.0, lat_ky=2 * np.pi / 2.0, ctrl_target=1,
             ctrl_t=np.array([0.0, 0.3, 0.6]), ctrl_v=np.array([0.0, 2.0, 0.5]))
    psi0 = gi.gaussian_state(32, 32, 8.0, 8.0, 1.2, 1e-2, seed=5)
    T = 0.6
    ref, _ = oracle.evolve(p, psi0, 7680, T / 7680, imag=False)
    errs = [rel_l2(oracle.evolve(p, psi0, n, T / n, imag=False)[0], ref) for n in (120, 240, 480)]
    assert 3.7 < errs[0] / errs[1] < 4.3
    assert 3.7 < errs[1] / errs[2] < 4.3


def test_paper_operator_order_agrees_to_second_order():
    """T/2-V-T/2 (Eq. 4) and V/2-T-V/2 differ by O(dt^2) globally."""
    p = base(32, 8.0, wx=1.0, wy=1.0, g=50.0)
    psi0 = gi.gaussian_state(32, 32, 8.0, 8.0, 1.2, 1e-2, seed=6)
    d = []
    for n in (40, 80):
        a, _ = oracle.evolve(p, psi0, n, 0.4 / n, imag=False)
        b, _ = oracle.evolve(p, psi0, n, 0.4 / n, imag=False, paper_order=True)
        d.append(rel_l2(a, b))
    assert 3.4 < d[0] / d[1] < 4.6
    # imaginary time: the two fixed points differ by O(dt) and meet as dt -> 0
    w = gi.harmonic_trap(n=32, L=12.0, g=20.0)
    gap = []
    for dt in (2e-3, 1e-3):
        n = int(8.0 / dt)
        ea = oracle.observables(w["params"], oracle.evolve(w["params"], w["psi0"](), n, dt, True)[0])
        eb = oracle.observables(w["params"], oracle.evolve(w["params"], w["psi0"](), n, dt, True,
                                                           paper_order=True)[0])
        gap.append(ea["mu"] - eb["mu"])
    assert 1.7 < gap[0] / gap[1] < 2.3


# ------------------------------------------------------------ lattice (Sec. 5.2)
def lattice_populations(psi, p, M):
    """Populations of |2 n k> for n = -M..M from the oracle state (via numpy.fft)."""
    f = np.fft.fft(psi[:, 0])                          # uniform in x: take one column
    dk = 2 * np.pi / p["Ly"]
    idx = [int(round(2 * n * p["lat_ky"] / dk)) % p["ny"] for n in range(-M, M + 1)]
    pops = np.abs(f[idx]) ** 2
    return pops / np.sum(np.abs(f) ** 2)


def test_lattice_pulse_matches_momentum_basis_evolution():
    """g = 0, no trap, uniform BEC, V = V0 cos^2(k y): exact in the basis |2nk>
    with H_nn = (2nk)^2/2 + V0/2 and H_n,n+-1 = V0/4."""
    L, k, V0 = 2 * np.pi, 1.0, 8.0
    p = base(8, L, lat_V0y=V0, lat_ky=k)
    p["ny"] = 64
    psi0 = gi.uniform_state(8, 64, L, L)
    M = 12
    n = np.arange(-M, M + 1)
    H = np.diag((2 * n * k) ** 2 / 2 + V0 / 2) + np.diag(np.full(2 * M, V0 / 4), 1) \
        + np.diag(np.full(2 * M, V0 / 4), -1)
    c0 = (n == 0).astype(complex)
    t = 0.5
    exact = np.abs(scipy.linalg.expm(-1j * H * t) @ c0) ** 2
    out, _ = oracle.evolve(p, psi0, 2000, t / 2000, imag=False)
    got = lattice_populations(out, p, M)
    assert np.max(np.abs(got - exact)) < 2e-6


def test_lattice_pulse_raman_nath_short_time():
    """Short pulses: P_n = J_n(V0 t/2)^2 up to the kinetic phase (Sec. 5.2)."""
    L, k, V0, t = 2 * np.pi, 1.0, 100.0, 0.02
    p = base(8, L, lat_V0y=V0, lat_ky=k)
    p["ny"] = 64
    out, _ = oracle.evolve(p, gi.uniform_state(8, 64, L, L), 200, t / 200, imag=False)
    got = lattice_populations(out, p, 3)
    rn = scipy.special.jv(np.arange(-3, 4), V0 * t / 2) ** 2
    assert np.max(np.abs(got - rn)) < 2e-3


# ------------------------------------------------------------ cavity (Sec. 5.3)
def cavity_params(n=32, L=8.0, eta=1.0, **kw):
    p = base(n, L, wx=1.0, wy=1.0, g=20.0, cavity=1, eta=eta, U0=-0.5, dc=-2.0,
             kappa=1.0, kc=2 * np.pi / 2.0, Nat=1.0, pump_lattice=1)
    p.update(kw)
    return p


def test_cavity_eta_zero_reduces_to_plain_gpe():
    pc = cavity_params(eta=0.0)
    pp = dict(pc, cavity=0)
    psi0 = gi.gaussian_state(32, 32, 8.0, 8.0, 1.2, 1e-2, seed=8)
    a, al = oracle.evolve(pc, psi0, 50, 1e-3, imag=False)
    b, _ = oracle.evolve(pp, psi0, 50, 1e-3, imag=False)
    assert al == 0
    assert np.array_equal(a, b)


def test_cavity_overlaps_of_a_known_density():
    """n ~ 1 + a cos(kc x) cos(kc y) on a box of whole periods: O = a/4, B = 1/2,
    so alpha = N eta (a/4) / (Delta_c - U0/2 + i kappa) (Eqs. 14-15)."""
    p = cavity_params(n=64, eta=1.7, Nat=2.0)
    x, y = grid(p)
    a = 0.6
    dens = 1 + a * np.cos(p["kc"] * x) * np.cos(p["kc"] * y)
    psi = np.sqrt(dens / (dens.sum() * (8.0 / 64) ** 2)).astype(complex)
    o = oracle.observables(p, psi)
    assert abs(o["O"] - a / 4) < 1e-12 and abs(o["B"] - 0.5) < 1e-12
    alpha = p["Nat"] * p["eta"] * (a / 4) / (p["dc"] - p["U0"] / 2 + 1j * p["kappa"])
    assert abs(complex(o["alpha_re"], o["alpha_im"]) - alpha) < 1e-12


def test_cavity_symmetric_density_has_no_field_and_keeps_norm():
    """A density invariant under x -> x + pi/kc has O = 0, hence alpha = 0; the
    real-time cavity step is unitary, so the norm is kept."""
    p = cavity_params(n=32, eta=2.0)
    x, y = grid(p)
    psi = (np.exp(-y ** 2 / 2) * (1 + 0.3 * np.cos(2 * p["kc"] * x))).astype(complex)
    psi /= np.sqrt(np.sum(abs(psi) ** 2) * (8.0 / 32) ** 2)
    o = oracle.observables(p, psi)
    assert abs(o["O"]) < 1e-14 and abs(complex(o["alpha_re"], o["alpha_im"])) < 1e-13
    noisy = gi.gaussian_state(32, 32, 8.0, 8.0, 1.2, 1e-2, seed=9)
    out, al = oracle.evolve(p, noisy, 200, 1e-3, imag=False)
    assert abs(oracle.observables(p, out)["norm"] - 1.0) < 1e-12
    assert al != 0


def test_cavity_potential_terms_at_lattice_points():
    """Eqs. (11)-(13) at x = y = 0 (all cosines 1) and at x = pi/(2 kc) (cos kc x = 0)."""
    p = cavity_params(n=16, L=8.0, eta=1.5, wx=0.0, wy=0.0)
    alpha = 0.3 - 0.2j
    V = oracle.potential(p, 0.0, alpha)
    i0 = 8                                             # x_8 = 0 on a 16-point box of 8
    vp = p["eta"] ** 2 / p["U0"]
    assert abs(V[i0, i0] - (vp + p["U0"] * abs(alpha) ** 2 + 2 * p["eta"] * alpha.real)) < 1e-12
    i1 = 8 + 1                                         # x = 0.5 = pi/(2 kc) for kc = pi
    assert abs(V[i0, i1] - vp) < 1e-12


# ------------------------------------------------------------ momentum populations (Sec. 5.2)
def test_momentum_populations_of_plane_wave_superpositions():
    """sum_n c_n exp(2 i n k y) times any x envelope has populations |c_n|^2 / sum |c|^2."""
    L, k = 2 * np.pi, 2.0
    x, y = gi.grid_axis(32, L), gi.grid_axis(64, L)
    c = {-2: 0.3, -1: 0.5j, 0: 1.0, 1: -0.4, 3: 0.2}
    psi = sum(v * np.exp(2j * n * k * y)[:, None] for n, v in c.items()) * np.exp(-x ** 2)[None, :]
    p = base(32, L)
    p["ny"] = 64
    got = oracle.momentum_populations(p, psi, 1, k, 3)
    w = np.array([abs(c.get(n, 0.0)) ** 2 for n in range(-3, 4)])
    assert np.max(np.abs(got - w / w.sum())) < 1e-12
    # along x the same state has everything in n = 0 (the x envelope is narrow in k only
    # up to its own width, so use a wide window)
    assert oracle.momentum_populations(p, psi, 0, 50.0, 1)[1] > 1 - 1e-12


def test_momentum_populations_raman_nath_flash():
    L, k, V0, t = 2 * np.pi, 1.0, 100.0, 0.02
    p = base(8, L, lat_V0y=V0, lat_ky=k)
    p["ny"] = 64
    out, _ = oracle.evolve(p, gi.uniform_state(8, 64, L, L), 200, t / 200, imag=False)
    got = oracle.momentum_populations(p, out, 1, k, 3)
    assert np.max(np.abs(got - lattice_populations(out, p, 3))) < 1e-12
    rn = scipy.special.jv(np.arange(-3, 4), V0 * t / 2) ** 2
    assert np.max(np.abs(got - rn)) < 2e-3


# ------------------------------------------------------------ cavity probe (Sec. 5.4)
def test_probe_alone_gives_the_driven_cavity_field():
    """eta = 0: the field is only the probe's, Omega exp(i(Dp t + phi)) / (Delta_c - U0 B + i kappa),
    with B the density overlap of the state (direct quadrature here)."""
    p = cavity_params(eta=0.0, probe_omega=0.3, probe_delta=7.0, probe_phi=0.4)
    psi = gi.gaussian_state(32, 32, p["Lx"], p["Ly"], 1.0, 1e-2, seed=31, checker=0.2, kc=p["kc"])
    t = 0.123
    o = oracle.observables(p, psi, t=t)
    x, y = gi.grid_axis(32, p["Lx"]), gi.grid_axis(32, p["Ly"])
    d = np.abs(psi) ** 2
    B = np.sum(np.cos(p["kc"] * x)[None, :] ** 2 * d) / np.sum(d)
    want = 0.3 * np.exp(1j * (7.0 * t + 0.4)) / (p["dc"] - p["U0"] * B + 1j * p["kappa"])
    assert abs(complex(o["alpha_re"], o["alpha_im"]) - want) < 1e-14


def test_probe_response_is_linear_for_weak_probes():
    """The change of the field trajectory scales with Omega_c for weak probes."""
    p = cavity_params(eta=1.5)
    psi0 = gi.gaussian_state(32, 32, p["Lx"], p["Ly"], 1.0, 1e-2, seed=32, checker=0.2, kc=p["kc"])
    a0 = oracle.evolve(p, psi0, 60, 1e-3, False)[1]
    d = [oracle.evolve(dict(p, probe_omega=om, probe_delta=5.0, probe_phi=0.2), psi0, 60, 1e-3, False)[1] - a0
         for om in (1e-4, 2e-4)]
    assert abs(d[0]) > 1e-6
    assert abs(d[1] / d[0] - 2.0) < 1e-3


def test_zero_probe_is_the_plain_cavity():
    p = cavity_params(eta=1.5)
    psi0 = gi.gaussian_state(32, 32, p["Lx"], p["Ly"], 1.0, 1e-2, seed=33, checker=0.2, kc=p["kc"])
    a, _ = oracle.evolve(p, psi0, 20, 1e-3, False)
    b, _ = oracle.evolve(dict(p, probe_omega=0.0, probe_delta=5.0, probe_phi=1.0), psi0, 20, 1e-3, False)
    assert np.array_equal(a, b)
