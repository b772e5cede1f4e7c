"""Probe workloads on the GPU (Sec. 5.2 Kapitza-Dirac flash).

The momentum-population readout (gpe_momentum_populations) is compared with
the oracle's on the same state, and a whole flash (trap + lattice pulse
through the control table, then the readout) with the oracle's flash; with
g = 0 and a short pulse both follow the Raman-Nath Bessel populations.
"""
import numpy as np
import pytest
import scipy.special

import gpe_inputs as gi
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def sim(p, psi):
    from paper_2404_14401_b300 import Simulation
    s = Simulation(p["nx"], p["ny"], p["Lx"], p["Ly"], p["m"], p["g"])
    s.set_potential(p)
    s.set_psi(np.asarray(psi, dtype=np.complex64))
    return s


def test_population_readout_matches_oracle_on_a_given_state():
    w = gi.kapitza_dirac(n=128, L=16.0)
    p = w["params"]
    x, y = gi.grid_axis(128, 16.0), gi.grid_axis(128, 16.0)
    k = w["k"]
    c = {-2: 0.3, -1: 0.5j, 0: 1.0, 1: -0.4}
    psi = (sum(v * np.exp(2j * n * k * y)[:, None] for n, v in c.items())
           * np.exp(-(x ** 2)[None, :] / 4 - (y ** 2)[:, None] / 8)).astype(np.complex64)
    s = sim(p, psi)
    got = s.momentum_populations(1, k, 3)
    ref = oracle.momentum_populations(p, psi.astype(np.complex128), 1, k, 3)
    assert np.max(np.abs(got - ref)) < 1e-6
    assert np.array_equal(s.get_psi(), psi)                       # psi untouched


@pytest.mark.parametrize("g", [0.0, 50.0])
def test_kapitza_dirac_flash_matches_oracle(g):
    w = gi.kapitza_dirac(g=g)
    p, steps, dt, k = w["params"], w["steps"], w["dt"], w["k"]
    psi0 = w["psi0"]()
    s = sim(p, psi0)
    s.step(steps + 20, dt, False)                                 # flash, then 20 steps with the lattice off
    got = s.momentum_populations(1, k, 3)
    ref_psi, _ = oracle.evolve(p, psi0.astype(np.complex64).astype(np.complex128), steps + 20, dt, False)
    ref = oracle.momentum_populations(p, ref_psi, 1, k, 3)
    assert np.max(np.abs(got - ref)) < 1e-5
    if g == 0.0:
        rn = scipy.special.jv(np.arange(-3, 4), p["lat_V0y"] * w["steps"] * dt / 2) ** 2
        assert np.max(np.abs(got - rn)) < 2e-2                     # Raman-Nath, up to kinetic and trap phases


def test_bragg_probe_cavity_field_matches_oracle():
    """On-axis probe (Sec. 5.4): the cavity field alpha(t), sampled every 40
    steps, follows the oracle's; the probe visibly changes it."""
    w = gi.bragg_probe(n=128, L=16.0, steps=400)
    p, dt = w["params"], w["dt"]
    psi0 = w["psi0"]().astype(np.complex64)
    s = sim(p, psi0)
    quiet = sim(dict(p, probe_omega=0.0), psi0)
    ref = psi0.astype(np.complex128)
    t = 0.0
    for _ in range(10):
        s.step(40, dt, False)
        quiet.step(40, dt, False)
        ref, _ = oracle.evolve(p, ref, 40, dt, False, t0=t)
        t += 40 * dt
        got, q = s.observables(), quiet.observables()
        want = oracle.observables(p, ref, t=t)
        a, b = complex(got["alpha_re"], got["alpha_im"]), complex(want["alpha_re"], want["alpha_im"])
        assert abs(a - b) < 1e-5 * abs(b) + 1e-7, (t, a, b)
        assert abs(a - complex(q["alpha_re"], q["alpha_im"])) > 1e-3 * abs(b)
    assert float(np.linalg.norm(s.get_psi() - ref) / np.linalg.norm(ref)) < 1e-5


def test_probed_batch_in_lockstep_matches_single_stepping():
    """A batch of small cavity grids under the probe, stepped by gpe_step_many:
    the probe makes every step's cavity-field update depend on time, so the
    batch must not replay one captured step; each context equals its own
    single-context stepping bit for bit."""
    from paper_2404_14401_b300 import Simulation
    w = gi.bragg_probe(n=64, L=12.0, steps=30)
    p, dt = w["params"], w["dt"]
    psi0 = w["psi0"]().astype(np.complex64)
    etas = (1.0, 1.5, 2.0)
    batch = [sim(dict(p, eta=e), psi0) for e in etas]
    Simulation.step_many(batch, 30, dt)
    for e, s in zip(etas, batch):
        one = sim(dict(p, eta=e), psi0)
        one.step(30, dt, False)
        assert s.sync() == 0
        assert np.array_equal(s.get_psi(), one.get_psi())
