"""Pins of the oracle's discrete adjoint (lattice-depth control, Sec. 5.2).

The gradient of J = E(psi_T) + |<phi|psi_T>|^2 with respect to the control
values comes from a reverse sweep of phase and kinetic adjoints.  It is
checked against central finite differences of the forward oracle (FP64,
h = 1e-4: truncation ~h^2, roundoff ~1e-12), which exercises every term of
the adjoint: the conjugate kinetic phase, both half-phase adjoints with the
nonlinear correction, the terminal adjoint of E and of the overlap, and the
piecewise-linear control weights.
"""
import numpy as np
import pytest

import gpe_inputs as gi
import oracle


def small_case(g=20.0, npts=6, steps=24, dt=1e-3, extra_points=0):
    w = gi.adjoint_control(n=32, L=8.0, steps=steps, dt=dt, npts=npts, g=g, seed=7)
    p = dict(w["params"])
    T = steps * dt
    if extra_points:
        t = np.concatenate([p["ctrl_t"], T * (1.0 + np.arange(1, extra_points + 1))])
        v = np.concatenate([p["ctrl_v"], 3.0 + np.arange(extra_points)])
        p.update(ctrl_t=t, ctrl_v=v)
    psi0 = gi.gaussian_state(32, 32, 8.0, 8.0, 1.2, 1e-2, seed=8, x0=0.3, kx0=1.0)
    return p, psi0, w["phi"](), steps, dt


def objective(p, psi0, phi, steps, dt):
    psi, _ = oracle.evolve(p, psi0, steps, dt, False)
    o = oracle.observables(p, psi, t=steps * dt)
    c = np.vdot(phi, psi) * (p["Lx"] / p["nx"]) * (p["Ly"] / p["ny"])
    return o["energy"] + abs(c) ** 2


@pytest.mark.parametrize("g", [0.0, 20.0])
def test_adjoint_gradient_matches_central_differences(g):
    p, psi0, phi, steps, dt = small_case(g=g)
    J, grad = oracle.adjoint(p, psi0, phi, steps, dt)
    assert abs(J - objective(p, psi0, phi, steps, dt)) < 1e-12 * max(1.0, abs(J))
    h = 1e-4
    for i in range(len(p["ctrl_v"])):
        vp, vm = p["ctrl_v"].copy(), p["ctrl_v"].copy()
        vp[i] += h
        vm[i] -= h
        fd = (objective(dict(p, ctrl_v=vp), psi0, phi, steps, dt)
              - objective(dict(p, ctrl_v=vm), psi0, phi, steps, dt)) / (2 * h)
        assert abs(grad[i] - fd) < 1e-7 + 1e-6 * abs(fd), (i, grad[i], fd)
    assert np.max(np.abs(grad)) > 1e-4                      # the test is not vacuous


def test_adjoint_control_points_after_the_run_get_no_gradient():
    p, psi0, phi, steps, dt = small_case(extra_points=2)
    _, grad = oracle.adjoint(p, psi0, phi, steps, dt)
    assert np.all(grad[-2:] == 0.0)
    assert np.max(np.abs(grad[:-2])) > 1e-4


def test_adjoint_rejects_other_controls():
    p, psi0, phi, steps, dt = small_case()
    with pytest.raises(ValueError):
        oracle.adjoint(dict(p, ctrl_target=2), psi0, phi, steps, dt)
