"""GPU adjoint of the real-time split step against the FP64 oracle adjoint.

The oracle's gradient is pinned to finite differences on the CPU
(test_oracle_adjoint.py); here the library's checkpointed reverse sweep
(ROW_ADJ / COL_ADJ passes, FP32 arithmetic with FP64 reductions) must give
the same J and dJ/dv_i.  Tolerances: J to 1e-6 relative and each gradient
component to 1e-5 of the largest one.  FP32 rounding in the forward states
and in the adjoint passes left 2e-7 and 1.2e-7 on the 64^2 cases of 40 steps
and 6e-9 / 5e-8 at 512^2 after 400 steps (measured on B300).
"""
import numpy as np
import pytest

import gpe_inputs as gi
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def case(n=64, L=8.0, steps=40, dt=1e-3, npts=8, g=20.0):
    w = gi.adjoint_control(n=n, L=L, steps=steps, dt=dt, npts=npts, g=g, seed=9)
    psi0 = gi.gaussian_state(n, n, L, L, 1.2, 1e-2, seed=10, x0=0.3, kx0=1.0)
    return w["params"], psi0, w["phi"](), steps, dt


def run_gpu(p, psi0, phi, steps, dt):
    from paper_2404_14401_b300 import Simulation
    s = Simulation(p["nx"], p["ny"], p["Lx"], p["Ly"], p["m"], p["g"])
    s.set_potential(p)
    s.set_psi(np.asarray(psi0, dtype=np.complex64))
    J, grad = s.adjoint_lattice(phi, steps, dt)
    return s, J, np.array(grad)


def close(J, grad, Jr, gr):
    assert abs(J - Jr) < 1e-6 * abs(Jr), (J, Jr)
    assert np.max(np.abs(grad - gr)) < 1e-5 * np.max(np.abs(gr)), (grad, gr)


@pytest.mark.parametrize("g", [0.0, 20.0])
def test_adjoint_matches_oracle(g):
    p, psi0, phi, steps, dt = case(g=g)
    _, J, grad = run_gpu(p, psi0, phi, steps, dt)
    Jr, gr = oracle.adjoint(p, psi0.astype(np.complex64).astype(np.complex128), phi, steps, dt)
    close(J, grad, Jr, gr)


@pytest.mark.parametrize("steps", [1, 7, 16])
def test_adjoint_segments_of_every_length(steps):
    # 1 step (one segment of one), 7 (segments 3 + 3 + 1), 16 (4 x 4)
    p, psi0, phi, _, dt = case(steps=steps, npts=5)
    _, J, grad = run_gpu(p, psi0, phi, steps, dt)
    Jr, gr = oracle.adjoint(p, psi0.astype(np.complex64).astype(np.complex128), phi, steps, dt)
    close(J, grad, Jr, gr)


def test_adjoint_ragged_grid():
    w = gi.adjoint_control(n=64, L=8.0, steps=20, dt=1e-3, npts=6, g=20.0, seed=11)
    p = dict(w["params"], nx=128, ny=32, Lx=16.0, Ly=4.0)
    psi0 = gi.gaussian_state(128, 32, 16.0, 4.0, 1.0, 1e-2, seed=12)
    phi = gi.target_gaussian(128, 32, 16.0, 4.0)
    _, J, grad = run_gpu(p, psi0, phi, 20, 1e-3)
    Jr, gr = oracle.adjoint(p, psi0.astype(np.complex64).astype(np.complex128), phi, 20, 1e-3)
    close(J, grad, Jr, gr)


def test_adjoint_leaves_the_state_of_single_steps():
    from paper_2404_14401_b300 import Simulation
    p, psi0, phi, steps, dt = case(steps=10)
    s, _, _ = run_gpu(p, psi0, phi, steps, dt)
    ref = Simulation(p["nx"], p["ny"], p["Lx"], p["Ly"], p["m"], p["g"])
    ref.set_potential(p)
    ref.set_psi(np.asarray(psi0, dtype=np.complex64))
    for _ in range(steps):
        ref.step(1, dt, False)
    assert np.array_equal(s.get_psi(), ref.get_psi())
    assert abs(s.t - steps * dt) < 1e-15


def test_autograd_function_returns_the_adjoint_gradient():
    from paper_2404_14401_b300 import Simulation
    from paper_2404_14401_b300.adjoint import lattice_control_objective
    p, psi0, phi, steps, dt = case(steps=12, npts=6)
    sim = Simulation(p["nx"], p["ny"], p["Lx"], p["Ly"], p["m"], p["g"])
    v = torch.tensor(p["ctrl_v"], dtype=torch.float64, requires_grad=True)
    J = lattice_control_objective(v, sim, p, np.asarray(psi0, dtype=np.complex64), phi, steps, dt)
    (3.0 * J).backward()
    _, Jc, gc = run_gpu(p, psi0, phi, steps, dt)
    assert J.detach().item() == Jc
    assert np.allclose(v.grad.numpy(), 3.0 * gc, rtol=0, atol=0)


def test_adjoint_argument_errors():
    from paper_2404_14401_b300 import Simulation, gpe as abi
    p, psi0, phi, steps, dt = case(steps=4)
    s = Simulation(p["nx"], p["ny"], p["Lx"], p["Ly"], p["m"], p["g"])
    s.set_potential(dict(p, ctrl_target=0, ctrl_t=None, ctrl_v=None))
    with pytest.raises(abi.GPEError) as e:
        s.adjoint_lattice(phi, steps, dt)
    assert e.value.status == abi.GPE_EINVAL
    s.set_potential(p)
    f = torch.from_numpy(phi.astype(np.complex64)).cuda()
    small = torch.empty(1024, dtype=torch.uint8, device="cuda")
    with pytest.raises(abi.GPEError) as e:
        abi.gpe_adjoint_lattice(s.ctx, steps, dt, f.data_ptr(), small.data_ptr(), 1024, len(p["ctrl_v"]))
    assert e.value.status == abi.GPE_ENOMEM


def test_adjoint_passes_are_profiled_per_kind():
    from paper_2404_14401_b300 import gpe as abi
    from paper_2404_14401_b300 import Simulation
    p, psi0, phi, steps, dt = case(steps=9)
    s = Simulation(p["nx"], p["ny"], p["Lx"], p["Ly"], p["m"], p["g"])
    s.set_potential(p)
    s.set_psi(np.asarray(psi0, dtype=np.complex64))
    s.profile(True)
    s.adjoint_lattice(phi, steps, dt)
    for kind in (abi.GPE_PASS_ADJ_ROW, abi.GPE_PASS_ADJ_COL):
        ms, n = abi.gpe_profile_read_kind(s.ctx, kind)
        assert n == steps and ms > 0.0
    assert abi.gpe_profile_read_kind(s.ctx, abi.GPE_PASS_ADJ_ROW) == (0.0, 0)     # reset by the read
    with pytest.raises(abi.GPEError):
        abi.gpe_profile_read_kind(s.ctx, 5)


# ------------------------------------------------------------------ reverse sweep without checkpoints
def run_gpu_reverse(p, psi0, phi, steps, dt):
    from paper_2404_14401_b300 import Simulation
    s = Simulation(p["nx"], p["ny"], p["Lx"], p["Ly"], p["m"], p["g"])
    s.set_potential(p)
    s.set_psi(np.asarray(psi0, dtype=np.complex64))
    J, grad = s.adjoint_lattice(phi, steps, dt, reverse=True)
    return s, J, np.array(grad)


@pytest.mark.parametrize("g", [0.0, 20.0])
def test_reverse_sweep_matches_oracle(g):
    """States recovered by stepping backward in time give the oracle's J and
    gradient within the checkpointed tolerances; J, computed before the
    reverse sweep, is the checkpointed call's bit for bit."""
    p, psi0, phi, steps, dt = case(g=g)
    s, J, grad = run_gpu_reverse(p, psi0, phi, steps, dt)
    Jr, gr = oracle.adjoint(p, psi0.astype(np.complex64).astype(np.complex128), phi, steps, dt)
    close(J, grad, Jr, gr)
    _, Jc, _ = run_gpu(p, psi0, phi, steps, dt)
    assert J == Jc
    assert s.sync() == 0


def test_reverse_sweep_leaves_the_state_of_single_steps():
    from paper_2404_14401_b300 import Simulation
    p, psi0, phi, steps, dt = case(steps=10)
    s, _, _ = run_gpu_reverse(p, psi0, phi, steps, dt)
    ref = Simulation(p["nx"], p["ny"], p["Lx"], p["Ly"], p["m"], p["g"])
    ref.set_potential(p)
    ref.set_psi(np.asarray(psi0, dtype=np.complex64))
    for _ in range(steps):
        ref.step(1, dt, False)
    assert np.array_equal(s.get_psi(), ref.get_psi())
    assert abs(s.t - steps * dt) < 1e-15


def test_reverse_sweep_on_the_control_workload_grid():
    """512^2, 400 steps of the adjoint-control workload: the gradient from the
    reverse sweep against the checkpointed one.  The recovered states carry the
    FP32 rounding of up to 400 steps taken back (a few 1e-5 at most if every
    step's rounding added up), so the bound is 1e-3 of the largest component."""
    w = gi.adjoint_control(n=512, L=20.0, steps=400, npts=40, seed=13)
    p, dt = w["params"], w["dt"]
    psi0 = w["psi0"]()
    phi = w["phi"]()
    _, Jc, gc = run_gpu(p, psi0, phi, 400, dt)
    _, J, g = run_gpu_reverse(p, psi0, phi, 400, dt)
    assert J == Jc
    assert np.max(np.abs(g - gc)) < 1e-3 * np.max(np.abs(gc))


def test_reverse_sweep_workspace_and_errors():
    from paper_2404_14401_b300 import Simulation, gpe as abi
    n = 4000
    ck = abi.gpe_adjoint_workspace_size_ex(512, 512, n, abi.GPE_ADJ_CHECKPOINT)
    rv = abi.gpe_adjoint_workspace_size_ex(512, 512, n, abi.GPE_ADJ_REVERSE)
    assert ck == abi.gpe_adjoint_workspace_size(512, 512, n)
    # by time reversal: 4 states on 512^2 (psi_T, lambda and the two extra
    # buffers of the step back) plus small tables, against ~200 checkpointed
    assert rv < 5 * 512 * 512 * 8 < 5 * 512 * 512 * 8 + 64 * 1024 < ck
    assert abi.gpe_adjoint_workspace_size_ex(512, 512, n, 2) == 0
    p, psi0, phi, steps, dt = case(steps=4)
    s = Simulation(p["nx"], p["ny"], p["Lx"], p["Ly"], p["m"], p["g"])
    s.set_potential(p)
    f = torch.from_numpy(phi.astype(np.complex64)).cuda()
    need = abi.gpe_adjoint_workspace_size_ex(p["nx"], p["ny"], steps, abi.GPE_ADJ_REVERSE)
    ws = torch.empty(need, dtype=torch.uint8, device="cuda")
    with pytest.raises(abi.GPEError) as e:
        abi.gpe_adjoint_lattice_ex(s.ctx, steps, dt, 2, f.data_ptr(), ws.data_ptr(), need, len(p["ctrl_v"]))
    assert e.value.status == abi.GPE_EINVAL
    with pytest.raises(abi.GPEError) as e:
        abi.gpe_adjoint_lattice_ex(s.ctx, steps, dt, abi.GPE_ADJ_REVERSE, f.data_ptr(), ws.data_ptr(), need - 256,
                                   len(p["ctrl_v"]))
    assert e.value.status == abi.GPE_ENOMEM


def test_autograd_function_with_the_reverse_sweep():
    from paper_2404_14401_b300 import Simulation
    from paper_2404_14401_b300.adjoint import lattice_control_objective
    p, psi0, phi, steps, dt = case(steps=12, npts=6)
    sim = Simulation(p["nx"], p["ny"], p["Lx"], p["Ly"], p["m"], p["g"])
    v = torch.tensor(p["ctrl_v"], dtype=torch.float64, requires_grad=True)
    J = lattice_control_objective(v, sim, p, np.asarray(psi0, dtype=np.complex64), phi, steps, dt, reverse=True)
    J.backward()
    _, Jc, gc = run_gpu_reverse(p, psi0, phi, steps, dt)
    assert J.detach().item() == Jc
    assert np.array_equal(v.grad.numpy(), gc)
