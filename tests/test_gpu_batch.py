"""The persistent batch (gpe_batch_*): n lockstep steps of many contexts in
one kernel launch, against the FP64 oracle and against gpe_step_many.

Tolerances as in test_gpu_parity: state relative L2 1e-4 * n / 1000 (floor
1e-5), norm drift 1e-6, energies and cavity observables relative 1e-5.  The
batch groups its FP64 reductions by items instead of CTAs, so it equals
gpe_step_many to rounding, not bit for bit.
"""
import numpy as np
import pytest

import gpe_inputs as gi
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def rel_l2(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def state_tol(n):
    return max(1e-5, 1e-4 * n / 1000)


def c64(a):
    return np.asarray(a, dtype=np.complex64)


def sim_for(p):
    from paper_2404_14401_b300 import Simulation
    s = Simulation(p["nx"], p["ny"], p["Lx"], p["Ly"], p["m"], p["g"])
    s.set_potential(p)
    return s


def check_against_oracle(s, p, psi0, n, dt, imag, t0=0.0, cavity=False):
    got, obs = s.get_psi(), s.observables()
    assert s.sync() == 0
    ref, _ = oracle.evolve(p, c64(psi0).astype(np.complex128), n, dt, imag, t0=t0)
    ro = oracle.observables(p, ref, t=s.t)
    assert abs(s.t - (t0 + n * dt)) < 1e-12
    assert rel_l2(got, ref) < state_tol(n)
    assert abs(obs["norm"] - (1.0 if imag else ro["norm"])) < 1e-6
    for k in ("energy", "mu"):
        assert abs(obs[k] - ro[k]) < 1e-5 * abs(ro[k]), k
    if cavity:
        a_gpu = complex(obs["alpha_re"], obs["alpha_im"])
        a_ref = complex(ro["alpha_re"], ro["alpha_im"])
        assert abs(a_ref) > 1e-3
        assert abs(a_gpu - a_ref) < 1e-5 * abs(a_ref)
        for k in ("O", "B"):
            assert abs(obs[k] - ro[k]) < 1e-5 * abs(ro[k]), k


def test_batch_of_sweep_instances_matches_oracle():
    """The phase-diagram sweep's instances of each grid size (256^2, 512^2,
    1024^2, imaginary time with a cavity; of each size the strongest pump),
    50 steps of 1e-3 in one persistent launch."""
    from paper_2404_14401_b300 import Batch
    ws = gi.phase_diagram_sweep()
    picks = [max((w for w in ws if w["params"]["nx"] == n), key=lambda w: w["params"]["eta"])
             for n in (256, 512, 1024)]
    sims, psis = [], []
    for w in picks:
        s = sim_for(w["params"])
        x = c64(w["psi0"]())
        s.set_psi(x)
        sims.append(s)
        psis.append(x)
    b = Batch(sims)
    b.step(25, 1e-3, imag=True)                 # also sets each context's kinetic factors for this dt
    l0 = [s.launches for s in sims]
    b.step(25, 1e-3, imag=True)
    assert [s.launches - a for s, a in zip(sims, l0)] == [1, 0, 0]      # one kernel for the whole batch
    for s, w, x in zip(sims, picks, psis):
        check_against_oracle(s, w["params"], x, 50, 1e-3, True, cavity=True)


@pytest.mark.parametrize("window", ["start of the ramp", "organised end of the ramp"])
def test_batch_cavity_ramp_512_matches_oracle(window):
    """The 512^2 self-consistent cavity ramp (eta(t) from the control table,
    evaluated on the device) for 200 real-time steps of 2e-4 in one launch."""
    from paper_2404_14401_b300 import Batch
    w = gi.cavity_ramp()
    p, dt, n = w["params"], w["dt"], 200
    if window == "start of the ramp":
        t0, psi0 = 0.0, w["psi0"]()
    else:
        t0 = 18000 * dt
        psi0 = gi.gaussian_state(512, 512, 40.0, 40.0, 1.5, 1e-3, seed=2, checker=0.3, kc=p["kc"])
    s = sim_for(p)
    s.set_psi(c64(psi0))
    s.t = t0
    b = Batch([s])
    b.step(n, dt)
    check_against_oracle(s, p, psi0, n, dt, False, t0=t0, cavity=(window != "start of the ramp"))


def test_batch_real_time_lattice_and_harmonic_trap_match_oracle():
    """Real time without a cavity (merged half phases, closing phase in the
    last column pass) on an uneven pair, 2 calls of 60 steps; then the 128^2
    imaginary-time trap workload (g = 100, 2000 steps) as a batch of one."""
    from paper_2404_14401_b300 import Batch
    w = gi.lattice_real_time(n=64, L=16.0)
    sims, ps, psis = [], [], []
    for nx, ny, seed in ((256, 256, 70), (128, 512, 71)):
        p = dict(w["params"], nx=nx, ny=ny, Lx=16.0 * nx / 256, Ly=16.0 * ny / 256)
        x = gi.gaussian_state(nx, ny, p["Lx"], p["Ly"], 1.2, 1e-3, seed=seed)
        s = sim_for(p)
        s.set_psi(c64(x))
        sims.append(s)
        ps.append(p)
        psis.append(x)
    b = Batch(sims)
    b.step(60, 5e-4)
    b.step(60, 5e-4)
    for s, p, x in zip(sims, ps, psis):
        got = s.get_psi()
        ref, _ = oracle.evolve(p, c64(x).astype(np.complex128), 60, 5e-4, False)
        ref, _ = oracle.evolve(p, ref, 60, 5e-4, False, t0=0.03)
        assert rel_l2(got, ref) < state_tol(120)
        assert abs(s.observables()["norm"] - oracle.observables(p, ref)["norm"]) < 1e-6
    h = gi.harmonic_trap(g=100.0)
    s = sim_for(h["params"])
    s.set_psi(c64(h["psi0"]()))
    Batch([s]).step(2000, h["dt"], imag=True)
    check_against_oracle(s, h["params"], h["psi0"](), 2000, h["dt"], True)


@pytest.mark.parametrize("imag", [False, True])
def test_batch_agrees_with_step_many(imag):
    """Same contexts, same steps: the batch and gpe_step_many agree to FP32
    rounding (the reductions are grouped differently)."""
    from paper_2404_14401_b300 import Batch, Simulation
    w = gi.harmonic_trap(n=64, L=10.0, g=100.0) if imag else gi.lattice_real_time(n=64, L=16.0)
    cases = [(256, 256), (512, 128), (64, 1024)]
    dt = 2e-3 if imag else 5e-4
    outs = []
    for use_batch in (False, True):
        sims = []
        for k, (nx, ny) in enumerate(cases):
            p = dict(w["params"], nx=nx, ny=ny, Lx=0.02 * nx if nx >= 512 else 10.0, Ly=0.02 * ny if ny >= 512 else 10.0)
            s = sim_for(p)
            s.set_psi(c64(gi.gaussian_state(nx, ny, p["Lx"], p["Ly"], 1.5, 1e-2, seed=80 + k)))
            sims.append(s)
        if use_batch:
            Batch(sims).step(25, dt, imag)
        else:
            Simulation.step_many(sims, 25, dt, imag)
        outs.append([s.get_psi() for s in sims])
    for a, b in zip(*outs):
        assert rel_l2(b, a) < 1e-6


def test_batch_picks_up_a_changed_potential():
    from paper_2404_14401_b300 import Batch
    w = gi.lattice_real_time(n=128, L=16.0)
    p = dict(w["params"])
    x = c64(gi.gaussian_state(128, 128, 16.0, 16.0, 1.5, 1e-3, seed=90))
    s = sim_for(p)
    s.set_psi(x)
    b = Batch([s])
    b.step(20, 5e-4)
    q = dict(p, lat_V0x=2.0, lat_V0y=7.0, g=500.0)
    s.set_potential(q)
    b.step(20, 5e-4)
    ref, _ = oracle.evolve(p, x.astype(np.complex128), 20, 5e-4, False)
    ref, _ = oracle.evolve(q, ref, 20, 5e-4, False, t0=0.01)
    assert rel_l2(s.get_psi(), ref) < state_tol(40)


def test_batch_wait_limit_runs_out_and_contexts_recover():
    """With a wait limit of 0 an item that has to wait gives up at once: the
    launch ends with GPE_ETIMEOUT latched instead of waiting.  After gpe_sync
    and a normal limit, the next batch step matches the oracle from the state
    psi then holds."""
    from paper_2404_14401_b300 import Batch
    from paper_2404_14401_b300 import gpe as abi
    w = gi.cavity_ramp(n=256, L=16.0, steps=40, dt=2e-4)
    p = dict(w["params"], ctrl_target=0, eta=2.0, ctrl_t=None, ctrl_v=None)
    s = sim_for(p)
    s.set_psi(c64(gi.gaussian_state(256, 256, 16.0, 16.0, 1.5, 1e-2, seed=91, checker=0.3, kc=p["kc"])))
    b = Batch([s])
    abi.gpe_set_wait_limit(s.ctx, 0)
    b.step(5, 2e-4)
    assert s.sync() == abi.GPE_ETIMEOUT
    assert s.sync() == abi.GPE_OK
    abi.gpe_set_wait_limit(s.ctx, 1 << 24)
    cur, t0 = s.get_psi(), s.t
    assert np.all(np.isfinite(cur))
    b.step(20, 2e-4)
    assert s.sync() == abi.GPE_OK
    ref, _ = oracle.evolve(p, cur.astype(np.complex128), 20, 2e-4, False, t0=t0)
    assert rel_l2(s.get_psi(), ref) < state_tol(20)


def test_batch_argument_errors():
    from paper_2404_14401_b300 import Batch, GPEError
    from paper_2404_14401_b300 import gpe as abi
    w = gi.lattice_real_time(n=64, L=16.0)
    small = sim_for(dict(w["params"], nx=32, ny=32))
    with pytest.raises(GPEError):
        Batch([small])                                             # 32 points: below the batch's 64
    a = sim_for(dict(w["params"], nx=64, ny=64))
    thin = sim_for(dict(w["params"], nx=2048, ny=64, Lx=40.0))     # a 2048-point row item needs 2 rows: fine
    a.set_psi(c64(gi.gaussian_state(64, 64, 16.0, 16.0, 1.5, 1e-3, seed=92)))
    thin.set_psi(c64(gi.gaussian_state(2048, 64, 40.0, 16.0, 1.5, 1e-3, seed=93)))
    Batch([a, thin]).step(3, 5e-4)
    assert a.sync() == 0 and thin.sync() == 0
    cav = sim_for(dict(w["params"], nx=64, ny=64, cavity=1, eta=1.0, U0=-0.5, dc=-2.0, kappa=1.0, kc=2 * np.pi))
    with pytest.raises(GPEError):
        Batch([a, cav]).step(2, 5e-4)                              # cavity and no cavity in one batch
    with pytest.raises(GPEError):
        Batch([a, a])                                              # repeated context
    ctxs = [a.ctx]
    need = abi.gpe_batch_workspace_size(ctxs)
    ws = torch.empty(need, dtype=torch.uint8, device="cuda")
    with pytest.raises(GPEError) as e:
        abi.gpe_batch_create(ctxs, ws.data_ptr(), need - 256)
    assert e.value.status == abi.GPE_ENOMEM
