"""GPU parity: the sm_103a kernels (through the C ABI) against the FP64 oracle.

Both sides get the same seeded inputs from gpe_inputs; the GPU receives them
rounded to complex64.  Tolerances come from the FP32 arithmetic of the GPU
path: one forward + inverse FP32 FFT pair has a relative L2 error of a few
1e-7 (~eps32 sqrt(log2 N)); a split step adds the phase and kinetic factors,
each rounded once, so after n steps the state error grows at most linearly,
bounded by 1e-4 after 1000 steps (the propagator's stated tolerance) and
scaled as 1e-4 n / 1000 (floor 1e-5) below that.  Observables are FP64
reductions of FP32 products: relative 1e-5.
"""
import numpy as np
import pytest

import gpe_inputs as gi
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def sim_for(p):
    from paper_2404_14401_b300 import Simulation
    s = Simulation(p["nx"], p["ny"], p["Lx"], p["Ly"], p["m"], p["g"])
    s.set_potential(p)
    return s


def rel_l2(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def state_tol(n):
    return max(1e-5, 1e-4 * n / 1000)


def c64(a):
    return np.asarray(a, dtype=np.complex64)


def rand_state(nx, ny, seed):
    z = gi.normal(seed, 2 * nx * ny).reshape(2, ny, nx)
    return z[0] + 1j * z[1]


# ------------------------------------------------------------------ FFT passes
FFT_SHAPES = [(8, 8), (16, 8), (8, 16), (32, 64), (64, 32), (128, 128), (256, 512), (512, 256),
              (1024, 64), (2048, 32), (4096, 16), (8192, 8), (8, 8192), (16, 4096), (32, 2048),
              (1024, 1024), (2048, 2048)]


@pytest.mark.parametrize("nx,ny", FFT_SHAPES)
def test_fft2_passes_match_oracle(nx, ny):
    p = gi.potential_defaults()
    p.update(nx=nx, ny=ny, Lx=1.0, Ly=1.0, m=1.0, g=0.0)
    s = sim_for(p)
    a = c64(rand_state(nx, ny, nx * 131 + ny))
    s.set_psi(a)
    s.fft2(-1)
    got = s.get_psi()
    ref = oracle.fft2(a.astype(np.complex128), -1)
    assert rel_l2(got, ref) < 1e-6
    assert np.max(np.abs(got - ref)) < 1e-5 * np.max(np.abs(ref))
    s.fft2(+1)
    back = s.get_psi()
    assert rel_l2(back, a) < 1e-6
    assert s.sync() == 0


# ------------------------------------------------------------------ split steps
def run_both(p, psi0, n, dt, imag, t0=0.0, streaming=False):
    s = sim_for(p)
    if streaming:                       # the streaming passes where they apply (the pair passes off)
        from paper_2404_14401_b300 import gpe as abi
        pairs = abi.GPE_VARIANT_PAIR_ROWS | abi.GPE_VARIANT_PAIR_COLS
        s.variants = (s.variants & ~pairs) | abi.GPE_VARIANT_STREAM_ROWS | abi.GPE_VARIANT_STREAM_COLS
    s.set_psi(c64(psi0))
    s.t = t0
    s.step(n, dt, imag)
    got = s.get_psi()
    obs = s.observables()
    ref, alpha = oracle.evolve(p, c64(psi0).astype(np.complex128), n, dt, imag, t0=t0)
    return s, got, obs, ref, alpha


@pytest.mark.parametrize("nx,ny,n", [(64, 64, 1), (64, 64, 2), (64, 64, 100), (128, 64, 100),
                                     (32, 256, 100), (256, 256, 1000)])
def test_real_time_lattice_matches_oracle(nx, ny, n):
    w = gi.lattice_real_time(n=64, L=16.0)
    p = dict(w["params"], nx=nx, ny=ny, Lx=16.0 * nx / 64, Ly=16.0 * ny / 64)
    psi0 = gi.gaussian_state(nx, ny, p["Lx"], p["Ly"], 1.5, 1e-3, seed=1)
    s, got, obs, ref, _ = run_both(p, psi0, n, 5e-4, False)
    assert rel_l2(got, ref) < state_tol(n)
    ro = oracle.observables(p, ref, t=s.t)
    assert abs(obs["norm"] - 1.0) < 1e-6                      # norm drift
    assert abs(obs["norm"] - ro["norm"]) < 1e-6
    assert abs(obs["energy"] - ro["energy"]) < 1e-5 * abs(ro["energy"])
    assert abs(obs["mu"] - ro["mu"]) < 1e-5 * abs(ro["mu"])


def component_bounds(p, ref, got):
    """Bounds on |E_kin(got) - E_kin(ref)| and |E_pot(got) - E_pot(ref)| that
    follow from the state difference d = got - ref alone (Cauchy-Schwarz):
    for a Hermitian operator A, <got|A|got> - <ref|A|ref> = 2 Re <ref|A|d> +
    <d|A|d>, so its size is at most 2 ||A ref|| ||d|| + ||A|| ||d||^2, with
    A = k^2/2m (spectral) or A = V (pointwise) and norms with the cell area.
    Added: the GPU's own rounding of the sum itself, at most 2e-6 of the value
    (an FP32 transform of relative error <= 1e-6, test_fft2_passes_match_oracle,
    squared; FP64 accumulation)."""
    nx, ny, Lx, Ly, m = p["nx"], p["ny"], p["Lx"], p["Ly"], p["m"]
    da = (Lx / nx) * (Ly / ny)
    kx = 2 * np.pi * np.fft.fftfreq(nx, Lx / nx)[None, :]
    ky = 2 * np.pi * np.fft.fftfreq(ny, Ly / ny)[:, None]
    t = (kx ** 2 + ky ** 2) / (2 * m)
    d = got.astype(np.complex128) - ref
    nd = np.sqrt(np.sum(np.abs(d) ** 2) * da)
    Tref = np.fft.ifft2(t * np.fft.fft2(ref))
    V = oracle.potential(p)
    out = {}
    for k, Aref, Anorm in (("ekin", Tref, t.max()), ("epot", V * ref, np.abs(V).max())):
        out[k] = 2 * np.sqrt(np.sum(np.abs(Aref) ** 2) * da) * nd + Anorm * nd ** 2
    return out


@pytest.mark.parametrize("g", [0.0, 100.0])
def test_imaginary_time_harmonic_trap_matches_oracle(g):
    """128^2, box 20, V = r^2/2, imaginary dt = 1e-3 for 2000 steps (Sec. 4.1 / 5.1).
    E and mu are stationary at the fixed point (second order in the state
    error) and are held to 1e-5; E_kin and E_pot alone are first order in it,
    so each is held to the bound that the measured state difference implies
    (component_bounds), and to 1e-4 outright."""
    w = gi.harmonic_trap(g=g)
    p = w["params"]
    s, got, obs, ref, _ = run_both(p, w["psi0"](), 2000, w["dt"], True)
    assert rel_l2(got, ref) < 1e-4
    ro = oracle.observables(p, ref, t=s.t)
    for k in ("energy", "mu"):
        assert abs(obs[k] - ro[k]) < 1e-5 * abs(ro[k]), k
    cb = component_bounds(p, ref, got)
    for k in ("ekin", "epot"):
        assert abs(obs[k] - ro[k]) < cb[k] + 2e-6 * abs(ro[k]), (k, abs(obs[k] - ro[k]), cb[k])
        assert abs(obs[k] - ro[k]) < 1e-4 * abs(ro[k]), k
    assert abs(obs["norm"] - 1.0) < 1e-6
    if g == 0.0:
        assert abs(obs["energy"] - 1.0) < 2e-4                # closed form E = 1


def test_imaginary_then_real_time_switches_kinetic_factors():
    w = gi.harmonic_trap(n=64, L=16.0, g=50.0)
    p = w["params"]
    psi0 = w["psi0"]()
    s = sim_for(p)
    s.set_psi(c64(psi0))
    s.step(300, 2e-3, True)
    s.step(200, 1e-3, False)
    ref, _ = oracle.evolve(p, c64(psi0).astype(np.complex128), 300, 2e-3, True)
    ref, _ = oracle.evolve(p, ref, 200, 1e-3, False, t0=0.6)
    assert rel_l2(s.get_psi(), ref) < state_tol(500)


def cavity_close(obs, ro):
    """O, B and alpha (FP64 sums of FP32 products, alpha formed in FP64):
    relative 1e-5, the bound stated for the observables."""
    a_gpu = complex(obs["alpha_re"], obs["alpha_im"])
    a_ref = complex(ro["alpha_re"], ro["alpha_im"])
    assert abs(obs["O"] - ro["O"]) < 1e-5 * abs(ro["O"])
    assert abs(obs["B"] - ro["B"]) < 1e-5 * abs(ro["B"])
    assert abs(a_gpu - a_ref) < 1e-5 * abs(a_ref)


def test_cavity_ramp_matches_oracle():
    """Self-consistent cavity (Sec. 5.3) with eta ramped in time, from a density
    with a seeded checkerboard modulation so that alpha is of order one."""
    w = gi.cavity_ramp(n=64, L=16.0, steps=400, dt=2e-4)
    p = w["params"]
    p["ctrl_v"] = np.array([1.0, 4.0])
    psi0 = gi.gaussian_state(64, 64, 16.0, 16.0, 1.5, 1e-2, seed=2, checker=0.3, kc=p["kc"])
    s, got, obs, ref, alpha = run_both(p, psi0, 400, 2e-4, False)
    assert rel_l2(got, ref) < state_tol(400)
    ro = oracle.observables(p, ref, t=s.t)
    assert abs(complex(ro["alpha_re"], ro["alpha_im"])) > 0.05
    cavity_close(obs, ro)
    assert abs(obs["norm"] - 1.0) < 1e-6


def test_cavity_imaginary_time_matches_oracle():
    w = gi.cavity_ramp(n=64, L=16.0, steps=300, dt=1e-3)
    p = dict(w["params"], ctrl_target=0, eta=10.0, ctrl_t=None, ctrl_v=None)   # organised phase
    psi0 = gi.gaussian_state(64, 64, 16.0, 16.0, 1.5, 1e-2, seed=3, checker=0.3, kc=p["kc"])
    s, got, obs, ref, _ = run_both(p, psi0, 300, 1e-3, True)
    assert rel_l2(got, ref) < 1e-4
    ro = oracle.observables(p, ref, t=s.t)
    cavity_close(obs, ro)
    assert abs(obs["energy"] - ro["energy"]) < 1e-5 * abs(ro["energy"])


def test_time_dependent_lattice_control_and_potential_array():
    """V0(t) from 200 seeded piecewise-linear control points (the adjoint-control
    workload's potential) plus a static array term, real time."""
    n = 64
    p = gi.potential_defaults()
    t, v = gi.control_points(seed=4, n=200, T=0.2, lo=0.0, hi=8.0)
    Varr = (0.5 * gi.normal(7, n * n).reshape(n, n)).astype(np.float32).astype(np.float64)
    p.update(nx=n, ny=n, Lx=16.0, Ly=16.0, m=1.0, g=500.0, wx=1.0, wy=1.0, lat_V0x=1.0, lat_V0y=1.0,
             lat_kx=2 * np.pi, lat_ky=2 * np.pi, ctrl_target=1, ctrl_t=t, ctrl_v=v, Varr=Varr, V_scale=0.7)
    psi0 = gi.gaussian_state(n, n, 16.0, 16.0, 1.5, 1e-3, seed=4)
    s, got, obs, ref, _ = run_both(p, psi0, 400, 5e-4, False)
    assert rel_l2(got, ref) < state_tol(400)


def test_observables_of_a_given_state():
    w = gi.lattice_real_time(n=128, L=20.0)
    p = w["params"]
    psi = gi.gaussian_state(128, 128, 20.0, 20.0, 1.2, 5e-2, seed=9, kx0=1.0)
    s = sim_for(p)
    s.set_psi(c64(psi))
    obs = s.observables()
    ro = oracle.observables(p, c64(psi).astype(np.complex128))
    for k in ("norm", "ekin", "epot", "eint", "energy", "mu"):
        assert abs(obs[k] - ro[k]) < 1e-5 * abs(ro[k]), k


def test_runs_are_bitwise_deterministic():
    w = gi.cavity_ramp(n=128, L=16.0, steps=50, dt=2e-4)
    p = w["params"]
    psi0 = c64(gi.gaussian_state(128, 128, 16.0, 16.0, 1.5, 1e-2, seed=5))
    outs = []
    for _ in range(2):
        s = sim_for(p)
        s.set_psi(psi0)
        s.step(50, 2e-4, False)
        outs.append(s.get_psi())
    assert np.array_equal(outs[0], outs[1])


def test_zero_steps_and_bad_arguments():
    from paper_2404_14401_b300 import GPEError
    w = gi.harmonic_trap(n=32, L=10.0)
    s = sim_for(w["params"])
    psi0 = c64(w["psi0"]())
    s.set_psi(psi0)
    s.step(0, 1e-3, False)
    assert np.array_equal(s.get_psi(), psi0)
    for bad in [(1, 0.0), (1, -1e-3), (-1, 1e-3), (1, float("nan"))]:
        with pytest.raises(GPEError):
            s.step(bad[0], bad[1], False)


def test_bounded_wait_times_out_and_context_stays_usable():
    from paper_2404_14401_b300 import gpe as abi
    w = gi.harmonic_trap(n=32, L=10.0)
    s = sim_for(w["params"])
    s.set_psi(c64(w["psi0"]()))
    abi.gpe_debug_timeout_probe(s.ctx, 64)
    assert s.sync() == abi.GPE_ETIMEOUT
    assert s.sync() == abi.GPE_OK                             # latched status was cleared
    s.step(10, 1e-3, True)
    assert abs(s.observables()["norm"] - 1.0) < 1e-6


@pytest.mark.parametrize("spins", [0, 1])
def test_real_pass_waits_run_out_and_reductions_recover(spins):
    """The bounded waits of real passes run out: with limit 0 every TMA wait
    gives up at once, with limit 1 after one poll (so some CTAs may finish and
    others not).  The context latches GPE_ETIMEOUT (limit 0 always), every
    CTA still takes its turn at the reduction counters, and after gpe_sync the
    observables and further steps match the oracle from the state psi then
    holds.  The cavity keeps a reducing pass in every step."""
    from paper_2404_14401_b300 import gpe as abi
    w = gi.cavity_ramp(n=64, L=16.0, steps=40, dt=2e-4)
    p = dict(w["params"], ctrl_target=0, eta=2.0, ctrl_t=None, ctrl_v=None)
    psi0 = c64(gi.gaussian_state(64, 64, 16.0, 16.0, 1.5, 1e-2, seed=64, checker=0.3, kc=p["kc"]))
    s = sim_for(p)
    s.set_psi(psi0)
    assert abi.gpe_get_wait_limit(s.ctx) == 1 << 24
    abi.gpe_set_wait_limit(s.ctx, spins)
    s.step(3, 2e-4)
    st = s.sync()
    assert st in (abi.GPE_OK, abi.GPE_ETIMEOUT)
    if spins == 0:
        assert st == abi.GPE_ETIMEOUT
    assert s.sync() == abi.GPE_OK                              # status and counters cleared
    abi.gpe_set_wait_limit(s.ctx, 1 << 24)
    cur, t0 = s.get_psi(), s.t
    assert np.all(np.isfinite(cur))
    obs = s.observables()
    ro = oracle.observables(p, cur.astype(np.complex128), t=t0)
    for k in ("norm", "energy", "O", "B"):
        assert abs(obs[k] - ro[k]) < 1e-5 * abs(ro[k]), k
    s.step(20, 2e-4)
    assert s.sync() == abi.GPE_OK
    ref, _ = oracle.evolve(p, cur.astype(np.complex128), 20, 2e-4, False, t0=t0)
    assert rel_l2(s.get_psi(), ref) < state_tol(20)


@pytest.mark.parametrize("n", [1024, 2048])
def test_full_size_real_time_lattice_first_100_steps(n):
    """The real-time throughput workload at full size (trap + lattice, g = 500,
    box 40, dt = 5e-4): the first 100 steps element by element against the
    oracle, plus norm and energy drift."""
    w = gi.lattice_real_time(n=n, L=40.0)
    p = w["params"]
    psi0 = w["psi0"]()
    s, got, obs, ref, _ = run_both(p, psi0, 100, w["dt"], False)
    assert rel_l2(got, ref) < state_tol(100)
    ro = oracle.observables(p, ref, t=s.t)
    r0 = oracle.observables(p, c64(psi0).astype(np.complex128))
    assert abs(obs["norm"] - ro["norm"]) < 1e-6
    assert abs(obs["energy"] - ro["energy"]) < 1e-5 * abs(ro["energy"])
    assert abs(obs["energy"] - r0["energy"]) < 1e-3 * abs(r0["energy"])     # conserved to O(dt^2)


@pytest.mark.parametrize("n", [4096, 8192])
def test_grids_larger_than_l2_match_oracle_and_conserve(n):
    """The same workload on grids whose state exceeds the 126 MB L2 (128 MB
    and 512 MB): the first 10 steps element by element against the oracle;
    then on the GPU alone the energy after 100 steps (conserved to O(dt^2),
    bound as at 2048^2) and the norm after 1000 (exact for the unitary step)."""
    w = gi.lattice_real_time(n=n, L=40.0)
    p = w["params"]
    psi0 = c64(w["psi0"]())
    s, got, obs, ref, _ = run_both(p, psi0, 10, w["dt"], False)
    assert rel_l2(got, ref) < state_tol(10)
    del got, ref
    ro = oracle.observables(p, psi0.astype(np.complex128))
    assert abs(obs["norm"] - ro["norm"]) < 1e-6
    s.step(90, w["dt"])
    o = s.observables()
    assert abs(o["energy"] - ro["energy"]) < 1e-3 * abs(ro["energy"])
    s.step(900, w["dt"])
    o = s.observables()
    assert s.sync() == 0
    assert abs(o["norm"] - ro["norm"]) < 1e-6


# ------------------------------------------------------------------ streaming passes
# Axes of 4096 points run the persistent, double-buffered row (nx = 4096) and
# column (ny = 4096) passes by default, 2048-point columns when the autotuner
# picks them; these cases cover their imaginary-time, cavity and real-time
# paths against the oracle and against the one-shot passes.
STREAM_SHAPES = [(4096, 64), (64, 4096), (64, 2048)]


def box(n):
    return 0.02 * n if n >= 1024 else 10.0


@pytest.mark.parametrize("nx,ny", STREAM_SHAPES)
def test_streaming_imaginary_time_matches_oracle(nx, ny):
    w = gi.harmonic_trap(n=64, L=10.0, g=100.0)
    p = dict(w["params"], nx=nx, ny=ny, Lx=box(nx), Ly=box(ny))
    psi0 = gi.gaussian_state(nx, ny, p["Lx"], p["Ly"], 1.5, 1e-3, seed=11)
    s, got, obs, ref, _ = run_both(p, psi0, 40, 2e-3, True, streaming=True)
    assert rel_l2(got, ref) < 1e-5
    ro = oracle.observables(p, ref, t=s.t)
    assert abs(obs["energy"] - ro["energy"]) < 1e-5 * abs(ro["energy"])
    assert abs(obs["norm"] - 1.0) < 1e-6


@pytest.mark.parametrize("nx,ny", STREAM_SHAPES)
def test_streaming_cavity_real_time_matches_oracle(nx, ny):
    w = gi.cavity_ramp(n=64, L=16.0, steps=40, dt=2e-4)
    p = dict(w["params"], nx=nx, ny=ny, Lx=box(nx), Ly=box(ny), ctrl_v=np.array([1.0, 4.0]))
    psi0 = gi.gaussian_state(nx, ny, p["Lx"], p["Ly"], 1.5, 1e-2, seed=12, checker=0.3, kc=p["kc"])
    s, got, obs, ref, _ = run_both(p, psi0, 40, 2e-4, False, streaming=True)
    assert rel_l2(got, ref) < 1e-5
    cavity_close(obs, oracle.observables(p, ref, t=s.t))


@pytest.mark.parametrize("nx,ny", STREAM_SHAPES)
def test_streaming_real_time_matches_oracle(nx, ny):
    w = gi.lattice_real_time(n=64, L=16.0)
    p = dict(w["params"], nx=nx, ny=ny, Lx=box(nx), Ly=box(ny))
    psi0 = gi.gaussian_state(nx, ny, p["Lx"], p["Ly"], 1.5, 1e-3, seed=13)
    s, got, obs, ref, _ = run_both(p, psi0, 30, 5e-4, False, streaming=True)
    assert rel_l2(got, ref) < 1e-5


@pytest.mark.parametrize("nx,ny", STREAM_SHAPES)
def test_streaming_and_one_shot_passes_agree_bitwise(nx, ny, monkeypatch):
    w = gi.lattice_real_time(n=64, L=16.0)
    p = dict(w["params"], nx=nx, ny=ny, Lx=box(nx), Ly=box(ny))
    psi0 = c64(gi.gaussian_state(nx, ny, p["Lx"], p["Ly"], 1.5, 1e-3, seed=14))
    from paper_2404_14401_b300 import gpe as abi
    outs = []
    for env in (None, "1"):
        if env:
            monkeypatch.setenv("GPE_NO_STREAM_PASSES", env)
        s = sim_for(p)
        pairs = abi.GPE_VARIANT_PAIR_ROWS | abi.GPE_VARIANT_PAIR_COLS      # one-pencil passes on both sides
        if not env:
            s.variants = (s.variants & ~pairs) | abi.GPE_VARIANT_STREAM_ROWS | abi.GPE_VARIANT_STREAM_COLS
        else:
            assert s.variants & (abi.GPE_VARIANT_STREAM_ROWS | abi.GPE_VARIANT_STREAM_COLS) == 0
            s.variants = s.variants & ~pairs
        s.set_psi(psi0)
        s.step(10, w["dt"], False)
        outs.append(s.get_psi())
    assert np.array_equal(outs[0], outs[1])



# ------------------------------------------------------------------ grouped row pass
# Rows of 512..2048 points run the grouped persistent row pass (tables in
# shared memory, TMA double buffering per group of warps); it must give
# exactly the one-shot row pass's result.  (512, 4096) gives groups several
# items, so both buffers and the store/reload hand-over are exercised.
@pytest.mark.parametrize("nx,ny,imag", [(512, 16, False), (1024, 8, True), (2048, 8, False),
                                        (2048, 64, True), (512, 4096, False)])
def test_grouped_and_one_shot_row_passes_agree_bitwise(nx, ny, imag):
    from paper_2404_14401_b300 import gpe as abi
    w = gi.harmonic_trap(n=64, L=10.0, g=100.0) if imag else gi.lattice_real_time(n=64, L=16.0)
    p = dict(w["params"], nx=nx, ny=ny, Lx=box(nx), Ly=box(ny))
    psi0 = c64(gi.gaussian_state(nx, ny, p["Lx"], p["Ly"], 1.5, 1e-3, seed=15))
    outs = []
    for grouped in (True, False):
        s = sim_for(p)
        # the column variant stays as it is; the pair row pass (which takes
        # precedence where it is on) is off on both sides
        base = s.variants & ~(abi.GPE_VARIANT_GROUP_ROWS | abi.GPE_VARIANT_PAIR_ROWS)
        s.variants = base | (abi.GPE_VARIANT_GROUP_ROWS if grouped else 0)
        s.set_psi(psi0)
        s.step(10, 2e-3 if imag else w["dt"], imag)
        outs.append(s.get_psi())
    assert np.array_equal(outs[0], outs[1])


def test_default_row_variants_follow_the_row_length():
    from paper_2404_14401_b300 import gpe as abi
    w = gi.lattice_real_time(n=64, L=16.0)
    for nx in (256, 512, 1024, 2048, 4096):
        s = sim_for(dict(w["params"], nx=nx, ny=16, Lx=box(nx), Ly=box(16)))
        assert bool(s.variants & abi.GPE_VARIANT_GROUP_ROWS) == (nx == 2048)
        assert bool(s.variants & abi.GPE_VARIANT_STREAM_ROWS)      # applies where row_stream_ok holds
        assert (s.variants >> abi.GPE_VARIANT_ROW_TILE_SHIFT) & 3 == (1 if nx in (512, 1024) else 0)
        assert bool(s.variants & abi.GPE_VARIANT_PAIR_ROWS) == (nx >= 512)
        assert not s.variants & abi.GPE_VARIANT_PAIR_COLS                  # 16-point columns
    for ny in (512, 1024, 2048, 4096, 8192):            # pencil-pair column passes from 1024 points on
        s = sim_for(dict(w["params"], nx=64, ny=ny, Lx=box(64), Ly=box(ny)))
        assert bool(s.variants & abi.GPE_VARIANT_PAIR_COLS) == (ny >= 1024)
        assert not s.variants & abi.GPE_VARIANT_STREAM_COLS



# ------------------------------------------------------------------ lockstep lanes
# gpe_step_many runs the contexts on two library streams.  Each trajectory
# must come out exactly as when stepped alone, including a context whose
# state was set by an asynchronous device copy on its own stream just before
# the call (the lanes must wait for it) and contexts of different sizes,
# modes of imaginary and real time, with and without a cavity.
@pytest.mark.parametrize("imag", [False, True])
def test_lockstep_lanes_match_single_context_stepping(imag):
    import torch
    from paper_2404_14401_b300 import Simulation
    cases = [(256, 256, False), (512, 128, True), (2048, 64, False)]
    dt = 2e-3 if imag else 5e-4
    w = gi.harmonic_trap(n=64, L=10.0, g=100.0) if imag else gi.lattice_real_time(n=64, L=16.0)
    sims, alone, states = [], [], []
    for k, (nx, ny, cav) in enumerate(cases):
        p = dict(w["params"], nx=nx, ny=ny, Lx=box(nx), Ly=box(ny))
        if cav:
            p.update(cavity=1, eta=2.0, U0=-0.5, dc=-2.0, kappa=1.0, kc=2 * np.pi, Nat=1.0, pump_lattice=1)
        psi0 = c64(gi.gaussian_state(nx, ny, p["Lx"], p["Ly"], 1.5, 1e-2, seed=40 + k, checker=0.2,
                                     kc=p.get("kc", 0.0)))
        a = sim_for(p)
        a.set_psi(psi0)
        a.step(20, dt, imag)
        alone.append(a.get_psi())
        s = sim_for(p)
        dev = torch.from_numpy(psi0).cuda()
        torch.cuda.synchronize()
        s.set_psi(dev)                       # asynchronous copy on the context's stream
        sims.append(s)
        states.append(dev)
    Simulation.step_many(sims, 20, dt, imag)
    for s, ref in zip(sims, alone):
        assert np.array_equal(s.get_psi(), ref)


def test_throughput_configuration_in_lockstep_matches_single_stepping_and_oracle():
    """The launch configuration the benchmark times: 8 trajectories of the
    2048^2 real-time lattice workload stepped in lockstep by gpe_step_many
    (one lane each).  Every trajectory equals its single-context stepping bit
    for bit, and one of them matches the oracle element by element."""
    from paper_2404_14401_b300 import Simulation
    w = gi.lattice_real_time(n=2048, L=40.0)
    p, dt, n = w["params"], w["dt"], 10
    base = w["psi0"]()
    states = []
    for b in range(8):
        z = gi.normal(100 + b, 2 * 2048 * 2048).reshape(2, 2048, 2048)
        x = base * (1 + 1e-3 * (z[0] + 1j * z[1]))
        states.append(c64(x / np.sqrt(np.sum(np.abs(x) ** 2) * (40.0 / 2048) ** 2)))
    sims = []
    for x in states:
        s = sim_for(p)
        s.set_psi(x)
        sims.append(s)
    Simulation.step_many(sims, n, dt)
    for s, x in zip(sims, states):
        assert s.sync() == 0
        one = sim_for(p)
        one.set_psi(x)
        one.step(n, dt)
        assert np.array_equal(s.get_psi(), one.get_psi())
    ref, _ = oracle.evolve(p, states[3].astype(np.complex128), n, dt, False)
    assert rel_l2(sims[3].get_psi(), ref) < state_tol(n)


def test_step_many_from_two_host_threads_matches_one_context_alone():
    """Two host threads stepping their own batches of small grids at once (the
    graph-replay path on the shared lanes) give each context's single-stream
    result bit for bit."""
    import threading
    from paper_2404_14401_b300 import Simulation
    w = gi.lattice_real_time(n=64, L=16.0)
    p = dict(w["params"])
    dt = 5e-4

    def batch(seed):
        out = []
        for b in range(4):
            s = sim_for(p)
            s.set_psi(c64(gi.gaussian_state(64, 64, 16.0, 16.0, 1.5, 1e-2, seed=seed + b)))
            out.append(s)
        return out

    batches = [batch(60), batch(70)]
    alone = []
    for seed in (60, 70):
        for s in batch(seed):
            for _ in range(3):
                s.step(12, dt)
            alone.append(s.get_psi())
    errors = []

    def run(sims):
        try:
            for _ in range(3):
                Simulation.step_many(sims, 12, dt)
            for s in sims:
                s.sync()
        except Exception as e:          # reported below, on the main thread
            errors.append(e)

    threads = [threading.Thread(target=run, args=(b,)) for b in batches]
    for t in threads:
        t.start()
    for t in threads:
        t.join()
    assert not errors, errors
    got = [s.get_psi() for b in batches for s in b]
    for g, ref in zip(got, alone):
        assert np.array_equal(g, ref)


def test_context_on_its_own_stream_matches_the_default_stream():
    """A context created on a side stream (its tensors then tell torch's
    allocator about that stream) steps exactly as one on the current stream."""
    from paper_2404_14401_b300 import Simulation
    w = gi.lattice_real_time(n=128, L=20.0)
    p = dict(w["params"])
    psi0 = c64(gi.gaussian_state(128, 128, 20.0, 20.0, 1.5, 1e-2, seed=62))
    a = sim_for(p)
    a.set_psi(psi0)
    a.step(25, w["dt"])
    side = torch.cuda.Stream()
    b = Simulation(128, 128, p["Lx"], p["Ly"], p["m"], p["g"], stream=side)
    b.set_potential(p)
    b.set_psi(psi0)
    b.step(25, w["dt"])
    assert b.sync() == 0
    assert np.array_equal(a.get_psi(), b.get_psi())
    b.close()
    side.synchronize()


def test_step_many_on_contexts_with_their_own_streams_and_uploads():
    """Lockstep steps of contexts on streams of their own, each uploaded from
    pinned host memory on its stream just before the call (each lane starts
    after its own context's upload), then each read back: bit for bit the
    trajectories of the same contexts on the current stream, twice in a row
    (the second call replays the per-lane graphs of the first)."""
    import torch
    from paper_2404_14401_b300 import Simulation
    from paper_2404_14401_b300 import gpe as abi
    w = gi.lattice_real_time(n=64, L=16.0)
    shapes = [(256, 256), (512, 128), (128, 512), (256, 256)]
    ref, got = [], []
    for own in (False, True):
        sims, hosts = [], []
        for k, (nx, ny) in enumerate(shapes):
            p = dict(w["params"], nx=nx, ny=ny, Lx=box(nx), Ly=box(ny))
            s = Simulation(nx, ny, p["Lx"], p["Ly"], p["m"], p["g"], stream=torch.cuda.Stream() if own else None)
            s.set_potential(p)
            hosts.append(torch.from_numpy(c64(gi.gaussian_state(nx, ny, p["Lx"], p["Ly"], 1.5, 1e-3,
                                                                   seed=300 + k))).pin_memory())
            sims.append(s)
        outs = []
        for call in range(2):
            for s, h in zip(sims, hosts):
                abi.gpe_set_psi(s.ctx, h.data_ptr(), False)
            Simulation.step_many(sims, 20, 5e-4)
            outs.append([s.get_psi() for s in sims])
            assert all(s.sync() == 0 for s in sims)
        (got if own else ref).append(outs)
    for a_call, b_call in zip(ref[0], got[0]):
        for a, b in zip(a_call, b_call):
            assert np.array_equal(a, b)
    for a, b in zip(got[0][0], got[0][1]):
        assert np.array_equal(a, b)                     # same upload, same steps


# ------------------------------------------------------------------ graph replay
# With two or more contexts and no time-dependent control, gpe_step_many
# captures the interior lockstep steps of each lane into a CUDA graph and
# replays it.  The result and the launch count must equal those of per-pass
# launches.
@pytest.mark.parametrize("imag", [False, True])
def test_graph_replay_matches_per_pass_launches(imag, monkeypatch):
    from paper_2404_14401_b300 import Simulation
    cases = [(256, 256, False), (128, 512, True), (64, 64, False)]
    dt = 2e-3 if imag else 5e-4
    w = gi.harmonic_trap(n=64, L=10.0, g=100.0) if imag else gi.lattice_real_time(n=64, L=16.0)
    runs = []
    for env in (None, "1"):
        if env:
            monkeypatch.setenv("GPE_NO_GRAPH", env)
        sims = []
        for k, (nx, ny, cav) in enumerate(cases):
            p = dict(w["params"], nx=nx, ny=ny, Lx=box(nx), Ly=box(ny))
            if cav:
                p.update(cavity=1, eta=2.0, U0=-0.5, dc=-2.0, kappa=1.0, kc=2 * np.pi, Nat=1.0, pump_lattice=1)
            s = sim_for(p)
            s.set_psi(c64(gi.gaussian_state(nx, ny, p["Lx"], p["Ly"], 1.5, 1e-2, seed=50 + k, checker=0.2,
                                            kc=p.get("kc", 0.0))))
            sims.append(s)
        l0 = [s.launches for s in sims]
        Simulation.step_many(sims, 12, dt, imag)
        runs.append(([s.get_psi() for s in sims], [s.launches - a for s, a in zip(sims, l0)]))
    for a, b in zip(runs[0][0], runs[1][0]):
        assert np.array_equal(a, b)
    assert runs[0][1] == runs[1][1]


@pytest.mark.parametrize("steps", [4, 11, 30])
def test_one_context_graph_replay_matches_per_pass_launches(steps, monkeypatch):
    """gpe_step on one small grid replays its interior steps from graphs of up
    to 8 steps on a library lane (4 steps: one 2-step graph; 11: one 8-step
    graph and a leftover step; 30: three replays and leftovers); state and
    launch count equal those of per-pass launches on the context's stream."""
    w = gi.cavity_ramp(n=64, L=16.0, steps=400, dt=2e-4)
    p = dict(w["params"], ctrl_target=0, eta=2.0, ctrl_t=None, ctrl_v=None)     # a cavity, no control
    psi0 = c64(gi.gaussian_state(64, 64, 16.0, 16.0, 1.5, 1e-2, seed=63, checker=0.3, kc=p["kc"]))
    runs = []
    for env in (None, "1"):
        if env:
            monkeypatch.setenv("GPE_NO_GRAPH", env)
        s = sim_for(p)
        s.set_psi(psi0)
        l0 = s.launches
        s.step(steps, 2e-4, False)
        assert s.sync() == 0
        runs.append((s.get_psi(), s.launches - l0, s.t))
    assert np.array_equal(runs[0][0], runs[1][0])
    assert runs[0][1] == runs[1][1] and runs[0][2] == runs[1][2]


# ------------------------------------------------------------------ autotuner
@pytest.mark.parametrize("nx,ny", [(2048, 64), (4096, 64), (64, 4096), (128, 128), (64, 2048), (64, 512)])
def test_autotuner_picks_an_applicable_fastest_variant_and_keeps_psi(nx, ny):
    from paper_2404_14401_b300 import gpe as abi
    w = gi.lattice_real_time(n=64, L=16.0)
    p = dict(w["params"], nx=nx, ny=ny, Lx=box(nx), Ly=box(ny))
    s = sim_for(p)
    psi0 = c64(gi.gaussian_state(nx, ny, p["Lx"], p["Ly"], 1.5, 1e-3, seed=60))
    s.set_psi(psi0)
    r = s.tune(w["dt"], reps=3)
    v, ms = r["variants"], {k: (np.nan if x is None else x) for k, x in r["ms"].items()}
    assert np.array_equal(s.get_psi(), psi0)                     # the tuner worked on a copy
    assert s.variants == v
    group_ok = nx in (512, 1024, 2048)
    assert np.isnan(ms["row_grouped"]) != group_ok
    assert np.isnan(ms["row_streaming"]) != (nx == 4096)
    assert np.isnan(ms["col_streaming"]) != (ny in (2048, 4096) and nx >= 16)
    rows = [ms["row_one_shot"], ms["row_grouped"], ms["row_streaming"]]
    best = 0                                    # a persistent variant must be 3% faster
    for k in (1, 2):
        if not np.isnan(rows[k]) and rows[k] < 0.97 * rows[best]:
            best = k
    assert (v & abi.GPE_VARIANT_GROUP_ROWS != 0) == (best == 1)
    assert (v & abi.GPE_VARIANT_STREAM_ROWS != 0) == (best == 2)
    assert (v & abi.GPE_VARIANT_STREAM_COLS != 0) == (not np.isnan(ms["col_streaming"])
                                                       and ms["col_streaming"] < ms["col_one_shot"])
    if ny not in (512, 1024, 2048, 4096, 8192) or v & abi.GPE_VARIANT_STREAM_COLS:
        assert not v & abi.GPE_VARIANT_PAIR_COLS       # no pair form here, or the streaming pass won
    assert r["row_tile"] in (0, 1) and (r["row_tile"] == 0 or best == 0)
    if nx not in (512, 1024, 2048, 4096, 8192) or best != 0:
        assert not v & abi.GPE_VARIANT_PAIR_ROWS       # no pair form here, or a persistent pass won
    if v & abi.GPE_VARIANT_PAIR_ROWS:
        assert r["row_tile"] == 0
    # stepping with the chosen variants still matches the oracle
    s.step(20, w["dt"], False)
    ref, _ = oracle.evolve(p, psi0.astype(np.complex128), 20, w["dt"], False)
    assert rel_l2(s.get_psi(), ref) < 1e-5


@pytest.mark.parametrize("nx,ny,imag", [(256, 256, False), (512, 128, True), (1024, 64, True), (2048, 32, False)])
def test_row_tiles_give_identical_steps(nx, ny, imag):
    """The one-shot row pass with 1/2 and 1/4 of its default rows per CTA
    (more, smaller CTAs) computes every row the same way: bit for bit the
    same trajectory, in real and imaginary time."""
    from paper_2404_14401_b300 import gpe as abi
    w = gi.harmonic_trap(n=64, L=10.0, g=100.0) if imag else gi.lattice_real_time(n=64, L=16.0)
    p = dict(w["params"], nx=nx, ny=ny, Lx=box(nx), Ly=box(ny))
    psi0 = c64(gi.gaussian_state(nx, ny, p["Lx"], p["Ly"], 1.5, 1e-2, seed=61))
    dt = 2e-3 if imag else 5e-4
    out = []
    for tile in (0, 1, 2):
        s = sim_for(p)
        s.variants = tile << abi.GPE_VARIANT_ROW_TILE_SHIFT        # one-shot passes only
        assert s.variants == tile << abi.GPE_VARIANT_ROW_TILE_SHIFT
        s.set_psi(psi0)
        s.step(15, dt, imag)
        assert s.sync() == 0
        out.append(s.get_psi())
    assert np.array_equal(out[0], out[1]) and np.array_equal(out[0], out[2])
    with pytest.raises(abi.GPEError):
        s.variants = 3 << abi.GPE_VARIANT_ROW_TILE_SHIFT
