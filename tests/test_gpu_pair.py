"""Pencil-pair column passes (GPE_VARIANT_PAIR_COLS): both columns of a
2-column tile transformed as one packed f32x2 pencil pair, in every mode the
pair form has (T_y; T_y + reductions; T_y + closing phase + reductions),
against the FP64 oracle and against the one-pencil passes.

Tolerances as in test_gpu_parity (state relative L2 1e-4 n / 1000, floor
1e-5; norm drift 1e-6; energy, mu and the cavity observables relative
1e-5).  The pair transform makes the one-pencil transform's roundings; the
kinetic factor and phase may contract their products differently, so the
two forms agree to FP32 rounding (relative 1e-6), not necessarily bit for
bit.
"""
import numpy as np
import pytest

import gpe_inputs as gi
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def sim_for(p, pair):
    from paper_2404_14401_b300 import Simulation
    from paper_2404_14401_b300 import gpe as abi
    s = Simulation(p["nx"], p["ny"], p["Lx"], p["Ly"], p["m"], p["g"])
    s.set_potential(p)
    v = s.variants & ~(abi.GPE_VARIANT_PAIR_COLS | abi.GPE_VARIANT_STREAM_COLS)
    s.variants = v | (abi.GPE_VARIANT_PAIR_COLS if pair else 0)
    return s


def rel_l2(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def state_tol(n):
    return max(1e-5, 1e-4 * n / 1000)


def c64(a):
    return np.asarray(a, dtype=np.complex64)


def box(n):
    return 0.02 * n if n >= 1024 else 10.0


# the narrowest grid (8 columns: 4 tiles), wide and square grids, and every
# column length the pair pass takes
PAIR_SHAPES = [(8, 512), (16, 1024), (64, 2048), (256, 512), (128, 1024), (512, 512), (8, 4096), (8, 8192)]


@pytest.mark.parametrize("nx,ny", PAIR_SHAPES)
def test_pair_columns_real_time_match_oracle(nx, ny):
    w = gi.lattice_real_time(n=64, L=16.0)
    p = dict(w["params"], nx=nx, ny=ny, Lx=box(nx), Ly=box(ny))
    psi0 = gi.gaussian_state(nx, ny, p["Lx"], p["Ly"], 1.5, 1e-3, seed=200 + nx)
    n = 40
    s = sim_for(p, True)
    assert s.variants & 32
    s.set_psi(c64(psi0))
    s.step(n, 5e-4)
    got, obs = s.get_psi(), s.observables()
    assert s.sync() == 0
    ref, _ = oracle.evolve(p, c64(psi0).astype(np.complex128), n, 5e-4, False)
    ro = oracle.observables(p, ref, t=s.t)
    assert rel_l2(got, ref) < state_tol(n)
    assert abs(obs["norm"] - ro["norm"]) < 1e-6
    assert abs(obs["energy"] - ro["energy"]) < 1e-5 * abs(ro["energy"])
    assert abs(obs["mu"] - ro["mu"]) < 1e-5 * abs(ro["mu"])


def test_pair_columns_1000_real_time_steps_hold_the_norm():
    """1000 real-time steps on 64 x 512 (every column pass but the last one
    a pair pass): state within 1e-4 of the oracle, norm drift below 1e-6."""
    w = gi.lattice_real_time(n=64, L=16.0)
    p = dict(w["params"], nx=64, ny=512, Lx=10.0, Ly=10.0)
    psi0 = gi.gaussian_state(64, 512, 10.0, 10.0, 1.5, 1e-3, seed=210)
    s = sim_for(p, True)
    s.set_psi(c64(psi0))
    n0 = s.observables()["norm"]
    s.step(1000, 5e-4)
    got, obs = s.get_psi(), s.observables()
    ref, _ = oracle.evolve(p, c64(psi0).astype(np.complex128), 1000, 5e-4, False)
    assert rel_l2(got, ref) < state_tol(1000)
    assert abs(obs["norm"] - n0) < 1e-6
    assert abs(obs["norm"] - oracle.observables(p, ref)["norm"]) < 1e-6


@pytest.mark.parametrize("nx,ny", [(64, 2048), (2048, 2048), (256, 512), (8, 1024), (16, 4096)])
def test_pair_and_one_pencil_columns_agree(nx, ny):
    """The same 12 real-time steps with and without the pair pass: equal to
    FP32 rounding; the launch count is the same (one column pass per step)."""
    w = gi.lattice_real_time(n=64, L=16.0)
    p = dict(w["params"], nx=nx, ny=ny, Lx=box(nx), Ly=box(ny))
    psi0 = c64(gi.gaussian_state(nx, ny, p["Lx"], p["Ly"], 1.5, 1e-3, seed=220))
    outs, launches = [], []
    for pair in (False, True):
        s = sim_for(p, pair)
        s.set_psi(psi0)
        s.step(12, 5e-4)
        outs.append(s.get_psi())
        launches.append(s.launches)
        assert s.sync() == 0
    assert rel_l2(outs[1], outs[0]) < 1e-6
    assert launches[0] == launches[1]


def test_pair_variant_bits():
    from paper_2404_14401_b300 import gpe as abi
    w = gi.lattice_real_time(n=64, L=16.0)
    s = sim_for(dict(w["params"], nx=64, ny=512, Lx=10.0, Ly=10.0), False)
    v = s.variants
    s.variants = v | abi.GPE_VARIANT_PAIR_COLS
    assert s.variants == v | 32
    s.variants = v | abi.GPE_VARIANT_PAIR_COLS | abi.GPE_VARIANT_PAIR_ROWS
    assert s.variants == v | 32 | 64
    s.variants = v | abi.GPE_VARIANT_PAIR_COLS
    with pytest.raises(Exception):
        s.variants = 256                      # unknown bit
    with pytest.raises(Exception):
        s.variants = 3 << 3                   # row-tile value 3
    assert s.variants == v | 32




def check_against_oracle(p, psi0, n, dt, imag, cavity=False):
    s = sim_for(p, True)
    s.set_psi(c64(psi0))
    s.step(n, dt, imag)
    got, obs = s.get_psi(), s.observables()
    assert s.sync() == 0
    ref, _ = oracle.evolve(p, c64(psi0).astype(np.complex128), n, dt, imag)
    ro = oracle.observables(p, ref, t=s.t)
    assert rel_l2(got, ref) < state_tol(n)
    assert abs(obs["norm"] - (1.0 if imag else ro["norm"])) < 1e-6
    for k in ("energy", "mu"):
        assert abs(obs[k] - ro[k]) < 1e-5 * abs(ro[k]), k
    if cavity:
        a_gpu, a_ref = complex(obs["alpha_re"], obs["alpha_im"]), complex(ro["alpha_re"], ro["alpha_im"])
        assert abs(a_ref) > 1e-3
        assert abs(a_gpu - a_ref) < 1e-5 * abs(a_ref)
        for k in ("O", "B"):
            assert abs(obs[k] - ro[k]) < 1e-5 * abs(ro[k]), k


@pytest.mark.parametrize("nx,ny", [(16, 2048), (64, 512), (32, 1024), (8, 4096)])
def test_pair_columns_imaginary_time_match_oracle(nx, ny):
    """Imaginary time: every column pass applies the closing half phase and
    reduces the norm (the pair form of T_y + phase + reductions)."""
    w = gi.harmonic_trap(n=64, L=10.0, g=100.0)
    p = dict(w["params"], nx=nx, ny=ny, Lx=10.0, Ly=box(ny))
    check_against_oracle(p, gi.gaussian_state(nx, ny, 10.0, p["Ly"], 1.5, 1e-3, seed=250 + ny), 40, 2e-3, True)


@pytest.mark.parametrize("nx,ny", [(16, 2048), (64, 512), (8, 4096)])
def test_pair_columns_cavity_real_time_match_oracle(nx, ny):
    """Real time with the self-consistent cavity: every column pass reduces
    the norm and the overlaps O, B for the next alpha (T_y + reductions)."""
    w = gi.cavity_ramp(n=64, L=16.0, steps=40, dt=2e-4)
    p = dict(w["params"], nx=nx, ny=ny, Lx=16.0, Ly=box(ny), ctrl_v=np.array([1.0, 4.0]))
    psi0 = gi.gaussian_state(nx, ny, 16.0, p["Ly"], 1.5, 1e-2, seed=260 + ny, checker=0.3, kc=p["kc"])
    check_against_oracle(p, psi0, 40, 2e-4, False, cavity=True)


@pytest.mark.parametrize("nx,ny", [(16, 2048), (64, 512)])
def test_pair_columns_cavity_imaginary_time_match_oracle(nx, ny):
    """Imaginary time with the cavity: closing phase, norm and overlaps in
    the column pass, the alpha of the result for the row pass after it."""
    w = gi.cavity_ramp(n=64, L=16.0, steps=40, dt=1e-3)
    p = dict(w["params"], nx=nx, ny=ny, Lx=16.0, Ly=box(ny), ctrl_target=0, eta=10.0, ctrl_t=None, ctrl_v=None)
    psi0 = gi.gaussian_state(nx, ny, 16.0, p["Ly"], 1.5, 1e-2, seed=270 + ny, checker=0.3, kc=p["kc"])
    check_against_oracle(p, psi0, 40, 1e-3, True, cavity=True)


def test_pair_columns_lattice_control_and_potential_array():
    """Time-dependent lattice depth and a static potential array read by the
    closing phase of the last column pass (two columns of the array per tile)."""
    nx, ny = 16, 2048
    p = gi.potential_defaults()
    t, v = gi.control_points(seed=280, n=200, T=0.2, lo=0.0, hi=8.0)
    Varr = (0.5 * gi.normal(281, nx * ny).reshape(ny, nx)).astype(np.float32).astype(np.float64)
    p.update(nx=nx, ny=ny, Lx=10.0, Ly=40.0, m=1.0, g=500.0, wx=1.0, wy=1.0, lat_V0x=1.0, lat_V0y=1.0,
             lat_kx=2 * np.pi, lat_ky=2 * np.pi, ctrl_target=1, ctrl_t=t, ctrl_v=v, Varr=Varr, V_scale=0.7)
    check_against_oracle(p, gi.gaussian_state(nx, ny, 10.0, 40.0, 1.5, 1e-3, seed=282), 60, 5e-4, False)


@pytest.mark.parametrize("imag,cavity", [(True, False), (False, True), (True, True)])
def test_pair_and_one_pencil_reducing_columns_agree(imag, cavity):
    """64 x 2048: the same 12 steps with and without the pair form, in the
    modes whose column pass reduces: states equal to FP32 rounding, norm,
    energy and alpha relative 1e-6."""
    if cavity:
        w = gi.cavity_ramp(n=64, L=16.0, steps=12, dt=1e-3 if imag else 2e-4)
        p = dict(w["params"], nx=64, ny=2048, Lx=16.0, Ly=40.0, ctrl_target=0, eta=6.0, ctrl_t=None, ctrl_v=None)
    else:
        w = gi.harmonic_trap(n=64, L=10.0, g=100.0)
        p = dict(w["params"], nx=64, ny=2048, Lx=10.0, Ly=40.0)
    psi0 = c64(gi.gaussian_state(64, 2048, p["Lx"], p["Ly"], 1.5, 1e-2, seed=290, checker=0.3, kc=2 * np.pi))
    dt = 1e-3 if imag else 2e-4
    outs, obs = [], []
    for pair in (False, True):
        s = sim_for(p, pair)
        s.set_psi(psi0)
        s.step(12, dt, imag)
        outs.append(s.get_psi())
        obs.append(s.observables())
        assert s.sync() == 0
    assert rel_l2(outs[1], outs[0]) < 1e-6
    for k in ("norm", "energy") + (("alpha_re", "O", "B") if cavity else ()):
        assert abs(obs[1][k] - obs[0][k]) < 1e-6 * abs(obs[0][k]), k


# ------------------------------------------------------------------ row pairs
def sim_rows(p, pair):
    from paper_2404_14401_b300 import gpe as abi
    s = sim_for(p, p["ny"] >= 2048)
    s.variants = (s.variants & ~abi.GPE_VARIANT_PAIR_ROWS) | (abi.GPE_VARIANT_PAIR_ROWS if pair else 0)
    return s


@pytest.mark.parametrize("nx,ny", [(512, 16), (1024, 8), (2048, 8), (4096, 16), (8192, 8), (2048, 64), (512, 512)])
def test_pair_rows_real_time_match_oracle(nx, ny):
    w = gi.lattice_real_time(n=64, L=16.0)
    p = dict(w["params"], nx=nx, ny=ny, Lx=box(nx), Ly=box(ny))
    psi0 = gi.gaussian_state(nx, ny, p["Lx"], p["Ly"], 1.5, 1e-3, seed=310 + ny)
    s = sim_rows(p, True)
    assert s.variants & 64
    s.set_psi(c64(psi0))
    s.step(40, 5e-4)
    got, obs = s.get_psi(), s.observables()
    assert s.sync() == 0
    ref, _ = oracle.evolve(p, c64(psi0).astype(np.complex128), 40, 5e-4, False)
    ro = oracle.observables(p, ref, t=s.t)
    assert rel_l2(got, ref) < state_tol(40)
    assert abs(obs["norm"] - ro["norm"]) < 1e-6
    for k in ("energy", "mu"):
        assert abs(obs[k] - ro[k]) < 1e-5 * abs(ro[k]), k


def check_rows_oracle(p, psi0, n, dt, imag, cavity=False):
    s = sim_rows(p, True)
    s.set_psi(c64(psi0))
    s.step(n, dt, imag)
    got, obs = s.get_psi(), s.observables()
    assert s.sync() == 0
    ref, _ = oracle.evolve(p, c64(psi0).astype(np.complex128), n, dt, imag)
    ro = oracle.observables(p, ref, t=s.t)
    assert rel_l2(got, ref) < state_tol(n)
    assert abs(obs["norm"] - (1.0 if imag else ro["norm"])) < 1e-6
    for k in ("energy", "mu"):
        assert abs(obs[k] - ro[k]) < 1e-5 * abs(ro[k]), k
    if cavity:
        a_gpu, a_ref = complex(obs["alpha_re"], obs["alpha_im"]), complex(ro["alpha_re"], ro["alpha_im"])
        assert abs(a_ref) > 1e-3
        assert abs(a_gpu - a_ref) < 1e-5 * abs(a_ref)


@pytest.mark.parametrize("nx", [512, 1024, 2048, 4096])
def test_pair_rows_imaginary_time_match_oracle(nx):
    """Imaginary time: the row pass scales by 1/sqrt(norm) of the previous
    column pass before its phase."""
    w = gi.harmonic_trap(n=64, L=10.0, g=100.0)
    p = dict(w["params"], nx=nx, ny=16, Lx=box(nx), Ly=10.0)
    check_rows_oracle(p, gi.gaussian_state(nx, 16, p["Lx"], 10.0, 1.5, 1e-3, seed=320), 40, 2e-3, True)


@pytest.mark.parametrize("nx", [512, 1024, 2048, 4096])
def test_pair_rows_cavity_real_time_match_oracle(nx):
    """The V_c and V_i terms of the row phase differ between the two rows of
    a pair through cos(kc y)."""
    w = gi.cavity_ramp(n=64, L=16.0, steps=40, dt=2e-4)
    p = dict(w["params"], nx=nx, ny=16, Lx=box(nx), Ly=16.0, ctrl_v=np.array([1.0, 4.0]))
    psi0 = gi.gaussian_state(nx, 16, p["Lx"], 16.0, 1.5, 1e-2, seed=330, checker=0.3, kc=p["kc"])
    check_rows_oracle(p, psi0, 40, 2e-4, False, cavity=True)


def test_pair_rows_lattice_control_and_potential_array():
    """Time-dependent lattice depth and a static potential array (the two
    rows of a pair read different array rows)."""
    nx, ny = 4096, 8
    p = gi.potential_defaults()
    t, v = gi.control_points(seed=340, n=200, T=0.2, lo=0.0, hi=8.0)
    Varr = (0.5 * gi.normal(341, nx * ny).reshape(ny, nx)).astype(np.float32).astype(np.float64)
    p.update(nx=nx, ny=ny, Lx=box(nx), Ly=10.0, m=1.0, g=500.0, wx=1.0, wy=1.0, lat_V0x=1.0, lat_V0y=1.0,
             lat_kx=2 * np.pi, lat_ky=2 * np.pi, ctrl_target=1, ctrl_t=t, ctrl_v=v, Varr=Varr, V_scale=0.7)
    check_rows_oracle(p, gi.gaussian_state(nx, ny, p["Lx"], 10.0, 1.5, 1e-3, seed=342), 60, 5e-4, False)


@pytest.mark.parametrize("nx,ny,imag", [(512, 64, True), (1024, 1024, False), (2048, 2048, False), (4096, 64, False),
                                        (4096, 64, True)])
def test_pair_rows_and_default_rows_agree(nx, ny, imag):
    """The same 12 steps with the pair row pass and with the default row
    pass of the length (one-shot at 512 and 1024, grouped at 2048, streaming
    at 4096): equal to FP32 rounding, one row pass per step either way."""
    w = gi.harmonic_trap(n=64, L=10.0, g=100.0) if imag else gi.lattice_real_time(n=64, L=16.0)
    p = dict(w["params"], nx=nx, ny=ny, Lx=box(nx), Ly=box(ny))
    psi0 = c64(gi.gaussian_state(nx, ny, p["Lx"], p["Ly"], 1.5, 1e-3, seed=350))
    outs, launches = [], []
    for pair in (False, True):
        s = sim_rows(p, pair)
        s.set_psi(psi0)
        s.step(12, 2e-3 if imag else 5e-4, imag)
        outs.append(s.get_psi())
        launches.append(s.launches)
        assert s.sync() == 0
    assert rel_l2(outs[1], outs[0]) < 1e-6
    assert launches[0] == launches[1]
