"""GPU runs of the debug bounds-check build (libgpe_debug.so, GPE_DEBUG_BOUNDS=1).

Its kernels check each thread's global row / column index and each CTA's
shared-memory regions against their buffers and latch GPE_EBOUNDS (skipping
the access) instead of making an out-of-bounds access.  A child process
loads that library (GPE_LIBRARY=debug) and runs cases through every pass
kernel family -- the one-shot row and column passes on short pencils (the
32 x 256 and 64 x 64 grids among them), the grouped, streaming, adjoint and
readout passes, the pencil-pair column passes (2048-point columns by
default, 512 by choice), the persistent batch, the cooperative step kernel
and the cooperative adjoint kernels -- each checked against the FP64 oracle
and for a clean device status.
"""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SCRIPT = r'''
import sys
import numpy as np
sys.path.insert(0, sys.argv[1])
import gpe_inputs as gi
import oracle
from paper_2404_14401_b300 import Batch, Simulation
from paper_2404_14401_b300 import gpe as abi
assert abi.lib_path().endswith("libgpe_debug.so")

def sim(p):
    s = Simulation(p["nx"], p["ny"], p["Lx"], p["Ly"], p["m"], p["g"])
    s.set_potential(p)
    return s

def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))

w = gi.lattice_real_time(n=64, L=16.0)
h = gi.harmonic_trap(n=64, L=10.0, g=100.0)
cav = dict(cavity=1, eta=2.0, U0=-0.5, dc=-2.0, kappa=1.0, kc=2 * np.pi, Nat=1.0, pump_lattice=1)
cases = [(32, 256, w, False, {}), (64, 64, w, False, {}), (64, 64, h, True, cav), (8, 8, h, True, {}),
         (2048, 8, w, False, {}), (4096, 64, w, False, {}), (64, 4096, h, True, {}), (128, 128, w, False, cav),
         (8, 2048, w, False, {}), (16, 2048, h, True, cav), (8, 512, h, True, {})]
pair = {(8, 512)}                       # pencil-pair column passes also off their default column length
for nx, ny, ww, imag, extra in cases:
    p = dict(ww["params"], nx=nx, ny=ny, Lx=max(0.02 * nx, 8.0), Ly=max(0.02 * ny, 8.0), **extra)
    x = gi.gaussian_state(nx, ny, p["Lx"], p["Ly"], 1.2, 1e-2, seed=nx + ny, checker=0.2, kc=2 * np.pi)
    x = x.astype(np.complex64)
    s = sim(p)
    if (nx, ny) in pair:
        s.variants = s.variants | abi.GPE_VARIANT_PAIR_COLS
    s.set_psi(x)
    dt = 1e-3 if imag else 5e-4
    s.step(20, dt, imag)
    o = s.observables()
    assert s.sync() == 0, (nx, ny)
    ref, _ = oracle.evolve(p, x.astype(np.complex128), 20, dt, imag)
    assert rel(s.get_psi(), ref) < 1e-5, (nx, ny, rel(s.get_psi(), ref))
    s.fft2(-1)
    s.fft2(+1)
    assert s.sync() == 0
# adjoint and readout passes
a = gi.adjoint_control(n=64, L=16.0, steps=12, npts=5)
s = sim(a["params"])
s.set_psi(a["psi0"]().astype(np.complex64))
J, g = s.adjoint_lattice(a["phi"]().astype(np.complex64), 12, a["dt"])
assert s.sync() == 0 and np.isfinite(J) and np.all(np.isfinite(g))
pops = s.momentum_populations(1, 2 * np.pi, 2)
assert s.sync() == 0 and 0.9 < sum(pops) <= 1.0 + 1e-9
# the persistent batch
sims = []
for nx, ny in ((256, 256), (64, 1024)):
    p = dict(w["params"], nx=nx, ny=ny, Lx=max(0.02 * nx, 8.0), Ly=max(0.02 * ny, 8.0))
    q = sim(p)
    q.set_psi(gi.gaussian_state(nx, ny, p["Lx"], p["Ly"], 1.2, 1e-3, seed=5).astype(np.complex64))
    sims.append(q)
Batch(sims).step(10, 5e-4)
assert all(q.sync() == 0 for q in sims)
# the cooperative step kernel: real time with the cavity on a rectangular grid
p = dict(w["params"], nx=1024, ny=512, Lx=20.48, Ly=10.24, **cav)
x = gi.gaussian_state(1024, 512, 20.48, 10.24, 1.2, 1e-2, seed=7, checker=0.2, kc=2 * np.pi).astype(np.complex64)
s = sim(p)
s.variants = s.variants | abi.GPE_VARIANT_COOP
s.set_psi(x)
l0 = s.launches
s.step(20, 5e-4)
assert s.launches - l0 <= 2 and s.sync() == 0
ref, _ = oracle.evolve(p, x.astype(np.complex128), 20, 5e-4, False)
assert rel(s.get_psi(), ref) < 1e-5, rel(s.get_psi(), ref)
# the cooperative adjoint kernels, checkpointed (states and segment kernels)
# and by time reversal (in-place states kernel, reverse-sweep kernel): 512^2
# (8 elements per thread, the packed pointwise adjoint) and 1024 x 512 (16)
a = gi.adjoint_control(n=512, L=20.0, steps=9, npts=5, seed=3)
for nx, ny, rev in ((512, 512, False), (512, 512, True), (1024, 512, False), (1024, 512, True)):
    p = dict(a["params"], nx=nx, ny=ny, Lx=20.0 * nx / 512, Ly=20.0 * ny / 512)
    x = gi.gaussian_state(nx, ny, p["Lx"], p["Ly"], 1.2, 1e-2, seed=8, x0=0.3, kx0=1.0).astype(np.complex64)
    f = gi.target_gaussian(nx, ny, p["Lx"], p["Ly"])
    s = sim(p)
    s.variants = s.variants | abi.GPE_VARIANT_COOP
    s.set_psi(x)
    l0 = s.launches
    J, g = s.adjoint_lattice(f.astype(np.complex64), 9, a["dt"], reverse=rev)
    assert s.sync() == 0 and s.launches - l0 < 30, (nx, ny, rev, s.launches - l0)
    Jr, gr = oracle.adjoint(p, x.astype(np.complex128), f, 9, a["dt"])
    assert abs(J - Jr) < 1e-6 * abs(Jr), (nx, ny, rev, J, Jr)
    assert np.max(np.abs(np.array(g) - gr)) < 1e-5 * np.max(np.abs(gr)), (nx, ny, rev)
print("debug bounds build: all cases clean")
'''


def test_bounds_check_build_runs_clean_and_matches_oracle():
    from paper_2404_14401_b300 import build
    build.build(debug=True)
    env = dict(os.environ, GPE_LIBRARY="debug")
    r = subprocess.run([sys.executable, "-c", SCRIPT, ROOT], env=env, capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-4000:]
    assert "all cases clean" in r.stdout
