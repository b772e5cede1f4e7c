"""gpe_overlaps_static: the allocation-free reduction, checked on the GPU.

Callers embedded in another program's memory management (which owns every
device allocation) or on paths that must not call cudaMalloc/cudaFree (which
can synchronise the device) cannot hand the library a workspace.  For them
the row-pass density reduction runs with scratch held in a fixed array
inside the library.  This file checks it, through the C ABI, against the
norm and cavity overlaps that gpe_observables computes with a normal
context, on two calls in a row (the second on a different grid, so the
shared scratch must be reset between calls).  It is collected last so that a
run stopping at its first failure has already run every other test.
"""
import numpy as np
import pytest

import gpe_inputs as gi

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def reference_overlaps(nx, ny, Lx, Ly, kc, psi):
    """(norm, O, B) from gpe_observables of a context with a cavity potential."""
    from paper_2404_14401_b300 import Simulation
    p = gi.potential_defaults()
    p.update(nx=nx, ny=ny, Lx=Lx, Ly=Ly, m=1.0, g=0.0, cavity=1, eta=1.0, U0=-0.5, dc=-2.0, kappa=1.0,
             kc=kc, pump_lattice=0)
    s = Simulation(nx, ny, Lx, Ly, 1.0, 0.0)
    s.set_potential(p)
    s.set_psi(psi)
    o = s.observables()
    return o["norm"], o["O"], o["B"]


def check_against_context_path(nx, ny, Lx, Ly, seed):
    from paper_2404_14401_b300 import gpe as abi
    stream = torch.cuda.current_stream().cuda_stream
    kc = 2 * np.pi
    psi = gi.gaussian_state(nx, ny, Lx, Ly, 1.5, 1e-2, seed=seed, checker=0.3, kc=kc).astype(np.complex64)
    dev = torch.from_numpy(psi).cuda()
    torch.cuda.synchronize()
    norm, O, B = abi.gpe_overlaps_static(dev.data_ptr(), nx, ny, Lx, Ly, kc, stream)
    rn, rO, rB = reference_overlaps(nx, ny, Lx, Ly, kc, psi)
    assert abs(rO) > 1e-2                                  # the checkerboard makes O non-trivial
    assert abs(norm - rn) < 1e-6
    assert abs(O - rO) < 1e-5 * abs(rO)
    assert abs(B - rB) < 1e-5 * abs(rB)


def test_static_scratch_reduction_matches_context_path_twice():
    for n, L, seed in ((256, 16.0, 21), (1024, 40.0, 22)):
        check_against_context_path(n, n, L, L, seed)


@pytest.mark.parametrize("nx,ny", [(2048, 2048), (2048, 8), (8, 2048)])
def test_static_scratch_at_the_largest_and_thinnest_grids(nx, ny):
    """2048 x 2048 needs every partial-sum slot of the scratch (1024 CTAs of
    the reducing row pass); the thin grids take the fewest and the most rows
    per CTA."""
    check_against_context_path(nx, ny, 0.02 * nx if nx > 8 else 4.0, 0.02 * ny if ny > 8 else 4.0, nx + ny)


def test_static_scratch_rejects_grids_beyond_its_size():
    from paper_2404_14401_b300 import gpe as abi
    big = torch.zeros((8, 4096), dtype=torch.complex64, device="cuda")
    with pytest.raises(abi.GPEError) as e:
        abi.gpe_overlaps_static(big.data_ptr(), 4096, 8, 1.0, 1.0, 1.0, 0)
    assert e.value.status == abi.GPE_ENOMEM
    with pytest.raises(abi.GPEError) as e:
        abi.gpe_overlaps_static(big.data_ptr(), 12, 8, 1.0, 1.0, 1.0, 0)
    assert e.value.status == abi.GPE_EINVAL
