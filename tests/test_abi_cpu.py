"""CPU-side checks of the C ABI library: it builds for sm_103a, loads without a
GPU, exports every entry point of include/gpe.h and validates arguments that
need no device (no kernel is launched here)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def header_functions():
    src = open(os.path.join(ROOT, "include", "gpe.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(gpe_[a-z0-9_]+)\s*\(", src)))


def test_library_exports_every_declared_entry_point():
    from paper_2404_14401_b300 import gpe as abi
    lib = abi.load()
    names = header_functions()
    assert len(names) >= 15
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) == set(abi.EXPORTS)


def test_workspace_size_rules():
    from paper_2404_14401_b300 import gpe as abi
    assert abi.gpe_workspace_size(128, 128) > 0
    for bad in [(0, 8), (4, 8), (12, 16), (16384, 8), (8, 3)]:
        assert abi.gpe_workspace_size(*bad) == 0
    assert abi.gpe_workspace_size(8192, 8192) < (1 << 21)


def test_create_rejects_bad_arguments_without_touching_the_device():
    from paper_2404_14401_b300 import gpe as abi
    lib = abi.load()
    ctx = ctypes.c_void_p()
    ws = abi.gpe_workspace_size(64, 64)
    cases = [
        (63, 64, 1.0, 1.0, 1.0, 0.0, 256, 256, ws),       # not a power of two
        (64, 64, -1.0, 1.0, 1.0, 0.0, 256, 256, ws),      # negative box
        (64, 64, 1.0, 1.0, 0.0, 0.0, 256, 256, ws),       # m = 0
        (64, 64, 1.0, 1.0, 1.0, 0.0, 0, 256, ws),         # null psi
        (64, 64, 1.0, 1.0, 1.0, 0.0, 264, 256, ws),       # psi not 16-byte aligned
        (64, 64, 1.0, 1.0, 1.0, 0.0, 256, 128, ws),       # workspace not 256-byte aligned
    ]
    for nx, ny, Lx, Ly, m, g, p, w, n in cases:
        s = lib.gpe_create(nx, ny, Lx, Ly, m, g, ctypes.c_void_p(p), ctypes.c_void_p(w), n, None,
                           ctypes.byref(ctx))
        assert s == abi.GPE_EINVAL and not ctx.value
    s = lib.gpe_create(64, 64, 1.0, 1.0, 1.0, 0.0, ctypes.c_void_p(256), ctypes.c_void_p(256), ws - 1, None,
                       ctypes.byref(ctx))
    assert s == abi.GPE_ENOMEM


def test_status_strings():
    from paper_2404_14401_b300 import gpe as abi
    assert abi.status_string(abi.GPE_ETIMEOUT) == "GPE_ETIMEOUT"
    assert abi.status_string(abi.GPE_OK) == "GPE_OK"


def test_null_context_calls_fail_cleanly():
    from paper_2404_14401_b300 import gpe as abi
    lib = abi.load()
    assert lib.gpe_step(None, 1, 0.1, 0) == abi.GPE_EINVAL
    assert lib.gpe_sync(None) == abi.GPE_EINVAL
    assert lib.gpe_last_error(None) == b"null context"


def test_bounds_check_build_compiles_and_exports_the_same_entry_points():
    """The debug bounds-check build (-DGPE_DEBUG_BOUNDS=1: kernels check their
    global indices and shared-memory regions and latch GPE_EBOUNDS instead of
    making an out-of-bounds access) builds for sm_103a and exports the same
    C ABI as the normal library."""
    from paper_2404_14401_b300 import build
    from paper_2404_14401_b300 import gpe as abi
    path = build.build(debug=True)
    assert path == build.DEBUG_LIB and os.path.exists(path)
    lib = ctypes.CDLL(path)
    for n in header_functions():
        assert hasattr(lib, n), n
    lib.gpe_status_string.restype = ctypes.c_char_p
    assert lib.gpe_status_string(abi.GPE_EBOUNDS) == b"GPE_EBOUNDS"
    assert abi.status_string(abi.GPE_EBOUNDS) == "GPE_EBOUNDS"


def test_adjoint_workspace_layout():
    """The adjoint workspace sizes include/gpe.h states, without a GPU:
    checkpointed, ceil(n/S) + S + 3 copies of psi (S + 1 more on 512^2 grids,
    the second segment buffer) plus 2n + 1 doubles, S = ceil(sqrt(n)); by time
    reversal, 2 copies (psi_T, lambda; 2 more on 512^2 grids, the rotating
    state buffers of the step back), the kinetic factors of -dt along each axis
    and the doubles.  Every region starts on a 256-byte boundary."""
    from paper_2404_14401_b300 import gpe as abi

    def a256(x):
        return (x + 255) // 256 * 256

    for nx, ny, n in ((512, 512, 4000), (256, 256, 4000), (512, 1024, 100), (512, 512, 1), (512, 512, 7),
                      (1024, 1024, 10), (64, 2048, 3)):
        P = a256(8 * nx * ny)
        S = 1
        while S * S < n:
            S += 1
        K = -(-n // S)
        copies = K + S + 3 + (S + 1 if (nx, ny) == (512, 512) else 0)
        g = a256(8 * (2 * n + 1))
        assert abi.gpe_adjoint_workspace_size_ex(nx, ny, n, abi.GPE_ADJ_CHECKPOINT) == copies * P + g, (nx, ny, n)
        assert abi.gpe_adjoint_workspace_size(nx, ny, n) == copies * P + g
        rev = (2 + (2 if (nx, ny) == (512, 512) else 0)) * P + a256(8 * nx) + a256(8 * ny) + g
        assert abi.gpe_adjoint_workspace_size_ex(nx, ny, n, abi.GPE_ADJ_REVERSE) == rev, (nx, ny, n)
    assert abi.gpe_adjoint_workspace_size_ex(512, 512, 0, abi.GPE_ADJ_CHECKPOINT) == 0
    assert abi.gpe_adjoint_workspace_size_ex(500, 512, 10, abi.GPE_ADJ_CHECKPOINT) == 0
