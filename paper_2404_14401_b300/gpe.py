"""Thin ctypes binding of the C ABI in include/gpe.h.

Functions keep the C names and only marshal arguments (torch tensors are
passed as device pointers, streams as handles).  Every step of the split-step
propagator runs in the sm_103a kernels of libgpe.so; there is no Python or
CPU fallback: if the library is missing or fails to load, this module raises.
"""
from __future__ import annotations

import ctypes
import os

from . import build as _build

c_int, c_double, c_size_t, c_void_p, c_char_p = (ctypes.c_int, ctypes.c_double, ctypes.c_size_t,
                                                  ctypes.c_void_p, ctypes.c_char_p)

GPE_OK, GPE_EINVAL, GPE_ENOMEM, GPE_ECUDA, GPE_ETIMEOUT, GPE_ENONFINITE, GPE_EILLCOND, GPE_EBOUNDS = range(8)
GPE_REAL, GPE_IMAG = 0, 1
GPE_CTRL_NONE, GPE_CTRL_LATTICE, GPE_CTRL_ETA = 0, 1, 2

EXPORTS = ("gpe_workspace_size", "gpe_create", "gpe_set_potential", "gpe_step", "gpe_step_many",
           "gpe_observables", "gpe_set_psi", "gpe_get_psi", "gpe_set_time", "gpe_get_time", "gpe_fft2",
           "gpe_sync", "gpe_set_wait_limit", "gpe_get_wait_limit", "gpe_debug_timeout_probe", "gpe_profile", "gpe_profile_read", "gpe_profile_read_kind", "gpe_launch_count",
           "gpe_overlaps_static", "gpe_momentum_populations", "gpe_get_pass_variants", "gpe_set_pass_variants", "gpe_tune",
           "gpe_adjoint_workspace_size", "gpe_adjoint_lattice", "gpe_adjoint_workspace_size_ex",
           "gpe_adjoint_lattice_ex", "gpe_batch_workspace_size", "gpe_batch_create", "gpe_batch_step",
           "gpe_batch_destroy", "gpe_destroy",
           "gpe_last_error", "gpe_status_string")


class gpe_potential(ctypes.Structure):
    _fields_ = [("wx", c_double), ("wy", c_double),
                ("lat_V0x", c_double), ("lat_V0y", c_double), ("lat_kx", c_double), ("lat_ky", c_double),
                ("V", c_void_p), ("V_scale", c_double),
                ("cavity", c_int),
                ("eta", c_double), ("U0", c_double), ("dc", c_double), ("kappa", c_double),
                ("kc", c_double), ("N", c_double),
                ("pump_lattice", c_int), ("ctrl_target", c_int), ("nctrl", c_int),
                ("ctrl_t", ctypes.POINTER(c_double)), ("ctrl_v", ctypes.POINTER(c_double)),
                ("probe_omega", c_double), ("probe_delta", c_double), ("probe_phi", c_double)]


class gpe_obs(ctypes.Structure):
    _fields_ = [(k, c_double) for k in ("norm", "ekin", "epot", "eint", "energy", "mu", "O", "B",
                                        "alpha_re", "alpha_im", "t")] + [("status", c_int)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


class GPEError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{status_string(status)}: {msg}")
        self.status = status


_lib = None


def lib_path() -> str:
    """libgpe.so, or with GPE_LIBRARY=debug the bounds-check build libgpe_debug.so."""
    return _build.DEBUG_LIB if os.environ.get("GPE_LIBRARY") == "debug" else _build.LIB


def load() -> ctypes.CDLL:
    """Load libgpe.so (built in-tree by build.py).  Raises if it cannot."""
    global _lib
    if _lib is not None:
        return _lib
    path = lib_path()
    if not os.path.exists(path):
        _build.build(debug=path == _build.DEBUG_LIB)
    L = ctypes.CDLL(path)
    P = ctypes.POINTER
    sig = {
        "gpe_workspace_size": (c_size_t, [c_int, c_int]),
        "gpe_create": (c_int, [c_int, c_int, c_double, c_double, c_double, c_double, c_void_p, c_void_p,
                               c_size_t, c_void_p, P(c_void_p)]),
        "gpe_set_potential": (c_int, [c_void_p, P(gpe_potential)]),
        "gpe_step": (c_int, [c_void_p, c_int, c_double, c_int]),
        "gpe_step_many": (c_int, [P(c_void_p), c_int, c_int, c_double, c_int]),
        "gpe_profile": (c_int, [c_void_p, c_int]),
        "gpe_profile_read": (c_int, [c_void_p, P(c_double), P(c_int), P(c_double), P(c_int)]),
        "gpe_profile_read_kind": (c_int, [c_void_p, c_int, P(c_double), P(c_int)]),
        "gpe_launch_count": (ctypes.c_longlong, [c_void_p]),
        "gpe_observables": (c_int, [c_void_p, P(gpe_obs)]),
        "gpe_set_psi": (c_int, [c_void_p, c_void_p, c_int]),
        "gpe_get_psi": (c_int, [c_void_p, c_void_p, c_int]),
        "gpe_set_time": (c_int, [c_void_p, c_double]),
        "gpe_get_time": (c_double, [c_void_p]),
        "gpe_fft2": (c_int, [c_void_p, c_int]),
        "gpe_sync": (c_int, [c_void_p]),
        "gpe_set_wait_limit": (c_int, [c_void_p, c_int]),
        "gpe_get_wait_limit": (c_int, [c_void_p]),
        "gpe_debug_timeout_probe": (c_int, [c_void_p, c_int]),
        "gpe_overlaps_static": (c_int, [c_void_p, c_int, c_int, c_double, c_double, c_double, c_void_p,
                                        P(c_double)]),
        "gpe_momentum_populations": (c_int, [c_void_p, c_int, c_double, c_int, c_void_p, c_size_t, P(c_double)]),
        "gpe_get_pass_variants": (c_int, [c_void_p]),
        "gpe_set_pass_variants": (c_int, [c_void_p, c_int]),
        "gpe_tune": (c_int, [c_void_p, c_double, c_int, c_void_p, c_size_t, c_int, P(c_int), P(c_double)]),
        "gpe_adjoint_workspace_size": (c_size_t, [c_int, c_int, c_int]),
        "gpe_adjoint_lattice": (c_int, [c_void_p, c_int, c_double, c_void_p, c_void_p, c_size_t, P(c_double),
                                        P(c_double)]),
        "gpe_adjoint_workspace_size_ex": (c_size_t, [c_int, c_int, c_int, c_int]),
        "gpe_adjoint_lattice_ex": (c_int, [c_void_p, c_int, c_double, c_int, c_void_p, c_void_p, c_size_t,
                                           P(c_double), P(c_double)]),
        "gpe_batch_workspace_size": (c_size_t, [P(c_void_p), c_int]),
        "gpe_batch_create": (c_int, [P(c_void_p), c_int, c_void_p, c_size_t, P(c_void_p)]),
        "gpe_batch_step": (c_int, [c_void_p, c_int, c_double, c_int]),
        "gpe_batch_destroy": (None, [c_void_p]),
        "gpe_destroy": (None, [c_void_p]),
        "gpe_last_error": (c_char_p, [c_void_p]),
        "gpe_status_string": (c_char_p, [c_int]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype, f.argtypes = res, args
    _lib = L
    return L


def status_string(s: int) -> str:
    return load().gpe_status_string(int(s)).decode()


def _check(ctx, s: int):
    if s != GPE_OK:
        msg = load().gpe_last_error(ctx).decode() if ctx else ""
        raise GPEError(s, msg)


# ---------------------------------------------------------------- C names
def gpe_workspace_size(nx: int, ny: int) -> int:
    return load().gpe_workspace_size(nx, ny)


def gpe_create(nx, ny, Lx, Ly, m, g, psi_ptr, ws_ptr, ws_bytes, stream_handle) -> c_void_p:
    ctx = c_void_p()
    _check(None, load().gpe_create(nx, ny, Lx, Ly, m, g, c_void_p(psi_ptr), c_void_p(ws_ptr), ws_bytes,
                                   c_void_p(stream_handle), ctypes.byref(ctx)))
    return ctx


def gpe_set_potential(ctx, pot: gpe_potential):
    _check(ctx, load().gpe_set_potential(ctx, ctypes.byref(pot)))


def gpe_step(ctx, n: int, dt: float, mode: int):
    _check(ctx, load().gpe_step(ctx, int(n), float(dt), int(mode)))


def gpe_step_many(ctxs, n: int, dt: float, mode: int):
    arr = (c_void_p * len(ctxs))(*[c.value for c in ctxs])
    _check(ctxs[0] if ctxs else None, load().gpe_step_many(arr, len(ctxs), int(n), float(dt), int(mode)))


def gpe_profile(ctx, enable: bool):
    _check(ctx, load().gpe_profile(ctx, int(enable)))


def gpe_profile_read(ctx) -> dict:
    rm, cm = c_double(), c_double()
    rn, cn = c_int(), c_int()
    _check(ctx, load().gpe_profile_read(ctx, ctypes.byref(rm), ctypes.byref(rn), ctypes.byref(cm),
                                        ctypes.byref(cn)))
    return dict(row_ms=rm.value, row_launches=rn.value, col_ms=cm.value, col_launches=cn.value)


GPE_PASS_ROW, GPE_PASS_COL, GPE_PASS_OTHER, GPE_PASS_ADJ_ROW, GPE_PASS_ADJ_COL = range(5)


def gpe_profile_read_kind(ctx, kind: int) -> tuple:
    """(milliseconds, launches) of one pass kind since its last read."""
    ms, n = c_double(), c_int()
    _check(ctx, load().gpe_profile_read_kind(ctx, int(kind), ctypes.byref(ms), ctypes.byref(n)))
    return ms.value, n.value


def gpe_launch_count(ctx) -> int:
    return int(load().gpe_launch_count(ctx))


def gpe_observables(ctx, check: bool = True) -> dict:
    o = gpe_obs()
    s = load().gpe_observables(ctx, ctypes.byref(o))
    if check:
        _check(ctx, s)
    return o.as_dict()


def gpe_set_psi(ctx, src_ptr: int, is_dev: bool):
    _check(ctx, load().gpe_set_psi(ctx, c_void_p(src_ptr), int(is_dev)))


def gpe_get_psi(ctx, dst_ptr: int, is_dev: bool):
    _check(ctx, load().gpe_get_psi(ctx, c_void_p(dst_ptr), int(is_dev)))


def gpe_set_time(ctx, t: float):
    _check(ctx, load().gpe_set_time(ctx, float(t)))


def gpe_get_time(ctx) -> float:
    return load().gpe_get_time(ctx)


def gpe_fft2(ctx, sign: int):
    _check(ctx, load().gpe_fft2(ctx, int(sign)))


def gpe_sync(ctx) -> int:
    """Wait for the stream; returns (does not raise) the latched device status."""
    return load().gpe_sync(ctx)


def gpe_set_wait_limit(ctx, spins: int):
    _check(ctx, load().gpe_set_wait_limit(ctx, int(spins)))


def gpe_get_wait_limit(ctx) -> int:
    return load().gpe_get_wait_limit(ctx)


def gpe_debug_timeout_probe(ctx, spins: int):
    _check(ctx, load().gpe_debug_timeout_probe(ctx, int(spins)))


def gpe_overlaps_static(psi_ptr: int, nx: int, ny: int, Lx: float, Ly: float, kc: float,
                        stream_handle: int):
    """Norm and cavity overlaps (norm, O, B) of a device psi with the library's
    fixed scratch instead of a workspace; raises GPEError on a bad status."""
    out = (c_double * 3)()
    s = load().gpe_overlaps_static(c_void_p(psi_ptr), nx, ny, Lx, Ly, kc, c_void_p(stream_handle), out)
    _check(None, s)
    return out[0], out[1], out[2]


def gpe_momentum_populations(ctx, axis: int, k0: float, nmax: int, scratch_ptr: int, scratch_bytes: int) -> list:
    """Populations of the momentum windows around 2 n k0 along `axis`, n = -nmax..nmax."""
    out = (c_double * (2 * nmax + 1))()
    _check(ctx, load().gpe_momentum_populations(ctx, int(axis), float(k0), int(nmax), c_void_p(scratch_ptr),
                                                scratch_bytes, out))
    return [out[i] for i in range(2 * nmax + 1)]


GPE_VARIANT_GROUP_ROWS, GPE_VARIANT_STREAM_ROWS, GPE_VARIANT_STREAM_COLS = 1, 2, 4
GPE_VARIANT_ROW_TILE_SHIFT = 3          # bits 3-4: one-shot row pass at 2^-value of its default rows per CTA
GPE_VARIANT_PAIR_COLS = 32              # column passes as pencil pairs (512..8192-point columns)
GPE_VARIANT_PAIR_ROWS = 64              # row pass (phase + T_x) on pairs of rows (512..8192 points)
GPE_VARIANT_COOP = 128                  # gpe_step of one 512/1024-point grid: one cooperative persistent launch


def gpe_get_pass_variants(ctx) -> int:
    return load().gpe_get_pass_variants(ctx)


def gpe_set_pass_variants(ctx, variants: int):
    _check(ctx, load().gpe_set_pass_variants(ctx, int(variants)))


def gpe_tune(ctx, dt: float, mode: int, scratch_ptr: int, scratch_bytes: int, reps: int = 5):
    """(variant bits chosen, [ms: row one-shot, row grouped, row streaming, col one-shot, col streaming])."""
    v = c_int()
    t = (c_double * 5)()
    _check(ctx, load().gpe_tune(ctx, float(dt), int(mode), c_void_p(scratch_ptr), scratch_bytes, int(reps),
                                ctypes.byref(v), t))
    return v.value, [t[k] for k in range(5)]


def gpe_adjoint_workspace_size(nx: int, ny: int, nsteps: int) -> int:
    return load().gpe_adjoint_workspace_size(nx, ny, nsteps)


def gpe_adjoint_lattice(ctx, nsteps: int, dt: float, phi_ptr: int, ws_ptr: int, ws_bytes: int, nctrl: int):
    """(J, [dJ/dv_i]) of the lattice-depth control; raises GPEError on a bad status."""
    J = c_double()
    grad = (c_double * max(nctrl, 1))()
    _check(ctx, load().gpe_adjoint_lattice(ctx, int(nsteps), float(dt), c_void_p(phi_ptr), c_void_p(ws_ptr),
                                           ws_bytes, ctypes.byref(J), grad))
    return J.value, [grad[i] for i in range(nctrl)]


GPE_ADJ_CHECKPOINT, GPE_ADJ_REVERSE = 0, 1


def gpe_adjoint_workspace_size_ex(nx: int, ny: int, nsteps: int, variant: int) -> int:
    return load().gpe_adjoint_workspace_size_ex(nx, ny, nsteps, variant)


def gpe_adjoint_lattice_ex(ctx, nsteps: int, dt: float, variant: int, phi_ptr: int, ws_ptr: int, ws_bytes: int,
                           nctrl: int):
    """gpe_adjoint_lattice with the reverse-sweep variant (GPE_ADJ_CHECKPOINT or GPE_ADJ_REVERSE)."""
    J = c_double()
    grad = (c_double * max(nctrl, 1))()
    _check(ctx, load().gpe_adjoint_lattice_ex(ctx, int(nsteps), float(dt), int(variant), c_void_p(phi_ptr),
                                              c_void_p(ws_ptr), ws_bytes, ctypes.byref(J), grad))
    return J.value, [grad[i] for i in range(nctrl)]


def _ctx_array(ctxs):
    arr = (c_void_p * len(ctxs))()
    for i, c in enumerate(ctxs):
        arr[i] = c.value if isinstance(c, c_void_p) else c
    return arr


def gpe_batch_workspace_size(ctxs) -> int:
    return load().gpe_batch_workspace_size(_ctx_array(ctxs), len(ctxs))


def gpe_batch_create(ctxs, ws_ptr: int, ws_bytes: int) -> c_void_p:
    b = c_void_p()
    _check(ctxs[0] if ctxs else None, load().gpe_batch_create(_ctx_array(ctxs), len(ctxs), c_void_p(ws_ptr), ws_bytes,
                                                              ctypes.byref(b)))
    return b


def gpe_batch_step(batch, ctx0, n: int, dt: float, mode: int):
    """ctx0: the batch's first context (for the error message)."""
    _check(ctx0, load().gpe_batch_step(batch, int(n), float(dt), int(mode)))


def gpe_batch_destroy(batch):
    load().gpe_batch_destroy(batch)


def gpe_destroy(ctx):
    load().gpe_destroy(ctx)


def gpe_last_error(ctx) -> str:
    return load().gpe_last_error(ctx).decode()


def gpe_status_string(s: int) -> str:
    return status_string(s)
