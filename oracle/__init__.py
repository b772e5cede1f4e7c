"""FP64 CPU oracle for the split-step GPE -- test infrastructure only.

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product library never does, and
this package imports nothing from the product.  The arithmetic lives in
``gpe_oracle.c`` (plain C, double precision, own radix-2 FFT); this file
only builds that library, mirrors its parameter struct and converts numpy
arrays.

Parity status per function (pins live in tests/test_oracle_*.py):
  fft1 / fft2     pinned: brute-force DFT, numpy.fft, Parseval, round trip
  evolve (real)   pinned: free-Gaussian closed form, norm conservation,
                  energy conservation, trapped coherent-state motion,
                  lattice momentum-basis exact evolution, 2nd order in dt
  evolve (imag)   pinned: harmonic ground state E = 1, Thomas-Fermi mu,
                  virial identity, unit norm
  potential array pinned: a trap written into V_scale * V[y][x] gives the
                  analytic-trap trajectory to 1e-12 on a non-square grid
                  (transposed, shifted or unscaled arrays fail)
  cavity alpha    pinned: eta = 0 gives alpha = 0 and the plain GPE;
                  symmetric density gives O = 0; alpha formula against a
                  direct quadrature of Eqs. (14)-(15) on a known density;
                  the update order in imaginary time (alpha from the density
                  at the start of each half phase) against a plain numpy
                  restatement of two steps on 8x8, to 1e-14.
                  The full self-consistent trajectory over many steps has
                  no closed form: its pieces are pinned, the trajectory as
                  a whole is compared with the GPU only.
  observables     pinned: E = mu = 1 for the oscillator ground state,
                  kinetic energy of a Gaussian in closed form
  momentum pops   pinned: plane-wave superpositions give |c_n|^2 exactly;
                  the Raman-Nath populations of a lattice flash
  adjoint         pinned: gradient of J = E(psi_T) + |<phi|psi_T>|^2 with
                  respect to the lattice control values against central
                  finite differences of the forward oracle; zero gradient
                  for control points the evolution never reaches
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gpe_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")


def build(force: bool = False) -> str:
    """Compile gpe_oracle.c into liboracle.so (gcc, -O2, OpenMP)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        cmd = ["gcc", "-O2", "-fopenmp", "-shared", "-fPIC", _SRC, "-o", _LIB, "-lm"]
        subprocess.run(cmd, check=True)
    return _LIB


class _Params(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int), ("ny", ctypes.c_int),
        ("Lx", ctypes.c_double), ("Ly", ctypes.c_double),
        ("m", ctypes.c_double), ("g", ctypes.c_double),
        ("wx", ctypes.c_double), ("wy", ctypes.c_double),
        ("lat_V0x", ctypes.c_double), ("lat_V0y", ctypes.c_double),
        ("lat_kx", ctypes.c_double), ("lat_ky", ctypes.c_double),
        ("Varr", ctypes.POINTER(ctypes.c_double)), ("V_scale", ctypes.c_double),
        ("cavity", ctypes.c_int),
        ("eta", ctypes.c_double), ("U0", ctypes.c_double), ("dc", ctypes.c_double),
        ("kappa", ctypes.c_double), ("kc", ctypes.c_double), ("Nat", ctypes.c_double),
        ("pump_lattice", ctypes.c_int),
        ("ctrl_target", ctypes.c_int), ("nctrl", ctypes.c_int),
        ("ctrl_t", ctypes.POINTER(ctypes.c_double)), ("ctrl_v", ctypes.POINTER(ctypes.c_double)),
        ("paper_order", ctypes.c_int),
        ("probe_omega", ctypes.c_double), ("probe_delta", ctypes.c_double), ("probe_phi", ctypes.c_double),
    ]


_lib = None


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        dp = ctypes.POINTER(ctypes.c_double)
        pp = ctypes.POINTER(_Params)
        lib.orc_fft1.argtypes = [dp, ctypes.c_int, ctypes.c_int]
        lib.orc_fft2.argtypes = [dp, ctypes.c_int, ctypes.c_int, ctypes.c_int]
        lib.orc_evolve.argtypes = [pp, dp, ctypes.c_int, ctypes.c_double, ctypes.c_int,
                                   ctypes.c_double, dp]
        lib.orc_observables.argtypes = [pp, dp, ctypes.c_double, dp]
        lib.orc_potential.argtypes = [pp, ctypes.c_double, ctypes.c_double, ctypes.c_double, dp]
        lib.orc_threads.argtypes = []
        lib.orc_adjoint.argtypes = [pp, dp, dp, ctypes.c_int, ctypes.c_double, ctypes.c_double, dp, dp]
        lib.orc_momentum_populations.argtypes = [pp, dp, ctypes.c_int, ctypes.c_double, ctypes.c_int, dp]
        for f in (lib.orc_fft1, lib.orc_fft2, lib.orc_evolve, lib.orc_observables,
                  lib.orc_potential, lib.orc_threads, lib.orc_adjoint, lib.orc_momentum_populations):
            f.restype = ctypes.c_int
        _lib = lib
    return _lib


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


class Params:
    """Owns the ctypes struct and the arrays it points into."""

    def __init__(self, p: dict, paper_order: bool = False):
        self._keep = []
        s = _Params()
        for name, _ in _Params._fields_:
            if name in ("Varr", "ctrl_t", "ctrl_v", "nctrl", "paper_order"):
                continue
            setattr(s, name, p.get(name, 0.0) if name.startswith("probe_") else p[name])
        if p.get("Varr") is not None:
            v = np.ascontiguousarray(p["Varr"], dtype=np.float64)
            assert v.shape == (p["ny"], p["nx"])
            self._keep.append(v)
            s.Varr = _dptr(v)
        if p.get("ctrl_t") is not None:
            t = np.ascontiguousarray(p["ctrl_t"], dtype=np.float64)
            v = np.ascontiguousarray(p["ctrl_v"], dtype=np.float64)
            assert t.shape == v.shape and t.ndim == 1
            self._keep += [t, v]
            s.ctrl_t, s.ctrl_v, s.nctrl = _dptr(t), _dptr(v), t.size
        s.paper_order = int(paper_order)
        self.s = s
        self.shape = (p["ny"], p["nx"])

    def ref(self):
        return ctypes.byref(self.s)


def threads() -> int:
    """OpenMP threads the oracle uses (OMP_NUM_THREADS, else all cores)."""
    return _load().orc_threads()


def fft1(a: np.ndarray, sign: int = -1) -> np.ndarray:
    """Unnormalised 1D DFT by the oracle's radix-2 FFT (sign -1 forward)."""
    x = np.array(a, dtype=np.complex128, copy=True)
    if _load().orc_fft1(_dptr(x.view(np.float64)), x.size, sign):
        raise ValueError("orc_fft1: size must be a power of two")
    return x


def fft2(a: np.ndarray, sign: int = -1) -> np.ndarray:
    """2D transform of a[ny][nx]; the inverse (sign +1) divides by nx*ny."""
    x = np.array(a, dtype=np.complex128, copy=True, order="C")
    ny, nx = x.shape
    if _load().orc_fft2(_dptr(x.view(np.float64)), nx, ny, sign):
        raise ValueError("orc_fft2: sizes must be powers of two")
    return x


def evolve(p: dict, psi: np.ndarray, steps: int, dt: float, imag: bool,
           t0: float = 0.0, paper_order: bool = False):
    """Run `steps` split steps from psi; returns (psi_new, alpha_last)."""
    P = Params(p, paper_order)
    x = np.array(psi, dtype=np.complex128, copy=True, order="C")
    assert x.shape == P.shape
    a = np.zeros(2)
    rc = _load().orc_evolve(P.ref(), _dptr(x.view(np.float64)), int(steps), float(dt),
                            int(bool(imag)), float(t0), _dptr(a))
    if rc:
        raise ValueError("orc_evolve failed")
    return x, complex(a[0], a[1])


OBS_KEYS = ("norm", "ekin", "epot", "eint", "energy", "mu", "O", "B", "alpha_re", "alpha_im")


def observables(p: dict, psi: np.ndarray, t: float = 0.0) -> dict:
    """Norm, energies, mu, cavity overlaps and alpha of psi at time t."""
    P = Params(p)
    x = np.ascontiguousarray(psi, dtype=np.complex128)
    out = np.zeros(10)
    _load().orc_observables(P.ref(), _dptr(x.view(np.float64)), float(t), _dptr(out))
    return dict(zip(OBS_KEYS, out.tolist()))


def potential(p: dict, t: float = 0.0, alpha: complex = 0.0) -> np.ndarray:
    """The potential V(x, y, t) on the grid for a given cavity field."""
    P = Params(p)
    V = np.zeros(P.shape)
    _load().orc_potential(P.ref(), float(t), float(np.real(alpha)), float(np.imag(alpha)), _dptr(V))
    return V


def adjoint(p: dict, psi0: np.ndarray, phi: np.ndarray, steps: int, dt: float, t0: float = 0.0):
    """J = E(psi_T) + |<phi|psi_T>|^2 after `steps` real-time steps from psi0,
    and dJ/dv_i for the lattice control values p["ctrl_v"] (discrete adjoint,
    reverse sweep over stored states).  Returns (J, grad)."""
    P = Params(p)
    x = np.ascontiguousarray(psi0, dtype=np.complex128)
    f = np.ascontiguousarray(phi, dtype=np.complex128)
    assert x.shape == P.shape and f.shape == P.shape
    J = np.zeros(1)
    grad = np.zeros(max(int(P.s.nctrl), 1))
    rc = _load().orc_adjoint(P.ref(), _dptr(x.view(np.float64)), _dptr(f.view(np.float64)), int(steps),
                             float(dt), float(t0), _dptr(J), _dptr(grad))
    if rc:
        raise ValueError("orc_adjoint needs a lattice control table and no cavity")
    return float(J[0]), grad[:int(P.s.nctrl)]


def momentum_populations(p: dict, psi: np.ndarray, axis: int, k0: float, nmax: int) -> np.ndarray:
    """Fractions of |F psi|^2 in the momentum windows |k - 2 n k0| < k0 along
    `axis` (0: x, 1: y), n = -nmax..nmax (Kapitza-Dirac readout, Sec. 5.2)."""
    P = Params(p)
    x = np.ascontiguousarray(psi, dtype=np.complex128)
    out = np.zeros(2 * nmax + 1)
    rc = _load().orc_momentum_populations(P.ref(), _dptr(x.view(np.float64)), int(axis), float(k0), int(nmax),
                                          _dptr(out))
    if rc:
        raise ValueError("orc_momentum_populations: bad arguments")
    return out
