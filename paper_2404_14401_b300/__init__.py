"""B300-native (sm_103a) split-step Fourier propagator for the 2D Gross-Pitaevskii
equation (TorchGPE, arXiv 2404.14401): symmetric splitting in real and
imaginary time, with the self-consistent cavity potential of Sec. 5.3.

The compute path is the C ABI of include/gpe.h implemented by hand-written
CUDA kernels in csrc/ (libgpe.so).  PyTorch provides only device memory and
streams.  `Simulation` owns the torch allocations a context borrows.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import gpe as abi
from .gpe import GPE_CTRL_ETA, GPE_CTRL_LATTICE, GPE_CTRL_NONE, GPE_IMAG, GPE_REAL, GPEError  # noqa: F401


class Simulation:
    """One grid: psi (complex64 [ny][nx]) and workspace allocated with torch on
    `device`, a gpe context bound to `stream` (torch.cuda.Stream or None for
    the current stream).  Methods are one C call each."""

    def __init__(self, nx, ny, Lx, Ly, m=1.0, g=0.0, device="cuda", stream=None):
        import torch
        self.torch = torch
        self.nx, self.ny, self.Lx, self.Ly, self.m, self.g = nx, ny, Lx, Ly, m, g
        self.device = torch.device(device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        ws = abi.gpe_workspace_size(nx, ny)
        if ws == 0:
            raise GPEError(abi.GPE_EINVAL, f"unsupported grid {nx}x{ny}")
        self.psi = self._borrow(torch.zeros((ny, nx), dtype=torch.complex64, device=self.device))
        self.ws = self._borrow(torch.empty(ws, dtype=torch.uint8, device=self.device))
        self._keep = []
        self._ctrl = None
        self._order_after_current()
        self.ctx = abi.gpe_create(nx, ny, Lx, Ly, m, g, self.psi.data_ptr(), self.ws.data_ptr(), ws,
                                  self.stream.cuda_stream)

    def _order_after_current(self):
        """Make the context's stream wait for the work torch enqueued on the
        current stream (allocations, fills, uploads) before it uses them."""
        cur = self.torch.cuda.current_stream(self.device)
        if self.stream != cur:
            self.stream.wait_stream(cur)

    def _borrow(self, t):
        """A device tensor the context will use on its stream: when that stream
        is not the one the tensor was allocated on, tell torch's caching
        allocator, so that the memory is not handed out again before the
        context's work on it has finished."""
        if self.stream != self.torch.cuda.current_stream(self.device):
            t.record_stream(self.stream)
        return t

    # ------------------------------------------------------------ set-up
    def set_potential(self, p: dict):
        """p uses the keys of gpe_inputs.potential_defaults(); a `Varr` array is
        copied to a float32 device tensor that the context borrows."""
        torch = self.torch
        pot = abi.gpe_potential()
        for k in ("wx", "wy", "lat_V0x", "lat_V0y", "lat_kx", "lat_ky", "V_scale", "cavity", "eta", "U0",
                  "dc", "kappa", "kc", "pump_lattice", "ctrl_target", "probe_omega", "probe_delta", "probe_phi"):
            setattr(pot, k, p.get(k, 0) if k != "V_scale" else p.get(k, 1.0))
        pot.N = p.get("Nat", p.get("N", 1.0))
        keep = []
        self._ctrl = None
        if p.get("Varr") is not None:
            V = self._borrow(torch.as_tensor(np.asarray(p["Varr"], dtype=np.float32)).to(self.device))
            self._order_after_current()
            keep.append(V)
            pot.V = V.data_ptr()
        if p.get("ctrl_t") is not None:
            t = np.ascontiguousarray(p["ctrl_t"], dtype=np.float64)
            v = np.ascontiguousarray(p["ctrl_v"], dtype=np.float64)
            keep += [t, v]
            pot.nctrl = t.size
            self._ctrl = v
            pot.ctrl_t = t.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
            pot.ctrl_v = v.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        abi.gpe_set_potential(self.ctx, pot)
        self._keep = keep                                    # the device V array stays borrowed

    def set_psi(self, psi):
        """psi: numpy array (copied from host) or a complex64 cuda tensor."""
        torch = self.torch
        if isinstance(psi, np.ndarray):
            h = torch.from_numpy(np.ascontiguousarray(psi, dtype=np.complex64))
            abi.gpe_set_psi(self.ctx, h.data_ptr(), False)
            self.sync()
        else:
            t = self._borrow(psi.to(device=self.device, dtype=torch.complex64).contiguous())
            self._order_after_current()
            abi.gpe_set_psi(self.ctx, t.data_ptr(), True)
            self._tmp = t

    def get_psi(self) -> np.ndarray:
        out = np.empty((self.ny, self.nx), dtype=np.complex64)
        abi.gpe_get_psi(self.ctx, out.ctypes.data, False)
        return out

    # ------------------------------------------------------------ evolution
    def step(self, n: int, dt: float, imag: bool = False):
        abi.gpe_step(self.ctx, n, dt, abi.GPE_IMAG if imag else abi.GPE_REAL)

    @staticmethod
    def step_many(sims, n: int, dt: float, imag: bool = False):
        """n lockstep steps on several simulations (one pass schedule)."""
        abi.gpe_step_many([s.ctx for s in sims], n, dt, abi.GPE_IMAG if imag else abi.GPE_REAL)

    def momentum_populations(self, axis: int, k0: float, nmax: int = 3) -> np.ndarray:
        """Kapitza-Dirac readout: fractions of the momentum distribution in the
        windows |k - 2 n k0| < k0 along `axis`, n = -nmax..nmax."""
        torch = self.torch
        scratch = self._borrow(torch.empty(8 * self.nx * self.ny, dtype=torch.uint8, device=self.device))
        return np.array(abi.gpe_momentum_populations(self.ctx, axis, k0, nmax, scratch.data_ptr(), scratch.numel()))

    def tune(self, dt: float, imag: bool = False, reps: int = 5) -> dict:
        """Time the applicable kernel variants of the interior passes on a copy
        of psi and keep the fastest (gpe_tune).  Returns the chosen variant bits
        and the per-variant milliseconds."""
        torch = self.torch
        scratch = self._borrow(torch.empty(8 * self.nx * self.ny, dtype=torch.uint8, device=self.device))
        v, t = abi.gpe_tune(self.ctx, dt, abi.GPE_IMAG if imag else abi.GPE_REAL, scratch.data_ptr(),
                            scratch.numel(), reps)
        keys = ("row_one_shot", "row_grouped", "row_streaming", "col_one_shot", "col_streaming")
        return {"variants": v, "row_tile": (v >> abi.GPE_VARIANT_ROW_TILE_SHIFT) & 3,
                "ms": {k: (None if x != x else x) for k, x in zip(keys, t)}}

    @property
    def variants(self) -> int:
        return abi.gpe_get_pass_variants(self.ctx)

    @variants.setter
    def variants(self, v: int):
        abi.gpe_set_pass_variants(self.ctx, v)

    def adjoint_lattice(self, phi, nsteps: int, dt: float, reverse: bool = False):
        """J = E(psi_T) + |<phi|psi_T>|^2 after nsteps real-time steps from the
        current state, and dJ/dv_i for the lattice control values set with
        set_potential (ctrl_target = GPE_CTRL_LATTICE).  One C call (forward,
        then the reverse sweep, whose states come from sqrt(nsteps)
        checkpoints, or with reverse=True from steps backward in time); psi is
        the final state afterwards.  phi: complex64 cuda tensor or numpy array
        [ny][nx]."""
        torch = self.torch
        phi_t = torch.as_tensor(np.asarray(phi, dtype=np.complex64) if isinstance(phi, np.ndarray) else phi)
        phi_t = self._borrow(phi_t.to(device=self.device, dtype=torch.complex64).contiguous())
        self._order_after_current()
        variant = abi.GPE_ADJ_REVERSE if reverse else abi.GPE_ADJ_CHECKPOINT
        nbytes = abi.gpe_adjoint_workspace_size_ex(self.nx, self.ny, nsteps, variant)
        if getattr(self, "_adj_ws", None) is None or self._adj_ws.numel() < nbytes:
            self._adj_ws = self._borrow(torch.empty(nbytes, dtype=torch.uint8, device=self.device))
        nctrl = 0 if self._ctrl is None else len(self._ctrl)
        return abi.gpe_adjoint_lattice_ex(self.ctx, nsteps, dt, variant, phi_t.data_ptr(), self._adj_ws.data_ptr(),
                                          self._adj_ws.numel(), nctrl)

    def profile(self, enable: bool):
        abi.gpe_profile(self.ctx, enable)

    def profile_read(self) -> dict:
        return abi.gpe_profile_read(self.ctx)

    @property
    def launches(self) -> int:
        return abi.gpe_launch_count(self.ctx)

    def observables(self, check: bool = True) -> dict:
        return abi.gpe_observables(self.ctx, check)

    def fft2(self, sign: int):
        abi.gpe_fft2(self.ctx, sign)

    @property
    def t(self) -> float:
        return abi.gpe_get_time(self.ctx)

    @t.setter
    def t(self, value: float):
        abi.gpe_set_time(self.ctx, value)

    def sync(self) -> int:
        return abi.gpe_sync(self.ctx)

    def close(self):
        if getattr(self, "ctx", None):
            abi.gpe_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """A persistent batch over Simulations (gpe_batch_create): each step() is one
    kernel launch for n lockstep steps of every simulation.  Owns the batch
    workspace (a torch allocation on the first simulation's device); the
    simulations must outlive it."""

    def __init__(self, sims):
        torch = sims[0].torch
        self.sims = list(sims)
        ctxs = [s.ctx for s in self.sims]
        nbytes = abi.gpe_batch_workspace_size(ctxs)
        if nbytes == 0:
            raise GPEError(abi.GPE_EINVAL, "empty batch")
        self.ws = self.sims[0]._borrow(torch.empty(nbytes, dtype=torch.uint8, device=self.sims[0].device))
        self.sims[0]._order_after_current()
        self.batch = abi.gpe_batch_create(ctxs, self.ws.data_ptr(), nbytes)

    def step(self, n: int, dt: float, imag: bool = False):
        abi.gpe_batch_step(self.batch, self.sims[0].ctx, n, dt, abi.GPE_IMAG if imag else abi.GPE_REAL)

    def close(self):
        if getattr(self, "batch", None):
            abi.gpe_batch_destroy(self.batch)
            self.batch = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
