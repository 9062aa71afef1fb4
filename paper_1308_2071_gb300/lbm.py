"""Python face of liblbm: a cavity of the porous-media MRT lattice Boltzmann
model (arXiv:1308.2071, Section 3 and 4) driven through the C-ABI.

PyTorch supplies device memory (field outputs, porosity input) and the CUDA
stream; every step of the method runs in the library's kernels.
"""
from __future__ import annotations

import ctypes as C

import torch

from . import _lib as L

PRECISIONS = {"f64": L.LBM_F64, "f32": L.LBM_F32, "f16": L.LBM_F32_STORE_F16, "f32t": L.LBM_F32_FRAMED}


def make_params(nx: int, ny: int, Ra: float, Da: float, phi: float, precision: str = "f32",
                **kw) -> L.Params:
    """lbm_params with the Section 4 defaults, overridden by keyword arguments
    (Pr, J, Ma, sigma, varpi, Th, Tc, Qppp, use_phi_field, forchheimer,
    thermal_bc, adiabatic_order, collision, block_x, block_y)."""
    p = L.Params()
    L.load().lbm_params_default(C.byref(p), nx, ny, Ra, Da, phi)
    p.precision = PRECISIONS[precision]
    for k, v in kw.items():
        if not hasattr(p, k):
            raise TypeError(f"unknown parameter {k}")
        setattr(p, k, v)
    return p


class Cavity:
    """One cavity on the current CUDA device.  Work runs on `stream`
    (default: the current torch stream)."""

    def __init__(self, nx: int, ny: int, Ra: float, Da: float, phi: float, precision: str = "f32",
                 stream: torch.cuda.Stream | None = None, phi_field: torch.Tensor | None = None, **kw):
        if not torch.cuda.is_available():
            raise RuntimeError("liblbm needs a CUDA device")
        lib = L.load()
        if phi_field is not None:
            kw.setdefault("use_phi_field", 1)
        self.params = make_params(nx, ny, Ra, Da, phi, precision, **kw)
        self.nx, self.ny = nx, ny
        self.precision = precision
        self.stream = stream or torch.cuda.current_stream()
        self.device = self.stream.device
        self._h = C.c_void_p()
        with torch.cuda.device(self.device):
            rc = lib.lbm_init(C.byref(self.params), C.c_void_p(self.stream.cuda_stream), C.byref(self._h))
        L.check(rc, None)
        if phi_field is not None:
            self.set_porous_field(phi_field)

    # -- lifetime --
    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            L.load().lbm_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    @property
    def handle(self) -> C.c_void_p:
        return self._h

    @property
    def field_dtype(self) -> torch.dtype:
        return torch.float64 if self.precision == "f64" else torch.float32

    # -- operations --
    def set_porous_field(self, phi: torch.Tensor):
        """Per-cell porosity (ny, nx) on this device, float32 or float64; resets to t = 0."""
        phi = phi.to(self.device).contiguous()
        if phi.shape != (self.ny, self.nx):
            raise ValueError(f"porosity field must be ({self.ny}, {self.nx})")
        dt = {torch.float64: L.LBM_F64, torch.float32: L.LBM_F32}[phi.dtype]
        self._sync_inputs(phi)
        L.check(L.load().lbm_set_porous_field(self._h, C.c_void_p(phi.data_ptr()), dt), self._h)

    def tune(self, cache_path: str | None = None):
        """Picks the fastest launch shape for this lattice (resets to t = 0);
        returns (block_x, block_y, nodes_per_thread)."""
        bx, by, npt = C.c_int(), C.c_int(), C.c_int()
        path = cache_path.encode() if cache_path else None
        L.check(L.load().lbm_tune(self._h, path, C.byref(bx), C.byref(by), C.byref(npt)), self._h)
        return bx.value, by.value, npt.value

    def reset(self) -> "Cavity":
        """Back to the initial state (t = 0), same parameters, field and launch shape."""
        L.check(L.load().lbm_reset(self._h), self._h)
        return self

    def step(self, n: int = 1) -> "Cavity":
        L.check(L.load().lbm_step(self._h, int(n)), self._h)
        return self

    def observables(self, fields: bool = False, check: bool = True) -> dict:
        """Nusselt numbers, residual, |u|max, mass and heat sums (FP64); with
        fields=True also ux, uy, T, p as (ny, nx) tensors."""
        obs = L.Obs()
        ptrs = [None] * 4
        out = {}
        if fields:
            ts = [torch.empty((self.ny, self.nx), dtype=self.field_dtype, device=self.device)
                  for _ in range(4)]
            out.update(zip(("ux", "uy", "T", "p"), ts))
            ptrs = [C.c_void_p(t.data_ptr()) for t in ts]
        rc = L.load().lbm_observables(self._h, C.byref(obs), *ptrs)
        if rc != L.LBM_ERR_DIVERGED or check:
            L.check(rc, self._h)
        out.update(t=obs.t, nu_hot=obs.nu_hot, nu_cold=obs.nu_cold, residual=obs.residual,
                   umax=obs.umax, mass=obs.mass, heat=obs.heat, status=obs.status)
        return out

    def adjoint(self, nsteps: int, ckpt_every: int = 100):
        """(J, dJ/dphi): J = mean Nu of the hot wall after nsteps from the
        initial state, and its gradient with respect to the porosity field,
        as a (ny, nx) tensor.  Leaves the cavity at t = nsteps."""
        out = torch.empty((self.ny, self.nx), dtype=self.field_dtype, device=self.device)
        J = C.c_double()
        L.check(L.load().lbm_adjoint_step(self._h, int(nsteps), int(ckpt_every), C.byref(J),
                                          C.c_void_p(out.data_ptr())), self._h)
        return J.value, out

    def run_steady(self, tol: float = 1e-9, check_every: int = 1000, max_steps: int = 10_000_000):
        """Steps until both wall Nusselt numbers change by less than tol
        (relative) between checks, on the device; returns (steps, change)."""
        n, ch = C.c_long(), C.c_double()
        L.check(L.load().lbm_run_steady(self._h, float(tol), int(check_every), int(max_steps), C.byref(n),
                                        C.byref(ch)), self._h)
        return n.value, ch.value

    def extrema(self):
        """(T max, psi min, psi max) of the current state, lattice units."""
        a, b, c = C.c_double(), C.c_double(), C.c_double()
        L.check(L.load().lbm_field_extrema(self._h, C.byref(a), C.byref(b), C.byref(c)), self._h)
        return a.value, b.value, c.value

    def nusselt(self):
        """(Nu of the hot wall, Nu of the cold wall), FP64 (Eq. 38)."""
        a, b = C.c_double(), C.c_double()
        L.check(L.load().lbm_nusselt(self._h, C.byref(a), C.byref(b)), self._h)
        return a.value, b.value

    def nusselt_async(self, out2_ptr: int):
        """Enqueues (nu_hot, nu_cold) of the current state into 2 doubles at
        out2_ptr (pinned host or device memory) without waiting."""
        L.check(L.load().lbm_nusselt_async(self._h, C.c_void_p(out2_ptr)), self._h)

    def step_nusselt(self, n: int, out=None):
        """Advances n steps; row k of the (n, 2) FP64 result holds (Nu of the
        hot wall, Nu of the cold wall) after step k (Eq. 38), as nusselt()
        would give there.  out: optional float64 tensor of 2n elements on this
        device or in pinned host memory; written asynchronously (complete once
        the handle's stream is)."""
        n = int(n)
        if out is None:
            out = torch.empty((n, 2), dtype=torch.float64, device=self.device)
        elif out.dtype != torch.float64 or not out.is_contiguous() or out.numel() < 2 * n:
            raise ValueError("out must be a contiguous float64 tensor of at least 2n elements")
        L.check(L.load().lbm_step_nusselt(self._h, n, C.c_void_p(out.data_ptr())), self._h)
        return out

    def read_state(self):
        """Full FP64 post-stream populations f (9, ny, nx) and g (5, ny, nx)."""
        f = torch.empty((9, self.ny, self.nx), dtype=torch.float64, device=self.device)
        g = torch.empty((5, self.ny, self.nx), dtype=torch.float64, device=self.device)
        L.check(L.load().lbm_read_state(self._h, C.c_void_p(f.data_ptr()), C.c_void_p(g.data_ptr())),
                self._h)
        self.stream.synchronize()
        return f, g

    def save(self) -> bytearray:
        """Checkpoint as host bytes: a header and the state buffer the current
        post-stream state is pulled from (lbm_save)."""
        n = C.c_size_t()
        L.check(L.load().lbm_checkpoint_size(self._h, C.byref(n)), self._h)
        buf = bytearray(n.value)
        ptr = (C.c_char * n.value).from_buffer(buf)
        L.check(L.load().lbm_save(self._h, C.addressof(ptr), n.value), self._h)
        return buf

    def load(self, blob: bytearray):
        """Restores a checkpoint of a cavity with the same nx, ny and precision."""
        ptr = (C.c_char * len(blob)).from_buffer(blob)
        L.check(L.load().lbm_load(self._h, C.addressof(ptr), len(blob)), self._h)

    def query(self):
        t, st = C.c_long(), C.c_int()
        L.check(L.load().lbm_query(self._h, C.byref(t), C.byref(st)), self._h)
        return t.value, st.value

    def _sync_inputs(self, *tensors):
        # inputs produced on torch's current stream must be ready on ours
        cur = torch.cuda.current_stream(self.device)
        if cur.cuda_stream != self.stream.cuda_stream:
            self.stream.wait_stream(cur)


class Batch:
    """Many independent cavities advanced by one persistent launch per call.

    cavities: list of dicts with nx, ny, Ra, Da, phi and optional Section 4
    overrides (Pr, J, Ma, ...); all share one precision ("f32" or "f64")."""

    def __init__(self, cavities, precision: str = "f32", stream: torch.cuda.Stream | None = None):
        if not torch.cuda.is_available():
            raise RuntimeError("liblbm needs a CUDA device")
        lib = L.load()
        n = len(cavities)
        arr = (L.Params * n)()
        for k, cv in enumerate(cavities):
            cv = dict(cv)
            p = make_params(cv.pop("nx"), cv.pop("ny"), cv.pop("Ra"), cv.pop("Da"), cv.pop("phi"), precision,
                            **cv)
            arr[k] = p
        self.params = arr
        self.ncav = n
        self.sizes = [(c["nx"], c["ny"]) for c in cavities]
        self.stream = stream or torch.cuda.current_stream()
        self.device = self.stream.device
        self._b = C.c_void_p()
        with torch.cuda.device(self.device):
            rc = lib.lbm_batch_init(arr, n, C.c_void_p(self.stream.cuda_stream), C.byref(self._b))
        L.check(rc, None)

    def close(self):
        if getattr(self, "_b", None) and self._b.value:
            L.load().lbm_batch_destroy(self._b)
            self._b = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, rc):
        L.check(rc, batch=self._b)

    def step(self, n: int = 1) -> "Batch":
        self._check(L.load().lbm_batch_step(self._b, int(n)))
        return self

    def nusselt(self):
        import numpy as np

        hot = np.zeros(self.ncav)
        cold = np.zeros(self.ncav)
        self._check(L.load().lbm_batch_nusselt(self._b, hot.ctypes.data, cold.ctypes.data))
        return hot, cold

    def status(self):
        """(return code, per-cavity status array)."""
        import numpy as np

        st = np.zeros(self.ncav, dtype=np.int32)
        rc = L.load().lbm_batch_status(self._b, st.ctypes.data)
        return rc, st

    def read_state(self, cav: int):
        nx, ny = self.sizes[cav]
        f = torch.empty((9, ny, nx), dtype=torch.float64, device=self.device)
        g = torch.empty((5, ny, nx), dtype=torch.float64, device=self.device)
        self._check(L.load().lbm_batch_read_state(self._b, cav, C.c_void_p(f.data_ptr()), C.c_void_p(g.data_ptr())))
        self.stream.synchronize()
        return f, g

    def set_wait_limit(self, polls: int):
        self._check(L.load().lbm_batch_set_wait_limit(self._b, int(polls)))

    def tune(self, cache_path: str | None = None):
        tw, th, bps = C.c_int(), C.c_int(), C.c_int()
        path = cache_path.encode() if cache_path else None
        self._check(L.load().lbm_batch_tune(self._b, path, C.byref(tw), C.byref(th), C.byref(bps)))
        return tw.value, th.value, bps.value

    def set_tiles(self, tile_w: int, tile_h: int, blocks_per_sm: int = 0, dynamic: int = 0):
        """tile_h = 0: runs of tile_w consecutive nodes in row-major order.
        dynamic: 0 static runs of tiles, 1 chunks from a per-step counter,
        2 dataflow with per-cavity step dependencies (no grid barrier)."""
        self._check(L.load().lbm_batch_set_tiles(self._b, tile_w, tile_h, blocks_per_sm, int(dynamic)))

    def query(self):
        t, nt, nb = C.c_long(), C.c_int(), C.c_int()
        self._check(L.load().lbm_batch_query(self._b, C.byref(t), C.byref(nt), C.byref(nb)))
        return dict(t=t.value, ntiles=nt.value, nblocks=nb.value)
