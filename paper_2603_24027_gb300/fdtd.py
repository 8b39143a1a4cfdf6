"""Python front end: a Simulation handle and the autograd Function.

PyTorch supplies device memory (the workspace is a uint8 CUDA tensor) and the
stream; every step of the computation runs in the library's CUDA kernels,
called through the C ABI in `_capi`.
"""
from __future__ import annotations

import ctypes as C
from typing import Optional

import numpy as np
import torch

from . import _capi as A


def _fill_structs(w):
    grid = A.Grid(w.nx, w.ny, w.nz)
    pml = A.Pml(w.pml_thickness, w.pml_order, w.pml_sigma_factor, w.pml_kappa_max,
                w.pml_alpha_factor)
    src = A.Source()
    src.kind = w.src_kind
    src.component = w.src_component
    src.pos[:] = list(w.src_pos)
    src.axis = w.src_axis
    src.sigma_uv[:] = list(w.src_sigma_uv)
    src.lambda0 = w.lambda0
    src.rel_bandwidth = w.rel_bandwidth
    src.t0_over_tau = w.t0_over_tau
    src.amplitude = w.amplitude
    det = A.Detector()
    det.kind = w.det_kind
    det.axis = w.det_axis
    det.index = w.det_index
    det.lo[:] = list(w.det_lo)
    det.hi[:] = list(w.det_hi)
    return grid, pml, src, det


def _detector2(w):
    d = A.Detector()
    d.kind = w.det2_kind
    d.axis = w.det2_axis
    d.index = w.det2_index
    d.lo[:] = list(w.det2_lo)
    d.hi[:] = list(w.det2_hi)
    return d


class Simulation:
    """One FDTD gradient problem on one GPU.

    `workload` carries the grid, dx, dt, CPML, source, detector, step count
    and design box (see `inputs.Workload`).  Creating the handle touches no
    device; the workspace is allocated on first use.
    """

    def __init__(self, workload, device: Optional[torch.device] = None, stream=None):
        self.w = workload
        self.device = torch.device(device) if device is not None else None
        self._stream = stream
        grid, pml, src, det = _fill_structs(workload)
        lo = (C.c_int * 3)(*workload.design_lo)
        hi = (C.c_int * 3)(*workload.design_hi)
        h = C.c_void_p()
        s = None if stream is None else C.c_void_p(stream.cuda_stream)
        A.check(A.lib().fdtd_create(C.byref(grid), workload.dx, workload.dt, C.byref(pml),
                                    C.byref(src), C.byref(det), workload.n_steps, lo, hi, s,
                                    C.byref(h)))
        self.h = h
        self._ws = None
        self._ws_bytes = 0
        if workload.det2_kind:
            self._check(A.lib().fdtd_set_detector2(self.h, C.byref(_detector2(workload))))

    # ------------------------------------------------------------ lifetime --
    def close(self):
        if getattr(self, "h", None):
            A.lib().fdtd_destroy(self.h)
            self.h = None
        self._ws = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, status):
        A.check(status, self.h)

    # ---------------------------------------------------------- workspace --
    def workspace_bytes(self, rec=None) -> int:
        n = C.c_size_t()
        self._check(A.lib().fdtd_workspace_bytes(self.h, C.byref(rec) if rec else None, C.byref(n)))
        return n.value

    def tape_bytes(self, rec) -> int:
        n = C.c_size_t()
        self._check(A.lib().fdtd_tape_bytes(self.h, C.byref(rec), C.byref(n)))
        return n.value

    def ensure_workspace(self, rec, device=None):
        need = self.workspace_bytes(rec)
        if self._ws is None or self._ws_bytes < need:
            dev = torch.device(device or self.device or "cuda")
            self._ws = torch.empty(need, dtype=torch.uint8, device=dev)
            self._ws_bytes = need
            self._check(A.lib().fdtd_bind_workspace(self.h, C.c_void_p(self._ws.data_ptr()), need))
        return self._ws

    def set_option(self, option: int, value: int):
        self._check(A.lib().fdtd_set_option(self.h, option, int(value)))

    def get_option(self, option: int) -> int:
        v = C.c_int()
        self._check(A.lib().fdtd_get_option(self.h, option, C.byref(v)))
        return v.value

    # -------------------------------------------------------------- runs ----
    @property
    def design_shape(self):
        return self.w.design_shape

    def forward(self, eps: torch.Tensor, rec) -> float:
        """L(eps) with the boundary tape recorded; eps float32 [nz][ny][nx] on CUDA."""
        assert eps.is_cuda and eps.dtype == torch.float32 and eps.is_contiguous()
        assert tuple(eps.shape) == self.w.shape
        self.ensure_workspace(rec, eps.device)
        out = C.c_double()
        self._check(A.lib().fdtd_forward(self.h, C.c_void_p(eps.data_ptr()), C.byref(rec),
                                         C.byref(out)))
        return out.value

    # --------------------------------------------------------- checkpoint --
    def save_state(self) -> "np.ndarray":
        """The last forward's state (fields, cb, tape, objectives) as a host
        byte array that load_state restores, in this or another handle of the
        same problem."""
        import numpy as np
        n = C.c_size_t()
        self._check(A.lib().fdtd_state_bytes(self.h, C.byref(n)))
        buf = np.empty(n.value, np.uint8)
        self._check(A.lib().fdtd_save_state(self.h, C.c_void_p(buf.ctypes.data), n.value))
        return buf

    def load_state(self, buf, rec) -> None:
        """Make this handle ready for backward() from a saved forward state
        (rec: the record config it was saved with, for the workspace size)."""
        import numpy as np
        buf = np.ascontiguousarray(buf, dtype=np.uint8)
        self.ensure_workspace(rec)
        self._check(A.lib().fdtd_load_state(self.h, C.c_void_p(buf.ctypes.data), buf.size))

    def backward(self, seed: float = 1.0, out: Optional[torch.Tensor] = None,
                 seed2: Optional[float] = None) -> torch.Tensor:
        """d(seed L + seed2 M)/d(eps) over the design box, float32 [dz][dy][dx]
        (M: the second detector's objective; seed2 only with one)."""
        if out is None:
            out = torch.empty(self.design_shape, dtype=torch.float32, device=self._ws.device)
        if seed2 is None:
            self._check(A.lib().fdtd_backward(self.h, float(seed), C.c_void_p(out.data_ptr())))
        else:
            self._check(A.lib().fdtd_backward2(self.h, float(seed), float(seed2),
                                               C.c_void_p(out.data_ptr())))
        return out

    def objectives(self):
        """(L, M) of the last forward; M is 0 without a second detector."""
        L, M = C.c_double(), C.c_double()
        self._check(A.lib().fdtd_objectives(self.h, C.byref(L), C.byref(M)))
        return L.value, M.value

    def value_and_grad_host(self, eps_host: torch.Tensor, rec, seed: float = 1.0,
                            grad_host: Optional[torch.Tensor] = None):
        """Host buffers in and out (pinned memory makes the copies async)."""
        assert eps_host.device.type == "cpu" and eps_host.dtype == torch.float32
        self.ensure_workspace(rec)
        if grad_host is None:
            grad_host = torch.empty(self.design_shape, dtype=torch.float32,
                                    pin_memory=eps_host.is_pinned())
        out = C.c_double()
        self._check(A.lib().fdtd_value_and_grad_host(self.h, C.c_void_p(eps_host.data_ptr()),
                                                     C.byref(rec), float(seed), C.byref(out),
                                                     C.c_void_p(grad_host.data_ptr())))
        return out.value, grad_host

    def read_fields(self) -> torch.Tensor:
        out = torch.empty((6,) + self.w.shape, dtype=torch.float32, device=self._ws.device)
        self._check(A.lib().fdtd_read_fields(self.h, C.c_void_p(out.data_ptr())))
        return out

    def objective_history(self) -> np.ndarray:
        out = np.zeros(self.w.n_steps)
        self._check(A.lib().fdtd_objective_history(self.h, out.ctypes.data_as(C.c_void_p)))
        return out

    def last_timing(self):
        f, b = C.c_float(), C.c_float()
        lf, lb = C.c_int(), C.c_int()
        self._check(A.lib().fdtd_last_timing(self.h, C.byref(f), C.byref(b), C.byref(lf),
                                             C.byref(lb)))
        return dict(fwd_ms=f.value, bwd_ms=b.value, fwd_launches=lf.value, bwd_launches=lb.value)

    def last_host_call_ms(self) -> float:
        """Device time of the last value_and_grad_host between its input and
        output copies (ms)."""
        ms = C.c_float()
        self._check(A.lib().fdtd_last_host_call_ms(self.h, C.byref(ms)))
        return ms.value

    def kernel_timing(self):
        """{kernel name: (average ms, sampled launches)} of the last runs."""
        out = {}
        for kind, name in enumerate(A.KERNEL_NAMES):
            ms, n = C.c_float(), C.c_int()
            self._check(A.lib().fdtd_kernel_timing(self.h, kind, C.byref(ms), C.byref(n)))
            if n.value:
                out[name] = (ms.value, n.value)
        return out

    # ----------------------------------------------------- host-side plan ---
    def pml_profile(self, axis: int, which: int) -> np.ndarray:
        n = (self.w.nx, self.w.ny, self.w.nz)[axis]
        out = np.zeros(n, np.float32)
        self._check(A.lib().fdtd_pml_profile(self.h, axis, which, out.ctypes.data_as(C.c_void_p)))
        return out

    def source_waveform(self) -> np.ndarray:
        out = np.zeros(self.w.n_steps, np.float32)
        self._check(A.lib().fdtd_source_waveform(self.h, out.ctypes.data_as(C.c_void_p)))
        return out

    def interp_weights(self, rec, step: int, field: int):
        slot = (C.c_int * 4)()
        wt = (C.c_float * 4)()
        self._check(A.lib().fdtd_interp_weights(self.h, C.byref(rec), step, field, slot, wt))
        return list(slot), list(wt)


def _first_error(sims, status):
    """Raise for a failed group call with the message of the handle that set one."""
    for s in sims:
        msg = A.lib().fdtd_last_error(s.h)
        if msg:
            raise A.FdtdError(status, msg.decode())
    A.check(status)


def group_forward(sims, eps_list, rec, batched: bool = False):
    """Forward runs of several designs together: concurrent time loops
    (fdtd_group_forward), or with batched=True one launch per half-step over
    all designs (fdtd_batch_forward)."""
    n = len(sims)
    hs = (C.c_void_p * n)(*[s.h.value for s in sims])
    for s, e in zip(sims, eps_list):
        s.ensure_workspace(rec, e.device)
    eps = (C.c_void_p * n)(*[e.data_ptr() for e in eps_list])
    objs = (C.c_double * n)()
    fn = A.lib().fdtd_batch_forward if batched else A.lib().fdtd_group_forward
    st = fn(hs, n, eps, C.byref(rec), objs)
    if st != A.FDTD_OK:
        _first_error(sims, st)
    return list(objs)


def group_backward(sims, seeds=None, outs=None, batched: bool = False):
    n = len(sims)
    hs = (C.c_void_p * n)(*[s.h.value for s in sims])
    seeds = [1.0] * n if seeds is None else seeds
    if outs is None:
        outs = [torch.empty(s.design_shape, dtype=torch.float32, device=s._ws.device) for s in sims]
    sd = (C.c_double * n)(*seeds)
    gp = (C.c_void_p * n)(*[o.data_ptr() for o in outs])
    fn = A.lib().fdtd_batch_backward if batched else A.lib().fdtd_group_backward
    st = fn(hs, n, sd, gp)
    if st != A.FDTD_OK:
        _first_error(sims, st)
    return outs


class FDTDGrad(torch.autograd.Function):
    """L(eps_design) with eps outside the design box held fixed.

    forward(eps_design, eps_background, sim, rec) -> 0-d float64 tensor L
    backward: dL/d(eps_design) from the time-reversed run (hand-written
    adjoint kernels; no autodiff through the time loop).
    """

    @staticmethod
    def forward(ctx, eps_design, eps_background, sim, rec):
        eps = eps_background.detach().clone()
        eps[sim.w.design_slice()] = eps_design.detach().to(torch.float32)
        eps = eps.contiguous()
        L = sim.forward(eps, rec)
        ctx.sim = sim
        ctx.dtype = eps_design.dtype
        return torch.tensor(L, dtype=torch.float64, device=eps.device)

    @staticmethod
    def backward(ctx, g):
        grad = ctx.sim.backward(float(g))
        return grad.to(ctx.dtype), None, None, None


def objective(eps_design, eps_background, sim, rec):
    return FDTDGrad.apply(eps_design, eps_background, sim, rec)


class FDTDGrad2(torch.autograd.Function):
    """(L, M)(eps_design) for a simulation with a second detector.

    forward(eps_design, eps_background, sim, rec) -> float64 tensor [L, M]
    backward: d(gL L + gM M)/d(eps_design) from one time-reversed run with the
    two detectors' seeds (gL, gM) = the incoming gradient.
    """

    @staticmethod
    def forward(ctx, eps_design, eps_background, sim, rec):
        eps = eps_background.detach().clone()
        eps[sim.w.design_slice()] = eps_design.detach().to(torch.float32)
        sim.forward(eps.contiguous(), rec)
        L, M = sim.objectives()
        ctx.sim = sim
        ctx.dtype = eps_design.dtype
        return torch.tensor([L, M], dtype=torch.float64, device=eps.device)

    @staticmethod
    def backward(ctx, g):
        gl, gm = (float(v) for v in g.detach().cpu())
        grad = ctx.sim.backward(gl, seed2=gm)
        return grad.to(ctx.dtype), None, None, None


def objectives(eps_design, eps_background, sim, rec):
    """Differentiable (L, M) of a simulation with a second detector."""
    return FDTDGrad2.apply(eps_design, eps_background, sim, rec)
