"""Python binding of the adjoint of the collisionless EC explicit step
(pic_adj_* in include/pic.h) and its torch.autograd.Function.

``AdjointRun`` owns the device arena (a torch uint8 tensor) and forwards to
libpic.so; ``ECStepFn.apply(rf_volt, vx0, run, cell0, off0)`` returns the
time-averaged absorbed power and current density of a K-step run as a
float64 tensor [2], and its backward gives d/d rf_volt and d/d vx0 from one
reverse sweep of the library's adjoint kernels.  PyTorch only supplies
memory, streams and the autograd bookkeeping.
"""
from __future__ import annotations

import ctypes

from . import _abi


def make_adj_config(spec: dict) -> _abi.PicAdjConfig:
    c = _abi.PicAdjConfig()
    c.boundary = _abi.BOUNDARY_PERIODIC if spec.get("periodic", False) else _abi.BOUNDARY_ELECTRODES
    c.n_cells = int(spec["n_cells"])
    c.checkpoint_every = int(spec.get("checkpoint_every", 20))
    c.n_particles = int(spec["n_particles"])
    c.nsteps = int(spec["nsteps"])
    c.step0 = int(spec.get("step0", 0))
    c.length = float(spec["length"])
    c.dt = float(spec["dt"])
    c.rf_freq = float(spec.get("rf_freq", 0.0))
    c.n0 = float(spec["n0"])
    c.bg_density = float(spec.get("bg_density", spec["n0"]))
    return c


class AdjointRun:
    """A collisionless EC run of n_particles electrons on a frozen ion
    background, K steps, with checkpointed reverse-mode derivatives."""

    def __init__(self, spec: dict, device="cuda", stream=None):
        import torch

        self.spec = dict(spec)
        self._c = make_adj_config(spec)
        self.n = int(self._c.n_particles)
        self.device = torch.device(device)
        s = _abi.PicSizes()
        _abi.check(_abi.lib().pic_adj_required_sizes(ctypes.byref(self._c), ctypes.byref(s)))
        with torch.cuda.device(self.device):
            self.arena = torch.empty(int(s.arena_bytes), dtype=torch.uint8, device=self.device)
            self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        bufs = _abi.PicBuffers(self.arena.data_ptr(), int(s.arena_bytes))
        h = ctypes.c_void_p()
        with torch.cuda.device(self.device):
            _abi.check(_abi.lib().pic_adj_init(ctypes.byref(self._c), ctypes.byref(bufs),
                                               ctypes.c_void_p(self.stream.cuda_stream), ctypes.byref(h)))
        self._h = h
        self.generation = 0  # bumped by every forward run (the checkpoints it owns)

    def close(self):
        h = getattr(self, "_h", None)
        if h:
            _abi.lib().pic_adj_free(h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _dev(self, t, dtype):
        import torch
        t = t.to(device=self.device, dtype=dtype).contiguous()
        if t.numel() != self.n:
            raise ValueError("expected %d entries, got %d" % (self.n, t.numel()))
        return t

    def forward(self, rf_volt: float, cell0, off0, vx0) -> tuple[float, float]:
        """Run K steps from (cell0, off0, vx0 = v^{-1/2}); returns (<P>, <G>)."""
        import torch
        cell0 = self._dev(cell0, torch.int32)
        off0 = self._dev(off0, torch.float32)
        vx0 = self._dev(vx0, torch.float32)
        out = (ctypes.c_double * 2)()
        _abi.check(_abi.lib().pic_adj_forward(self._h, float(rf_volt), ctypes.c_void_p(cell0.data_ptr()),
                                              ctypes.c_void_p(off0.data_ptr()), ctypes.c_void_p(vx0.data_ptr()),
                                              out))
        self.generation += 1
        return float(out[0]), float(out[1])

    def backward(self, c_power: float, c_flux: float, want_x0: bool = False):
        """dJ/dv^{-1/2} (float32 tensor), dJ/dx^0 per metre (or None) and dJ/d rf_volt
        for J = c_power <P> + c_flux <G> of the last forward run."""
        import torch
        g_v = torch.empty(self.n, dtype=torch.float32, device=self.device)
        g_x = torch.empty(self.n, dtype=torch.float32, device=self.device) if want_x0 else None
        dv = ctypes.c_double()
        _abi.check(_abi.lib().pic_adj_backward(self._h, float(c_power), float(c_flux),
                                               ctypes.c_void_p(g_v.data_ptr()),
                                               ctypes.c_void_p(g_x.data_ptr()) if g_x is not None else None,
                                               ctypes.byref(dv)))
        return g_v, g_x, float(dv.value)

    def final_state(self):
        import numpy as np
        cell = np.zeros(self.n, np.int32)
        off = np.zeros(self.n, np.float32)
        vx = np.zeros(self.n, np.float32)
        _abi.check(_abi.lib().pic_adj_final_state(self._h, cell.ctypes.data, off.ctypes.data, vx.ctypes.data))
        return {"cell": cell, "off": off, "vx": vx}


def _ec_step_fn():
    import torch

    class ECStepFn(torch.autograd.Function):
        """(rf_volt, vx0) -> [<P>, <G>] of a collisionless EC run; gradients by
        the library's reverse sweep (absorptions held fixed)."""

        @staticmethod
        def forward(ctx, rf_volt, vx0, run: AdjointRun, cell0, off0):
            p, g = run.forward(float(rf_volt), cell0, off0, vx0.detach())
            ctx.run = run
            ctx.inputs = (float(rf_volt), cell0, off0, vx0.detach())
            ctx.generation = run.generation
            ctx.vx_dtype = vx0.dtype
            return torch.tensor([p, g], dtype=torch.float64, device=vx0.device)

        @staticmethod
        def backward(ctx, grad_out):
            run = ctx.run
            if run.generation != ctx.generation:  # another forward run took the checkpoints
                v, c0, o0, x0 = ctx.inputs
                run.forward(v, c0, o0, x0)
                ctx.generation = run.generation
            go = grad_out.detach().to("cpu", torch.float64)
            g_v, _, d_volt = run.backward(float(go[0]), float(go[1]))
            return (torch.tensor(d_volt, dtype=torch.float64), g_v.to(ctx.vx_dtype), None, None, None)

    return ECStepFn


def __getattr__(name):
    if name == "ECStepFn":
        fn = _ec_step_fn()
        globals()["ECStepFn"] = fn
        return fn
    raise AttributeError(name)
