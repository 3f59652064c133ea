"""Discrete-adjoint driver: binomial checkpoint replay and the torch.autograd.Function.

Sec. 3.2 of arxiv 2609.30039: the backward sweep replays the forward pass between
checkpoints, with C checkpoints and N steps placed by the binomial schedule of Griewank
(repetition number r = min{r : C(c + r, r) >= n}), checkpoints kept in GPU memory (FP32/FP64
exact copies or BF16 with per-slab scales).  Sec. 3.1: the transposed sweep is exposed to
PyTorch as a custom autograd function whose backward receives the cotangent of the monitor
spectra and returns d(objective)/d(eps^-1) of the design box.

Only scheduling lives here; every forward and transposed step runs in libgbfdtd's kernels.
"""
from __future__ import annotations

from math import comb
import numpy as np
from typing import Callable, Dict, List, Tuple

from . import fdtd as F


def beta(c: int, t: int) -> int:
    """Number of steps reversible with c free checkpoints and t repetitions: C(c + t, t)."""
    return comb(c + t, t)


def repetitions(n: int, c: int) -> int:
    if c <= 0:
        return max(n - 1, 0)    # no free checkpoint: replay from the base for every step
    t = 0
    while beta(c, t) < n:
        t += 1
    return t


def split(l: int, r: int, c: int) -> int:
    """First checkpoint position inside (l, r): the left part keeps c checkpoints and t-1
    repetitions, the right part c-1 checkpoints and t repetitions (binomial schedule)."""
    n = r - l
    t = repetitions(n, c)
    m = min(beta(c, t - 1), n - 1)
    m = max(m, n - beta(c - 1, t), 1)
    return l + m


def spine(n: int, c: int) -> List[int]:
    """Checkpoint positions the first forward sweep stores (the right-most recursion path)."""
    out, l = [], 0
    while n - l > 1 and c > 0:
        s = split(l, n, c)
        out.append(s)
        l, c = s, c - 1
    return out


def schedule(n: int, slots: int) -> List[Tuple]:
    """Actions reversing n steps with `slots` checkpoint slots (slot 0 holds u^0).  Actions:
    ("save", slot, step), ("restore", slot), ("advance", k), ("adjoint", m), ("forward_done",).
    The first sweep runs 0 -> n saving the spine; the reversal then never replays past n."""
    if slots < 1:
        raise ValueError("need at least one checkpoint slot")
    acts: List[Tuple] = [("save", 0, 0)]
    sp = spine(n, slots - 1)
    pos = 0
    for k, s in enumerate(sp):
        acts.append(("advance", s - pos))
        acts.append(("save", k + 1, s))
        pos = s
    acts.append(("advance", n - pos))
    acts.append(("forward_done",))
    stored = {0: 0}
    for k, s in enumerate(sp):
        stored[s] = k + 1
    free = [k for k in range(1, slots) if k not in stored.values()]

    def rev(l: int, r: int, c: int, slot_l: int):
        while r > l:
            if r - l == 1 or c == 0:
                for m in range(r - 1, l - 1, -1):
                    acts.append(("restore", slot_l))
                    if m - l:
                        acts.append(("advance", m - l))
                    acts.append(("adjoint", m))
                return
            s = split(l, r, c)
            if s in stored:
                sl = stored[s]
                own = False
            else:
                sl = free.pop()
                own = True
                acts.append(("restore", slot_l))
                acts.append(("advance", s - l))
                acts.append(("save", sl, s))
                stored[s] = sl
            rev(s, r, c - 1, sl)
            del stored[s]
            free.append(sl)
            r = s

    rev(0, n, slots - 1, 0)
    return acts


def encode(acts) -> np.ndarray:
    """The schedule as (kind, arg) int32 rows for the native executor (fdtd_run_schedule)."""
    rows = []
    for a in acts:
        kind = a[0]
        if kind == "save":
            rows.append((F.FDTD_ACT_SAVE, a[1]))
        elif kind == "restore":
            rows.append((F.FDTD_ACT_RESTORE, a[1]))
        elif kind == "advance":
            rows.append((F.FDTD_ACT_ADVANCE, a[1]))
        elif kind == "adjoint":
            rows.append((F.FDTD_ACT_ADJOINT, 1))
        elif kind == "forward_done":
            rows.append((F.FDTD_ACT_STOP, 0))
        else:
            raise ValueError(f"unknown action {kind}")
    return np.asarray(rows, dtype=np.int32).reshape(-1, 2)


def run_schedule(ctx: "F.Context", acts, objective: Callable, codec: int = F.FDTD_CODEC_NATIVE):
    """Executes a schedule on a Context whose forward state is u^0, in the library's native
    executor (two calls: the forward sweep up to its end, then the reversal).  `objective(ctx)` is
    called in between and must register adjoint sources and design buffers; it returns what
    run_schedule returns."""
    c = ctx.ctx
    rows = encode(acts)
    nxt = F.fdtd_run_schedule(c, rows, 0, codec)
    result = None
    if nxt > 0 and rows[nxt - 1, 0] == F.FDTD_ACT_STOP:
        result = objective(ctx)
        F.fdtd_adjoint_begin(c)
        F.fdtd_dft_enable(c, 0)
        try:
            F.fdtd_run_schedule(c, rows, nxt, codec)
        finally:
            F.fdtd_dft_enable(c, 1)
    return result


def replay_stats(acts) -> Dict[str, int]:
    fwd = sum(a[1] for a in acts if a[0] == "advance")
    return {"forward_steps": fwd, "adjoint_steps": sum(1 for a in acts if a[0] == "adjoint"),
            "saves": sum(1 for a in acts if a[0] == "save"), "restores": sum(1 for a in acts if a[0] == "restore")}


class DesignAdjoint:
    """Gradient of a real objective of the monitor spectra w.r.t. eps^-1 in each domain's design
    box, by one forward sweep and one checkpointed transposed sweep on the GPU."""

    def __init__(self, ctx: "F.Context", slots: int = 32, codec: int = F.FDTD_CODEC_NATIVE,
                 pole_grads: bool = False):
        """pole_grads: also collect d J / d(delta_eps, omega_dt, gamma_dt) of the poles of every
        dispersive domain (read from self.pole_grads after run)."""
        self.ctx = ctx
        self.slots = slots
        self.codec = codec
        torch = ctx.torch
        self.pole_domains = []
        if pole_grads:
            for d, sc in enumerate(ctx.scenes):
                if sc.pole_mask is not None and len(sc.poles):
                    F.fdtd_set_pole_grad(ctx.ctx, d, 1)
                    self.pole_domains.append(d)
        self.pole_grads = {}
        self.grads = []
        for d, sc in enumerate(ctx.scenes):
            if sc.design is None:
                self.grads.append(None)
                continue
            lo, hi = sc.design
            n = (hi[0] - lo[0]) * (hi[1] - lo[1]) * (hi[2] - lo[2])
            # [3][cells] of the diagonal eps^-1, or [6][nodes] of a tensor domain (Sec. 2.3)
            ncomp = 6 if getattr(sc, "tensor", None) is not None else 3
            g = torch.zeros(ncomp * n, dtype=torch.float64, device=ctx.device)
            F.fdtd_set_design(ctx.ctx, d, lo, hi, g.data_ptr())
            self.grads.append(g)

    def run(self, n_steps: int, loss_of_spectra: Callable):
        """loss_of_spectra(list of complex spectra tensors) -> (J float, list of cotangent tensors)."""
        ctx = self.ctx
        acts = schedule(n_steps, self.slots)
        keep = {}

        def objective(cx):
            specs = [cx.dft(k) for k in range(len(cx.monitors))]
            J, cots = loss_of_spectra(specs)
            keep["cots"] = [ct.contiguous() if ct is not None else None for ct in cots]
            for k, ct in enumerate(keep["cots"]):
                F.fdtd_set_adjoint_source(cx.ctx, cx.monitors[k][0], ct.data_ptr() if ct is not None else None)
            for g in self.grads:
                if g is not None:
                    g.zero_()
            return J, specs

        out = run_schedule(ctx, acts, objective, self.codec)
        ctx.synchronize()
        self.pole_grads = {d: F.fdtd_pole_grad(ctx.ctx, d, len(ctx.scenes[d].poles)) for d in self.pole_domains}
        return out, self.grads, replay_stats(acts)


class ReversibleAdjoint(DesignAdjoint):
    """The same gradient without checkpoints, for nondispersive domains (Sec. 3.2: the forward
    fields are rebuilt by stepping Eq. (yee) backward): one forward sweep, then for m = n-1 .. 0 a
    backward step (u^(m+1) -> u^m) and the transposed step m.  Lossless domains step back whole;
    domains with CPML faces use the absorbing-face variant: the forward sweep records the fields at
    the interface between interior and absorber, and the interior -- where every design box lies --
    steps back from it.  Memory: the state plus the interface record; work: one extra step per
    transposed step instead of the binomial replays."""

    def __init__(self, ctx: "F.Context"):
        super().__init__(ctx, slots=1)

    def run(self, n_steps: int, loss_of_spectra: Callable):
        ctx = self.ctx
        c = ctx.ctx
        if any(any(sc.cpml) for sc in ctx.scenes):
            F.fdtd_record_interface(c, n_steps)
        F.fdtd_step_forward(c, n_steps)
        specs = [ctx.dft(k) for k in range(len(ctx.monitors))]
        J, cots = loss_of_spectra(specs)
        keep = [ct.contiguous() if ct is not None else None for ct in cots]
        for k, ct in enumerate(keep):
            F.fdtd_set_adjoint_source(c, ctx.monitors[k][0], ct.data_ptr() if ct is not None else None)
        for g in self.grads:
            if g is not None:
                g.zero_()
        F.fdtd_adjoint_begin(c)
        F.fdtd_dft_enable(c, 0)
        for _ in range(n_steps):
            F.fdtd_step_backward(c, 1)
            F.fdtd_step_adjoint(c, 1)
        F.fdtd_dft_enable(c, 1)
        if any(any(sc.cpml) for sc in ctx.scenes):
            F.fdtd_record_interface(c, 0)
        ctx.synchronize()
        return (J, specs), self.grads, {"forward_steps": n_steps, "backward_steps": n_steps,
                                        "adjoint_steps": n_steps}


class StreamedAdjoint(DesignAdjoint):
    """The same gradient on a host-streamed context (Sec. 4.2: the transposed sweep runs the slab
    tiling in reverse): one forward sweep that keeps its state at every batch start in pinned host
    memory, then the transposed sweep batch by batch, last to first, each slab window replaying its
    batch on the device from the checkpoint.  Device memory: the stepping workspaces, the adjoint
    window and the replayed windows of one batch; host memory: the state, two adjoint state sets and
    one checkpoint per batch, whose pinned buffers are kept for the next run until release() or the
    context's close."""

    def __init__(self, ctx: "F.Context"):
        super().__init__(ctx, slots=1)

    def run(self, n_steps: int, loss_of_spectra: Callable):
        ctx = self.ctx
        c = ctx.ctx
        F.fdtd_stream_checkpoints(c, 1)
        F.fdtd_step_forward(c, n_steps)
        specs = [ctx.dft(k) for k in range(len(ctx.monitors))]
        J, cots = loss_of_spectra(specs)
        keep = [ct.contiguous() if ct is not None else None for ct in cots]
        for k, ct in enumerate(keep):
            F.fdtd_set_adjoint_source(c, ctx.monitors[k][0], ct.data_ptr() if ct is not None else None)
        for g in self.grads:
            if g is not None:
                g.zero_()
        F.fdtd_adjoint_begin(c)
        F.fdtd_step_adjoint(c, n_steps)
        ctx.synchronize()
        # checkpoints off; their pinned buffers stay for the next run (freed with the context)
        F.fdtd_stream_checkpoints(c, 2)
        return (J, specs), self.grads, {"forward_steps": n_steps, "adjoint_steps": n_steps}

    def release(self):
        """Frees the pinned host checkpoint buffers kept between runs."""
        F.fdtd_stream_checkpoints(self.ctx.ctx, 0)


def _make_function():
    import torch

    class FDTDSpectra(torch.autograd.Function):
        """inv_eps of the design box (3 x box, FP64 view) -> monitor spectra (complex128).

        forward runs the sweep on the GPU (storing the spine checkpoints); backward receives
        d(loss)/d(spectra) (torch's convention for a real loss: dL/dRe + i dL/dIm), replays
        with the binomial schedule and returns d(loss)/d(inv_eps of the box)."""

        @staticmethod
        def forward(fctx, inv_eps_box, runner, n_steps):
            runner.set_design_values(inv_eps_box)
            specs = runner.forward(n_steps)
            fctx.runner = runner
            fctx.n_steps = n_steps
            return tuple(specs)

        @staticmethod
        def backward(fctx, *grad_specs):
            g = fctx.runner.backward(grad_specs)
            return g, None, None

    return FDTDSpectra


class Runner:
    """State shared by FDTDSpectra's forward and backward for one domain with a design box."""

    def __init__(self, ctx: "F.Context", domain: int = 0, slots: int = 32, codec: int = F.FDTD_CODEC_NATIVE):
        self.ctx = ctx
        self.domain = domain
        self.slots = slots
        self.codec = codec
        torch = ctx.torch
        sc = ctx.scenes[domain]
        self.lo, self.hi = sc.design
        n = (self.hi[0] - self.lo[0]) * (self.hi[1] - self.lo[1]) * (self.hi[2] - self.lo[2])
        self.ncell = n
        self.grad = torch.zeros(3 * n, dtype=torch.float64, device=ctx.device)
        F.fdtd_set_design(ctx.ctx, domain, self.lo, self.hi, self.grad.data_ptr())
        self.base = [t.clone() for t in ctx.inv_eps[domain]]
        self.acts = None

    def set_design_values(self, box):
        """box: (3, bz, by, bx) tensor of eps^-1 inside the design box."""
        torch = self.ctx.torch
        (lx, ly, lz), (hx, hy, hz) = self.lo, self.hi
        ie = [b.clone() for b in self.base]
        for a in range(3):
            ie[a][lz:hz, ly:hy, lx:hx] = box[a].to(ie[a].dtype)
        self.ctx.set_inv_eps(self.domain, ie)

    def forward(self, n_steps):
        ctx = self.ctx
        F.fdtd_reset(ctx.ctx)
        F.fdtd_dft_reset(ctx.ctx)
        self.acts = schedule(n_steps, self.slots)
        self.rows = encode(self.acts)
        self.cut = F.fdtd_run_schedule(ctx.ctx, self.rows, 0, self.codec)   # up to the STOP
        return [ctx.dft(k).clone() for k in range(len(ctx.monitors))]

    def backward(self, grad_specs):
        torch = self.ctx.torch
        ctx = self.ctx
        cots = []
        for k, g in enumerate(grad_specs):
            ct = torch.zeros_like(ctx.dft(k)) if g is None else g.to(torch.complex128).contiguous()
            cots.append(torch.view_as_real(ct).contiguous())
            F.fdtd_set_adjoint_source(ctx.ctx, ctx.monitors[k][0], cots[-1].data_ptr())
        self.grad.zero_()
        F.fdtd_adjoint_begin(ctx.ctx)
        F.fdtd_dft_enable(ctx.ctx, 0)
        try:
            F.fdtd_run_schedule(ctx.ctx, self.rows, self.cut, self.codec)
        finally:
            F.fdtd_dft_enable(ctx.ctx, 1)
        ctx.synchronize()
        (lx, ly, lz), (hx, hy, hz) = self.lo, self.hi
        out = self.grad.view(3, hz - lz, hy - ly, hx - lx).clone()
        for k in range(len(cots)):
            F.fdtd_set_adjoint_source(ctx.ctx, ctx.monitors[k][0], None)
        return out


_FN = None


def spectra(inv_eps_box, runner: Runner, n_steps: int):
    """Differentiable map eps^-1(design box) -> tuple of monitor spectra (complex128)."""
    global _FN
    if _FN is None:
        _FN = _make_function()
    return _FN.apply(inv_eps_box, runner, n_steps)
