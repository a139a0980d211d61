"""PyTorch-facing API over the C ABI: device buffers, streams and autograd.

PyTorch supplies device memory (output tensors and the workspace are torch
allocations owned by the caller of the C ABI) and the current CUDA stream.
Every step of the simulation runs in the CUDA library.
"""
from __future__ import annotations

import ctypes
from typing import Dict, Optional

import numpy as np
import torch

from . import capi
from .workloads import Batch, Model


class CompiledModel:
    """A model compiled and uploaded by cwc_model_create."""

    def __init__(self, model: Model):
        m = model.contiguous()
        self.model = m
        self._keep = (m.kind, m.ctx_label, m.child_label, m.lhs, m.rhs, m.grand_label, m.lhs_ext, m.rhs_ext,
                      m.rate_law, m.rate_par)

        def ptr(a):
            return None if a is None else a.ctypes.data

        desc = capi.cwc_model_desc(m.n_species, m.n_labels, m.n_rules, m.max_compartments,
                                   m.kind.ctypes.data, m.ctx_label.ctypes.data, m.child_label.ctypes.data,
                                   m.lhs.ctypes.data, m.rhs.ctypes.data,
                                   ptr(m.grand_label), ptr(m.lhs_ext), ptr(m.rhs_ext),
                                   ptr(m.rate_law), ptr(m.rate_par))
        self.handle = capi.cwc_model_create(desc)
        self.n_observables = capi.cwc_model_num_observables(self.handle)
        self.flat = m.n_labels == 1 and m.max_compartments == 1

    def close(self) -> None:
        if getattr(self, "handle", None):
            capi.cwc_model_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _p(t: Optional[torch.Tensor]):
    return None if t is None else t.data_ptr()


def _stream_handle(stream: Optional[torch.cuda.Stream]) -> int:
    s = stream if stream is not None else torch.cuda.current_stream()
    return s.cuda_stream


def device_inputs(batch: Batch, device="cuda"):
    """Copy a batch's inputs to the device: rates [P,M] f64, init int32, grid [G] f64."""
    return (torch.from_numpy(np.ascontiguousarray(batch.rates)).to(device),
            torch.from_numpy(np.ascontiguousarray(batch.init)).to(device),
            torch.from_numpy(np.ascontiguousarray(batch.grid)).to(device))


def _sim_args(cm: CompiledModel, rates, init, grid, R, seed, max_events, layout, block_threads, deadline_ns,
              replica_offset=0, lanes=0):
    P = rates.shape[0]
    a = capi.cwc_sim_args()
    a.P, a.R, a.G, a.Pi = P, R, grid.shape[0], init.shape[0]
    a.replica_offset = replica_offset
    a.rates, a.init, a.grid = _p(rates), _p(init), _p(grid)
    a.seed = seed & 0xFFFFFFFFFFFFFFFF
    a.max_events = max_events
    a.layout, a.block_threads, a.deadline_ns = layout, block_threads, deadline_ns
    a.lanes = lanes
    return a


def _check_inputs(cm, rates, init, grid):
    for name, t, dt in (("rates", rates, torch.float64), ("init", init, torch.int32), ("grid", grid, torch.float64)):
        if not t.is_cuda or t.dtype != dt or not t.is_contiguous():
            raise ValueError("%s must be a contiguous CUDA %s tensor" % (name, dt))
    if rates.dim() != 2 or rates.shape[1] != cm.model.n_rules:
        raise ValueError("rates must be [P, M]")


def _workspace(nbytes: int, device) -> Optional[torch.Tensor]:
    if nbytes == 0:
        return None
    return torch.empty(nbytes + 256, dtype=torch.uint8, device=device)


def _aligned(ws: Optional[torch.Tensor]) -> int:
    if ws is None:
        return 0
    p = ws.data_ptr()
    return (p + 255) & ~255


def simulate(cm: CompiledModel, rates: torch.Tensor, init: torch.Tensor, grid: torch.Tensor, R: int, seed: int,
             max_events: int = (1 << 32) - 1, *, states: bool = True, sums: bool = False, means: bool = False,
             sumsq: bool = False, variance: bool = False, ci90: bool = False,
             traj: bool = True, log_cap: int = 0, layout: int = capi.CWC_LAYOUT_AUTO, block_threads: int = 0,
             lanes: int = 0, deadline_ns: int = 0, replica_offset: int = 0, checkpoint: bool = False,
             resume: bool = False, tail_threshold: int = 0, term_bits: int = 0,
             stream: Optional[torch.cuda.Stream] = None,
             out: Optional[Dict[str, torch.Tensor]] = None) -> Dict[str, torch.Tensor]:
    """Run P x R trajectories (cwc_simulate) and return the requested outputs.

    ``out`` may hold preallocated output tensors of the right shapes (reused
    across calls, e.g. by a benchmark loop or a CUDA graph).
    """
    _check_inputs(cm, rates, init, grid)
    dev = rates.device
    P, G, O, M = rates.shape[0], grid.shape[0], cm.n_observables, cm.model.n_rules
    res: Dict[str, torch.Tensor] = {} if out is None else dict(out)

    def get(name, shape, dtype):
        t = res.get(name)
        if t is None:
            t = torch.empty(shape, dtype=dtype, device=dev)
            res[name] = t
        return t

    a = _sim_args(cm, rates, init, grid, R, seed, max_events, layout, block_threads, deadline_ns, replica_offset, lanes)
    a.tail_threshold = tail_threshold
    a.term_bits = term_bits
    if states:
        a.states = _p(get("states", (P, R, G, O), torch.int32))
    if sums:
        a.sums = _p(get("sums", (P, G, O), torch.int64))
    if means:
        a.means = _p(get("means", (P, G, O), torch.float64))
    if sumsq:
        a.sumsq = _p(get("sumsq", (P, G, O, 2), torch.int64))
    if variance:
        a.variance = _p(get("variance", (P, G, O), torch.float64))
    if ci90:
        a.ci90 = _p(get("ci90", (P, G, O), torch.float64))
    if traj:
        a.traj_status = _p(get("status", (P, R), torch.int32))
        a.traj_events = _p(get("events", (P, R), torch.int64))
        a.traj_hash = _p(get("hash", (P, R), torch.int64))
        a.traj_final_t = _p(get("final_t", (P, R), torch.float64))
    if log_cap > 0:
        a.log_cap = log_cap
        a.log_rule = _p(get("log_rule", (P, R, log_cap), torch.int32))
        a.log_slot = _p(get("log_slot", (P, R, log_cap), torch.int32))
        a.log_t = _p(get("log_t", (P, R, log_cap), torch.float64))
    if checkpoint or resume:
        words = capi.cwc_checkpoint_words(cm.handle)
        a.checkpoint = _p(get("checkpoint", (P, R, words), torch.int32))
        a.resume = 1 if resume else 0
    nbytes = capi.cwc_simulate_workspace_size(cm.handle, a)
    ws = res.get("_workspace")
    if nbytes and (ws is None or ws.numel() < nbytes + 256):
        ws = _workspace(nbytes, dev)
        res["_workspace"] = ws
    a.workspace = _aligned(ws) if nbytes else None
    a.workspace_bytes = nbytes
    capi.cwc_simulate(cm.handle, a, _stream_handle(stream))
    return res


def simulate_sliced(cm: CompiledModel, rates: torch.Tensor, init: torch.Tensor, grid: torch.Tensor, R: int,
                    seed: int, max_events: int = (1 << 32) - 1, *, slice_ns: int, max_slices: int = 1 << 20,
                    on_slice=None, stream: Optional[torch.cuda.Stream] = None, **kw):
    """Run the batch as a sequence of launches of at most ``slice_ns`` of
    device time each: every launch stops the trajectories still running at
    its deadline and saves them in the checkpoint buffer, the next resumes
    them (the time-sliced, stoppable instances of Sec. 5.2).  Between slices
    the GPU is free for other work on other streams, and ``on_slice(i,
    remaining)`` sees the number of trajectories still to finish.  Returns
    (outputs, slices); the outputs equal one uninterrupted ``simulate`` bit
    for bit.  Takes ``simulate``'s keyword arguments except the reductions
    over replicas (which checkpoints exclude)."""
    if slice_ns <= 0:
        raise ValueError("slice_ns must be > 0")
    kw.pop("traj", None)
    out = simulate(cm, rates, init, grid, R, seed, max_events, traj=True, checkpoint=True, deadline_ns=slice_ns,
                   stream=stream, **kw)
    slices = 1
    while True:
        (stream or torch.cuda.current_stream(rates.device)).synchronize()
        remaining = int((out["status"] == capi.CWC_TRAJ_TIMEOUT).sum().item())
        if on_slice is not None:
            on_slice(slices, remaining)
        if remaining == 0:
            return out, slices
        if slices >= max_slices:
            raise RuntimeError("%d trajectories still running after %d slices" % (remaining, slices))
        out = simulate(cm, rates, init, grid, R, seed, max_events, traj=True, resume=True, deadline_ns=slice_ns,
                       stream=stream, out=out, **kw)
        slices += 1


def sensitivity(cm: CompiledModel, rates, init, grid, R: int, seed: int, means: torch.Tensor,
                grad_means: torch.Tensor, max_events: int = (1 << 32) - 1, *, partials: bool = False,
                layout: int = capi.CWC_LAYOUT_AUTO, block_threads: int = 0, lanes: int = 0,
                stream: Optional[torch.cuda.Stream] = None) -> Dict[str, torch.Tensor]:
    """d L / d k by likelihood-ratio replay (cwc_sensitivity); returns grad_rates [P, M]."""
    _check_inputs(cm, rates, init, grid)
    dev = rates.device
    P, M = rates.shape
    means = means.contiguous()
    grad_means = grad_means.contiguous().to(torch.float64)
    a = _sim_args(cm, rates, init, grid, R, seed, max_events, layout, block_threads, 0, 0, lanes)
    s = capi.cwc_sens_args()
    grad = torch.empty((P, M), dtype=torch.float64, device=dev)
    s.means, s.grad_means, s.grad_rates = _p(means), _p(grad_means), _p(grad)
    part = None
    if partials:
        part = torch.empty((P, R, M), dtype=torch.float64, device=dev)
        s.partials = _p(part)
    nbytes = capi.cwc_sensitivity_workspace_size(cm.handle, a, s)
    ws = _workspace(nbytes, dev)
    a.workspace = _aligned(ws) if nbytes else None
    a.workspace_bytes = nbytes
    capi.cwc_sensitivity(cm.handle, a, s, _stream_handle(stream))
    out = {"grad_rates": grad, "_workspace": ws}
    if part is not None:
        out["partials"] = part
    return out


class MeanObservables(torch.autograd.Function):
    """Forward: E[X_o(g)] per sweep point (exact int64 sums over R replicas /
    R), [P, G, O] float64.  Backward: likelihood-ratio gradient with respect
    to the rates, by replaying each trajectory's Philox stream."""

    @staticmethod
    def forward(ctx, rates, cm, init, grid, R, seed, max_events=(1 << 32) - 1):
        res = simulate(cm, rates.detach().contiguous(), init, grid, R, seed, max_events,
                       states=False, means=True, traj=False)
        m = res["means"]
        ctx.save_for_backward(rates.detach(), init, grid, m)
        ctx.cm, ctx.R, ctx.seed, ctx.max_events = cm, R, seed, max_events
        return m

    @staticmethod
    def backward(ctx, grad_means):
        rates, init, grid, m = ctx.saved_tensors
        g = sensitivity(ctx.cm, rates.contiguous(), init, grid, ctx.R, ctx.seed, m, grad_means, ctx.max_events)
        return g["grad_rates"], None, None, None, None, None, None


def mean_observables(rates, cm, init, grid, R, seed, max_events=(1 << 32) - 1):
    return MeanObservables.apply(rates, cm, init, grid, R, seed, max_events)


def simulate_host(cm: CompiledModel, rates_h: torch.Tensor, init_h: torch.Tensor, grid_h: torch.Tensor, R: int,
                  seed: int, max_events: int = (1 << 32) - 1, *, dev_bufs: Optional[dict] = None,
                  host_out: Optional[torch.Tensor] = None, stream: Optional[torch.cuda.Stream] = None,
                  direct: bool = True, **kw) -> torch.Tensor:
    """End-to-end call from host (pinned) tensors: copy the inputs to the
    device, simulate, and return the grid states in ``host_out`` (page-locked
    host memory).  With ``direct`` the kernel writes the states into
    ``host_out`` itself while it runs (over NVLink-C2C on Grace systems);
    otherwise they go to device memory and are copied back afterwards."""
    st = stream if stream is not None else torch.cuda.current_stream()
    bufs = dev_bufs if dev_bufs is not None else {}
    with torch.cuda.stream(st):
        d_rates = bufs.setdefault("rates", torch.empty_like(rates_h, device="cuda"))
        d_init = bufs.setdefault("init", torch.empty_like(init_h, device="cuda"))
        d_grid = bufs.setdefault("grid", torch.empty_like(grid_h, device="cuda"))
        d_rates.copy_(rates_h, non_blocking=True)
        d_init.copy_(init_h, non_blocking=True)
        d_grid.copy_(grid_h, non_blocking=True)
        P, G = rates_h.shape[0], grid_h.shape[0]
        if host_out is None:
            host_out = torch.empty((P, R, G, cm.n_observables), dtype=torch.int32, pin_memory=True)
        out = dict(bufs.get("out") or {})
        if direct:
            out["states"] = host_out
        elif "states" in out and out["states"].device.type != "cuda":
            del out["states"]
        res = simulate(cm, d_rates, d_init, d_grid, R, seed, max_events, out=out, stream=st, **kw)
        bufs["out"] = res
        if not direct:
            host_out.copy_(res["states"], non_blocking=True)
    return host_out


def autotune(cm: CompiledModel, rates, init, grid, R: int, seed: int, max_events: int = (1 << 32) - 1,
             tune_events: int = 0, stream: Optional[torch.cuda.Stream] = None):
    """cwc_autotune on this batch: returns (layout, block_threads, lanes, ms)
    and caches the choice for later automatic calls on the same shape."""
    _check_inputs(cm, rates, init, grid)
    nbytes = 0
    for lanes in ((1,) if cm.flat else (1, 4, 8)):
        for lay in (capi.CWC_LAYOUT_STATIC, capi.CWC_LAYOUT_QUEUE):
            for T in range(32, 257, 32):
                a = _sim_args(cm, rates, init, grid, R, seed, max_events, lay, T, 0, 0, lanes)
                try:
                    nbytes = max(nbytes, capi.cwc_simulate_workspace_size(cm.handle, a))
                except capi.CwcError:
                    pass
    ws = _workspace(nbytes, rates.device)
    a = _sim_args(cm, rates, init, grid, R, seed, max_events, capi.CWC_LAYOUT_AUTO, 0, 0)
    a.workspace = _aligned(ws) if nbytes else None
    a.workspace_bytes = nbytes
    return capi.cwc_autotune(cm.handle, a, tune_events, _stream_handle(stream))


class GraphedSimulation:
    """One cwc_simulate call captured in a CUDA graph over static buffers.

    ``replay(rates=..., init=..., grid=...)`` copies new inputs (same shapes)
    into the captured buffers and relaunches the graph; the outputs are the
    tensors in ``self.out`` (overwritten by every replay).  The seed and the
    batch shape are part of the capture.
    """

    def __init__(self, cm: CompiledModel, rates, init, grid, R: int, seed: int,
                 max_events: int = (1 << 32) - 1, **kw):
        self.rates = rates.clone()
        self.init = init.clone()
        self.grid = grid.clone()
        side = torch.cuda.Stream()
        side.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(side):
            self.out = simulate(cm, self.rates, self.init, self.grid, R, seed, max_events, stream=side, **kw)
        torch.cuda.current_stream().wait_stream(side)
        torch.cuda.synchronize()
        self.graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(self.graph, capture_error_mode="thread_local"):
            self.out = simulate(cm, self.rates, self.init, self.grid, R, seed, max_events, out=self.out,
                                stream=torch.cuda.current_stream(), **kw)

    def replay(self, rates=None, init=None, grid=None) -> Dict[str, torch.Tensor]:
        if rates is not None:
            self.rates.copy_(rates)
        if init is not None:
            self.init.copy_(init)
        if grid is not None:
            self.grid.copy_(grid)
        self.graph.replay()
        return self.out
