"""CPU oracle for batched Gillespie / CWC simulation -- TEST INFRASTRUCTURE.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline legs of
``bench.py`` may import this package.  The CUDA library never does, and the
oracle imports nothing from it (inputs come from
``paper_1010_2438_gb300.workloads``, which holds no simulation arithmetic).

The arithmetic lives in ``cwc_oracle.c`` (plain sequential C, built without
FMA contraction); this module only marshals numpy arrays through ctypes.
ctypes releases the GIL during foreign calls, so ``threads > 1`` runs
disjoint trajectory ranges in parallel.
"""
from __future__ import annotations

import ctypes
import itertools
import os
import threading
from concurrent.futures import ThreadPoolExecutor
from typing import Dict, Optional

import numpy as np

from . import build as _build

ST_OK, ST_ABSORBED, ST_INT_OVERFLOW, ST_PROP_OVERFLOW, ST_CAPACITY, ST_EVENT_LIMIT, ST_BAD_INPUT = range(7)

_lib = None
_lib_lock = threading.Lock()


class _Model(ctypes.Structure):
    _fields_ = [
        ("S", ctypes.c_int32), ("L", ctypes.c_int32), ("C", ctypes.c_int32), ("M", ctypes.c_int32),
        ("kind", ctypes.c_void_p), ("ctx_label", ctypes.c_void_p), ("child_label", ctypes.c_void_p),
        ("grand_label", ctypes.c_void_p), ("lhs", ctypes.c_void_p), ("rhs", ctypes.c_void_p),
        ("rate_law", ctypes.c_void_p), ("rate_par", ctypes.c_void_p),
    ]


def lib():
    global _lib
    with _lib_lock:
        return _lib if _lib is not None else _load()


# A patched copy of the oracle, loaded instead of the built one when this
# variable names it: tests/test_oracle_mutants.py plants one mistake per copy
# (in the C source, on the CPU) to show that the pins catch it.  Unset
# otherwise.
LIBRARY_ENV = "CWC_ORACLE_LIBRARY"


def _load():
    global _lib
    path = os.environ.get(LIBRARY_ENV) or _build.build()
    L = ctypes.CDLL(path)
    vp, i32, i64, u64, dbl = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64, ctypes.c_double
    L.oracle_philox4x32_10.argtypes = [vp, vp, vp]
    L.oracle_philox_array.argtypes = [vp, vp, vp, i64]
    L.oracle_u52.argtypes = [ctypes.c_uint32, ctypes.c_uint32]
    L.oracle_u52.restype = dbl
    L.oracle_log_spec.argtypes = [dbl]
    L.oracle_log_spec.restype = dbl
    L.oracle_log_spec_array.argtypes = [vp, vp, i64]
    L.oracle_tree_sum.argtypes = [vp, i32]
    L.oracle_tree_sum.restype = dbl
    L.oracle_select.argtypes = [vp, i32, dbl]
    L.oracle_select.restype = i32
    L.oracle_num_observables.argtypes = [vp]
    L.oracle_num_observables.restype = i32
    L.oracle_rule_totals.argtypes = [vp, vp, vp]
    L.oracle_rule_totals.restype = ctypes.c_int
    L.oracle_rule_h.argtypes = [vp, vp, vp]
    L.oracle_rule_h.restype = ctypes.c_int
    L.oracle_simulate.argtypes = [
        vp, vp, i32, i32, vp, i32, vp, i32, u64, i64, i64, i64,
        vp, vp, vp, vp, vp, i32, vp, vp, vp, vp, vp, vp]
    L.oracle_simulate.restype = ctypes.c_int
    _lib = L
    return _lib


def _ptr(a: Optional[np.ndarray]):
    return None if a is None else a.ctypes.data


class _ModelHandle:
    """Keeps the numpy arrays alive while the C struct points at them."""

    def __init__(self, model):
        m = model.contiguous()
        lhs5, rhs5, grand = m.rows5()        # pattern rows 0-4 (rows 3-4 zero for the 3-row kinds)
        law = None if m.rate_law is None else np.ascontiguousarray(m.rate_law, np.int32)
        par = None if m.rate_par is None else np.ascontiguousarray(m.rate_par, np.float64)
        self.arrays = (m.kind, m.ctx_label, m.child_label, grand, lhs5, rhs5, law, par)
        self.struct = _Model(m.n_species, m.n_labels, m.max_compartments, m.n_rules,
                             _ptr(m.kind), _ptr(m.ctx_label), _ptr(m.child_label), _ptr(grand),
                             _ptr(lhs5), _ptr(rhs5), _ptr(law), _ptr(par))

    @property
    def ref(self):
        return ctypes.byref(self.struct)


# ---------------------------------------------------------------------------
# Scalar routines
# ---------------------------------------------------------------------------

def philox(ctr, key) -> np.ndarray:
    """Philox4x32-10 of counters ``ctr`` [n, 4] (uint32) under ``key`` (2 words)."""
    c = np.ascontiguousarray(np.atleast_2d(np.asarray(ctr, dtype=np.uint32)))
    k = np.ascontiguousarray(np.asarray(key, dtype=np.uint32))
    out = np.empty_like(c)
    lib().oracle_philox_array(_ptr(c), _ptr(k), _ptr(out), c.shape[0])
    return out


def u52(wa: int, wb: int) -> float:
    return lib().oracle_u52(wa & 0xFFFFFFFF, wb & 0xFFFFFFFF)


def log_spec(u) -> np.ndarray:
    x = np.ascontiguousarray(np.asarray(u, dtype=np.float64).ravel())
    out = np.empty_like(x)
    lib().oracle_log_spec_array(_ptr(x), _ptr(out), x.size)
    return out


def tree_sum(a) -> float:
    x = np.ascontiguousarray(np.asarray(a, dtype=np.float64))
    return lib().oracle_tree_sum(_ptr(x), x.size)


def select(a, x: float) -> int:
    arr = np.ascontiguousarray(np.asarray(a, dtype=np.float64))
    return lib().oracle_select(_ptr(arr), arr.size, float(x))


def num_observables(model) -> int:
    h = _ModelHandle(model)
    return lib().oracle_num_observables(h.ref)


def rule_totals(model, term) -> np.ndarray:
    """H_j (combinatorial counts summed over contexts) of every rule at ``term``."""
    h = _ModelHandle(model)
    t = np.ascontiguousarray(np.asarray(term, dtype=np.int32))
    out = np.zeros(model.n_rules, np.int64)
    rc = lib().oracle_rule_totals(h.ref, _ptr(t), _ptr(out))
    if rc != 0:
        raise ValueError("invalid term or int64 overflow")
    return out


def rule_h(model, counts) -> np.ndarray:
    """h_j of every rule of a flat model at ``counts`` [S], as doubles: the
    number of reactant combinations, or the Michaelis-Menten value."""
    h = _ModelHandle(model)
    x = np.ascontiguousarray(np.asarray(counts, dtype=np.int32))
    out = np.zeros(model.n_rules, np.float64)
    if lib().oracle_rule_h(h.ref, _ptr(x), _ptr(out)) != 0:
        raise ValueError("int64 overflow")
    return out


# ---------------------------------------------------------------------------
# Simulation
# ---------------------------------------------------------------------------

def simulate(batch, q_begin: int = 0, q_end: Optional[int] = None, *, states: bool = True,
             log_cap: int = 0, means: Optional[np.ndarray] = None,
             grad_means: Optional[np.ndarray] = None, threads: int = 1,
             rates: Optional[np.ndarray] = None, seed: Optional[int] = None,
             max_events: Optional[int] = None, schedule: str = "static") -> Dict[str, np.ndarray]:
    """Run trajectories q in [q_begin, q_end) (q = p*R + r) of ``batch``.

    With ``threads > 1`` the trajectories are split over threads either
    statically (``schedule="static"``: one contiguous range per thread) or on
    demand (``schedule="farm"``: each thread takes the next unstarted
    trajectory whenever it finishes one, the task farm of independent
    simulation instances of Sec. 5.2, so uneven trajectory lengths do not
    leave threads idle).  Results do not depend on the split.

    Returns a dict with ``status``, ``events``, ``hash``, ``final_t`` [nq],
    ``states`` [nq, G, O] (if requested), ``log_rule/log_slot/log_t``
    [nq, log_cap] (if log_cap > 0) and ``partials`` [nq, M] (if ``means`` and
    ``grad_means`` [P, G, O] are given).
    """
    model = batch.model
    h = _ModelHandle(model)
    P, R, G, M = batch.P, batch.R, batch.G, model.n_rules
    O = model.n_observables
    if q_end is None:
        q_end = P * R
    nq = q_end - q_begin
    rates = np.ascontiguousarray(batch.rates if rates is None else rates, dtype=np.float64)
    init = np.ascontiguousarray(batch.init, dtype=np.int32)
    Pi = init.shape[0]
    grid = np.ascontiguousarray(batch.grid, dtype=np.float64)
    seed = batch.seed if seed is None else seed
    max_events = batch.max_events if max_events is None else max_events
    out: Dict[str, np.ndarray] = {
        "status": np.zeros(nq, np.int32),
        "events": np.zeros(nq, np.int64),
        "hash": np.zeros(nq, np.uint64),
        "final_t": np.zeros(nq, np.float64),
    }
    if states:
        out["states"] = np.zeros((nq, G, O), np.int32)
    if log_cap > 0:
        out["log_rule"] = np.full((nq, log_cap), -1, np.int32)
        out["log_slot"] = np.full((nq, log_cap), -1, np.int32)
        out["log_t"] = np.zeros((nq, log_cap), np.float64)
    score = means is not None and grad_means is not None
    if score:
        means = np.ascontiguousarray(means, dtype=np.float64)
        grad_means = np.ascontiguousarray(grad_means, dtype=np.float64)
        out["partials"] = np.zeros((nq, M), np.float64)

    def run(lo: int, hi: int) -> int:
        off = lo - q_begin

        def sl(name, row_elems):
            a = out.get(name)
            return None if a is None else a.ctypes.data + off * row_elems * a.itemsize

        return lib().oracle_simulate(
            h.ref, _ptr(rates), P, R, _ptr(init), Pi, _ptr(grid), G,
            seed & 0xFFFFFFFFFFFFFFFF, max_events, lo, hi,
            sl("states", G * O), sl("status", 1), sl("events", 1), sl("hash", 1), sl("final_t", 1),
            log_cap, sl("log_rule", log_cap), sl("log_slot", log_cap), sl("log_t", log_cap),
            _ptr(means) if score else None, _ptr(grad_means) if score else None,
            sl("partials", M))

    if nq <= 0:
        return out
    threads = max(1, min(threads, nq))
    if threads == 1:
        rc = run(q_begin, q_end)
        if rc != 0:
            raise ValueError("oracle rejected the model")
    elif schedule == "farm":
        tickets = itertools.count(q_begin)
        lock = threading.Lock()

        def worker(_):
            rc = 0
            while True:
                with lock:
                    q = next(tickets)
                if q >= q_end:
                    return rc
                rc |= run(q, q + 1)

        with ThreadPoolExecutor(threads) as ex:
            rcs = list(ex.map(worker, range(threads)))
        if any(rcs):
            raise ValueError("oracle rejected the model")
    elif schedule == "static":
        bounds = [q_begin + (nq * i) // threads for i in range(threads + 1)]
        with ThreadPoolExecutor(threads) as ex:
            rcs = list(ex.map(lambda i: run(bounds[i], bounds[i + 1]), range(threads)))
        if any(rcs):
            raise ValueError("oracle rejected the model")
    else:
        raise ValueError("schedule must be 'static' or 'farm'")
    return out


def sums(states: np.ndarray, P: int, R: int) -> np.ndarray:
    """Exact per-sweep-point sums over replicas: [P, G, O] int64."""
    nq, G, O = states.shape
    return states.reshape(P, R, G, O).astype(np.int64).sum(axis=1)


Z90 = 1.6448536269514722   # the double nearest the 0.95 quantile of N(0, 1)


def replica_stats(states: np.ndarray, P: int, R: int):
    """Per (p, g, o): exact sum and sum of squares over replicas (Python
    integers), sample variance RN(R*sumsq - sum^2) / (R*(R-1)) and the 90 %
    normal-approximation half-width Z90 * sqrt(variance / R), each a single
    IEEE double operation (the on-line mean / variance / confidence reduction
    of the multi-instance simulator, Sec. 5.2)."""
    nq, G, O = states.shape
    x = states.reshape(P, R, G, O).astype(object)
    s = x.sum(axis=1)
    q = (x * x).sum(axis=1)
    num = R * q - s * s
    numf = np.array([float(v) for v in num.ravel()], dtype=np.float64).reshape(num.shape)
    if R > 1:
        var = numf / (np.float64(R) * np.float64(R - 1))
    else:
        var = np.zeros(num.shape, np.float64)
    ci = np.float64(Z90) * np.sqrt(var / np.float64(R))
    return s, q, var, ci


def mean_observables(batch, threads: int = 1) -> np.ndarray:
    """E[X(g)] estimate per sweep point: exact int64 sum over R, one division."""
    st = simulate(batch, states=True, threads=threads)["states"]
    return sums(st, batch.P, batch.R).astype(np.float64) / batch.R


def sensitivity(batch, means: np.ndarray, grad_means: np.ndarray, threads: int = 1):
    """dL/dk [P, M] = (1/R) sum_r partial_r, and the per-trajectory partials [P*R, M]."""
    res = simulate(batch, states=False, means=means, grad_means=grad_means, threads=threads)
    part = res["partials"]
    grad = part.reshape(batch.P, batch.R, -1).sum(axis=1) / batch.R
    return grad, part
