"""ctypes binding of the C ABI in include/cwcgpu.h (argument marshalling only).

Every function here has the name of the C entry point it calls.  Nothing is
computed in Python: all simulation work runs in the CUDA library
``_lib/libcwcgpu.so``, which must have been built for sm_103a
(``python -m paper_1010_2438_gb300.build``).  If it is missing, ``lib()``
raises; there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libcwcgpu.so")

CWC_OK, CWC_ERR_INVALID_ARG, CWC_ERR_UNSUPPORTED, CWC_ERR_CUDA, CWC_ERR_WORKSPACE, CWC_ERR_INTERNAL = range(6)
STATUS_NAMES = {0: "CWC_OK", 1: "CWC_ERR_INVALID_ARG", 2: "CWC_ERR_UNSUPPORTED", 3: "CWC_ERR_CUDA",
                4: "CWC_ERR_WORKSPACE", 5: "CWC_ERR_INTERNAL"}
(CWC_TRAJ_OK, CWC_TRAJ_ABSORBED, CWC_TRAJ_INT_OVERFLOW, CWC_TRAJ_PROP_OVERFLOW, CWC_TRAJ_CAPACITY,
 CWC_TRAJ_EVENT_LIMIT, CWC_TRAJ_BAD_INPUT, CWC_TRAJ_TIMEOUT) = range(8)
CWC_LAYOUT_AUTO, CWC_LAYOUT_STATIC, CWC_LAYOUT_QUEUE, CWC_LAYOUT_TAIL = range(4)

# Every symbol the header declares (checked by the CPU test-suite).
EXPORTED = ("cwc_model_create", "cwc_model_destroy", "cwc_model_num_observables", "cwc_simulate_workspace_size",
            "cwc_simulate", "cwc_simulate_noalloc", "cwc_sensitivity_workspace_size", "cwc_sensitivity",
            "cwc_autotune", "cwc_checkpoint_words", "cwc_log_spec", "cwc_last_error", "cwc_version",
            "cwc_fp64_peak")
CWC_NOALLOC_SCRATCH_BYTES = 1 << 20

_vp = ctypes.c_void_p
_i32 = ctypes.c_int32
_i64 = ctypes.c_int64
_u64 = ctypes.c_uint64


class cwc_model_desc(ctypes.Structure):
    _fields_ = [("n_species", _i32), ("n_labels", _i32), ("n_rules", _i32), ("max_compartments", _i32),
                ("kind", _vp), ("ctx_label", _vp), ("child_label", _vp), ("lhs", _vp), ("rhs", _vp),
                ("grand_label", _vp), ("lhs_ext", _vp), ("rhs_ext", _vp), ("rate_law", _vp), ("rate_par", _vp)]


class cwc_sim_args(ctypes.Structure):
    _fields_ = [("P", _i32), ("R", _i32), ("G", _i32), ("Pi", _i32), ("replica_offset", ctypes.c_uint32),
                ("rates", _vp), ("init", _vp), ("grid", _vp), ("seed", _u64), ("max_events", _i64),
                ("states", _vp), ("sums", _vp), ("means", _vp), ("sumsq", _vp), ("variance", _vp), ("ci90", _vp),
                ("traj_status", _vp), ("traj_events", _vp), ("traj_hash", _vp), ("traj_final_t", _vp),
                ("log_cap", _i32), ("log_rule", _vp), ("log_slot", _vp), ("log_t", _vp),
                ("checkpoint", _vp), ("resume", _i32),
                ("layout", _i32), ("block_threads", _i32), ("lanes", _i32), ("deadline_ns", _i64),
                ("workspace", _vp), ("workspace_bytes", ctypes.c_size_t), ("tail_threshold", _i32),
                ("term_bits", _i32)]


class cwc_sens_args(ctypes.Structure):
    _fields_ = [("means", _vp), ("grad_means", _vp), ("grad_rates", _vp), ("partials", _vp)]


_lib = None


class CwcError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__("%s: %s" % (STATUS_NAMES.get(status, str(status)), message))
        self.status = status


def lib_exists() -> bool:
    return os.path.exists(LIB_PATH)


def lib() -> ctypes.CDLL:
    """Load the CUDA library; raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("CUDA library %s is missing: run python -m paper_1010_2438_gb300.build "
                               "(there is no CPU fallback)" % LIB_PATH)
        L = ctypes.CDLL(LIB_PATH)
        L.cwc_model_create.argtypes = [ctypes.POINTER(cwc_model_desc), ctypes.POINTER(_vp)]
        L.cwc_model_create.restype = ctypes.c_int
        L.cwc_model_destroy.argtypes = [_vp]
        L.cwc_model_destroy.restype = None
        L.cwc_model_num_observables.argtypes = [_vp]
        L.cwc_model_num_observables.restype = _i32
        L.cwc_simulate_workspace_size.argtypes = [_vp, ctypes.POINTER(cwc_sim_args), ctypes.POINTER(ctypes.c_size_t)]
        L.cwc_simulate_workspace_size.restype = ctypes.c_int
        L.cwc_simulate.argtypes = [_vp, ctypes.POINTER(cwc_sim_args), _vp]
        L.cwc_simulate.restype = ctypes.c_int
        L.cwc_simulate_noalloc.argtypes = [_vp, ctypes.POINTER(cwc_sim_args), _vp]
        L.cwc_simulate_noalloc.restype = ctypes.c_int
        L.cwc_sensitivity_workspace_size.argtypes = [_vp, ctypes.POINTER(cwc_sim_args),
                                                     ctypes.POINTER(cwc_sens_args), ctypes.POINTER(ctypes.c_size_t)]
        L.cwc_sensitivity_workspace_size.restype = ctypes.c_int
        L.cwc_sensitivity.argtypes = [_vp, ctypes.POINTER(cwc_sim_args), ctypes.POINTER(cwc_sens_args), _vp]
        L.cwc_sensitivity.restype = ctypes.c_int
        L.cwc_autotune.argtypes = [_vp, ctypes.POINTER(cwc_sim_args), _i64, _vp, ctypes.POINTER(_i32),
                                   ctypes.POINTER(_i32), ctypes.POINTER(ctypes.c_double), ctypes.POINTER(_i32)]
        L.cwc_autotune.restype = ctypes.c_int
        L.cwc_checkpoint_words.argtypes = [_vp]
        L.cwc_checkpoint_words.restype = _i32
        L.cwc_log_spec.argtypes = [_vp, _vp, _i64, _vp]
        L.cwc_log_spec.restype = ctypes.c_int
        L.cwc_fp64_peak.argtypes = [_vp, ctypes.POINTER(ctypes.c_double)]
        L.cwc_fp64_peak.restype = ctypes.c_int
        L.cwc_last_error.argtypes = []
        L.cwc_last_error.restype = ctypes.c_char_p
        L.cwc_version.argtypes = []
        L.cwc_version.restype = ctypes.c_char_p
        _lib = L
    return _lib


def _check(status: int) -> None:
    if status != CWC_OK:
        raise CwcError(status, cwc_last_error())


def cwc_last_error() -> str:
    return lib().cwc_last_error().decode()


def cwc_version() -> str:
    return lib().cwc_version().decode()


def cwc_model_create(desc: cwc_model_desc) -> int:
    out = _vp()
    _check(lib().cwc_model_create(ctypes.byref(desc), ctypes.byref(out)))
    return out.value


def cwc_model_destroy(handle: Optional[int]) -> None:
    if handle:
        lib().cwc_model_destroy(handle)


def cwc_checkpoint_words(handle: int) -> int:
    return lib().cwc_checkpoint_words(handle)


def cwc_model_num_observables(handle: int) -> int:
    return lib().cwc_model_num_observables(handle)


def cwc_simulate_workspace_size(handle: int, args: cwc_sim_args) -> int:
    n = ctypes.c_size_t()
    _check(lib().cwc_simulate_workspace_size(handle, ctypes.byref(args), ctypes.byref(n)))
    return n.value


def cwc_simulate(handle: int, args: cwc_sim_args, stream: int = 0) -> None:
    _check(lib().cwc_simulate(handle, ctypes.byref(args), stream))


def cwc_simulate_noalloc(handle: int, args: cwc_sim_args, stream: int = 0) -> None:
    """cwc_simulate for callers that cannot allocate device memory (no
    workspace: the library's fixed CWC_NOALLOC_SCRATCH_BYTES device array is
    used instead; calls overlapping on the GPU race on it)."""
    _check(lib().cwc_simulate_noalloc(handle, ctypes.byref(args), stream))


def cwc_autotune(handle: int, args: cwc_sim_args, tune_events: int = 0, stream: int = 0):
    """Time the launch candidates on this batch; returns (layout, block_threads, lanes, ms) and caches them."""
    lay, thr, ms, lanes = _i32(), _i32(), ctypes.c_double(), _i32()
    _check(lib().cwc_autotune(handle, ctypes.byref(args), tune_events, stream, ctypes.byref(lay), ctypes.byref(thr),
                              ctypes.byref(ms), ctypes.byref(lanes)))
    return lay.value, thr.value, lanes.value, ms.value


def cwc_fp64_peak(stream: int = 0) -> float:
    """Measured FP64 lane-operations per second of the current GPU."""
    v = ctypes.c_double(0.0)
    _check(lib().cwc_fp64_peak(stream, ctypes.byref(v)))
    return v.value


def cwc_log_spec(u_ptr: int, out_ptr: int, n: int, stream: int = 0) -> None:
    """The device logarithm of the time step over n doubles (device pointers)."""
    _check(lib().cwc_log_spec(u_ptr, out_ptr, n, stream))


def cwc_sensitivity_workspace_size(handle: int, args: cwc_sim_args, sens: cwc_sens_args) -> int:
    n = ctypes.c_size_t()
    _check(lib().cwc_sensitivity_workspace_size(handle, ctypes.byref(args), ctypes.byref(sens), ctypes.byref(n)))
    return n.value


def cwc_sensitivity(handle: int, args: cwc_sim_args, sens: cwc_sens_args, stream: int = 0) -> None:
    _check(lib().cwc_sensitivity(handle, ctypes.byref(args), ctypes.byref(sens), stream))
