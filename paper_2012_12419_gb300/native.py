"""ctypes binding of ``libvcmdp.so`` (declared in ``include/vcmdp.h``).

Argument marshalling only: every step of the method runs in the library's CUDA kernels.
PyTorch supplies device memory and the current stream.  Without the built library (or
without a CUDA device) every call raises; there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np
import torch

from . import build as _build

VC_OK = 0
VC_ERR_ARG = 1
VC_ERR_NOT_STOCHASTIC = 2
VC_ERR_NO_FEASIBLE_ACTION = 3
VC_ERR_NOT_CONVERGED = 4
VC_ERR_TIMEOUT = 5
VC_ERR_OOM = 6
VC_ERR_CUDA = 7

VC_IMPLICIT = 0
VC_CSR_F32 = 1
VC_CSR_BF16 = 2
VC_PADDED = 16
VC_DIRECT = 32
VC_SLICED = 64
VC_VAL_F32 = 0
VC_VAL_BF16 = 1
VC_ITER_FP32_ONLY = 1
VC_ITER_ACCURATE = 2
VC_ITER_PLAIN_CORRECTION = 4
VC_ITER_SELF_LOOP = 8
VC_ITER_BLOCK = 16

FORMATS = {"implicit": VC_IMPLICIT, "csr_f32": VC_CSR_F32, "csr_bf16": VC_CSR_BF16}

EXPORTS = [
    "vc_last_error", "vc_build_mdp", "vc_build_mdp_csr", "vc_mdp_info", "vc_value_iterate", "vc_extract_policy",
    "vc_bellman64", "vc_evaluate_policy", "vc_destroy", "vc_mdp_export_csr", "vc_bellman32", "vc_kernel_launches", "vc_autotune", "vc_autotune_report", "vc_bellman32_noalloc",
    "vc_value_grad", "vc_build_batch", "vc_batch_info", "vc_batch_offsets", "vc_value_iterate_batch",
    "vc_batch_autotune", "vc_batch_autotune_report", "vc_batch_destroy", "vc_mdp_slice", "vc_greedy_policy",
    "vc_set_wait_limit", "vc_aaa_intervals", "vc_objective", "vc_build_binary_mdp", "vc_set_block_iteration",
    "vc_block_iteration_info", "vc_batch_set_block_iteration", "vc_batch_set_small_instances",
    "vc_batch_small_instances", "vc_sweep_schedule",
]


class VcError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"vcmdp error {code}: {msg}")
        self.code = code


class Params(ctypes.Structure):
    _fields_ = [
        ("H", ctypes.c_int32), ("C", ctypes.c_int32), ("Q", ctypes.c_int32), ("reserved", ctypes.c_int32),
        ("lam", ctypes.c_double), ("f", ctypes.c_double), ("gamma", ctypes.c_double),
        ("w_occ", ctypes.c_double), ("w_loss", ctypes.c_double), ("w_q", ctypes.c_double),
        ("mu", ctypes.POINTER(ctypes.c_double)), ("delta", ctypes.POINTER(ctypes.c_double)),
    ]


class BinaryParams(ctypes.Structure):
    _fields_ = [
        ("H", ctypes.c_int32), ("C", ctypes.c_int32), ("J", ctypes.c_int32), ("reserved", ctypes.c_int32),
        ("lam", ctypes.c_double), ("gamma", ctypes.c_double), ("beta_vc", ctypes.c_double),
        ("beta_tc", ctypes.c_double), ("gamma_vc", ctypes.c_double),
        ("mu", ctypes.POINTER(ctypes.c_double)), ("delta", ctypes.POINTER(ctypes.c_double)),
    ]


class Info(ctypes.Structure):
    _fields_ = [
        ("S", ctypes.c_int64), ("A", ctypes.c_int32), ("fmt", ctypes.c_int32),
        ("nnz_logical", ctypes.c_int64), ("nnz_stored", ctypes.c_int64), ("feasible_rows", ctypes.c_int64),
        ("device_bytes", ctypes.c_int64), ("sweep_bytes", ctypes.c_int64),
        ("has_model", ctypes.c_int32), ("csr_pipelined", ctypes.c_int32), ("csr_tile_states", ctypes.c_int32),
        ("csr_stages", ctypes.c_int32), ("csr_ctas_per_sm", ctypes.c_int32), ("csr_smem_bytes", ctypes.c_int32),
        ("csr_sliced", ctypes.c_int32), ("reserved", ctypes.c_int32), ("nnz_sliced", ctypes.c_int64),
    ]


class Stats(ctypes.Structure):
    _fields_ = [
        ("sweeps", ctypes.c_int64), ("residual", ctypes.c_double), ("eval_sweeps", ctypes.c_int64),
        ("bellman64", ctypes.c_int64), ("policy_rounds", ctypes.c_int32), ("certified", ctypes.c_int32),
        ("residual64", ctypes.c_double), ("ms_fp32", ctypes.c_double), ("ms_fp64", ctypes.c_double),
    ]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


class GradStats(ctypes.Structure):
    _fields_ = [
        ("sweeps", ctypes.c_int64), ("correction_sweeps", ctypes.c_int64), ("rounds", ctypes.c_int32),
        ("reserved", ctypes.c_int32), ("residual64", ctypes.c_double), ("J", ctypes.c_double),
        ("nnz_transpose", ctypes.c_int64),
    ]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_ if k != "reserved"}


class BatchInfo(ctypes.Structure):
    _fields_ = [
        ("n", ctypes.c_int32), ("tiles", ctypes.c_int32), ("total_states", ctypes.c_int64),
        ("tile_states", ctypes.c_int32), ("blocks_per_sm", ctypes.c_int32), ("grid", ctypes.c_int32),
        ("reserved", ctypes.c_int32), ("device_bytes", ctypes.c_int64),
    ]


class BatchStats(ctypes.Structure):
    _fields_ = [
        ("sweeps", ctypes.c_int64), ("correction_sweeps", ctypes.c_int64), ("residual64", ctypes.c_double),
        ("certified", ctypes.c_int32), ("termination", ctypes.c_int32), ("rounds", ctypes.c_int32),
        ("reserved", ctypes.c_int32),
    ]


_lib = None
_lock = threading.Lock()


def lib_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = False) -> ctypes.CDLL:
    """Load the library (optionally building it first).  Raises if it is missing."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        # VC_DEBUG_BOUNDS=1 selects the bounds-checking build of the same library
        debug = os.environ.get("VC_DEBUG_BOUNDS", "") == "1"
        path = _build.LIB_DEBUG if debug else _build.LIB
        if build_if_missing and not _build.up_to_date(debug):
            _build.build(debug=debug)
        if not os.path.exists(path):
            raise RuntimeError(f"{path} is not built: run __graft_entry__.build() (nvcc, sm_103a)")
        L = ctypes.CDLL(path)
        vp, i32, i64, dbl = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double
        L.vc_last_error.restype = ctypes.c_char_p
        L.vc_last_error.argtypes = []
        L.vc_build_mdp.argtypes = [ctypes.POINTER(Params), ctypes.c_int, vp, ctypes.POINTER(vp)]
        L.vc_build_mdp_csr.argtypes = [i64, i32, vp, vp, vp, ctypes.c_int, vp, vp, dbl, vp, ctypes.POINTER(vp)]
        L.vc_mdp_info.argtypes = [vp, ctypes.POINTER(Info)]
        L.vc_value_iterate.argtypes = [vp, vp, vp, vp, dbl, i64, ctypes.c_int, ctypes.POINTER(Stats), vp]
        L.vc_extract_policy.argtypes = [vp, vp, vp, vp, vp]
        L.vc_bellman64.argtypes = [vp, vp, vp, vp, vp, ctypes.POINTER(dbl), vp]
        L.vc_evaluate_policy.argtypes = [vp, vp, vp, dbl, i64, ctypes.POINTER(i64), vp]
        L.vc_destroy.argtypes = [vp]
        L.vc_mdp_export_csr.argtypes = [vp, vp, vp, vp, vp, vp, vp]
        L.vc_bellman32.argtypes = [vp, vp, vp, vp, vp, vp]
        L.vc_kernel_launches.argtypes = []
        L.vc_autotune.argtypes = [vp, ctypes.c_int, ctypes.POINTER(dbl), vp]
        L.vc_autotune_report.argtypes = [vp, ctypes.c_char_p, i64]
        L.vc_bellman32_noalloc.argtypes = [ctypes.POINTER(Params), vp, vp, vp, vp, vp]
        L.vc_value_grad.argtypes = [vp, vp, vp, vp, vp, vp, dbl, i64, ctypes.POINTER(GradStats), vp]
        L.vc_build_batch.argtypes = [ctypes.POINTER(Params), i32, vp, ctypes.POINTER(vp)]
        L.vc_batch_info.argtypes = [vp, ctypes.POINTER(BatchInfo)]
        L.vc_batch_offsets.argtypes = [vp, vp]
        L.vc_value_iterate_batch.argtypes = [vp, vp, vp, vp, dbl, i64, ctypes.c_int, ctypes.POINTER(BatchStats), vp]
        L.vc_batch_autotune.argtypes = [vp, ctypes.c_int, ctypes.POINTER(dbl), vp]
        L.vc_batch_autotune_report.argtypes = [vp, ctypes.c_char_p, i64]
        L.vc_batch_destroy.argtypes = [vp]
        L.vc_mdp_slice.argtypes = [vp, vp]
        L.vc_greedy_policy.argtypes = [vp, vp, vp]
        L.vc_set_wait_limit.argtypes = [vp, i64]
        L.vc_aaa_intervals.argtypes = [vp, vp, vp, i32, i32, i32, dbl, dbl, dbl, vp, vp, vp]
        L.vc_objective.argtypes = [vp, vp, i64, vp, vp]
        L.vc_build_binary_mdp.argtypes = [ctypes.POINTER(BinaryParams), ctypes.c_int, vp, ctypes.POINTER(vp)]
        L.vc_set_block_iteration.argtypes = [vp, i32, i32]
        L.vc_block_iteration_info.argtypes = [vp, vp, vp, vp]
        L.vc_batch_set_block_iteration.argtypes = [vp, i32, i32, vp]
        L.vc_batch_set_small_instances.argtypes = [vp, i32, vp]
        L.vc_batch_small_instances.argtypes = [vp, vp, vp]
        L.vc_sweep_schedule.argtypes = [vp, i32, ctypes.POINTER(i32), vp]
        for name in EXPORTS:
            if name not in ("vc_last_error", "vc_kernel_launches", "vc_autotune_report", "vc_batch_autotune_report"):
                getattr(L, name).restype = ctypes.c_int
        L.vc_kernel_launches.restype = ctypes.c_int64
        L.vc_autotune_report.restype = ctypes.c_int64
        L.vc_batch_autotune_report.restype = ctypes.c_int64
        _lib = L
        return _lib


def _check(rc: int, allow=()):
    if rc != VC_OK and rc not in allow:
        msg = load().vc_last_error().decode(errors="replace")
        raise VcError(rc, msg)
    return rc


def _stream(stream=None):
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _ptr(t):
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    return ctypes.c_void_p(t.data_ptr())


def _params(p: dict):
    H = int(p["H"])
    mu = (ctypes.c_double * H)(*[float(v) for v in p["mu"][:H]])
    delta = (ctypes.c_double * H)(*[float(v) for v in p["delta"][:H]])
    c = Params(H, int(p["C"]), int(p["Q"]), 0, float(p["lam"]), float(p["f"]), float(p["gamma"]),
               float(p["w_occ"]), float(p["w_loss"]), float(p["w_q"]),
               ctypes.cast(mu, ctypes.POINTER(ctypes.c_double)), ctypes.cast(delta, ctypes.POINTER(ctypes.c_double)))
    return c, (mu, delta)


def _binary_params(p: dict):
    H = int(p["H"])
    mu = (ctypes.c_double * H)(*[float(v) for v in p["mu"][:H]])
    delta = (ctypes.c_double * H)(*[float(v) for v in p["delta"][:H]])
    c = BinaryParams(H, int(p["C"]), int(p["J"]), 0, float(p["lam"]), float(p["gamma"]), float(p["beta_vc"]),
                     float(p["beta_tc"]), float(p["gamma_vc"]), ctypes.cast(mu, ctypes.POINTER(ctypes.c_double)),
                     ctypes.cast(delta, ctypes.POINTER(ctypes.c_double)))
    return c, (mu, delta)


def _dev():
    if not torch.cuda.is_available():
        raise RuntimeError("vcmdp needs a CUDA device")
    return torch.device("cuda", torch.cuda.current_device())


class MDP:
    """An instance on the device (a ``vc_mdp`` handle)."""

    def __init__(self, handle: ctypes.c_void_p):
        self._h = handle
        self._info = None

    # ------------------------------------------------------------------ construction
    @classmethod
    def build(cls, params: dict, fmt: str = "implicit", padded: bool = False, direct: bool = False,
              sliced: bool = False, stream=None) -> "MDP":
        L = load()
        _dev()
        code = (FORMATS[fmt] | (VC_PADDED if padded else 0) | (VC_DIRECT if direct else 0)
                | (VC_SLICED if sliced else 0))
        cp, keep = _params(params)
        h = ctypes.c_void_p()
        _check(L.vc_build_mdp(ctypes.byref(cp), code, _stream(stream), ctypes.byref(h)))
        del keep
        return cls(h)

    @classmethod
    def build_binary(cls, params: dict, fmt: str = "csr_f32", direct: bool = False, sliced: bool = False,
                     stream=None) -> "MDP":
        """The paper's binary-action model (A = {-1, 1}; action 0 is -1, the paid cloud)
        as an explicit CSR built on the device, exact FP64 rows kept for the refinement."""
        L = load()
        _dev()
        code = FORMATS[fmt] | (VC_DIRECT if direct else 0) | (VC_SLICED if sliced else 0)
        cp, keep = _binary_params(params)
        h = ctypes.c_void_p()
        _check(L.vc_build_binary_mdp(ctypes.byref(cp), code, _stream(stream), ctypes.byref(h)))
        del keep
        return cls(h)

    @classmethod
    def from_csr(cls, S: int, A: int, row_ptr, col, val, R, gamma: float, row_scale=None, stream=None) -> "MDP":
        """Arbitrary explicit MDP: CUDA tensors int64 row_ptr[S*A+1], int32 col, float32 or
        bfloat16 val, float32 R[S*A] (-inf = infeasible), optional float32 row_scale."""
        L = load()
        if val.dtype == torch.float32:
            vdt = VC_VAL_F32
        elif val.dtype == torch.bfloat16:
            vdt = VC_VAL_BF16
        else:
            raise ValueError("val must be float32 or bfloat16")
        assert row_ptr.dtype == torch.int64 and col.dtype == torch.int32 and R.dtype == torch.float32
        h = ctypes.c_void_p()
        _check(L.vc_build_mdp_csr(int(S), int(A), _ptr(row_ptr), _ptr(col), _ptr(val), vdt, _ptr(row_scale),
                                  _ptr(R), float(gamma), _stream(stream), ctypes.byref(h)))
        return cls(h)

    def set_wait_limit(self, polls: int = -1) -> None:
        """Cap the bounded shared-memory waits of the pipelined sweeps (fault injection;
        0 = give up at once, negative = the default)."""
        _check(load().vc_set_wait_limit(self._h, int(polls)))

    def slice(self, stream=None) -> "MDP":
        """Add the sliced copy of the stored matrix and sweep it from now on."""
        _check(load().vc_mdp_slice(self._h, _stream(stream)))
        self._info = None
        return self

    def close(self):
        if self._h is not None and self._h.value:
            load().vc_destroy(self._h)
        self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ------------------------------------------------------------------------ queries
    def info(self) -> dict:
        if self._info is None:
            inf = Info()
            _check(load().vc_mdp_info(self._h, ctypes.byref(inf)))
            self._info = {k: getattr(inf, k) for k, _ in Info._fields_ if k != "reserved"}
        return self._info

    @property
    def S(self) -> int:
        return int(self.info()["S"])

    @property
    def A(self) -> int:
        return int(self.info()["A"])

    # ------------------------------------------------------------------------- solve
    def value_iterate(self, V=None, tol: float = 1e-6, max_sweeps: int = 1_000_000, fp32_only: bool = False,
                      want_v64: bool = True, want_pi: bool = True, stream=None, raise_on_nonconvergence=True,
                      accurate: bool = False, plain_correction: bool = False, self_loop: bool = False,
                      block: bool = False):
        """Algorithm 3 on the device.  Returns (V fp32, V64 fp64 or None, pi int32 or None, stats dict).

        accurate=True certifies the error rather than the residual: max|V64 - V*| <= tol / 2.
        plain_correction=True solves the refinement's correction equation by fixed-point
        sweeps instead of BiCGSTAB.  self_loop=True runs the FP32 sweeps with each action's
        self-transition solved exactly (VC_ITER_SELF_LOOP: same V*, fewer sweeps).  block=True
        (implicit handles) adds Algorithm 4's in-block passes (VC_ITER_BLOCK, shaped by
        set_block_iteration)."""
        dev = _dev()
        S = self.S
        if V is None:
            V = torch.zeros(S, dtype=torch.float32, device=dev)
        V64 = torch.empty(S, dtype=torch.float64, device=dev) if want_v64 else None
        pi = torch.empty(S, dtype=torch.int32, device=dev) if want_pi else None
        st = Stats()
        flags = ((VC_ITER_FP32_ONLY if fp32_only else 0) | (VC_ITER_ACCURATE if accurate else 0)
                 | (VC_ITER_PLAIN_CORRECTION if plain_correction else 0) | (VC_ITER_SELF_LOOP if self_loop else 0)
                 | (VC_ITER_BLOCK if block else 0))
        rc = load().vc_value_iterate(self._h, _ptr(V), _ptr(V64), _ptr(pi), float(tol), int(max_sweeps),
                                     flags, ctypes.byref(st), _stream(stream))
        _check(rc, allow=() if raise_on_nonconvergence else (VC_ERR_NOT_CONVERGED,))
        d = st.as_dict()
        d["status"] = rc
        return V, V64, pi, d

    def set_block_iteration(self, inner_hosts: int = -1, passes: int = 4) -> None:
        """Blocks of 2(Q+1)(C+1)^inner_hosts states (-1: the largest up to 1024) and the local
        passes per global sweep of the in-block iteration."""
        _check(load().vc_set_block_iteration(self._h, int(inner_hosts), int(passes)))

    def block_iteration_info(self) -> dict:
        h, B, p = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
        _check(load().vc_block_iteration_info(self._h, ctypes.byref(h), ctypes.byref(B), ctypes.byref(p)))
        return {"inner_hosts": h.value, "block_states": B.value, "passes": p.value}

    def extract_policy(self, V, stream=None):
        dev = _dev()
        pi = torch.empty(self.S, dtype=torch.int32, device=dev)
        gap = torch.empty(self.S, dtype=torch.float32, device=dev)
        _check(load().vc_extract_policy(self._h, _ptr(V), _ptr(pi), _ptr(gap), _stream(stream)))
        return pi, gap

    def autotune(self, reps: int = 5, stream=None) -> float:
        """Time the CSR sweep schedules on this instance and keep the fastest (us per sweep)."""
        us = ctypes.c_double()
        _check(load().vc_autotune(self._h, int(reps), ctypes.byref(us), _stream(stream)))
        self._info = None
        return us.value

    def schedules(self, stream=None) -> int:
        """Number of candidate sweep schedules (the autotuner's rows, in its order)."""
        n = ctypes.c_int32()
        _check(load().vc_sweep_schedule(self._h, -1, ctypes.byref(n), _stream(stream)))
        return n.value

    def use_schedule(self, index: int, stream=None) -> None:
        """Switch later sweeps to candidate schedule `index` (no timing)."""
        n = ctypes.c_int32()
        _check(load().vc_sweep_schedule(self._h, int(index), ctypes.byref(n), _stream(stream)))
        self._info = None

    def autotune_report(self) -> str:
        """Candidates and times of the last autotune, one line each."""
        L = load()
        n = L.vc_autotune_report(self._h, None, 0)
        buf = ctypes.create_string_buffer(int(n))
        L.vc_autotune_report(self._h, buf, int(n))
        return buf.value.decode()

    def bellman32(self, V, V_out=None, pi=None, qgap=None, stream=None):
        """One FP32 Bellman sweep (outputs optional, preallocated CUDA tensors)."""
        _check(load().vc_bellman32(self._h, _ptr(V), _ptr(V_out), _ptr(pi), _ptr(qgap), _stream(stream)))
        return V_out

    def bellman64(self, V64, stream=None):
        dev = _dev()
        out = torch.empty(self.S, dtype=torch.float64, device=dev)
        pi = torch.empty(self.S, dtype=torch.int32, device=dev)
        gap = torch.empty(self.S, dtype=torch.float64, device=dev)
        r = ctypes.c_double()
        _check(load().vc_bellman64(self._h, _ptr(V64), _ptr(out), _ptr(pi), _ptr(gap), ctypes.byref(r),
                                   _stream(stream)))
        return out, pi, gap, r.value

    def export_csr(self, stream=None):
        """Copies of the stored CSR: (row_ptr, col, val, row_scale or None, R) CUDA tensors."""
        dev = _dev()
        inf = self.info()
        rows = int(inf["S"]) * int(inf["A"])
        nnz = int(inf["nnz_stored"])
        bf16 = (inf["fmt"] & 0xF) == VC_CSR_BF16
        row_ptr = torch.empty(rows + 1, dtype=torch.int64, device=dev)
        col = torch.empty(max(nnz, 1), dtype=torch.int32, device=dev)
        val = torch.empty(max(nnz, 1), dtype=torch.int16 if bf16 else torch.float32, device=dev)
        scale = torch.empty(rows, dtype=torch.float32, device=dev) if bf16 else None
        R = torch.empty(rows, dtype=torch.float32, device=dev)
        _check(load().vc_mdp_export_csr(self._h, _ptr(row_ptr), _ptr(col), _ptr(val), _ptr(scale), _ptr(R),
                                        _stream(stream)))
        torch.cuda.synchronize()
        return row_ptr, col[:nnz], val[:nnz], scale, R

    def value_grad(self, V64, pi, rho, tol: float = 1e-11, max_sweeps: int = 1_000_000, want_lambda=False,
                   stream=None):
        """dJ/dtheta of J = rho . V_pi (theta = lambda, mu.., delta.., f, w_occ, w_loss, w_q).

        Returns (dJ [2H+5] float64 CUDA tensor, lam [S] float64 or None, stats dict)."""
        dev = _dev()
        H = (int(self.info()["A"]) - 1)
        dJ = torch.empty(2 * H + 5, dtype=torch.float64, device=dev)
        lam = torch.empty(self.S, dtype=torch.float64, device=dev) if want_lambda else None
        gs = GradStats()
        _check(load().vc_value_grad(self._h, _ptr(V64), _ptr(pi), _ptr(rho), _ptr(dJ), _ptr(lam), float(tol),
                                    int(max_sweeps), ctypes.byref(gs), _stream(stream)))
        return dJ, lam, gs.as_dict()

    def greedy_policy(self, stream=None):
        """The greedy heuristic (Algorithm 2 read as a policy) as an int32 CUDA tensor."""
        pi = torch.empty(self.S, dtype=torch.int32, device=_dev())
        _check(load().vc_greedy_policy(self._h, _ptr(pi), _stream(stream)))
        return pi

    def evaluate_policy(self, pi, V0=None, tol: float = 1e-10, max_sweeps: int = 1_000_000, stream=None):
        dev = _dev()
        V = torch.zeros(self.S, dtype=torch.float64, device=dev) if V0 is None else V0.clone()
        n = ctypes.c_int64()
        _check(load().vc_evaluate_policy(self._h, _ptr(pi), _ptr(V), float(tol), int(max_sweeps), ctypes.byref(n),
                                         _stream(stream)))
        return V, n.value


def solve(params: dict, fmt: str = "implicit", padded: bool = False, tol: float = 1e-6,
          max_sweeps: int = 1_000_000):
    """End-to-end call from host inputs to host results: build, iterate, certify.

    Returns numpy (V64, pi) and the stats dict.  The instance is built and solved on the
    current CUDA device; the results are copied back to the host.
    """
    m = MDP.build(params, fmt=fmt, padded=padded)
    try:
        V, V64, pi, st = m.value_iterate(tol=tol, max_sweeps=max_sweeps)
        return V64.cpu().numpy(), pi.cpu().numpy(), st
    finally:
        m.close()


class Batch:
    """Many independent instances solved together (a ``vc_batch`` handle)."""

    def __init__(self, params_list, stream=None):
        L = load()
        _dev()
        n = len(params_list)
        arr = (Params * n)()
        self._keep = []
        for i, p in enumerate(params_list):
            cp, keep = _params(p)
            arr[i] = cp
            self._keep.append(keep)
        h = ctypes.c_void_p()
        _check(L.vc_build_batch(arr, n, _stream(stream), ctypes.byref(h)))
        self._h = h
        self.n = n
        off = np.zeros(n + 1, np.int64)
        _check(L.vc_batch_offsets(self._h, off.ctypes.data_as(ctypes.c_void_p)))
        self.offsets = off

    def info(self) -> dict:
        inf = BatchInfo()
        _check(load().vc_batch_info(self._h, ctypes.byref(inf)))
        return {k: getattr(inf, k) for k, _ in BatchInfo._fields_ if k != "reserved"}

    @property
    def total(self) -> int:
        return int(self.offsets[-1])

    def value_iterate(self, V=None, tol: float = 1e-6, max_sweeps: int = 1_000_000, fp32_only: bool = False,
                      stream=None, raise_on_nonconvergence=True, accurate: bool = False,
                      plain_correction: bool = False, self_loop: bool = False, block: bool = False):
        """Returns (V fp32 [total], V64 [total] or None, pi [total] or None, list of per-instance dicts, status).

        accurate=True certifies every instance's error: max|V64_i - V*_i| <= tol / 2.
        plain_correction=True solves the correction equations by fixed-point sweeps.
        self_loop=True runs the FP32 loop with each action's self-transition solved;
        block=True adds Algorithm 4's in-block passes (set_block_iteration)."""
        dev = _dev()
        if V is None:
            V = torch.zeros(self.total, dtype=torch.float32, device=dev)
        V64 = torch.empty(self.total, dtype=torch.float64, device=dev)
        pi = torch.empty(self.total, dtype=torch.int32, device=dev)
        st = (BatchStats * self.n)()
        flags = ((VC_ITER_FP32_ONLY if fp32_only else 0) | (VC_ITER_ACCURATE if accurate else 0)
                 | (VC_ITER_PLAIN_CORRECTION if plain_correction else 0) | (VC_ITER_SELF_LOOP if self_loop else 0)
                 | (VC_ITER_BLOCK if block else 0))
        rc = load().vc_value_iterate_batch(self._h, _ptr(V), _ptr(V64), _ptr(pi), float(tol), int(max_sweeps),
                                           flags, st, _stream(stream))
        _check(rc, allow=() if raise_on_nonconvergence else (VC_ERR_NOT_CONVERGED,))
        stats = [{k: getattr(s, k) for k, _ in BatchStats._fields_ if k != "reserved"} for s in st]
        return V, V64, pi, stats, rc

    def set_small_instances(self, max_states: int, stream=None) -> None:
        """Instances of at most max_states states are swept whole in one thread block
        before the graph loop (0: none; capped by shared memory)."""
        _check(load().vc_batch_set_small_instances(self._h, int(max_states), _stream(stream)))

    def small_instances(self) -> dict:
        n, mx = ctypes.c_int32(), ctypes.c_int32()
        _check(load().vc_batch_small_instances(self._h, ctypes.byref(n), ctypes.byref(mx)))
        return {"count": n.value, "max_states": mx.value}

    def set_block_iteration(self, threads: int = 512, passes: int = 4, stream=None) -> None:
        """In-block iteration of every instance: blocks of at most `threads` states (the
        largest 2(Q+1)(C+1)^h that fits), `passes` local passes per global sweep."""
        _check(load().vc_batch_set_block_iteration(self._h, int(threads), int(passes), _stream(stream)))

    def autotune(self, sweeps: int = 20, stream=None) -> float:
        ms = ctypes.c_double()
        _check(load().vc_batch_autotune(self._h, int(sweeps), ctypes.byref(ms), _stream(stream)))
        return ms.value

    def autotune_report(self) -> str:
        L = load()
        n = L.vc_batch_autotune_report(self._h, None, 0)
        buf = ctypes.create_string_buffer(int(n))
        L.vc_batch_autotune_report(self._h, buf, int(n))
        return buf.value.decode()

    def close(self):
        if self._h is not None and self._h.value:
            load().vc_batch_destroy(self._h)
        self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def bellman32_noalloc(params: dict, V, V_out, pi=None, residual=None, stream=None):
    """One FP32 Bellman sweep of the implicit model with no device allocation: the
    library's static scratch holds the intermediate values (S <= 1,048,576).  V, V_out,
    pi and residual (one float) are caller-owned CUDA tensors."""
    cp, keep = _params(params)
    _check(load().vc_bellman32_noalloc(ctypes.byref(cp), _ptr(V), _ptr(V_out), _ptr(pi), _ptr(residual),
                                       _stream(stream)))
    del keep
    return V_out


def objective(V, rho, stream=None):
    """J = rho . V in FP64 on the device (float64 CUDA tensors of one length); returns a
    one-element float64 CUDA tensor."""
    if V.dtype != torch.float64 or rho.dtype != torch.float64 or V.numel() != rho.numel():
        raise ValueError("V and rho must be float64 tensors of one length")
    J = torch.empty(1, dtype=torch.float64, device=V.device)
    _check(load().vc_objective(_ptr(V), _ptr(rho), int(V.numel()), _ptr(J), _stream(stream)))
    return J


def aaa_intervals(S_v, D_v, R_v, si_per_second: int = 10, si_ms: float = 100.0, dcchi_ms: float = 50.0,
                  dschi_ms: float = 50.0):
    """The AAA timer update (Algorithm 1) over a trace: S_v, D_v, R_v are [n_si, n_vehicles]
    arrays (BSMs sent and acknowledged, total delay in ms of the BSMs received, BSMs
    received).  Returns (CCHI, SCHI, f) per UTC second as float64 numpy arrays; f = SCHI/SI
    is the phase-flip parameter of the placement model.  Host routine of the library."""
    S = np.ascontiguousarray(S_v, dtype=np.float64)
    D = np.ascontiguousarray(D_v, dtype=np.float64)
    R = np.ascontiguousarray(R_v, dtype=np.float64)
    if S.ndim != 2 or S.shape != D.shape or S.shape != R.shape:
        raise ValueError("S_v, D_v, R_v must be [n_si, n_vehicles] arrays of one shape")
    n_si, n_v = S.shape
    n_out = n_si // int(si_per_second) if int(si_per_second) > 0 else 0
    cchi = np.zeros(max(n_out, 1), np.float64)
    schi = np.zeros(max(n_out, 1), np.float64)
    f = np.zeros(max(n_out, 1), np.float64)
    dp = lambda a: a.ctypes.data_as(ctypes.c_void_p)
    _check(load().vc_aaa_intervals(dp(S), dp(D), dp(R), int(n_v), int(n_si), int(si_per_second), float(si_ms),
                                   float(dcchi_ms), float(dschi_ms), dp(cchi), dp(schi), dp(f)))
    return cchi[:n_out], schi[:n_out], f[:n_out]


def kernel_launches() -> int:
    """Kernels the library has enqueued since it was loaded (process-wide)."""
    return int(load().vc_kernel_launches())


def exported_symbols(path: str | None = None):
    """Names of the vc_* symbols the shared object exports (no CUDA needed)."""
    L = ctypes.CDLL(path or _build.LIB)
    return [n for n in EXPORTS if hasattr(L, n)]


def fmt_name(code: int) -> str:
    inv = {v: k for k, v in FORMATS.items()}
    return inv[code & 0xF] + ("+padded" if code & VC_PADDED else "") + ("+sliced" if code & VC_SLICED else "")


__all__ = ["MDP", "solve", "VcError", "load", "exported_symbols", "np"]
