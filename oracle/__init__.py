"""FP64 CPU oracle for value iteration on the vehicular-cloud task-placement MDP.

TEST INFRASTRUCTURE ONLY.  This package is the independent reference the CUDA library
is checked against (arxiv 2012.12419, Section V: Eq. 18 and Algorithm 3).  Only
``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may
import it; the library itself never does, and nothing here imports the library.

Two layers:

* ``vc_oracle.c`` (loaded through ctypes): successor enumeration of the model, explicit
  CSR construction, Jacobi value iteration (with Eq. 18's backup, and with each action's
  self-transition solved exactly, also inside Algorithm 4's blocks of consecutive states),
  single-state backups, policies, policy evaluation,
  analytic transition derivatives and a bfloat16 rounding routine.
* numpy helpers below for tiny problems: dense policy evaluation by a linear solve,
  exhaustive policy enumeration, value iteration on dense random MDPs and the
  dense-solve adjoint gradient; and the AAA timer update of Section II (Algorithm 1)
  in plain Python.

Parity status: every function here is pinned by a CPU test (``tests/test_oracle_*``)
against hand-derived transition rows, closed forms, brute force, or invariants.
"""
from __future__ import annotations

import ctypes
import itertools
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "vc_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

MAXH = 16


class _Params(ctypes.Structure):
    _fields_ = [
        ("H", ctypes.c_int32),
        ("C", ctypes.c_int32),
        ("Q", ctypes.c_int32),
        ("pad_", ctypes.c_int32),
        ("lam", ctypes.c_double),
        ("f", ctypes.c_double),
        ("gamma", ctypes.c_double),
        ("w_occ", ctypes.c_double),
        ("w_loss", ctypes.c_double),
        ("w_q", ctypes.c_double),
        ("mu", ctypes.c_double * MAXH),
        ("delta", ctypes.c_double * MAXH),
    ]


def build(force: bool = False) -> str:
    """Compile ``vc_oracle.c`` into ``liboracle.so`` next to it (plain gcc, -O2)."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(_LIB_PATH)
            P = ctypes.POINTER(_Params)
            i64, i32, dbl = ctypes.c_int64, ctypes.c_int32, ctypes.c_double
            vp = ctypes.c_void_p
            L.or_num_states.argtypes = [P]
            L.or_num_states.restype = i64
            L.or_decode.argtypes = [P, i64, vp, vp, vp]
            L.or_encode.argtypes = [P, vp, i32, i32]
            L.or_encode.restype = i64
            L.or_uniformisation.argtypes = [P]
            L.or_uniformisation.restype = dbl
            L.or_feasible.argtypes = [P, i64, ctypes.c_int]
            L.or_feasible.restype = ctypes.c_int
            L.or_transitions.argtypes = [P, i64, ctypes.c_int, vp, vp, vp]
            L.or_transitions.restype = ctypes.c_int
            L.or_transition_grads.argtypes = [P, i64, ctypes.c_int, vp, vp, vp]
            L.or_transition_grads.restype = ctypes.c_int
            L.or_build_csr.argtypes = [P, ctypes.c_int, vp, vp, vp, vp]
            L.or_build_csr.restype = i64
            L.or_backup.argtypes = [P, vp, i64, vp, vp, vp]
            L.or_value_iteration.argtypes = [P, dbl, i64, vp, vp, vp, vp]
            L.or_value_iteration.restype = ctypes.c_int
            L.or_greedy_policy.argtypes = [P, vp]
            L.or_policy.argtypes = [P, vp, vp, vp]
            L.or_policy_eval_iter.argtypes = [P, vp, dbl, i64, vp, vp]
            L.or_policy_eval_iter.restype = ctypes.c_int
            L.or_vi_csr.argtypes = [i64, i32, vp, vp, vp, vp, dbl, dbl, i64, vp, vp, vp]
            L.or_vi_csr.restype = ctypes.c_int
            L.or_value_iteration_sl.argtypes = [P, dbl, i64, vp, vp, vp, vp]
            L.or_value_iteration_sl.restype = ctypes.c_int
            L.or_vi_csr_sl.argtypes = [i64, i32, vp, vp, vp, vp, dbl, dbl, i64, vp, vp, vp]
            L.or_vi_csr_sl.restype = ctypes.c_int
            L.or_block_vi_csr_sl.argtypes = [i64, i32, vp, vp, vp, vp, dbl, i64, i32, dbl, i64, vp, vp, vp]
            L.or_block_vi_csr_sl.restype = ctypes.c_int
            L.or_policy_csr.argtypes = [i64, i32, vp, vp, vp, vp, dbl, vp, vp, vp]
            L.or_bf16_rne.argtypes = [dbl]
            L.or_bf16_rne.restype = ctypes.c_uint16
            L.or_bf16_to_double.argtypes = [ctypes.c_uint16]
            L.or_bf16_to_double.restype = dbl
            L.or_bf16_round_array.argtypes = [i64, vp, vp]
            L.or_bf16_renormalise_csr.argtypes = [i64, vp, vp, vp, vp, vp]
            _lib = L
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _params(p: dict) -> _Params:
    H = int(p["H"])
    if not 1 <= H <= MAXH:
        raise ValueError("H out of range")
    c = _Params()
    c.H, c.C, c.Q = H, int(p["C"]), int(p["Q"])
    c.lam, c.f, c.gamma = float(p["lam"]), float(p["f"]), float(p["gamma"])
    c.w_occ, c.w_loss, c.w_q = float(p["w_occ"]), float(p["w_loss"]), float(p["w_q"])
    for k in range(H):
        c.mu[k] = float(p["mu"][k])
        c.delta[k] = float(p["delta"][k])
    return c


# --------------------------------------------------------------------------- model


def num_states(p: dict) -> int:
    return int(lib().or_num_states(ctypes.byref(_params(p))))


def num_actions(p: dict) -> int:
    return int(p["H"]) + 1


def decode(p: dict, s: int):
    occ = np.zeros(MAXH, np.int32)
    q = np.zeros(1, np.int32)
    ph = np.zeros(1, np.int32)
    lib().or_decode(ctypes.byref(_params(p)), int(s), _ptr(occ), _ptr(q), _ptr(ph))
    return occ[: int(p["H"])].tolist(), int(q[0]), int(ph[0])


def encode(p: dict, occ, q: int, ph: int) -> int:
    o = np.zeros(MAXH, np.int32)
    o[: len(occ)] = occ
    return int(lib().or_encode(ctypes.byref(_params(p)), _ptr(o), int(q), int(ph)))


def uniformisation(p: dict) -> float:
    return float(lib().or_uniformisation(ctypes.byref(_params(p))))


def feasible(p: dict, s: int, a: int) -> bool:
    return bool(lib().or_feasible(ctypes.byref(_params(p)), int(s), int(a)))


def transitions(p: dict, s: int, a: int):
    """Merged, sorted successor row of (s, a): (cols, probs, R), or None if infeasible."""
    cols = np.zeros(2 * MAXH + 4, np.int64)
    probs = np.zeros(2 * MAXH + 4, np.float64)
    R = np.zeros(1, np.float64)
    n = lib().or_transitions(ctypes.byref(_params(p)), int(s), int(a), _ptr(cols), _ptr(probs), _ptr(R))
    if n < 0:
        return None
    return cols[:n].copy(), probs[:n].copy(), float(R[0])


def transition_grads(p: dict, s: int, a: int):
    """(cols, dprobs[n, 2H+5], dR[2H+5]) for theta = (lam, mu.., delta.., f, w_occ, w_loss, w_q)."""
    H = int(p["H"])
    nt = 2 * H + 5
    cols = np.zeros(2 * MAXH + 4, np.int64)
    dprobs = np.zeros((2 * MAXH + 4) * nt, np.float64)
    dR = np.zeros(nt, np.float64)
    n = lib().or_transition_grads(ctypes.byref(_params(p)), int(s), int(a), _ptr(cols), _ptr(dprobs), _ptr(dR))
    if n < 0:
        return None
    return cols[:n].copy(), dprobs[: n * nt].reshape(n, nt).copy(), dR


def build_csr(p: dict, padded: bool = False):
    """Explicit CSR (row_ptr int64[S*A+1], col int32[nnz], val float64[nnz], R float64[S*A])."""
    cp = _params(p)
    L = lib()
    S = num_states(p)
    A = num_actions(p)
    nnz = L.or_build_csr(ctypes.byref(cp), int(padded), None, None, None, None)
    row_ptr = np.zeros(S * A + 1, np.int64)
    col = np.zeros(nnz, np.int32)
    val = np.zeros(nnz, np.float64)
    R = np.zeros(S * A, np.float64)
    L.or_build_csr(ctypes.byref(cp), int(padded), _ptr(row_ptr), _ptr(col), _ptr(val), _ptr(R))
    return row_ptr, col, val, R


def csr_nnz(p: dict, padded: bool = False) -> int:
    return int(lib().or_build_csr(ctypes.byref(_params(p)), int(padded), None, None, None, None))


# ------------------------------------------------------------------ value iteration


def value_iteration(p: dict, tol: float = 1e-6, max_sweeps: int = 100000, V0=None, record=False):
    """Jacobi VI (Algorithm 3) from V0 (zeros by default).

    Returns (V, sweeps, last_residual[, residuals]); raises if max_sweeps runs out.
    """
    S = num_states(p)
    V = np.zeros(S, np.float64) if V0 is None else np.array(V0, np.float64, copy=True)
    sweeps = np.zeros(1, np.int64)
    res = np.zeros(1, np.float64)
    hist = np.zeros(max_sweeps if record else 0, np.float64)
    st = lib().or_value_iteration(
        ctypes.byref(_params(p)), float(tol), int(max_sweeps), _ptr(V), _ptr(sweeps), _ptr(res),
        _ptr(hist) if record else None)
    if st != 0:
        raise RuntimeError("oracle value iteration did not converge")
    if record:
        return V, int(sweeps[0]), float(res[0]), hist[: int(sweeps[0])].copy()
    return V, int(sweeps[0]), float(res[0])


def value_iteration_self_loop(p: dict, tol: float = 1e-6, max_sweeps: int = 100000, V0=None, record=False,
                              strict=True):
    """Value iteration whose backup solves each action's self-transition exactly,
    Qs = (R + gamma sum_{s' != s} P V) / (1 - gamma P(s|s,a)) (Puterman 1994, Sec. 6.3.3;
    Algorithm 4's in-block iteration for a block of one state, iterated to its limit).
    Same fixed point V* as Eq. 18.  Returns (V, sweeps, last_change[, changes]); with
    strict=False a max_sweeps that runs out returns the iterate instead of raising.
    """
    S = num_states(p)
    V = np.zeros(S, np.float64) if V0 is None else np.array(V0, np.float64, copy=True)
    sweeps = np.zeros(1, np.int64)
    res = np.zeros(1, np.float64)
    hist = np.zeros(max_sweeps if record else 0, np.float64)
    st = lib().or_value_iteration_sl(
        ctypes.byref(_params(p)), float(tol), int(max_sweeps), _ptr(V), _ptr(sweeps), _ptr(res),
        _ptr(hist) if record else None)
    if st != 0 and strict:
        raise RuntimeError("oracle value iteration did not converge")
    if record:
        return V, int(sweeps[0]), float(res[0]), hist[: int(sweeps[0])].copy()
    return V, int(sweeps[0]), float(res[0])


def backup(p: dict, V: np.ndarray, s: int):
    """One Bellman backup of state s from V: (best value, argmax action, Q-gap)."""
    V = np.ascontiguousarray(V, np.float64)
    b = np.zeros(1, np.float64)
    a = np.zeros(1, np.int32)
    g = np.zeros(1, np.float64)
    lib().or_backup(ctypes.byref(_params(p)), _ptr(V), int(s), _ptr(b), _ptr(a), _ptr(g))
    return float(b[0]), int(a[0]), float(g[0])


def policy(p: dict, V: np.ndarray):
    """pi = argmax_a Q (lowest action on ties) and the Q-gap, from V (Algorithm 3 step 4)."""
    V = np.ascontiguousarray(V, np.float64)
    S = num_states(p)
    pi = np.zeros(S, np.int32)
    gap = np.zeros(S, np.float64)
    lib().or_policy(ctypes.byref(_params(p)), _ptr(V), _ptr(pi), _ptr(gap))
    return pi, gap


def greedy_policy(p: dict) -> np.ndarray:
    """Algorithm 2 read as a policy: feasible host with the largest service rate, else defer."""
    pi = np.zeros(num_states(p), np.int32)
    lib().or_greedy_policy(ctypes.byref(_params(p)), _ptr(pi))
    return pi


def policy_eval_iter(p: dict, pi: np.ndarray, tol: float = 1e-13, max_sweeps: int = 10**6, V0=None):
    pi = np.ascontiguousarray(pi, np.int32)
    V = np.zeros(len(pi), np.float64) if V0 is None else np.array(V0, np.float64, copy=True)
    sweeps = np.zeros(1, np.int64)
    st = lib().or_policy_eval_iter(ctypes.byref(_params(p)), _ptr(pi), float(tol), int(max_sweeps), _ptr(V),
                                   _ptr(sweeps))
    if st != 0:
        raise RuntimeError(f"oracle policy evaluation failed (status {st})")
    return V


def policy_matrices(p: dict, pi: np.ndarray):
    """Dense P_pi (S x S) and R_pi (S) of a deterministic policy (small S only)."""
    S = num_states(p)
    P = np.zeros((S, S), np.float64)
    R = np.zeros(S, np.float64)
    for s in range(S):
        row = transitions(p, s, int(pi[s]))
        if row is None:
            raise ValueError(f"policy action {pi[s]} infeasible in state {s}")
        cols, probs, r = row
        P[s, cols] = probs
        R[s] = r
    return P, R


def policy_eval_dense(p: dict, pi: np.ndarray) -> np.ndarray:
    """V_pi = (I - gamma P_pi)^-1 R_pi by a dense LU solve (S <= a few thousand)."""
    P, R = policy_matrices(p, pi)
    S = len(R)
    return np.linalg.solve(np.eye(S) - float(p["gamma"]) * P, R)


def solve(p: dict, tol: float = 1e-12):
    """Reference optimum: VI to tol, then the argmax policy evaluated exactly.

    Returns (V_star, pi, qgap, sweeps).  The final values come from evaluating the
    greedy policy of the converged V, by dense LU when S <= 5000 and otherwise by
    FP64 iteration to 1e-13.
    """
    V, sweeps, _ = value_iteration(p, tol=tol)
    pi, gap = policy(p, V)
    if num_states(p) <= 5000:
        Vs = policy_eval_dense(p, pi)
    else:
        Vs = policy_eval_iter(p, pi, tol=1e-13, V0=V)
    return Vs, pi, gap, sweeps


# ------------------------------------------------------------- explicit / dense MDPs


def vi_csr(S, A, row_ptr, col, val, R, gamma, tol=1e-12, max_sweeps=10**6, V0=None, strict=True):
    """Jacobi VI on an explicit CSR MDP (R = -inf marks infeasible rows); with strict=False
    a max_sweeps that runs out returns the iterate instead of raising."""
    row_ptr = np.ascontiguousarray(row_ptr, np.int64)
    col = np.ascontiguousarray(col, np.int32)
    val = np.ascontiguousarray(val, np.float64)
    R = np.ascontiguousarray(R, np.float64)
    V = np.zeros(S, np.float64) if V0 is None else np.array(V0, np.float64, copy=True)
    sweeps = np.zeros(1, np.int64)
    res = np.zeros(1, np.float64)
    st = lib().or_vi_csr(int(S), int(A), _ptr(row_ptr), _ptr(col), _ptr(val), _ptr(R), float(gamma), float(tol),
                         int(max_sweeps), _ptr(V), _ptr(sweeps), _ptr(res))
    if st != 0 and strict:
        raise RuntimeError("oracle CSR value iteration did not converge")
    return V, int(sweeps[0])


def vi_csr_self_loop(S, A, row_ptr, col, val, R, gamma, tol=1e-12, max_sweeps=10**6, V0=None, strict=True):
    """vi_csr with each row's self-transition solved exactly (entries whose column is the
    row's own state form P(s|s,a)); returns (V, sweeps)."""
    row_ptr = np.ascontiguousarray(row_ptr, np.int64)
    col = np.ascontiguousarray(col, np.int32)
    val = np.ascontiguousarray(val, np.float64)
    R = np.ascontiguousarray(R, np.float64)
    V = np.zeros(S, np.float64) if V0 is None else np.array(V0, np.float64, copy=True)
    sweeps = np.zeros(1, np.int64)
    res = np.zeros(1, np.float64)
    st = lib().or_vi_csr_sl(int(S), int(A), _ptr(row_ptr), _ptr(col), _ptr(val), _ptr(R), float(gamma),
                            float(tol), int(max_sweeps), _ptr(V), _ptr(sweeps), _ptr(res))
    if st != 0 and strict:
        raise RuntimeError("oracle CSR value iteration did not converge")
    return V, int(sweeps[0])


def block_vi_csr_self_loop(S, A, row_ptr, col, val, R, gamma, tile, passes, tol=1e-12, max_sweeps=10**6, V0=None,
                           strict=True):
    """Algorithm 4's in-block iteration over consecutive blocks of `tile` states, `passes`
    local passes of the self-transition-solved backup per global sweep (successors in the
    state's block from the previous local pass, others from the previous global iterate).
    Returns (V, global sweeps)."""
    row_ptr = np.ascontiguousarray(row_ptr, np.int64)
    col = np.ascontiguousarray(col, np.int32)
    val = np.ascontiguousarray(val, np.float64)
    R = np.ascontiguousarray(R, np.float64)
    V = np.zeros(S, np.float64) if V0 is None else np.array(V0, np.float64, copy=True)
    sweeps = np.zeros(1, np.int64)
    res = np.zeros(1, np.float64)
    st = lib().or_block_vi_csr_sl(int(S), int(A), _ptr(row_ptr), _ptr(col), _ptr(val), _ptr(R), float(gamma),
                                  int(tile), int(passes), float(tol), int(max_sweeps), _ptr(V), _ptr(sweeps),
                                  _ptr(res))
    if st != 0 and strict:
        raise RuntimeError("oracle block value iteration did not converge")
    return V, int(sweeps[0])


def policy_csr(S, A, row_ptr, col, val, R, gamma, V):
    row_ptr = np.ascontiguousarray(row_ptr, np.int64)
    col = np.ascontiguousarray(col, np.int32)
    val = np.ascontiguousarray(val, np.float64)
    R = np.ascontiguousarray(R, np.float64)
    V = np.ascontiguousarray(V, np.float64)
    pi = np.zeros(S, np.int32)
    gap = np.zeros(S, np.float64)
    lib().or_policy_csr(int(S), int(A), _ptr(row_ptr), _ptr(col), _ptr(val), _ptr(R), float(gamma), _ptr(V),
                        _ptr(pi), _ptr(gap))
    return pi, gap


def dense_value_iteration(P: np.ndarray, R: np.ndarray, gamma: float, tol: float = 1e-12, max_sweeps=10**6):
    """VI on a dense MDP: P[a, s, s'], R[s, a] (-inf = infeasible).  Plain loops; tiny S only."""
    A, S, _ = P.shape
    V = np.zeros(S)
    for _k in range(max_sweeps):
        Vn = np.empty(S)
        for s in range(S):
            best = -np.inf
            for a in range(A):
                if R[s, a] == -np.inf:
                    continue
                q = R[s, a] + gamma * sum(P[a, s, t] * V[t] for t in range(S))
                best = max(best, q)
            Vn[s] = best
        res = np.max(np.abs(Vn - V))
        V = Vn
        if res < tol:
            return V
    raise RuntimeError("dense VI did not converge")


def brute_force_optimum(P: np.ndarray, R: np.ndarray, gamma: float, max_policies: int = 200000):
    """V* as the elementwise max over every deterministic policy of (I - gamma P_pi)^-1 R_pi.

    P[a, s, s'], R[s, a] with -inf for infeasible actions.  Enumerates all policies.
    """
    A, S, _ = P.shape
    choices = [[a for a in range(A) if R[s, a] != -np.inf] for s in range(S)]
    count = 1
    for c in choices:
        count *= len(c)
    if count > max_policies:
        raise ValueError(f"{count} policies is too many to enumerate")
    best = np.full(S, -np.inf)
    for pol in itertools.product(*choices):
        Pp = np.array([P[pol[s], s] for s in range(S)])
        Rp = np.array([R[s, pol[s]] for s in range(S)])
        V = np.linalg.solve(np.eye(S) - gamma * Pp, Rp)
        best = np.maximum(best, V)
    return best


def model_dense(p: dict):
    """Dense P[a, s, s'] and R[s, a] (-inf where infeasible) of a small instance."""
    S = num_states(p)
    A = num_actions(p)
    P = np.zeros((A, S, S))
    R = np.full((S, A), -np.inf)
    for s in range(S):
        for a in range(A):
            row = transitions(p, s, a)
            if row is None:
                continue
            cols, probs, r = row
            P[a, s, cols] = probs
            R[s, a] = r
    return P, R


# --------------------------------------------------------------------------- gradient


def theta_names(H: int):
    return ["lam"] + [f"mu{k}" for k in range(H)] + [f"delta{k}" for k in range(H)] + ["f", "w_occ", "w_loss", "w_q"]


def theta_vector(p: dict) -> np.ndarray:
    H = int(p["H"])
    return np.array([p["lam"]] + list(p["mu"][:H]) + list(p["delta"][:H]) + [p["f"], p["w_occ"], p["w_loss"],
                                                                             p["w_q"]], np.float64)


def with_theta(p: dict, theta: np.ndarray) -> dict:
    H = int(p["H"])
    q = dict(p)
    q["lam"] = float(theta[0])
    q["mu"] = [float(v) for v in theta[1:1 + H]]
    q["delta"] = [float(v) for v in theta[1 + H:1 + 2 * H]]
    q["f"], q["w_occ"], q["w_loss"], q["w_q"] = (float(v) for v in theta[1 + 2 * H:5 + 2 * H])
    return q


def grad_dense(p: dict, V: np.ndarray, pi: np.ndarray, rho: np.ndarray) -> np.ndarray:
    """dJ/dtheta for J = rho . V_pi by the adjoint of a dense solve (small S only).

    lam_bar = (I - gamma P_pi)^-T rho, then
    dJ/dtheta_i = sum_s lam_bar(s) [dR_pi(s)/dtheta_i + gamma sum_s' dP_pi(s, s')/dtheta_i V(s')].
    """
    P, R = policy_matrices(p, pi)
    S = len(R)
    gamma = float(p["gamma"])
    lam_bar = np.linalg.solve((np.eye(S) - gamma * P).T, np.asarray(rho, np.float64))
    nt = 2 * int(p["H"]) + 5
    g = np.zeros(nt)
    for s in range(S):
        cols, dprobs, dR = transition_grads(p, s, int(pi[s]))
        g += lam_bar[s] * (dR + gamma * dprobs.T @ V[cols])
    return g


def bf16_rne(x: float) -> int:
    return int(lib().or_bf16_rne(float(x)))


def bf16_to_double(b: int) -> float:
    return float(lib().or_bf16_to_double(int(b)))


def bf16_round_array(x: np.ndarray) -> np.ndarray:
    x = np.ascontiguousarray(x, np.float64)
    bits = np.zeros(len(x), np.uint16)
    lib().or_bf16_round_array(len(x), _ptr(x), _ptr(bits))
    return bits


def bf16_renormalised(row_ptr, val, nrows):
    """The matrix the BF16 form solves: bf16(p) * scale32, scale = 1/sum bf16(p) in FP64
    (column order) rounded to FP32.  Returns (bf16 bit patterns, effective float64 values,
    float32 scales)."""
    row_ptr = np.ascontiguousarray(row_ptr, np.int64)
    val = np.ascontiguousarray(val, np.float64)
    bits = np.zeros(len(val), np.uint16)
    out = np.zeros(len(val), np.float64)
    scale = np.zeros(nrows, np.float32)
    lib().or_bf16_renormalise_csr(int(nrows), _ptr(row_ptr), _ptr(val), _ptr(bits), _ptr(out), _ptr(scale))
    return bits, out, scale


def sweep_states(p: dict, V: np.ndarray, Vn: np.ndarray, s0: int, s1: int, step: int = 1) -> int:
    """Backups of states s0, s0+step, ... < s1 from V into Vn; returns the updates done."""
    L = lib()
    L.or_sweep_states.argtypes = [ctypes.POINTER(_Params), ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64,
                                  ctypes.c_int64, ctypes.c_int64]
    L.or_sweep_states.restype = ctypes.c_int64
    return int(L.or_sweep_states(ctypes.byref(_params(p)), _ptr(V), _ptr(Vn), int(s0), int(s1), int(step)))


def backup_range(p: dict, V: np.ndarray, s0: int, s1: int, Vn: np.ndarray, pi: np.ndarray, gap: np.ndarray):
    """Backups of states s0 .. s1-1 of V into Vn, pi, gap (each indexed like V), by the
    single-state backup; the C routine runs outside the Python lock."""
    L = lib()
    L.or_backup_range.argtypes = [ctypes.POINTER(_Params), ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64,
                                  ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    L.or_backup_range.restype = None
    for a, t in ((V, np.float64), (Vn, np.float64), (pi, np.int32), (gap, np.float64)):
        if a.dtype != t or not a.flags.c_contiguous:
            raise ValueError("backup_range wants contiguous float64 V, Vn, gap and int32 pi")
    L.or_backup_range(ctypes.byref(_params(p)), _ptr(V), int(s0), int(s1), _ptr(Vn), _ptr(pi), _ptr(gap))


def backup_all(p: dict, V, threads: int | None = None):
    """Bellman backup, argmax and Q-gap of every state of V, on contiguous state ranges
    split over host threads (Jacobi: each state reads only V, so the result does not
    depend on the split).  Returns (Vn, pi, gap)."""
    V = np.ascontiguousarray(V, np.float64)
    S = len(V)
    Vn = np.empty(S, np.float64)
    pi = np.empty(S, np.int32)
    gap = np.empty(S, np.float64)
    n = max(1, min(threads or os.cpu_count() or 1, S))
    cuts = [S * i // n for i in range(n + 1)]
    ts = [threading.Thread(target=backup_range, args=(p, V, cuts[i], cuts[i + 1], Vn, pi, gap)) for i in range(n)]
    for t in ts:
        t.start()
    for t in ts:
        t.join()
    return Vn, pi, gap


def grad_contract(p: dict, V, pi, lam) -> np.ndarray:
    """sum_s lam[s] (dR/dtheta + gamma dP/dtheta V) over the policy's rows, in C (any size)."""
    L = lib()
    L.or_grad_contract.argtypes = [ctypes.POINTER(_Params), ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                   ctypes.c_void_p]
    L.or_grad_contract.restype = ctypes.c_int
    V = np.ascontiguousarray(V, np.float64)
    pi = np.ascontiguousarray(pi, np.int32)
    lam = np.ascontiguousarray(lam, np.float64)
    g = np.zeros(2 * MAXH + 5, np.float64)
    if L.or_grad_contract(ctypes.byref(_params(p)), _ptr(V), _ptr(pi), _ptr(lam), _ptr(g)) != 0:
        raise ValueError("policy infeasible")
    return g[: 2 * int(p["H"]) + 5].copy()


def adjoint_apply(p: dict, pi, lam) -> np.ndarray:
    """P_pi^T lam (push form), any size."""
    L = lib()
    L.or_adjoint_apply.argtypes = [ctypes.POINTER(_Params), ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    L.or_adjoint_apply.restype = ctypes.c_int
    pi = np.ascontiguousarray(pi, np.int32)
    lam = np.ascontiguousarray(lam, np.float64)
    out = np.zeros(len(lam), np.float64)
    if L.or_adjoint_apply(ctypes.byref(_params(p)), _ptr(pi), _ptr(lam), _ptr(out)) != 0:
        raise ValueError("policy infeasible")
    return out


# ------------------------------------------------------ AAA multichannel timers (Section II)


def aaa_intervals(S_v, D_v, R_v, si_per_second: int = 10, si_ms: float = 100.0, dcchi_ms: float = 50.0,
                  dschi_ms: float = 50.0):
    """Algorithm 1 (AAA multi-channel steps) over a trace, step by step in the paper's order.

    S_v[j][h], D_v[j][h], R_v[j][h]: BSMs vehicle h sent and had acknowledged in SI j
    (Eq. 2), the total end-to-end delay (ms) of the BSMs it received (the numerator of
    Eq. 3), and how many it received.  Every SI that is not the last of its UTC second
    updates the running S_V2V and D_V2V (Algorithm 1, the two averaging lines); the last SI
    of each second computes U_CCH = S_V2V * D_V2V (Eq. 4) and I_CCH = CCHI - U_CCH (Eq. 7),
    sets CCHI = U_CCH and SCHI = SCHI + I_CCH when U_CCH < DCCHI (else both defaults), and
    clears S_V2V and D_V2V.  Returns lists (CCHI, SCHI, SCHI / SI), one entry per second.
    """
    n_si = len(S_v)
    cchi, schi = float(dcchi_ms), float(dschi_ms)
    s_v2v = 0.0
    d_v2v = 0.0
    out_c, out_s, out_f = [], [], []
    for j in range(n_si):
        n_v = len(S_v[j])
        utc_second = (j + 1) % si_per_second == 0
        if not utc_second:
            sent = 0.0
            for h in range(n_v):
                sent += float(S_v[j][h])
            s_v2v = (s_v2v + sent) / (1 + n_v)
            delay = 0.0
            received = 0.0
            for h in range(n_v):
                delay += float(D_v[j][h])
                received += float(R_v[j][h])
            d_v2v = (d_v2v + delay) / (1 + received)
        else:
            u_cch = s_v2v * d_v2v
            i_cch = cchi - u_cch
            if u_cch < dcchi_ms:
                cchi = u_cch
                schi = schi + i_cch
            else:
                cchi = float(dcchi_ms)
                schi = float(dschi_ms)
            out_c.append(cchi)
            out_s.append(schi)
            out_f.append(schi / si_ms)
            s_v2v = 0.0
            d_v2v = 0.0
    return out_c, out_s, out_f


# ------------------------------------------------- the paper's binary-action model (NEXT)


class _BinParams(ctypes.Structure):
    _fields_ = [
        ("H", ctypes.c_int32),
        ("C", ctypes.c_int32),
        ("J", ctypes.c_int32),
        ("pad_", ctypes.c_int32),
        ("lam", ctypes.c_double),
        ("gamma", ctypes.c_double),
        ("beta_vc", ctypes.c_double),
        ("beta_tc", ctypes.c_double),
        ("gamma_vc", ctypes.c_double),
        ("mu", ctypes.c_double * MAXH),
        ("delta", ctypes.c_double * MAXH),
    ]


def _bin_params(p: dict) -> _BinParams:
    H, J = int(p["H"]), int(p["J"])
    if not 1 <= H <= MAXH or not 1 <= J <= 8:
        raise ValueError("H must be in 1..16 and J in 1..8")
    c = _BinParams()
    c.H, c.C, c.J = H, int(p["C"]), J
    c.lam, c.gamma = float(p["lam"]), float(p["gamma"])
    c.beta_vc, c.beta_tc, c.gamma_vc = float(p["beta_vc"]), float(p["beta_tc"]), float(p["gamma_vc"])
    for k in range(H):
        c.mu[k] = float(p["mu"][k])
        c.delta[k] = float(p["delta"][k])
    return c


def _bin_lib():
    L = lib()
    if not hasattr(L, "_bin_ready"):
        P = ctypes.POINTER(_BinParams)
        vp = ctypes.c_void_p
        L.or_bin_num_states.argtypes = [P]
        L.or_bin_num_states.restype = ctypes.c_int64
        L.or_bin_uniformisation.argtypes = [P]
        L.or_bin_uniformisation.restype = ctypes.c_double
        L.or_bin_transitions.argtypes = [P, ctypes.c_int64, ctypes.c_int, vp, vp, vp]
        L.or_bin_transitions.restype = ctypes.c_int
        L.or_bin_build_csr.argtypes = [P, vp, vp, vp, vp]
        L.or_bin_build_csr.restype = ctypes.c_int64
        L._bin_ready = True
    return L


def bin_num_states(p: dict) -> int:
    return int(_bin_lib().or_bin_num_states(ctypes.byref(_bin_params(p))))


def bin_uniformisation(p: dict) -> float:
    return float(_bin_lib().or_bin_uniformisation(ctypes.byref(_bin_params(p))))


def bin_transitions(p: dict, s: int, a: int):
    """Merged, sorted successor row of (s, a) of the binary-action model: (cols, probs, R),
    or None if a is infeasible in s (a = 0 is the paper's -1, a = 1 its +1)."""
    cols = np.zeros(162, np.int64)
    probs = np.zeros(162, np.float64)
    R = np.zeros(1, np.float64)
    n = _bin_lib().or_bin_transitions(ctypes.byref(_bin_params(p)), int(s), int(a), _ptr(cols), _ptr(probs), _ptr(R))
    if n < 0:
        return None
    return cols[:n].copy(), probs[:n].copy(), float(R[0])


def bin_build_csr(p: dict):
    """Explicit CSR of the binary-action model: (row_ptr int64[2S+1], col int32, val float64,
    R float64[2S] with -inf on infeasible rows); row r = 2 s + a."""
    cp = _bin_params(p)
    L = _bin_lib()
    S = bin_num_states(p)
    nnz = L.or_bin_build_csr(ctypes.byref(cp), None, None, None, None)
    row_ptr = np.zeros(2 * S + 1, np.int64)
    col = np.zeros(nnz, np.int32)
    val = np.zeros(nnz, np.float64)
    R = np.zeros(2 * S, np.float64)
    L.or_bin_build_csr(ctypes.byref(cp), _ptr(row_ptr), _ptr(col), _ptr(val), _ptr(R))
    return row_ptr, col, val, R


def bin_solve(p: dict, tol: float = 1e-12, val=None):
    """Optimum of the binary-action model: value iteration on its CSR (val replaces the
    exact FP64 probabilities, e.g. their FP32 rounding), then the argmax policy.
    Returns (V, pi, gap, sweeps)."""
    S = bin_num_states(p)
    rp, col, v, R = bin_build_csr(p)
    if val is not None:
        v = np.asarray(val, np.float64)
    V, n = vi_csr(S, 2, rp, col, v, R, p["gamma"], tol=tol)
    pi, gap = policy_csr(S, 2, rp, col, v, R, p["gamma"], V)
    return V, pi, gap, n


def bin_backup_all(p: dict, V, threads: int | None = None):
    """Bellman backup, argmax and Q-gap of every state of the binary-action model from V,
    on contiguous state ranges over host threads.  Returns (Vn, pi, gap)."""
    L = _bin_lib()
    L.or_bin_backup_range.argtypes = [ctypes.POINTER(_BinParams), ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64,
                                      ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    L.or_bin_backup_range.restype = None
    V = np.ascontiguousarray(V, np.float64)
    S = len(V)
    Vn = np.empty(S, np.float64)
    pi = np.empty(S, np.int32)
    gap = np.empty(S, np.float64)
    cp = _bin_params(p)
    n = max(1, min(threads or os.cpu_count() or 1, S))
    cuts = [S * i // n for i in range(n + 1)]

    def run(i):
        L.or_bin_backup_range(ctypes.byref(cp), _ptr(V), cuts[i], cuts[i + 1], _ptr(Vn), _ptr(pi), _ptr(gap))

    ts = [threading.Thread(target=run, args=(i,)) for i in range(n)]
    for t in ts:
        t.start()
    for t in ts:
        t.join()
    return Vn, pi, gap
