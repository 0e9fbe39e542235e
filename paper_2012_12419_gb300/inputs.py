"""Seeded synthetic instances of the vehicular-cloud placement MDP.

This module draws inputs only: model sizes, rates, reward weights and discount factors,
from a SplitMix64 stream.  It holds none of the method's arithmetic (no transition
probabilities, rewards or Bellman backups).  The CUDA library and the CPU oracle both
take the dictionaries it returns.

Instance recipe (the paper, Section V, leaves the instance unspecified):
  * hosts H (H-1 vehicles and one RSU), C VM slots per host, task queue 0..Q, and the
    SCHI/CCHI phase bit; S = 2 (Q+1) (C+1)^H states, A = H+1 actions;
  * per instance, in this order: mu_1..mu_H ~ U[0.2, 1], lambda ~ U[0.5, 2],
    delta_1..delta_H ~ U[0.01, 0.1], f ~ U[0.3, 0.7]; reward weights
    (w_occ, w_loss, w_q) = (1, -5, -0.1);
  * the batched workload first draws H in {2..5}, C in {2..6}, Q in {3..12} and
    gamma in {0.9, 0.95, 0.99} per instance, then the rates;
  * the binary-action model (the paper's A = {-1, 1}): H clouds of C VMs, requests of
    1..J VMs, mu_1..mu_H ~ U[0.2, 1], lambda ~ U[0.5, 2], delta_1..delta_H ~ U[0.01, 0.1],
    reward constants (beta_vc, beta_tc, gamma_vc) = (1, 1.2, 1).
Uniform doubles are the top 53 bits of SplitMix64 outputs; the seed of a named
workload is its index in the list below.
"""
from __future__ import annotations

import numpy as np

MASK64 = (1 << 64) - 1

# Named workloads: (H, C, Q, gamma).  S = 2(Q+1)(C+1)^H.
WORKLOADS = {
    "tiny": dict(seed=0, H=3, C=3, Q=4, gamma=0.95),          # S = 640,        A = 4
    "large": dict(seed=1, H=7, C=4, Q=15, gamma=0.95),        # S = 2,500,000,  A = 8
    "batched": dict(seed=2, n=512),                           # 512 instances,  S in [72, 436,982]
    "precision": dict(seed=3, H=8, C=4, Q=15, gamma=0.95),    # S = 12,500,000, A = 9
    "precision_sub": dict(seed=3, H=5, C=4, Q=15, gamma=0.95),  # S = 100,000,   A = 6
    "grad": dict(seed=4, H=6, C=4, Q=10, gamma=0.95),         # S = 343,750,    A = 7
    "medium": dict(seed=1, H=7, C=3, Q=15, gamma=0.95),       # S = 524,288,    A = 8
}

# The paper's binary-action model (A = {-1, 1}): H vehicular clouds of C VMs each, requests
# of 1..J VMs; S = (1 + H J) (C+1)^H, A = 2.
BINARY_WORKLOADS = {
    "binary": dict(seed=5, H=6, C=6, J=3, gamma=0.95),        # S = 2,235,331,  A = 2
    "binary_tiny": dict(seed=6, H=2, C=3, J=2, gamma=0.95),   # S = 80,         A = 2
    "binary_mid": dict(seed=7, H=4, C=4, J=2, gamma=0.95),    # S = 5,625,      A = 2
}

# Reward constants of the paper's numerical section: VM reward per VC, VM cost per paid
# traditional-cloud VM, penalty per idle VC VM.
BINARY_WEIGHTS = dict(beta_vc=1.0, beta_tc=1.2, gamma_vc=1.0)

WEIGHTS = dict(w_occ=1.0, w_loss=-5.0, w_q=-0.1)


class SplitMix64:
    """SplitMix64 (Steele, Lea, Flood 2014): 64-bit state, golden-ratio increment."""

    def __init__(self, seed: int):
        self.state = seed & MASK64

    def next_u64(self) -> int:
        self.state = (self.state + 0x9E3779B97F4A7C15) & MASK64
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
        return z ^ (z >> 31)

    def uniform(self, lo: float = 0.0, hi: float = 1.0) -> float:
        u = (self.next_u64() >> 11) * (1.0 / 9007199254740992.0)
        return lo + (hi - lo) * u

    def choice(self, values):
        values = list(values)
        return values[(self.next_u64() >> 11) * len(values) >> 53]


def num_states(H: int, C: int, Q: int) -> int:
    return 2 * (Q + 1) * (C + 1) ** H


def _draw_rates(rng: SplitMix64, H: int) -> dict:
    mu = [rng.uniform(0.2, 1.0) for _ in range(H)]
    lam = rng.uniform(0.5, 2.0)
    delta = [rng.uniform(0.01, 0.1) for _ in range(H)]
    f = rng.uniform(0.3, 0.7)
    return dict(mu=mu, lam=lam, delta=delta, f=f)


def make_params(H: int, C: int, Q: int, gamma: float, seed: int) -> dict:
    """One instance with rates drawn from SplitMix64(seed)."""
    rng = SplitMix64(seed)
    p = dict(H=H, C=C, Q=Q, gamma=gamma)
    p.update(_draw_rates(rng, H))
    p.update(WEIGHTS)
    return p


def workload(name: str) -> dict:
    """Parameters of a named single-instance workload."""
    w = WORKLOADS[name]
    if name == "batched":
        raise ValueError("use batch_params() for the batched workload")
    return make_params(w["H"], w["C"], w["Q"], w["gamma"], w["seed"])


def binary_params(H: int, C: int, J: int, gamma: float, seed: int) -> dict:
    """One instance of the binary-action model: per VC k a completion rate mu_k ~ U[0.2, 1]
    per busy VM, then the request rate lambda ~ U[0.5, 2], then departure rates
    delta_k ~ U[0.01, 0.1] (the placement model's draws without f), and the paper's reward
    constants."""
    rng = SplitMix64(seed)
    mu = [rng.uniform(0.2, 1.0) for _ in range(H)]
    lam = rng.uniform(0.5, 2.0)
    delta = [rng.uniform(0.01, 0.1) for _ in range(H)]
    p = dict(H=H, C=C, J=J, gamma=gamma, mu=mu, lam=lam, delta=delta)
    p.update(BINARY_WEIGHTS)
    return p


def binary_workload(name: str) -> dict:
    w = BINARY_WORKLOADS[name]
    return binary_params(w["H"], w["C"], w["J"], w["gamma"], w["seed"])


def binary_num_states(H: int, C: int, J: int) -> int:
    return (1 + H * J) * (C + 1) ** H


def batch_params(n: int = 512, seed: int = 2) -> list:
    """n independent uneven instances: H, C, Q, gamma drawn per instance, then the rates."""
    rng = SplitMix64(seed)
    out = []
    for _ in range(n):
        H = rng.choice(range(2, 6))
        C = rng.choice(range(2, 7))
        Q = rng.choice(range(3, 13))
        gamma = rng.choice([0.9, 0.95, 0.99])
        p = dict(H=H, C=C, Q=Q, gamma=gamma)
        p.update(_draw_rates(rng, H))
        p.update(WEIGHTS)
        out.append(p)
    return out


def random_csr_mdp(S: int, A: int, max_succ: int, seed: int, infeasible_frac: float = 0.2, gamma: float = 0.9):
    """A random explicit MDP in CSR form for the generic path.

    Row r = s*A + a holds 1..max_succ distinct successors with positive probabilities that
    sum to one (normalised in FP64), rewards in [-1, 1]; a fraction of rows is infeasible
    (empty, R = -inf) but action 0 is always feasible.  Returns a dict of numpy arrays.
    """
    g = np.random.default_rng(seed)
    row_ptr = [0]
    cols, vals = [], []
    R = np.empty(S * A, np.float64)
    for s in range(S):
        for a in range(A):
            r = s * A + a
            if a > 0 and g.random() < infeasible_frac:
                R[r] = -np.inf
                row_ptr.append(row_ptr[-1])
                continue
            n = int(g.integers(1, max_succ + 1))
            n = min(n, S)
            c = np.sort(g.choice(S, size=n, replace=False)).astype(np.int32)
            w = g.random(n) + 0.05
            v = w / w.sum()
            cols.extend(c.tolist())
            vals.extend(v.tolist())
            R[r] = g.uniform(-1.0, 1.0)
            row_ptr.append(row_ptr[-1] + n)
    return dict(S=S, A=A, gamma=gamma, row_ptr=np.array(row_ptr, np.int64), col=np.array(cols, np.int32),
                val=np.array(vals, np.float64), R=R)


def aaa_trace(n_vehicles: int, n_seconds: int, seed: int, si_per_second: int = 10):
    """A synthetic BSM trace for the AAA timer update: per SI (row) and vehicle (column),
    BSMs sent and acknowledged (one generated per 100 ms SI, each acknowledged with
    probability 0.9), BSMs received from the other vehicles (delivery ratio U[0.7, 1]), and
    their total end-to-end delay in ms (per BSM U[0.2, 2] ms scaled by n_vehicles / 10,
    so denser networks are slower).  Returns three float64 arrays [n_si, n_vehicles]."""
    rng = SplitMix64(seed)
    n_si = n_seconds * si_per_second
    S = np.zeros((n_si, n_vehicles))
    R = np.zeros((n_si, n_vehicles))
    D = np.zeros((n_si, n_vehicles))
    for j in range(n_si):
        for h in range(n_vehicles):
            S[j, h] = 1.0 if rng.uniform() < 0.9 else 0.0
            r = float(int((n_vehicles - 1) * rng.uniform(0.7, 1.0)))
            R[j, h] = r
            D[j, h] = r * rng.uniform(0.2, 2.0) * n_vehicles / 10.0
    return S, D, R
