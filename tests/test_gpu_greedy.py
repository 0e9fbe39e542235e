"""The greedy heuristic (Algorithm 2 read as a policy) on the device, and the comparison
with the optimum that the paper reports (the MDP schedule is never worse than greedy).

* the device policy equals the oracle's greedy policy exactly (tiny, mid, a one-host model
  and instances of the batched workload);
* its FP64 evaluation on the device equals the oracle's evaluation of the same policy to
  1e-9 relative, and never exceeds the oracle's optimum;
* on the large workload the evaluated greedy values stay below the certified optimum
  everywhere (the optimum's certificate bounds its own error by gamma/(1-gamma) 1e-6), and
  the gap is substantial in the initial-distribution objective;
* a handle without a model (user CSR) is rejected.
"""
import numpy as np
import pytest

import oracle
from paper_2012_12419_gb300 import inputs

from gpu_common import native_or_skip

pytestmark = pytest.mark.gpu


def _cases():
    ps = [inputs.workload("tiny"), inputs.make_params(4, 4, 6, 0.95, seed=7), inputs.make_params(1, 3, 5, 0.9, seed=3)]
    batch = inputs.batch_params(512, seed=2)
    small = [p for p in batch if inputs.num_states(p["H"], p["C"], p["Q"]) <= 3000][:4]
    return ps + small


@pytest.mark.parametrize("k", range(7))
def test_greedy_policy_and_value_match_oracle(k):
    native = native_or_skip()
    p = _cases()[k]
    m = native.MDP.build(p, fmt="implicit")
    pi = m.greedy_policy()
    pio = oracle.greedy_policy(p)
    assert np.array_equal(pi.cpu().numpy(), pio)
    Vg, _ = m.evaluate_policy(pi, tol=1e-12)
    Vgo = oracle.policy_eval_iter(p, pio, tol=1e-13)
    Vg = Vg.cpu().numpy()
    assert np.max(np.abs(Vg - Vgo) / np.maximum(np.abs(Vgo), 1.0)) <= 1e-9
    Vs, _, _, _ = oracle.solve(p, tol=1e-12)
    assert np.all(Vg <= Vs + 1e-9)
    m.close()


def test_greedy_below_certified_optimum_on_the_large_workload():
    native = native_or_skip()
    import torch

    p = inputs.workload("large")
    m = native.MDP.build(p, fmt="implicit")
    _, V64, pi_opt, st = m.value_iterate(tol=1e-6)
    assert st["certified"] == 1
    pig = m.greedy_policy()
    # spot-check the device policy against the oracle's rule on sampled states
    g = np.random.default_rng(0)
    full = oracle.greedy_policy(p)
    idx = g.choice(m.S, 5000, replace=False)
    assert np.array_equal(pig.cpu().numpy()[idx], full[idx])
    Vg, _ = m.evaluate_policy(pig, tol=1e-10)
    slack = p["gamma"] / (1 - p["gamma"]) * 1e-6 + 1e-9
    assert bool(torch.all(Vg <= V64 + slack))
    rho = torch.zeros(m.S, dtype=torch.float64, device="cuda")
    rho[: 2 * (p["Q"] + 1)] = 1.0 / (2 * (p["Q"] + 1))
    J_opt, J_greedy = float(rho @ V64), float(rho @ Vg)
    assert J_opt > J_greedy
    m.close()


def test_greedy_needs_a_model():
    native = native_or_skip()
    import torch

    mdp = inputs.random_csr_mdp(10, 3, max_succ=4, seed=1, gamma=0.9)
    m = native.MDP.from_csr(10, 3, torch.tensor(mdp["row_ptr"], device="cuda"), torch.tensor(mdp["col"], device="cuda"),
                            torch.tensor(mdp["val"].astype(np.float32), device="cuda"),
                            torch.tensor(mdp["R"].astype(np.float32), device="cuda"), 0.9)
    with pytest.raises(native.VcError):
        m.greedy_policy()
    m.close()
