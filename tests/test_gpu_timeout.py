"""Failure detection without a GPU fault: the bounded shared-memory waits of the pipelined
sweeps are capped from the host (0 polls: give up at once), the solve reports
VC_ERR_TIMEOUT, and the same handle then solves normally with the default cap (the kernels
drained their own copies and returned; the context is intact).  No wait is left unbounded:
a capped wait returns, it never spins."""
import numpy as np
import pytest

import oracle
from paper_2012_12419_gb300 import inputs

from gpu_common import native_or_skip, rel_err

pytestmark = pytest.mark.gpu

MID = inputs.make_params(4, 4, 6, 0.95, seed=7)


@pytest.mark.parametrize("sliced", [False, True])
def test_forced_wait_timeout_is_reported_and_recoverable(sliced):
    native = native_or_skip()
    m = native.MDP.build(MID, fmt="csr_f32", padded=True, sliced=sliced)
    assert m.info()["csr_pipelined"] == 1
    m.set_wait_limit(0)
    with pytest.raises(native.VcError) as e:
        m.value_iterate(tol=1e-6)
    assert e.value.code == native.VC_ERR_TIMEOUT
    m.set_wait_limit(-1)
    _, V64, pi, st = m.value_iterate(tol=1e-6)
    assert st["certified"] == 1
    Vs, _, _, _ = oracle.solve(MID, tol=1e-12)
    assert rel_err(V64.cpu().numpy(), Vs) <= 1e-6
    m.close()
