"""The AAA multichannel timer update (Section II, Algorithm 1) -- the library's host routine
and the oracle's plain transcription -- and the SCHI fraction it feeds to the placement
model.

Pins of the oracle (not taken from either implementation):
* a trace worked out by hand (two vehicles, three SIs per second);
* no BSM traffic: U_CCH = 0, so the CCH interval shrinks to 0 and f = 1;
* saturated traffic: U_CCH >= DCCHI restores the 50/50 defaults (f = 1/2);
* CCHI + SCHI = SI after every update (the update only moves the inactivity I_CCH).
Then the library equals the oracle exactly on synthetic traces of several densities, and
(on a GPU) the f of a trace is a valid model parameter that solves to the oracle's optimum.
"""
import numpy as np
import pytest

import oracle
from paper_2012_12419_gb300 import inputs


def _lib():
    from paper_2012_12419_gb300 import build, native

    if not build.up_to_date():
        pytest.skip("library not built")
    return native


def test_oracle_hand_example():
    # SI 0: S_V2V = (0 + 3 + 5) / (1 + 2) = 8/3;   D_V2V = (0 + 6 + 10) / (1 + 2 + 3) = 8/3
    # SI 1: S_V2V = (8/3 + 4 + 2) / 3 = 26/9;      D_V2V = (8/3 + 4 + 4) / (1 + 2 + 2) = 32/15
    # SI 2 (UTC second): U_CCH = 26/9 * 32/15 = 832/135 < 50, I_CCH = 50 - 832/135,
    #   CCHI = 832/135, SCHI = 50 + 50 - 832/135 = 100 - 832/135
    S = [[3, 5], [4, 2], [9, 9]]
    D = [[6, 10], [4, 4], [0, 0]]
    R = [[2, 3], [2, 2], [0, 0]]
    c, s, f = oracle.aaa_intervals(S, D, R, si_per_second=3)
    assert c == pytest.approx([832 / 135], rel=1e-15)
    assert s == pytest.approx([100 - 832 / 135], rel=1e-15)
    assert f == pytest.approx([(100 - 832 / 135) / 100], rel=1e-15)


def test_oracle_no_traffic_and_saturation():
    zero = [[0.0] * 4 for _ in range(20)]
    c, s, f = oracle.aaa_intervals(zero, zero, zero)
    assert c == [0.0, 0.0] and s == [100.0, 100.0] and f == [1.0, 1.0]
    # every vehicle sends one BSM per SI and each received BSM takes 200 ms: U >= DCCHI
    S = [[1.0] * 4 for _ in range(10)]
    R = [[3.0] * 4 for _ in range(10)]
    D = [[600.0] * 4 for _ in range(10)]
    c, s, f = oracle.aaa_intervals(S, D, R)
    assert c == [50.0] and s == [50.0] and f == [0.5]


def _library_equals_oracle(n_vehicles, seed):
    S, D, R = inputs.aaa_trace(n_vehicles, 6, seed)
    c, s, f = oracle.aaa_intervals(S.tolist(), D.tolist(), R.tolist())
    assert len(c) == 6
    for a, b, x in zip(c, s, f):
        assert a + b == pytest.approx(100.0, rel=1e-12)
        assert 0.0 <= a <= 50.0 and x == b / 100.0
    native = _lib()
    lc, ls, lf = native.aaa_intervals(S, D, R)
    assert np.array_equal(lc, np.array(c)) and np.array_equal(ls, np.array(s)) and np.array_equal(lf, np.array(f))


@pytest.mark.parametrize("n_vehicles,seed", [(5, 1), (40, 2), (200, 3)])
def test_intervals_sum_to_the_si_and_library_equals_oracle(n_vehicles, seed):
    _library_equals_oracle(n_vehicles, seed)


@pytest.mark.gpu
@pytest.mark.parametrize("n_vehicles,seed", [(5, 1), (40, 2), (200, 3), (1000, 4)])
def test_library_equals_oracle_in_the_gpu_build(n_vehicles, seed):
    """The same comparison in the GPU test run, against the library built on that machine
    (the routine is host code, so the GPU build is the one a user of the GPU path loads)."""
    from gpu_common import native_or_skip

    native_or_skip()
    _library_equals_oracle(n_vehicles, seed)


def test_library_argument_errors():
    native = _lib()
    z = np.zeros((10, 2))
    with pytest.raises(native.VcError):
        native.aaa_intervals(z, z, z, dcchi_ms=40.0, dschi_ms=50.0)
    with pytest.raises(native.VcError):
        native.aaa_intervals(z, z, z, si_per_second=0)


@pytest.mark.gpu
def test_trace_fraction_feeds_the_model():
    """The last second's f of a dense trace parameterises a model that solves to the
    oracle's optimum; a sparser network (larger f) changes the optimum."""
    native = _lib()
    from gpu_common import native_or_skip, rel_err

    native_or_skip()
    S, D, R = inputs.aaa_trace(200, 3, 7)
    _, _, f = native.aaa_intervals(S, D, R)
    assert 0.0 < f[-1] < 1.0
    p = dict(inputs.make_params(3, 3, 4, 0.95, seed=1), f=float(f[-1]))
    m = native.MDP.build(p, fmt="implicit")
    _, V64, _, st = m.value_iterate(tol=1e-6)
    assert st["certified"] == 1
    Vs = oracle.solve(p, tol=1e-12)[0]
    assert rel_err(V64.cpu().numpy(), Vs) <= 1e-6
    m.close()
