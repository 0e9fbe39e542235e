"""Helpers shared by the GPU parity tests (no oracle arithmetic here)."""
import numpy as np
import pytest


def native_or_skip():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2012_12419_gb300 import native

    native.load(build_if_missing=True)
    return native


def rel_err(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.max(np.abs(a - b) / np.maximum(np.abs(b), 1e-300)))


def policy_mismatches(pi, pi_ref, gap_ref, min_gap=1e-6):
    """Entries where the reference argmax is unique by more than min_gap and pi differs."""
    pi = np.asarray(pi)
    pi_ref = np.asarray(pi_ref)
    sel = np.asarray(gap_ref) > min_gap
    return int(np.sum(pi[sel] != pi_ref[sel])), int(np.sum(sel))
