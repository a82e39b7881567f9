"""Helpers shared by the GPU parity tests (comparison against the FP64 oracle)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")


def require_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def assert_same_tree(got, ref):
    """Edge lists equal entry by entry (both in K order), weights bit-exact."""
    gu, gv, gw = (np.asarray(got["u"]), np.asarray(got["v"]), np.asarray(got["w"]))
    assert len(gu) == len(ref["u"])
    bad = np.flatnonzero((gu != ref["u"]) | (gv != ref["v"]))
    assert bad.size == 0, f"first differing edge at {bad[:5]}: got {list(zip(gu[bad[:3]], gv[bad[:3]], gw[bad[:3]]))} " \
                          f"want {list(zip(ref['u'][bad[:3]], ref['v'][bad[:3]], ref['w'][bad[:3]]))}"
    assert np.array_equal(gw, ref["w"])


def to_np(x):
    if hasattr(x, "detach"):
        return x.detach().cpu().numpy()
    return np.asarray(x)
