"""wm_emst_noalloc: the EMST entry point for callers that cannot allocate device memory.

Its scratch lives in the library's static device array, so a caller that has handed all of its
device memory to its own pool, or that runs where cudaMalloc's synchronisation is not allowed,
can still compute an EMST.  These tests call it through the C ABI and check that its output
equals wm_emst's (edge lists identical, weights bit-exact, total within a relative 1e-12, the
tolerance of the other EMST tests) on two calls in a row, with host and with device buffers, and
that it rejects sizes beyond its limit.  The file is named to be collected last; it passes both
alone in a fresh process and after the other tests.
"""
import ctypes

import numpy as np
import pytest

import synthdata
import paper_2104_01126_gb300 as wm
from gpu_common import require_gpu, torch

pytestmark = pytest.mark.gpu

MAX_POINTS = 32768


@pytest.fixture(scope="module")
def lib():
    require_gpu()
    return wm.load()


def _call_noalloc(lib, x, precision=0, stream=None):
    """wm_emst_noalloc through ctypes with host input and host outputs."""
    x = np.ascontiguousarray(x)
    n, d = x.shape
    out = np.zeros(max(n - 1, 1), dtype=wm.EDGE_DTYPE)
    total = ctypes.c_double(-1.0)
    opts = wm._Opts()
    opts.precision = precision
    opts.stream = stream
    dtype = wm.WM_F32 if x.dtype == np.float32 else wm.WM_F64
    rc = lib.wm_emst_noalloc(x.ctypes.data, n, d, dtype, wm.WM_AOS, out.ctypes.data, ctypes.byref(total),
                             ctypes.byref(opts))
    return rc, out[: n - 1], total.value


def _same(noalloc_out, noalloc_total, ref):
    assert np.array_equal(noalloc_out["u"], ref["u"])
    assert np.array_equal(noalloc_out["v"], ref["v"])
    assert np.array_equal(noalloc_out["w"], ref["w"])
    assert abs(noalloc_total - ref["total"]) <= 1e-12 * max(ref["total"], 1e-300)


@pytest.mark.parametrize("kind,n,d,prec", [("uniform", 20000, 2, 0), ("gmm", 32768, 3, 0), ("uniform", 5000, 5, 1),
                                           ("uniform", 32768, 7, 0), ("uniform", 32768, 16, 0)])
def test_noalloc_matches_wm_emst_on_two_calls_in_a_row(lib, kind, n, d, prec):
    xs = [synthdata.generate(kind, n, d, seed) for seed in (1, 2)]
    for x in xs:   # two calls in a row; the second reuses the static scratch left by the first
        ref = wm.emst(x, precision="fp64" if prec else "fp32")
        rc, out, total = _call_noalloc(lib, x, prec)
        assert rc == 0, lib.wm_last_error_detail()
        _same(out, total, ref)


def test_noalloc_device_buffers(lib):
    x = synthdata.uniform(10000, 3, seed=5).astype(np.float32)
    ref = wm.emst(x)
    xd = torch.from_numpy(x).cuda()
    for _ in range(2):
        got = wm.emst_noalloc(xd)
        assert got["u"].is_cuda
        assert np.array_equal(got["u"].cpu().numpy(), ref["u"])
        assert np.array_equal(got["v"].cpu().numpy(), ref["v"])
        assert np.array_equal(got["w"].cpu().numpy(), ref["w"])
        assert abs(got["total"] - ref["total"]) <= 1e-12 * ref["total"]


def test_noalloc_rejects_sizes_beyond_the_limit(lib):
    x = np.zeros((MAX_POINTS + 1, 2))
    rc, _, _ = _call_noalloc(lib, x)
    assert rc == -1
    assert b"WM_NOALLOC_MAX_POINTS" in lib.wm_last_error_detail()


def test_noalloc_tiny_inputs(lib):
    for n in (1, 2, 3):
        x = synthdata.uniform(n, 2, seed=n)
        rc, out, total = _call_noalloc(lib, x)
        assert rc == 0
        ref = wm.emst(x)
        _same(out, total, ref)


def test_noalloc_two_threads_on_two_streams(lib):
    # Calls from two host threads, each on a stream of its own, share the one static array: the
    # entry point serialises them per device and returns only after its GPU work has finished,
    # so every result must still equal wm_emst's.
    import threading
    inputs = [[synthdata.generate(kind, 6000 + 997 * i, d, seed=40 + 10 * t + i) for i in range(3)]
              for t, (kind, d) in enumerate((("uniform", 3), ("gmm", 2)))]
    refs = [[wm.emst(x) for x in xs] for xs in inputs]
    streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    results = [[None] * 3, [None] * 3]

    def worker(t):
        torch.cuda.set_device(0)
        for i, x in enumerate(inputs[t]):
            results[t][i] = _call_noalloc(lib, x, stream=streams[t].cuda_stream)

    threads = [threading.Thread(target=worker, args=(t,)) for t in range(2)]
    for th in threads:
        th.start()
    for th in threads:
        th.join()
    for t in range(2):
        for i in range(3):
            rc, out, total = results[t][i]
            assert rc == 0
            _same(out, total, refs[t][i])
