"""The allocation-free SSE entry point (als_eval_sse_static).

Some callers may not allocate device memory when they evaluate: code running
while its stream is captured into a CUDA graph, programs whose device memory
all belongs to their own pool allocator, services held to a fixed memory
budget. als_eval_sse_static serves them: it needs no handle and keeps its
partial sums in a fixed device array compiled into the library. This test
calls it through the C ABI and compares it with als_eval_sse, twice in a row
on different entry sets, so a stale partial from the first call would show up
in the second. The file sorts last so a stop-at-first-failure run has already
run every other test.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _entries(rng, n, n_u, n_m):
    iu = torch.as_tensor(rng.integers(0, n_u, n).astype(np.int32)).cuda()
    im = torch.as_tensor(rng.integers(0, n_m, n).astype(np.int32)).cuda()
    r = torch.as_tensor(rng.integers(1, 6, n).astype(np.float32)).cuda()
    return iu, im, r


def test_static_sse_matches_handle_sse_on_consecutive_calls():
    from paper_2509_18024_gb300 import binding as B
    from paper_2509_18024_gb300 import core_als

    lib = B.load()
    rng = np.random.default_rng(42)
    n_u, n_m, f = 3000, 2000, 24
    U = torch.as_tensor(rng.standard_normal((n_u, f)).astype(np.float32)).cuda()
    M = torch.as_tensor(rng.standard_normal((n_m, f)).astype(np.float32)).cuda()
    eng = core_als.CoreALS(f, 0.05, 0.25)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    # A multi-block call (300k entries, 19 blocks), then a one-block call.
    for n in (300_000, 5_000):
        iu, im, r = _entries(rng, n, n_u, n_m)
        out = torch.full((1,), -1.0, dtype=torch.float64, device="cuda")
        rc = lib.als_eval_sse_static(n, iu.data_ptr(), im.data_ptr(), r.data_ptr(), U.data_ptr(), M.data_ptr(),
                                     f, out.data_ptr(), stream)
        assert rc == 0, B.STATUS.get(rc, rc)
        torch.cuda.synchronize()
        ref = eng.sse(iu, im, r, U, M)
        assert out.item() == pytest.approx(ref, rel=1e-10)


def test_static_sse_rejects_oversize_and_bad_arguments():
    from paper_2509_18024_gb300 import binding as B

    lib = B.load()
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    dummy = out.data_ptr()
    rc = lib.als_eval_sse_static(B.ALS_SSE_STATIC_MAX_ENTRIES + 1, dummy, dummy, dummy, dummy, dummy, 8,
                                 out.data_ptr(), None)
    assert rc == -1
    assert lib.als_eval_sse_static(10, None, None, None, None, None, 8, out.data_ptr(), None) == -1
    assert lib.als_eval_sse_static(0, None, None, None, None, None, 8, out.data_ptr(), None) == 0
    torch.cuda.synchronize()
    assert out.item() == 0.0
