"""perch_best_noalloc against perch_best, through the C ABI, on the GPU.

perch_best_noalloc serves callers that may not allocate device memory once
running (it needs no context and keeps its scratch in a static device array).
It must return exactly what the context-based perch_best returns, call after
call, since every call reuses the same scratch.  This file is collected last.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_noalloc_matches_best_on_consecutive_calls():
    import torch
    from paper_2008_00326_gb300 import build, perch as P
    build.build()
    P.load()
    rng = np.random.default_rng(11)
    with P.Context(0) as ctx:
        s = torch.cuda.Stream()
        for call, n in enumerate((300_001, 4_097, 1)):
            costs = rng.integers(0, 6, size=(n, 2)).astype(np.int32)
            ids = rng.permutation(n).astype(np.uint64) if call == 1 else None
            want = ctx.best(costs, ids)                      # existing entry point
            d_costs = torch.from_numpy(costs).cuda()
            d_ids = None if ids is None else torch.from_numpy(ids.view(np.int64)).cuda()
            with torch.cuda.stream(s):
                # filled on the stream the kernel runs on, so the fill is ordered before it
                bi = torch.full((1,), -7, dtype=torch.int64, device="cuda")
                bc = torch.full((1,), -7, dtype=torch.int32, device="cuda")
                s.wait_stream(torch.cuda.current_stream())
                P.perch_best_noalloc(d_costs, d_ids, bi, bc, stream=s)
            s.synchronize()
            assert (int(bi.item()), int(bc.item())) == want, (call, n)


def test_noalloc_rejects_sizes_beyond_the_maximum():
    from paper_2008_00326_gb300 import build, perch as P
    import ctypes as C
    build.build()
    L = P.load()
    dummy = C.c_void_p(16)   # never dereferenced: the size check comes first
    assert L.perch_best_noalloc(dummy, None, 1 << 31, dummy, dummy, None) == -1
    assert L.perch_best_noalloc(dummy, None, 0, dummy, dummy, None) == -1


def test_noalloc_refuses_host_memory():
    """A host pointer is refused before any launch (the kernel would fault on it)."""
    import ctypes as C
    import torch
    from paper_2008_00326_gb300 import build, perch as P
    build.build()
    L = P.load()
    torch.cuda.init()
    host = np.zeros((8, 2), np.int32)
    out_i = np.zeros(1, np.int64)
    out_c = np.zeros(1, np.int32)
    assert L.perch_best_noalloc(host.ctypes.data, None, 8, out_i.ctypes.data, out_c.ctypes.data, None) == -1
    with pytest.raises(TypeError):
        P.perch_best_noalloc(torch.zeros((8, 2), dtype=torch.int32), None,
                             torch.zeros(1, dtype=torch.int64, device="cuda"),
                             torch.zeros(1, dtype=torch.int32, device="cuda"))
