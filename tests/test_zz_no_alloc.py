"""ubt_count_threshold_noalloc, the threshold count for callers that cannot
allocate device memory where they query (code that may only use the buffers
it is handed): its per-call scratch is a fixed array inside the library.

Called through the C ABI and compared with ubt_count_threshold and with the
oracle, twice in a row on each graph (the fixed array keeps the previous
call's contents, so the second call checks that it is cleared).  Counts are
integers: the comparison is exact.  The traversal's self-checks of these
calls reach the graph's own self-check word, which must read 0 afterwards.
This file sorts last so that a run stopping at the first failure has already
run every other test.
"""
import ctypes

import numpy as np
import pytest

import oracle
import synth
from gpu_util import mixed_graph, require_gpu

pytestmark = pytest.mark.gpu


def call_noalloc(ubt, G, taus, prune, out):
    import torch
    t = np.ascontiguousarray(np.atleast_1d(taus), dtype=np.float64)
    return ubt.lib().ubt_count_threshold_noalloc(G.handle, t.ctypes.data_as(ctypes.c_void_p), t.size, int(prune),
                                                ctypes.c_void_p(out.data_ptr()),
                                                ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))


def graphs():
    s, d = synth.chung_lu(20000, 2.1, 20.0, 2000.0, 3)
    yield 20000, s, d, synth.quantise(synth.p_beta(s.size, 0.5, 0.5, 4))
    s, d = mixed_graph(3000, 30000, 5)
    yield 3000, s, d, synth.k_uniform(s.size, 6)


@pytest.mark.parametrize("taus", [[0.6], [0.55, 0.7], [0.55, 0.7, 0.85, 0.95],
                                  [0.5, 0.51, 0.6, 0.7, 0.75, 0.8, 0.9, 1.0]])
def test_noalloc_matches_count_threshold_twice(taus):
    ubt = require_gpu()
    import torch
    for n, s, d, k in graphs():
        G = ubt.Graph(n, s, d, k=k)
        ob, ou = oracle.count_threshold(n, s, d, k, taus)
        for prune in (0, 1):
            want_b, want_u = G.count_threshold(taus, prune=prune)
            want = np.concatenate([want_b, want_u])
            assert np.array_equal(want, np.concatenate([ob, ou]))
            for _ in range(2):
                out = torch.full((2 * len(taus),), -1, dtype=torch.int64, device="cuda")
                assert call_noalloc(ubt, G, taus, prune, out) == 0
                torch.cuda.synchronize()
                assert np.array_equal(out.cpu().numpy(), want), (n, taus, prune)
        assert G.guard() == 0


def test_noalloc_rejects_more_thresholds_than_its_scratch_holds():
    ubt = require_gpu()
    import torch
    s, d = synth.er_graph(200, 2000, 9)
    G = ubt.Graph(200, s, d, k=synth.k_uniform(s.size, 10))
    out = torch.zeros(18, dtype=torch.int64, device="cuda")
    st = call_noalloc(ubt, G, np.linspace(0.5, 0.9, 9), 1, out)
    assert st == -12
    assert "fixed scratch" in ubt.lib().ubt_status_str(st).decode()
