"""Host-side figures of the benchmark line, checked on the CPU against
brute force: the merge-model bytes of Alg. 1 (every forward edge reads both
forward lists, Sec. 4) on small graphs."""
import numpy as np

import bench
import synth


def brute_merge_bytes(n, src, dst):
    deg = [0] * n
    for a, b in zip(src.tolist(), dst.tolist()):
        deg[a] += 1
        deg[b] += 1
    fwd = []
    for a, b in zip(src.tolist(), dst.tolist()):
        fwd.append((a, b) if (deg[a], a) < (deg[b], b) else (b, a))
    dplus = [0] * n
    for u, _ in fwd:
        dplus[u] += 1
    return 8 * sum(dplus[u] + dplus[v] for u, v in fwd)


def test_merge_model_bytes_equal_brute_force():
    for seed in (1, 2, 3):
        s, d = synth.er_graph(300, 3000, seed)
        assert bench.merge_model_bytes(300, s, d) == brute_merge_bytes(300, s, d)
    s, d = synth.chung_lu(2000, 2.1, 10.0, 300.0, 4)
    assert bench.merge_model_bytes(2000, s, d) == brute_merge_bytes(2000, s, d)


def test_merge_model_bytes_of_a_star_and_a_triangle():
    # star K_{1,4}: leaves (degree 1) come first, each leaf's list is {centre}; the centre's is empty
    s = np.array([0, 0, 0, 0], dtype=np.uint32)
    d = np.array([1, 2, 3, 4], dtype=np.uint32)
    assert bench.merge_model_bytes(5, s, d) == 8 * 4 * (1 + 0)
    # triangle: lists of sizes 2, 1, 0 along Node Order; edges 0-1, 0-2, 1-2 read 3, 2, 1 entries
    s = np.array([0, 0, 1], dtype=np.uint32)
    d = np.array([1, 2, 2], dtype=np.uint32)
    assert bench.merge_model_bytes(3, s, d) == 8 * (3 + 2 + 1)
