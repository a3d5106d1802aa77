"""CPU oracle for uncertain balanced/unbalanced triangles -- TEST INFRASTRUCTURE.

Only the test suite, ``__graft_entry__.smoke()`` and the benchmark's CPU
baseline leg may import this package.  It is independent of the CUDA path:
the two share no code, and nothing in the product path calls it.

``ubt_oracle.c`` holds the arithmetic (see its header for the passages of
the paper each part follows); this module compiles it with the system C
compiler into ``liboracle.so`` next to the source and marshals numpy arrays.

Parity status of each function (what pins it, in the tests under
``tests/test_oracle_*.py``):
  num_triangles / list_triangles -- O(n^3) brute-force listing; trace(A^3)/6.
  count_threshold / enumerate    -- brute force over all 2^m sign worlds in
      exact rationals; closed forms on K_n; the boundary cases the paper
      describes in Sec. 3 and Sec. 5 (golden fixtures).
  expected_fixed / expected_real -- the same brute force (exact rationals).
  grad_real                      -- central finite differences (exact: the
      expected count is affine in each p_e); closed form on K_n.
  ResidentGraph.count            -- equals count_threshold (the serial pass) on
      several graphs for any thread count; its samples partition the counts.
  philox4x64_10                  -- numpy's Philox bit generator.
  local_counts                   -- sums over edges / vertices = 3 x the counts;
      brute-force classification in exact rationals; closed forms on K_n.
  world_counts                   -- per-world recount from numpy Philox draws
      and brute-force listing; binomial bounds on the sign frequencies.
The paper's worked example with numbers (Sec. 1, the two example triangles
with balance probabilities 0.77 and 0.468) is parity unpinned: its edge
probabilities exist only in a figure that is not in the text.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ubt_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None

STATUS = {0: "ok", -1: "vertex out of range", -2: "self-loop", -3: "duplicate edge",
          -4: "probability out of range", -5: "tau out of range", -6: "out of memory"}


class OracleError(RuntimeError):
    pass


def build(force: bool = False) -> str:
    """Compile the oracle (plain C, -O2, with OpenMP where the compiler has
    it, else single-threaded) into liboracle.so; returns its path."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".%d.tmp" % os.getpid()
        cc = os.environ.get("CC", "gcc")
        base = [cc, "-O2", "-std=c11", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
        r = subprocess.run(base[:1] + ["-fopenmp"] + base[1:], capture_output=True)
        if r.returncode != 0:
            subprocess.check_call(base)
        os.replace(tmp, _LIB)
    return _LIB


def _L():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        P = ctypes.c_void_p
        I64 = ctypes.c_int64
        lib.ubto_num_triangles.restype = I64
        lib.ubto_num_triangles.argtypes = [I64, I64, P, P]
        lib.ubto_list.restype = I64
        lib.ubto_list.argtypes = [I64, I64, P, P, I64, P, P]
        lib.ubto_count_threshold.restype = ctypes.c_int
        lib.ubto_count_threshold.argtypes = [I64, I64, P, P, P, ctypes.c_int, P, P, P]
        lib.ubto_enumerate.restype = I64
        lib.ubto_enumerate.argtypes = [I64, I64, P, P, P, ctypes.c_double, ctypes.c_int, I64, P, P, P]
        lib.ubto_expected_fixed.restype = ctypes.c_int
        lib.ubto_expected_fixed.argtypes = [I64, I64, P, P, P, P, P, P]
        lib.ubto_expected_real.restype = ctypes.c_int
        lib.ubto_expected_real.argtypes = [I64, I64, P, P, P, P]
        lib.ubto_grad_real.restype = ctypes.c_int
        lib.ubto_grad_real.argtypes = [I64, I64, P, P, P, P, P]
        lib.ubto_philox4x64_10.restype = None
        lib.ubto_philox4x64_10.argtypes = [P, P, P]
        lib.ubto_world_word.restype = ctypes.c_uint64
        lib.ubto_world_word.argtypes = [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32]
        lib.ubto_local_counts.restype = ctypes.c_int
        lib.ubto_local_counts.argtypes = [I64, I64, P, P, P, ctypes.c_int, P, P, P, P, P]
        lib.ubto_sample_class.restype = I64
        lib.ubto_sample_class.argtypes = [I64, I64]
        lib.ubto_threads.restype = ctypes.c_int
        lib.ubto_threads.argtypes = []
        lib.ubto_graph_new.restype = P
        lib.ubto_graph_new.argtypes = [I64, I64, P, P, ctypes.POINTER(ctypes.c_int)]
        lib.ubto_graph_free.restype = None
        lib.ubto_graph_free.argtypes = [P]
        lib.ubto_graph_count.restype = I64
        lib.ubto_graph_count.argtypes = [P, P, ctypes.c_int, P, I64, I64, ctypes.c_int, P, P]
        lib.ubto_world_counts.restype = ctypes.c_int
        lib.ubto_world_counts.argtypes = [I64, I64, P, P, P, P, ctypes.c_uint64, ctypes.c_int, P, P]
        _lib = lib
    return _lib


def _u32(a):
    return np.ascontiguousarray(a, dtype=np.uint32)


def _ptr(a):
    return None if a is None else a.ctypes.data


def _check(rc):
    if rc < 0:
        raise OracleError(STATUS.get(int(rc), str(rc)))
    return rc


def num_triangles(n, src, dst) -> int:
    s, d = _u32(src), _u32(dst)
    return int(_check(_L().ubto_num_triangles(n, s.size, _ptr(s), _ptr(d))))


def list_triangles(n, src, dst):
    """All triangles: (vtx (T,3) uint32 with a<b<c, eid (T,3) = (e_ab, e_ac, e_bc)),
    sorted lexicographically by vertex triple."""
    s, d = _u32(src), _u32(dst)
    t = int(_check(_L().ubto_list(n, s.size, _ptr(s), _ptr(d), 0, None, None)))
    vtx = np.zeros((max(t, 1), 3), dtype=np.uint32)
    eid = np.zeros((max(t, 1), 3), dtype=np.uint32)
    _check(_L().ubto_list(n, s.size, _ptr(s), _ptr(d), t, _ptr(vtx), _ptr(eid)))
    vtx, eid = vtx[:t], eid[:t]
    order = np.lexsort((vtx[:, 2], vtx[:, 1], vtx[:, 0]))
    return vtx[order], eid[order]


def count_threshold(n, src, dst, k, taus):
    """(bal[n_tau], unbal[n_tau]) int64 counts."""
    s, d, kk = _u32(src), _u32(dst), _u32(k)
    t = np.ascontiguousarray(np.atleast_1d(np.asarray(taus, dtype=np.float64)))
    bal = np.zeros(t.size, dtype=np.int64)
    unbal = np.zeros(t.size, dtype=np.int64)
    _check(_L().ubto_count_threshold(n, s.size, _ptr(s), _ptr(d), _ptr(kk), t.size, _ptr(t),
                                     _ptr(bal), _ptr(unbal)))
    return bal, unbal


def threads() -> int:
    """Threads the oracle's multi-threaded count can use (1 without OpenMP)."""
    return int(_L().ubto_threads())


def sample_class(u, sample_mod) -> int:
    """The sample a vertex u belongs to in ResidentGraph.count (a hash of u mod sample_mod)."""
    return int(_L().ubto_sample_class(int(u), int(sample_mod)))


class ResidentGraph:
    """The oracle's forward lists built once, for repeated counting queries
    (the CPU baseline times queries on a built graph, as the GPU side does).
    count() runs Alg. 1's outer loop over `threads` threads; with sample_mod
    > 1 it visits only the u with sample_class(u, sample_mod) == sample_rem
    (the triangles whose earliest vertex in Node Order is such a u)."""

    def __init__(self, n, src, dst):
        s, d = _u32(src), _u32(dst)
        st = ctypes.c_int(0)
        self.m = s.size
        self._g = _L().ubto_graph_new(n, s.size, _ptr(s), _ptr(d), ctypes.byref(st))
        _check(st.value)

    def count(self, k, taus, threads=1, sample_mod=1, sample_rem=0):
        """(bal[n_tau], unbal[n_tau], triangles visited)."""
        kk = _u32(k)
        assert kk.size == self.m
        t = np.ascontiguousarray(np.atleast_1d(np.asarray(taus, dtype=np.float64)))
        bal = np.zeros(t.size, dtype=np.int64)
        unbal = np.zeros(t.size, dtype=np.int64)
        tri = _check(_L().ubto_graph_count(self._g, _ptr(kk), t.size, _ptr(t), int(sample_mod), int(sample_rem),
                                           int(threads), _ptr(bal), _ptr(unbal)))
        return bal, unbal, int(tri)

    def close(self):
        if getattr(self, "_g", None):
            _L().ubto_graph_free(self._g)
            self._g = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def enumerate_records(n, src, dst, k, tau, which=3):
    """Records sorted by (u, v, w): (uvw (R,3) uint32, cls (R,) uint32, pbal (R,) float64)."""
    s, d, kk = _u32(src), _u32(dst), _u32(k)
    r = int(_check(_L().ubto_enumerate(n, s.size, _ptr(s), _ptr(d), _ptr(kk), float(tau), int(which),
                                       0, None, None, None)))
    uvw = np.zeros((max(r, 1), 3), dtype=np.uint32)
    cls = np.zeros(max(r, 1), dtype=np.uint32)
    pb = np.zeros(max(r, 1), dtype=np.float64)
    _check(_L().ubto_enumerate(n, s.size, _ptr(s), _ptr(d), _ptr(kk), float(tau), int(which),
                               r, _ptr(uvw), _ptr(cls), _ptr(pb)))
    uvw, cls, pb = uvw[:r], cls[:r], pb[:r]
    order = np.lexsort((uvw[:, 2], uvw[:, 1], uvw[:, 0]))
    return uvw[order], cls[order], pb[order]


def expected_fixed(n, src, dst, k):
    """Exact expected counts for fixed-point input.

    Returns (T, S) with S = sum over triangles of 2^48 * P_bal as a Python int;
    E_bal = S / 2^48 and E_unbal = T - E_bal exactly.
    """
    s, d, kk = _u32(src), _u32(dst), _u32(k)
    t = np.zeros(1, dtype=np.int64)
    lo = np.zeros(1, dtype=np.uint64)
    hi = np.zeros(1, dtype=np.uint64)
    _check(_L().ubto_expected_fixed(n, s.size, _ptr(s), _ptr(d), _ptr(kk), _ptr(t), _ptr(lo), _ptr(hi)))
    return int(t[0]), (int(hi[0]) << 64) | int(lo[0])


def expected_real(n, src, dst, p):
    """(E_bal, E_unbal, T) for float32 probabilities, double accumulation."""
    s, d = _u32(src), _u32(dst)
    pp = np.ascontiguousarray(p, dtype=np.float32)
    out = np.zeros(3, dtype=np.float64)
    _check(_L().ubto_expected_real(n, s.size, _ptr(s), _ptr(d), _ptr(pp), _ptr(out)))
    return float(out[0]), float(out[1]), int(out[2])


def grad_real(n, src, dst, p, with_abs=False):
    """dE_bal/dp_e for every edge (input order), float64; optionally also
    sum over triangles of |dP_bal/dp_e|."""
    s, d = _u32(src), _u32(dst)
    pp = np.ascontiguousarray(p, dtype=np.float32)
    g = np.zeros(s.size, dtype=np.float64)
    ga = np.zeros(s.size, dtype=np.float64) if with_abs else None
    _check(_L().ubto_grad_real(n, s.size, _ptr(s), _ptr(d), _ptr(pp), _ptr(g), _ptr(ga)))
    return (g, ga) if with_abs else g


def local_counts(n, src, dst, k, taus):
    """Per-edge (input order) and per-vertex local counts of t-balanced and
    t-unbalanced triangles: (edge_bal, edge_unbal) int64 (m, n_tau) and
    (vtx_bal, vtx_unbal) int64 (n, n_tau)."""
    s, d, kk = _u32(src), _u32(dst), _u32(k)
    t = np.ascontiguousarray(np.atleast_1d(np.asarray(taus, dtype=np.float64)))
    m = s.size
    eb = np.zeros((max(m, 1), t.size), dtype=np.int64)
    eu = np.zeros((max(m, 1), t.size), dtype=np.int64)
    vb = np.zeros((max(n, 1), t.size), dtype=np.int64)
    vu = np.zeros((max(n, 1), t.size), dtype=np.int64)
    _check(_L().ubto_local_counts(n, m, _ptr(s), _ptr(d), _ptr(kk), t.size, _ptr(t), _ptr(eb), _ptr(eu),
                                  _ptr(vb), _ptr(vu)))
    return eb[:m], eu[:m], vb[:n], vu[:n]


def philox4x64_10(ctr, key):
    c = np.ascontiguousarray(ctr, dtype=np.uint64)
    k = np.ascontiguousarray(key, dtype=np.uint64)
    out = np.zeros(4, dtype=np.uint64)
    _L().ubto_philox4x64_10(_ptr(c), _ptr(k), _ptr(out))
    return out


def world_word(seed, ekey, word, k) -> int:
    return int(_L().ubto_world_word(int(seed), int(ekey), int(word), int(k)))


def world_counts(n, src, dst, k, seed, words, ekey=None):
    """Per-world balanced counts for the given world words: (len(words)*64,) int64."""
    s, d, kk = _u32(src), _u32(dst), _u32(k)
    w = _u32(np.atleast_1d(words))
    ek = None if ekey is None else _u32(ekey)
    out = np.zeros(w.size * 64, dtype=np.int64)
    _check(_L().ubto_world_counts(n, s.size, _ptr(s), _ptr(d), _ptr(kk), _ptr(ek), int(seed),
                                  w.size, _ptr(w), _ptr(out)))
    return out
