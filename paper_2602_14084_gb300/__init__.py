"""Python binding of libubt -- uncertain balanced/unbalanced triangles on GB300.

Argument marshalling only: every step of the path runs in the CUDA kernels of
``libubt.so`` (built from ``csrc/`` by ``_build.py``), reached through the C
ABI declared in ``include/ubt.h``.  PyTorch provides device memory and
streams.  There is no CPU fallback: if the library is missing the import of
any entry point raises.

Paper: "Counting Balanced Triangles on Social Networks With Uncertain Edge
Signs" (arXiv 2602.14084): t-balanced triangles have P_bal >= t and
t-unbalanced ones P_unbal > t (Defs. 4-5, Sec. 3); counting and enumeration
problems (Defs. 7-8); exact algorithms Alg. 1 / Alg. 2 (Secs. 4-5).
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

__all__ = ["Graph", "expected_counts", "count_host", "set_tuning", "get_tuning", "lib",
           "UbtError", "TRI_REC_DTYPE", "FIXED", "REAL"]

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libubt.so")
FIXED, REAL = 0, 1
UBT_OPT_UNDIRECTED = 1
UBT_OPT_EDGE_INDEX = 2

# ubt_tri_rec: {uint32 u, v, w, cls; double p_bal}
TRI_REC_DTYPE = np.dtype([("u", "<u4"), ("v", "<u4"), ("w", "<u4"), ("cls", "<u4"), ("p_bal", "<f8")])

_lib = None


class UbtError(RuntimeError):
    def __init__(self, status, what=""):
        self.status = int(status)
        msg = lib().ubt_status_str(self.status).decode()
        super().__init__("%s: %s (status %d)" % (what, msg, self.status) if what else msg)


class _GraphOpts(ctypes.Structure):
    _fields_ = [("d_edge_key", ctypes.c_void_p), ("d_vertex_offsets", ctypes.c_void_p),
                ("n_graphs", ctypes.c_int64), ("flags", ctypes.c_int64)]


class _GraphInfo(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("m", ctypes.c_int64), ("max_out_degree", ctypes.c_int64),
                ("hub_vertices", ctypes.c_int64), ("wedges", ctypes.c_int64), ("kind", ctypes.c_int64),
                ("probes", ctypes.c_int64)]


def lib():
    """The loaded libubt.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libubt.so is not built (run __graft_entry__.build() or "
                               "python paper_2602_14084_gb300/_build.py)")
        L = ctypes.CDLL(LIB_PATH)
        P, I32, I64, SZ = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_size_t
        sig = {
            "ubt_status_str": (ctypes.c_char_p, [I32]),
            "ubt_version": (I32, []),
            "ubt_graph_workspace_size": (I32, [I64, I64, I32, P, ctypes.POINTER(SZ)]),
            "ubt_create_graph": (I32, [I64, I64, P, P, P, P, I32, P, P, SZ, P, ctypes.POINTER(P)]),
            "ubt_destroy_graph": (I32, [P]),
            "ubt_graph_get_info": (I32, [P, ctypes.POINTER(_GraphInfo)]),
            "ubt_count_threshold": (I32, [P, P, I32, I32, P, P]),
            "ubt_count_threshold_noalloc": (I32, [P, P, I32, I32, P, P]),
            "ubt_enumerate": (I32, [P, ctypes.c_double, I32, I32, P, I64, ctypes.POINTER(I64), P]),
            "ubt_expected_counts": (I32, [P, P, P, P]),
            "ubt_expected_counts_backward": (I32, [P, P, P, P]),
            "ubt_set_edge_values": (I32, [P, P, P]),
            "ubt_sample_worlds_workspace_size": (I32, [P, I64, ctypes.POINTER(SZ)]),
            "ubt_sample_worlds": (I32, [P, ctypes.c_uint64, I64, P, P, P, SZ, P]),
            "ubt_batch_query": (I32, [P, P, I32, ctypes.c_uint64, P, P, P, P]),
            "ubt_count_host_workspace_size": (I32, [I64, I64, ctypes.POINTER(SZ)]),
            "ubt_count_host": (I32, [I64, I64, P, P, P, P, I32, I32, P, P, SZ, P]),
            "ubt_traversal_stats": (I32, [P, P, I32, I32, P, P]),
            "ubt_query_guard": (I32, [P, ctypes.POINTER(I64), P]),
            "ubt_graph_export": (I32, [P, P, P, P, P, P, P]),
            "ubt_graph_export_pairs": (I32, [P, P, P, P]),
            "ubt_graph_export_undirected": (I32, [P, P, P, P, P, P, P, P]),
            "ubt_count_aeo": (I32, [P, P, I32, P, P]),
            "ubt_topk_workspace_size": (I32, [I64, ctypes.POINTER(SZ)]),
            "ubt_vertex_topk": (I32, [P, P, I64, I32, I32, P, P, P]),
            "ubt_topk": (I32, [P, I64, I32, P, ctypes.POINTER(I64), P, SZ, P]),
            "ubt_enumerate_aeo": (I32, [P, ctypes.c_double, I32, P, I64, ctypes.POINTER(I64), P]),
            "ubt_edge_local_counts": (I32, [P, P, I64, P, I32, P, P, P, P]),
            "ubt_vertex_local_counts": (I32, [P, P, I64, P, I32, P, P, P, P]),
            "ubt_set_tuning": (I32, [ctypes.c_char_p, I64]),
            "ubt_get_tuning": (I32, [ctypes.c_char_p, ctypes.POINTER(I64)]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def _check(st, what):
    if st != 0:
        raise UbtError(st, what)


def _torch():
    import torch
    return torch


def _stream(stream=None):
    torch = _torch()
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _dev_u32(x, device):
    torch = _torch()
    if isinstance(x, torch.Tensor):
        t = x.to(device=device)
        if t.dtype != torch.int32:
            t = t.to(torch.int64).to(torch.int32) if t.dtype != torch.uint32 else t.view(torch.int32)
        return t.contiguous()
    a = np.ascontiguousarray(np.asarray(x, dtype=np.uint32)).view(np.int32)
    return torch.from_numpy(a).to(device)


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else ctypes.c_void_p(0)


def set_tuning(name: str, value: int):
    _check(lib().ubt_set_tuning(name.encode(), int(value)), "ubt_set_tuning(%s)" % name)


def get_tuning(name: str) -> int:
    v = ctypes.c_int64(0)
    _check(lib().ubt_get_tuning(name.encode(), ctypes.byref(v)), "ubt_get_tuning(%s)" % name)
    return int(v.value)


class Graph:
    """An uncertain signed graph built on the GPU (ubt_create_graph).

    n: number of vertices; src, dst: endpoints (uint32, numpy or torch);
    exactly one of k (uint32 in [0, 65536], P+ = k/65536) or p (float32 in
    [0, 1]).  edge_key: optional Philox key per edge; vertex_offsets: int64
    [n_graphs + 1] for a batch of disjoint graphs.  undirected: also build
    the rows in Absolute Edge Order (AEO iteration, samplers, per-vertex
    top-k); edge_index (with undirected): also build the hash index of the
    edges that the vertex queries use for neighbours with long rows.  Device
    memory (the workspace) is a torch tensor owned by this object.
    """

    def __init__(self, n, src, dst, k=None, p=None, edge_key=None, vertex_offsets=None, device="cuda",
                 stream=None, undirected=False, edge_index=False):
        torch = _torch()
        if (k is None) == (p is None):
            raise ValueError("give exactly one of k or p")
        self.device = torch.device(device)
        if self.device.type == "cuda" and self.device.index is None:
            self.device = torch.device("cuda", torch.cuda.current_device())
        self.n = int(n)
        L = lib()
        s_dev = _dev_u32(src, self.device)
        d_dev = _dev_u32(dst, self.device)
        self.m = int(s_dev.numel())
        self.kind = FIXED if k is not None else REAL
        k_dev = _dev_u32(k, self.device) if k is not None else None
        p_dev = None
        if p is not None:
            p_dev = (p.to(self.device, torch.float32) if isinstance(p, torch.Tensor)
                     else torch.from_numpy(np.ascontiguousarray(p, dtype=np.float32)).to(self.device)).contiguous()
        opts = None
        self._keep = []
        self.undirected = bool(undirected)
        self.edge_index = bool(edge_index)
        if edge_key is not None or vertex_offsets is not None or undirected or edge_index:
            opts = _GraphOpts()
            opts.flags = (UBT_OPT_UNDIRECTED if undirected else 0) | (UBT_OPT_EDGE_INDEX if edge_index else 0)
            if edge_key is not None:
                ek = _dev_u32(edge_key, self.device)
                self._keep.append(ek)
                opts.d_edge_key = ek.data_ptr()
            if vertex_offsets is not None:
                vo = (vertex_offsets.to(self.device, torch.int64) if isinstance(vertex_offsets, torch.Tensor)
                      else torch.from_numpy(np.ascontiguousarray(vertex_offsets, dtype=np.int64)).to(self.device))
                self._keep.append(vo)
                opts.d_vertex_offsets = vo.data_ptr()
                opts.n_graphs = int(vo.numel()) - 1
        self.n_graphs = opts.n_graphs if (opts is not None and opts.d_vertex_offsets) else 1
        popts = ctypes.byref(opts) if opts is not None else None
        nbytes = ctypes.c_size_t(0)
        _check(L.ubt_graph_workspace_size(self.n, self.m, self.kind, popts, ctypes.byref(nbytes)),
               "ubt_graph_workspace_size")
        self.workspace = torch.empty(int(nbytes.value), dtype=torch.uint8, device=self.device)
        h = ctypes.c_void_p(0)
        _check(L.ubt_create_graph(self.n, self.m, _ptr(s_dev), _ptr(d_dev), _ptr(k_dev), _ptr(p_dev), self.kind,
                                  popts, _ptr(self.workspace), self.workspace.numel(), _stream(stream),
                                  ctypes.byref(h)), "ubt_create_graph")
        self._h = h
        self._keep = []  # the inputs are no longer needed after the build

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            lib().ubt_destroy_graph(self._h)
            self._h = ctypes.c_void_p(0)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def handle(self):
        return self._h

    def info(self) -> dict:
        i = _GraphInfo()
        _check(lib().ubt_graph_get_info(self._h, ctypes.byref(i)), "ubt_graph_get_info")
        return {f: int(getattr(i, f)) for f, _ in _GraphInfo._fields_}

    def traversal_stats(self, taus=(0.5,), prune=False, stream=None) -> dict:
        """Exact sizes of the traversal a query performs (ubt_traversal_stats)."""
        t = np.ascontiguousarray(np.atleast_1d(np.asarray(taus, dtype=np.float64)))
        out = np.zeros(4, dtype=np.int64)
        _check(lib().ubt_traversal_stats(self._h, t.ctypes.data_as(ctypes.c_void_p), t.size, int(bool(prune)),
                                         out.ctypes.data_as(ctypes.c_void_p), _stream(stream)),
               "ubt_traversal_stats")
        return {"table_entries": int(out[0]), "pairs": int(out[1]), "streamed": int(out[2]), "tasks": int(out[3])}

    def guard(self, stream=None) -> int:
        """Reads and clears the traversal self-check word (0 = all checks passed)."""
        w = ctypes.c_int64(0)
        _check(lib().ubt_query_guard(self._h, ctypes.byref(w), _stream(stream)), "ubt_query_guard")
        return int(w.value)

    def export(self, stream=None) -> dict:
        """The built forward CSR and work lists, copied to host numpy arrays."""
        sizes = np.zeros(4, dtype=np.int64)
        _check(lib().ubt_graph_export(self._h, None, None, None, None, sizes.ctypes.data_as(ctypes.c_void_p),
                                      _stream(stream)), "ubt_graph_export")
        rp = np.zeros(self.n + 1, dtype=np.uint32)
        adj = np.zeros(max(self.m, 1), dtype=np.uint64)
        eid = np.zeros(max(self.m, 1), dtype=np.uint32)
        lists = np.zeros(max(int(sizes.sum()), 1), dtype=np.uint32)
        c = lambda a: a.ctypes.data_as(ctypes.c_void_p)
        _check(lib().ubt_graph_export(self._h, c(rp), c(adj), c(eid), c(lists), None, _stream(stream)),
               "ubt_graph_export")
        pp = np.zeros(self.n + 1, dtype=np.uint32)
        pw = np.zeros(max(self.m, 1), dtype=np.uint64)
        _check(lib().ubt_graph_export_pairs(self._h, c(pp), c(pw), _stream(stream)), "ubt_graph_export_pairs")
        return {"row_ptr": rp, "col": (adj[: self.m] & 0xFFFFFFFF).astype(np.uint32),
                "val": (adj[: self.m] >> 32).astype(np.uint32).view(np.int32), "eid": eid[: self.m],
                "lists": lists[: int(sizes.sum())], "list_sizes": sizes, "pair_ptr": pp,
                "pair_streamed": (pw[: self.m] & 0xFFFFFFFF).astype(np.uint32),
                "pair_pos": (pw[: self.m] >> 32).astype(np.uint32)}

    # ---------------------------------------------------------------- queries

    def count_threshold_(self, taus, out, prune=True, stream=None):
        """ASYNC: writes int64 [2 * n_tau] (balanced counts, then unbalanced) into `out`."""
        t = np.ascontiguousarray(np.atleast_1d(np.asarray(taus, dtype=np.float64)))
        _check(lib().ubt_count_threshold(self._h, t.ctypes.data_as(ctypes.c_void_p), t.size, int(bool(prune)),
                                         _ptr(out), _stream(stream)), "ubt_count_threshold")
        return out

    def count_threshold(self, taus, prune=True, stream=None):
        """(balanced int64[n_tau], unbalanced int64[n_tau]) as numpy arrays."""
        torch = _torch()
        nt = int(np.atleast_1d(taus).size)
        out = torch.empty(2 * nt, dtype=torch.int64, device=self.device)
        self.count_threshold_(taus, out, prune, stream)
        h = out.cpu().numpy()
        return h[:nt].copy(), h[nt:].copy()

    def enumerate(self, tau, which=3, prune=True, capacity=None, stream=None):
        """Records as a numpy structured array (TRI_REC_DTYPE), unordered."""
        torch = _torch()
        L = lib()
        found = ctypes.c_int64(0)
        if capacity is None:
            st = L.ubt_enumerate(self._h, float(tau), int(which), int(bool(prune)), None, 0, ctypes.byref(found),
                                 _stream(stream))
            if st not in (0, -7):
                _check(st, "ubt_enumerate")
            capacity = int(found.value)
        buf = torch.empty(max(capacity, 1) * TRI_REC_DTYPE.itemsize, dtype=torch.uint8, device=self.device)
        st = L.ubt_enumerate(self._h, float(tau), int(which), int(bool(prune)), _ptr(buf), int(capacity),
                             ctypes.byref(found), _stream(stream))
        if st == -7:
            raise UbtError(st, "ubt_enumerate needs capacity %d" % found.value)
        _check(st, "ubt_enumerate")
        n = min(int(found.value), int(capacity))
        return buf[: n * TRI_REC_DTYPE.itemsize].cpu().numpy().view(TRI_REC_DTYPE)

    # ------------------------------------------- Absolute Edge Order / sampling

    def count_aeo_(self, taus, out, stream=None):
        """ASYNC: ubt_count_aeo into `out` (int64 [2 * n_tau])."""
        t = np.ascontiguousarray(np.atleast_1d(np.asarray(taus, dtype=np.float64)))
        _check(lib().ubt_count_aeo(self._h, t.ctypes.data_as(ctypes.c_void_p), t.size, _ptr(out), _stream(stream)),
               "ubt_count_aeo")
        return out

    def count_aeo(self, taus, stream=None):
        """(balanced, unbalanced) int64 counts by the Absolute-Edge-Order iteration (Alg. 2)."""
        torch = _torch()
        nt = int(np.atleast_1d(taus).size)
        out = torch.empty(2 * nt, dtype=torch.int64, device=self.device)
        self.count_aeo_(taus, out, stream)
        h = out.cpu().numpy()
        return h[:nt].copy(), h[nt:].copy()

    def enumerate_aeo(self, tau, which=3, capacity=None, stream=None):
        """Records (TRI_REC_DTYPE) found by the Absolute-Edge-Order iteration."""
        torch = _torch()
        L = lib()
        found = ctypes.c_int64(0)
        if capacity is None:
            st = L.ubt_enumerate_aeo(self._h, float(tau), int(which), None, 0, ctypes.byref(found), _stream(stream))
            if st not in (0, -7):
                _check(st, "ubt_enumerate_aeo")
            capacity = int(found.value)
        buf = torch.empty(max(capacity, 1) * TRI_REC_DTYPE.itemsize, dtype=torch.uint8, device=self.device)
        _check(L.ubt_enumerate_aeo(self._h, float(tau), int(which), _ptr(buf), int(capacity), ctypes.byref(found),
                                   _stream(stream)), "ubt_enumerate_aeo (found %d)" % found.value)
        return buf.cpu().numpy()[: int(found.value) * TRI_REC_DTYPE.itemsize].view(TRI_REC_DTYPE)

    def _local(self, fn, items, taus, stream):
        torch = _torch()
        it = _dev_u32(items, self.device)
        t = np.ascontiguousarray(np.atleast_1d(np.asarray(taus, dtype=np.float64)))
        k = int(it.numel())
        bal = torch.empty(max(k, 1) * t.size, dtype=torch.int64, device=self.device)
        unb = torch.empty(max(k, 1) * t.size, dtype=torch.int64, device=self.device)
        est = torch.empty(2 * t.size, dtype=torch.float64, device=self.device)
        _check(fn(self._h, _ptr(it), k, t.ctypes.data_as(ctypes.c_void_p), t.size, _ptr(bal), _ptr(unb), _ptr(est),
                  _stream(stream)), "local counts")
        nt = t.size
        return (bal.cpu().numpy()[: k * nt].reshape(k, nt), unb.cpu().numpy()[: k * nt].reshape(k, nt),
                est.cpu().numpy().reshape(2, nt))

    def edge_local_counts(self, edges, taus, stream=None):
        """Edge sampling (Algs. 5-6): per sampled edge (input index) the
        t-balanced / t-unbalanced triangles through it, and the estimator
        |E|/3 * mean: (bal (k, n_tau), unbal (k, n_tau), estimate (2, n_tau))."""
        return self._local(lib().ubt_edge_local_counts, edges, taus, stream)

    def vertex_local_counts(self, vertices, taus, stream=None):
        """Vertex sampling (Algs. 3-4): as edge_local_counts, per sampled vertex,
        estimator |V|/3 * mean."""
        return self._local(lib().ubt_vertex_local_counts, vertices, taus, stream)

    def topk(self, K, which=1, stream=None):
        """The K most balanced (which=1) or most unbalanced (which=2) triangles,
        as records (TRI_REC_DTYPE) in decreasing order of that probability."""
        torch = _torch()
        L = lib()
        nb = ctypes.c_size_t(0)
        _check(L.ubt_topk_workspace_size(int(K), ctypes.byref(nb)), "ubt_topk_workspace_size")
        work = torch.empty(int(nb.value), dtype=torch.uint8, device=self.device)
        out = torch.empty(int(K) * TRI_REC_DTYPE.itemsize, dtype=torch.uint8, device=self.device)
        n = ctypes.c_int64(0)
        _check(L.ubt_topk(self._h, int(K), int(which), _ptr(out), ctypes.byref(n), _ptr(work), work.numel(),
                          _stream(stream)), "ubt_topk")
        return out.cpu().numpy()[: int(n.value) * TRI_REC_DTYPE.itemsize].view(TRI_REC_DTYPE)

    def vertex_topk(self, vertices, K, which=1, stream=None):
        """Per vertex, its K most balanced (which=1) or unbalanced (which=2)
        triangles: a list of record arrays (TRI_REC_DTYPE), one per vertex."""
        torch = _torch()
        it = _dev_u32(vertices, self.device)
        k = int(it.numel())
        out = torch.empty(max(k * int(K), 1) * TRI_REC_DTYPE.itemsize, dtype=torch.uint8, device=self.device)
        cnt = torch.zeros(max(k, 1), dtype=torch.int32, device=self.device)
        _check(lib().ubt_vertex_topk(self._h, _ptr(it), k, int(K), int(which), _ptr(out), _ptr(cnt), _stream(stream)),
               "ubt_vertex_topk")
        rec = out.cpu().numpy()[: k * int(K) * TRI_REC_DTYPE.itemsize].view(TRI_REC_DTYPE).reshape(k, int(K))
        c = cnt.cpu().numpy()[:k]
        return [rec[i, : int(c[i])] for i in range(k)]

    def export_undirected(self, stream=None):
        """The undirected adjacency in Absolute Edge Order and the AEO edge owners."""
        n, m = self.n, self.m
        up = np.zeros(n + 1, dtype=np.uint32)
        ua = np.zeros(max(2 * m, 1), dtype=np.uint64)
        ue = np.zeros(max(2 * m, 1), dtype=np.uint32)
        um = np.zeros(max(2 * m, 1), dtype=np.uint32)
        ap = np.zeros(n + 1, dtype=np.uint32)
        aw = np.zeros(max(m, 1), dtype=np.uint64)
        c = lambda a: a.ctypes.data_as(ctypes.c_void_p)
        _check(lib().ubt_graph_export_undirected(self._h, c(up), c(ua), c(ue), c(um), c(ap), c(aw), _stream(stream)),
               "ubt_graph_export_undirected")
        return {"uptr": up, "col": (ua[: 2 * m] & 0xFFFFFFFF).astype(np.uint32),
                "val": (ua[: 2 * m] >> 32).astype(np.uint32).view(np.int32), "eid": ue[: 2 * m], "mirror": um[: 2 * m],
                "apair_ptr": ap, "apair_other": (aw[:m] & 0xFFFFFFFF).astype(np.uint32),
                "apair_pos": (aw[:m] >> 32).astype(np.uint32)}

    def expected_counts_(self, out, exact=None, stream=None):
        _check(lib().ubt_expected_counts(self._h, _ptr(out), _ptr(exact), _stream(stream)), "ubt_expected_counts")

    def expected_counts(self, with_exact=False, stream=None):
        """(E_bal, E_unbal) floats; with_exact also returns (T, 128-bit sum as Python int)."""
        torch = _torch()
        out = torch.empty(2, dtype=torch.float64, device=self.device)
        ex = torch.empty(4, dtype=torch.int64, device=self.device)
        self.expected_counts_(out, ex, stream)
        o = out.cpu().numpy()
        if not with_exact:
            return float(o[0]), float(o[1])
        e = ex.cpu().numpy().view(np.uint64)
        s = (int(e[2]) << 64) | int(e[1])
        if s >= 1 << 127:
            s -= 1 << 128
        return float(o[0]), float(o[1]), int(e[0]), s

    def set_edge_values_(self, p, stream=None):
        """ASYNC: new probabilities of a REAL graph (float32 [m], input edge
        order, on this graph's device) without a rebuild (ubt_set_edge_values).
        An entry outside [0, 1] keeps its old value and is reported by guard()."""
        torch = _torch()
        if not isinstance(p, torch.Tensor) or p.dtype != torch.float32 or p.device != self.device \
                or p.numel() != self.m or not p.is_contiguous():
            raise ValueError("p must be a contiguous float32 tensor of %d entries on %s" % (self.m, self.device))
        _check(lib().ubt_set_edge_values(self._h, _ptr(p), _stream(stream)), "ubt_set_edge_values")

    def expected_counts_backward_(self, gout, grad, stream=None):
        _check(lib().ubt_expected_counts_backward(self._h, _ptr(gout), _ptr(grad), _stream(stream)),
               "ubt_expected_counts_backward")

    def sample_worlds_workspace(self, W):
        nb = ctypes.c_size_t(0)
        _check(lib().ubt_sample_worlds_workspace_size(self._h, int(W), ctypes.byref(nb)),
               "ubt_sample_worlds_workspace_size")
        return int(nb.value)

    def sample_worlds_(self, seed, W, out, total=None, workspace=None, stream=None):
        torch = _torch()
        if workspace is None:
            workspace = torch.empty(self.sample_worlds_workspace(W), dtype=torch.uint8, device=self.device)
        _check(lib().ubt_sample_worlds(self._h, ctypes.c_uint64(int(seed)), int(W), _ptr(out), _ptr(total),
                                       _ptr(workspace), workspace.numel(), _stream(stream)), "ubt_sample_worlds")
        return out

    def sample_worlds(self, seed, W, stream=None):
        """Balanced-triangle count in each of W sign worlds: (int64[W], total)."""
        torch = _torch()
        out = torch.empty(int(W), dtype=torch.int64, device=self.device)
        tot = torch.empty(1, dtype=torch.int64, device=self.device)
        self.sample_worlds_(seed, W, out, tot, stream=stream)
        return out.cpu().numpy(), int(tot.cpu().item())

    def batch_query_(self, taus, seed, counts, expect=None, worlds=None, stream=None):
        t = np.ascontiguousarray(np.atleast_1d(np.asarray(taus, dtype=np.float64)))
        _check(lib().ubt_batch_query(self._h, t.ctypes.data_as(ctypes.c_void_p), t.size,
                                     ctypes.c_uint64(int(seed)), _ptr(counts), _ptr(expect), _ptr(worlds),
                                     _stream(stream)), "ubt_batch_query")

    def batch_query(self, taus, seed=0, expect=True, worlds=True, stream=None):
        """Per graph of a batch: counts [G, 2, n_tau], expected [G, 2], worlds [G, 64]."""
        torch = _torch()
        nt = int(np.atleast_1d(taus).size)
        G = self.n_graphs
        c = torch.empty(G * 2 * nt, dtype=torch.int64, device=self.device)
        e = torch.empty(G * 2, dtype=torch.float64, device=self.device) if expect else None
        w = torch.empty(G * 64, dtype=torch.int64, device=self.device) if worlds else None
        self.batch_query_(taus, seed, c, e, w, stream)
        return (c.cpu().numpy().reshape(G, 2, nt), None if e is None else e.cpu().numpy().reshape(G, 2),
                None if w is None else w.cpu().numpy().reshape(G, 64))


class _ExpectedCountsFn:
    _cls = None

    @classmethod
    def get(cls):
        if cls._cls is None:
            torch = _torch()

            class ExpectedCounts(torch.autograd.Function):
                """(E_bal, E_unbal) of a REAL graph at probabilities p; backward is
                the hand-written adjoint kernel.  Both load p into the graph first
                (ubt_set_edge_values), so they answer for the p they are given."""

                @staticmethod
                def forward(ctx, p, graph):
                    p32 = _p_for(graph, p)
                    graph.set_edge_values_(p32)
                    out = torch.empty(2, dtype=torch.float64, device=graph.device)
                    graph.expected_counts_(out)
                    ctx.graph = graph
                    ctx.p_dtype = p.dtype
                    ctx.save_for_backward(p)
                    return out[0].clone(), out[1].clone()

                @staticmethod
                def backward(ctx, g_bal, g_unbal):
                    graph = ctx.graph
                    (p,) = ctx.saved_tensors
                    # another forward on this graph may have loaded other values since
                    graph.set_edge_values_(_p_for(graph, p))
                    gout = torch.stack([g_bal.to(torch.float64).reshape(()), g_unbal.to(torch.float64).reshape(())])
                    grad = torch.empty(graph.m, dtype=torch.float32, device=graph.device)
                    graph.expected_counts_backward_(gout.contiguous(), grad)
                    return grad.to(ctx.p_dtype), None

            cls._cls = ExpectedCounts
        return cls._cls


def _p_for(graph, p):
    """p as the contiguous float32 device tensor ubt_set_edge_values takes."""
    torch = _torch()
    if graph.kind != REAL:
        raise ValueError("expected_counts(graph, p) needs a REAL graph (built with p=...)")
    if p.numel() != graph.m:
        raise ValueError("p has %d entries, the graph %d edges" % (p.numel(), graph.m))
    return p.detach().to(device=graph.device, dtype=torch.float32).contiguous().reshape(-1)


def expected_counts(graph: Graph, p):
    """Differentiable (E_bal, E_unbal) of the REAL graph `graph` at the edge
    probabilities `p` (one per input edge, in input order): p is loaded into
    the graph (no rebuild) before the forward traversal and again before the
    adjoint, so updating p between calls is enough.  Gradients flow to `p`
    through the adjoint kernel."""
    return _ExpectedCountsFn.get().apply(p, graph)


def count_host(n, src, dst, k, taus, prune=True, stream=None):
    """End to end from host arrays (ubt_count_host): H2D copies, build, count,
    D2H copy.  Returns (balanced, unbalanced) int64 numpy arrays."""
    torch = _torch()
    L = lib()
    s = np.ascontiguousarray(src, dtype=np.uint32)
    d = np.ascontiguousarray(dst, dtype=np.uint32)
    kk = np.ascontiguousarray(k, dtype=np.uint32)
    t = np.ascontiguousarray(np.atleast_1d(np.asarray(taus, dtype=np.float64)))
    nb = ctypes.c_size_t(0)
    _check(L.ubt_count_host_workspace_size(int(n), s.size, ctypes.byref(nb)), "ubt_count_host_workspace_size")
    ws = torch.empty(int(nb.value), dtype=torch.uint8, device="cuda")
    out = np.zeros(2 * t.size, dtype=np.int64)
    _check(L.ubt_count_host(int(n), s.size, s.ctypes.data_as(ctypes.c_void_p), d.ctypes.data_as(ctypes.c_void_p),
                            kk.ctypes.data_as(ctypes.c_void_p), t.ctypes.data_as(ctypes.c_void_p), t.size,
                            int(bool(prune)), out.ctypes.data_as(ctypes.c_void_p), _ptr(ws), ws.numel(),
                            _stream(stream)), "ubt_count_host")
    return out[: t.size], out[t.size:]
