"""The C-ABI library builds, loads and exports every symbol include/ubt.h
declares; host-side argument checks that need no GPU."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "ubt.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(ubt_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def L():
    from paper_2602_14084_gb300 import _build
    _build.build()
    import paper_2602_14084_gb300 as ubt
    return ubt.lib()


def test_header_declares_the_entry_points():
    names = declared_functions()
    for must in ["ubt_create_graph", "ubt_count_threshold", "ubt_enumerate", "ubt_expected_counts",
                 "ubt_expected_counts_backward", "ubt_sample_worlds", "ubt_batch_query", "ubt_count_host"]:
        assert must in names


def test_every_declared_symbol_is_exported(L):
    for name in declared_functions():
        assert hasattr(L, name), name
        assert ctypes.cast(getattr(L, name), ctypes.c_void_p).value


def test_status_strings_and_version(L):
    for code in range(0, -12, -1):
        s = L.ubt_status_str(code).decode()
        assert s and s != "unknown status"
    assert L.ubt_status_str(-99).decode() == "unknown status"
    assert L.ubt_version() >= 10000


def test_tuning_knobs(L):
    import paper_2602_14084_gb300 as ubt
    old = ubt.get_tuning("hub_threshold")
    ubt.set_tuning("hub_threshold", 96)
    assert ubt.get_tuning("hub_threshold") == 96
    ubt.set_tuning("hub_threshold", old)
    with pytest.raises(ubt.UbtError):
        ubt.set_tuning("no_such_knob", 1)
    with pytest.raises(ubt.UbtError):
        ubt.set_tuning("smem_table_max", 1000)  # not a power of two
    with pytest.raises(ubt.UbtError):
        ubt.set_tuning("world_words_per_pass", 3)


def test_workspace_size_argument_checks(L):
    sz = ctypes.c_size_t(0)
    assert L.ubt_graph_workspace_size(10, 20, 0, None, ctypes.byref(sz)) == 0
    assert sz.value > 0
    small = sz.value
    assert L.ubt_graph_workspace_size(1000, 200000, 0, None, ctypes.byref(sz)) == 0
    assert sz.value > small
    assert L.ubt_graph_workspace_size(-1, 20, 0, None, ctypes.byref(sz)) == -1
    assert L.ubt_graph_workspace_size(10, 1 << 33, 0, None, ctypes.byref(sz)) == -1
    assert L.ubt_graph_workspace_size(10, 20, 7, None, ctypes.byref(sz)) == -1
    # create_graph rejects bad arguments before touching the device
    h = ctypes.c_void_p(0)
    assert L.ubt_create_graph(10, 5, None, None, None, None, 0, None, None, 0, None, ctypes.byref(h)) == -1
    assert L.ubt_create_graph(10, 5, 256, 256, 256, 256, 0, None, 256, 1 << 20, None, ctypes.byref(h)) == -1
    assert L.ubt_count_threshold(None, None, 1, 0, None, None) == -1
    assert L.ubt_destroy_graph(None) == -1


def test_traversal_and_index_knobs(L):
    import paper_2602_14084_gb300 as ubt
    knobs = {"long_min": (1, 1 << 20, [0, (1 << 20) + 1]), "long_tail": (0, 1, [-1, 2]),
             "edge_index": (0, 2, [-1, 3]), "vertex_split": (1, 1 << 32, [0, (1 << 32) + 1]),
             "warp_sort_max": (128, 512, [64, 384, 1024])}
    for name, (lo, hi, bad) in knobs.items():
        old = ubt.get_tuning(name)
        try:
            for v in (lo, hi):
                ubt.set_tuning(name, v)
                assert ubt.get_tuning(name) == v, name
            for v in bad:
                with pytest.raises(ubt.UbtError):
                    ubt.set_tuning(name, v)
                assert ubt.get_tuning(name) == hi, name  # a rejected value leaves the knob as it was
        finally:
            ubt.set_tuning(name, old)


def test_workspace_grows_with_the_options(L):
    """The undirected rows add the AEO adjacency; the edge index adds 16
    bytes per slot for the power of two >= 4m slots."""
    import paper_2602_14084_gb300 as ubt
    n, m = 100000, 1000000

    def size(flags):
        opts = ubt._GraphOpts()
        opts.flags = flags
        sz = ctypes.c_size_t(0)
        assert L.ubt_graph_workspace_size(n, m, 0, ctypes.byref(opts), ctypes.byref(sz)) == 0
        return sz.value

    plain, und, idx = size(0), size(ubt.UBT_OPT_UNDIRECTED), size(ubt.UBT_OPT_UNDIRECTED | ubt.UBT_OPT_EDGE_INDEX)
    slots = 1 << (4 * m - 1).bit_length()
    assert und > plain + 2 * m * (8 + 4 + 4 + 4)   # uadj, ueid, umir, uepos at least
    assert idx - und >= 16 * slots and idx - und < 16 * slots + 4096
    # the index without the undirected rows is refused when the graph is created
    opts = ubt._GraphOpts()
    opts.flags = ubt.UBT_OPT_EDGE_INDEX
    h = ctypes.c_void_p(0)
    assert L.ubt_create_graph(10, 0, None, None, None, None, 0, ctypes.byref(opts), 256, 1 << 20, None,
                              ctypes.byref(h)) == -1
