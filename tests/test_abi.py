"""The C ABI library loads, exports every entry point include/fgim.h declares, and rejects
bad arguments on the host before any device work (no GPU needed)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    with open(os.path.join(ROOT, "include", "fgim.h")) as f:
        src = f.read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(fgim_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_2603_21710_gb300 import _lib
    return _lib.load()


def test_exports_every_declared_symbol(lib):
    names = _declared()
    assert "fgim_merge" in names and "fgim_search" in names
    for n in names:
        assert hasattr(lib, n), n


def test_binding_covers_header():
    from paper_2603_21710_gb300 import _lib
    assert set(_declared()) <= set(_lib.EXPORTS)


def test_struct_layouts_match_header():
    from paper_2603_21710_gb300 import _lib
    assert ctypes.sizeof(_lib.Shard) == 40
    assert ctypes.sizeof(_lib.Params) == 64
    assert ctypes.sizeof(_lib.KNNG) == 40
    assert ctypes.sizeof(_lib.Graph) == 40
    assert ctypes.sizeof(_lib.Stats) == 120


def _params(**kw):
    from paper_2603_21710_gb300 import _lib
    p = _lib.Params()
    p.dim, p.dtype, p.metric, p.k, p.R, p.alpha, p.L, p.iters = 32, 0, 0, 16, 32, 1.2, 0, 3
    for a, v in kw.items():
        setattr(p, a, v)
    return p


@pytest.mark.parametrize("kw", [dict(dim=30), dict(k=0), dict(k=200), dict(R=0), dict(alpha=float("nan")),
                                dict(L=500), dict(metric=7), dict(iters=-1), dict(dtype=3), dict(prune_rule=3),
                                dict(tau=-1.0), dict(tau=float("inf"))])
def test_bad_params_rejected_on_host(lib, kw):
    from paper_2603_21710_gb300 import _lib
    sh = (_lib.Shard * 2)()
    buf = ctypes.create_string_buffer(4096 + 16)
    base = (ctypes.addressof(buf) + 15) & ~15
    for i in range(2):
        sh[i] = _lib.Shard(base, base, 4, 4, 0, 0)
    g = _lib.Graph(base, base, base, 8, 32, 0)
    p = _params(**kw)
    st = lib.fgim_merge(sh, 2, ctypes.byref(p), None, ctypes.byref(g), None)
    assert st in (_lib.FGIM_EINVAL, _lib.FGIM_EUNSUPPORTED)
    assert lib.fgim_last_error()


def test_bad_shards_rejected_on_host(lib):
    from paper_2603_21710_gb300 import _lib
    buf = ctypes.create_string_buffer(4096 + 16)
    base = (ctypes.addressof(buf) + 15) & ~15
    g = _lib.Graph(base, base, base, 8, 32, 0)
    p = _params()
    sh = (_lib.Shard * 2)()
    sh[0] = _lib.Shard(base, base, 4, 4, 0, 0)
    sh[1] = _lib.Shard(base, base, 4, 4, 9, 0)       # entry out of range
    assert lib.fgim_merge(sh, 2, ctypes.byref(p), None, ctypes.byref(g), None) == _lib.FGIM_EINVAL
    sh[1] = _lib.Shard(base + 4, base, 4, 4, 0, 0)   # misaligned vectors
    assert lib.fgim_merge(sh, 2, ctypes.byref(p), None, ctypes.byref(g), None) == _lib.FGIM_EINVAL
    assert lib.fgim_merge(sh, 1, ctypes.byref(p), None, ctypes.byref(g), None) == _lib.FGIM_EINVAL  # h < 2
    g2 = _lib.Graph(base, base, base, 9, 32, 0)     # wrong output shape
    sh[1] = _lib.Shard(base, base, 4, 4, 0, 0)
    assert lib.fgim_merge(sh, 2, ctypes.byref(p), None, ctypes.byref(g2), None) == _lib.FGIM_EINVAL


def test_strerror_and_version(lib):
    assert lib.fgim_strerror(0) == b"ok"
    assert lib.fgim_strerror(-1) == b"invalid argument"
    assert b"sm_103a" in lib.fgim_version()


def test_newer_entry_points_reject_bad_arguments_on_host(lib):
    """Batches, HNSW levels / layers and the layered search check their arguments before any
    device work."""
    from paper_2603_21710_gb300 import _lib
    buf = ctypes.create_string_buffer(4096 + 16)
    base = (ctypes.addressof(buf) + 15) & ~15
    p = _params()
    # a batch with a negative count, and one whose descriptors are missing
    assert lib.fgim_merge_batch(None, None, -1, ctypes.byref(p), None, None) == _lib.FGIM_EINVAL
    assert lib.fgim_merge_batch(None, None, 2, ctypes.byref(p), None, None) == _lib.FGIM_EINVAL
    counts = (ctypes.c_int64 * (_lib.MAX_LEVELS + 1))()
    assert lib.fgim_hnsw_levels(100, 1, 0, base, counts, None) == _lib.FGIM_EINVAL      # M < 2
    assert lib.fgim_hnsw_levels(0, 8, 0, base, counts, None) == _lib.FGIM_EINVAL        # n < 1
    # layer 0 is the base graph, not an upper layer; M and ef out of range
    args = (base, 64, 16, 0, 0, base, 0, 8, 16, base, base, base, 4, None)
    assert lib.fgim_hnsw_layer(*args) == _lib.FGIM_EINVAL
    assert lib.fgim_hnsw_layer(base, 64, 16, 0, 0, base, 1, 65, 16, base, base, base, 4, None) == _lib.FGIM_EINVAL
    assert lib.fgim_hnsw_layer(base, 64, 16, 0, 0, base, 1, 8, 200, base, base, base, 4, None) == _lib.FGIM_EINVAL
    # the layered search: ef_up out of range, too many layers
    L = (_lib.Layer * 1)()
    L[0] = _lib.Layer(base, base, 4, 8, 0)
    assert lib.fgim_search_hnsw(base, 64, 16, 0, 0, base, 8, L, 1, 0, base, 4, 10, 64, 0, base, base, None,
                                None) == _lib.FGIM_EINVAL
    assert lib.fgim_search_hnsw(base, 64, 16, 0, 0, base, 8, L, 17, 0, base, 4, 10, 64, 8, base, base, None,
                                None) == _lib.FGIM_EINVAL
    assert ctypes.sizeof(_lib.Layer) == 32
    # the input-PG builder: M and ef out of range
    ent = ctypes.c_int32(0)
    assert lib.fgim_build_pg(base, 64, 16, 0, 0, 0, 16, base, base, ctypes.byref(ent), None) == _lib.FGIM_EINVAL
    assert lib.fgim_build_pg(base, 64, 16, 0, 0, 8, 129, base, base, ctypes.byref(ent), None) == _lib.FGIM_EINVAL
    assert lib.fgim_build_pg(base, 64, 16, 0, 0, 8, 16, base, base, None, None) == _lib.FGIM_EINVAL


def test_test_hooks_named_and_unknown(lib):
    """The test hooks exist by name, unknown names are refused; none touches the device."""
    for knob, off in (("prop_cap", 0), ("hop_budget", 0), ("fail_alloc_after", -1), ("join_sparse_nn", -1)):
        assert lib.fgim_test_set(knob.encode(), off) == 1
    assert lib.fgim_test_set(b"no_such_knob", 1) == 0
    assert lib.fgim_test_get(b"no_such_counter") == -1


def test_noalloc_search_refuses_bf16_storage_on_host(lib):
    """fgim_search_noalloc takes FP32 vectors only (a decoded BF16 copy would be an allocation):
    BF16 storage is refused with FGIM_EUNSUPPORTED before any device work."""
    buf = ctypes.create_string_buffer(4096 + 16)
    p = ctypes.c_void_p((ctypes.addressof(buf) + 15) & ~15)
    st = lib.fgim_search_noalloc(p, 16, 32, 1, 0, p, 8, 0, p, 4, 10, 64, p, p, None)
    assert st == -5


def test_graph_alloc_rejects_bad_shapes_on_host(lib):
    from paper_2603_21710_gb300 import _lib
    g = _lib.Graph()
    assert lib.fgim_graph_alloc(0, 32, ctypes.byref(g)) == -1
    assert lib.fgim_graph_alloc(10, 0, ctypes.byref(g)) == -1
    assert lib.fgim_graph_alloc(10, 32, None) == -1
    assert not g.ids and g.n == 0
    lib.fgim_graph_free(ctypes.byref(g))   # a zeroed graph is a no-op


def test_autotune_cache_parsing_on_host(lib, tmp_path):
    """fgim_autotune_load reads the cache's JSON lines without a device; unreadable input is refused."""
    assert lib.fgim_autotune_load(str(tmp_path / "missing.jsonl").encode()) == -1
    bad = tmp_path / "bad.jsonl"
    bad.write_text("not json\n")
    assert lib.fgim_autotune_load(str(bad).encode()) == -1
    good = tmp_path / "good.jsonl"
    good.write_text('{"key": 12345, "wpb": 2, "ht_bits": 9, "ms": 1.0}\n{"key": 12345, "wpb": 8, "ht_bits": 9}\n')
    assert lib.fgim_autotune_load(str(good).encode()) == 0   # the second line (wpb 8) is refused
    lib.fgim_autotune_clear()
