"""CPU-only checks of the C ABI library: it loads, exports every declared
symbol, and its host-side format builder (no GPU involved) agrees with the
oracle's CCSS enumeration and rejects malformed input."""
import os
import re

import numpy as np
import pytest

import s3synth
from oracle import ccss

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def s3():
    from paper_2311_08595_gb300 import build
    build.build()
    import paper_2311_08595_gb300 as mod
    return mod


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "s3ttvc.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(s3_[a-z0-9_]+)\s*\(", src)))


def test_every_declared_symbol_is_exported(s3):
    import ctypes
    lib = ctypes.CDLL(s3.lib_path())
    names = declared_symbols()
    assert len(names) >= 12
    for name in names:
        assert hasattr(lib, name), name
    from paper_2311_08595_gb300 import _lib
    assert set(names) <= set(_lib.SIGNATURES), set(names) - set(_lib.SIGNATURES)


def test_version_and_status_strings(s3):
    assert s3.s3_version() == 1
    from paper_2311_08595_gb300 import _lib
    assert _lib.status_name(0) == "S3_OK" and _lib.status_name(4) == "S3_ENOCONV"
    # every status of the header has its name, in the header's order
    names = ["S3_OK", "S3_EINVAL", "S3_ENOMEM", "S3_ECUDA", "S3_ENOCONV", "S3_ETIMEOUT", "S3_ERANGE", "S3_ENOTSUP"]
    assert [_lib.status_name(i) for i in range(8)] == names
    assert [getattr(_lib, k) for k in names] == list(range(8))


def test_inspect_fig1_matches_fig2_counts(s3):
    hg = s3synth.fig1_example()
    info = s3.s3_format_inspect(hg.n, hg.edge_ptr, hg.members, build_ccss=1, order=1)
    assert info["rank"] == 4 and info["nnz"] == 21 and info["m"] == 6
    assert info["edges_per_size"][2:5] == [1, 1, 4]
    assert info["ccss_nodes_per_level"][1:4] == [6, 10, 16]
    assert info["ccss_special_leaves"] == 21
    assert info["ccss_nodes"] == 32 and info["ccss_products"] == 26


@pytest.mark.parametrize("seed", range(6))
def test_inspect_ccss_matches_oracle_enumeration(s3, seed):
    hg = s3synth.tiny_case(seed=seed, n=9, m=25, rank=5)
    info = s3.s3_format_inspect(hg.n, hg.edge_ptr, hg.members, build_ccss=1, order=1)
    want = ccss.level_counts(ccss.trimmed_levels(hg.edges()))
    assert info["ccss_nodes_per_level"][1:1 + len(want)] == want
    assert info["ccss_nodes_per_level"][1 + len(want)] == 0
    assert info["ccss_special_leaves"] == hg.nnz


def test_inspect_sunflower_sharing(s3):
    hg = s3synth.sunflower(petals=50, k=8, core=5, n=400)
    info = s3.s3_format_inspect(hg.n, hg.edge_ptr, hg.members, build_ccss=1, order=1)
    want = ccss.level_counts(ccss.trimmed_levels(hg.edges()))
    assert info["ccss_nodes_per_level"][1:1 + len(want)] == want
    # shared prefixes make the forest smaller than one path set per edge ((k^2+k-2)/2 nodes each)
    assert info["ccss_nodes"] < 50 * (8 * 8 + 8 - 2) // 2


@pytest.mark.parametrize("seed", range(4))
def test_inspect_ccss_degree_order(s3, seed):
    # the default order sorts the nodes of every edge by decreasing degree (ties by id):
    # the forest equals the index-order forest of the relabelled hypergraph
    hg = s3synth.tiny_case(seed=seed, n=10, m=30, rank=5)
    deg = hg.degrees()
    order = sorted(range(hg.n), key=lambda v: (-deg[v], v))
    key = {v: r for r, v in enumerate(order)}
    relabelled = [tuple(key[v] for v in e) for e in hg.edges()]
    info = s3.s3_format_inspect(hg.n, hg.edge_ptr, hg.members, build_ccss=1)
    want = ccss.level_counts(ccss.trimmed_levels(relabelled))
    assert info["ccss_nodes_per_level"][1:1 + len(want)] == want


def test_inspect_buckets_and_degrees(s3):
    hg = s3synth.config_small(seed=1)
    info = s3.s3_format_inspect(hg.n, hg.edge_ptr, hg.members)
    sizes = np.bincount(hg.sizes(), minlength=6)
    assert info["edges_per_size"][:6] == list(sizes)
    assert info["max_degree"] == hg.degrees().max()
    assert info["ccss_levels"] == 0


@pytest.mark.parametrize("case", ["empty_edge", "bad_id", "repeat", "rank_small", "ptr_decreasing", "too_big"])
def test_inspect_rejects_malformed(s3, case):
    ep = np.array([0, 2, 4], dtype=np.int64)
    mem = np.array([0, 1, 1, 2], dtype=np.int32)
    n, kw = 3, {}
    if case == "empty_edge":
        ep = np.array([0, 2, 2], dtype=np.int64)
        mem = mem[:2]
    elif case == "bad_id":
        mem = np.array([0, 1, 1, 3], dtype=np.int32)
    elif case == "repeat":
        mem = np.array([0, 0, 1, 2], dtype=np.int32)
    elif case == "rank_small":
        kw = {"rank": 1}
    elif case == "ptr_decreasing":
        ep = np.array([0, 3, 2], dtype=np.int64)
    elif case == "too_big":
        n = 200
        ep = np.array([0, 129], dtype=np.int64)
        mem = np.arange(129, dtype=np.int32)
    with pytest.raises(s3.S3Error) as ei:
        s3.s3_format_inspect(n, ep, mem, **kw)
    assert ei.value.status == 1


def test_explicit_rank_and_size_one_edges(s3):
    hg = s3synth.from_edges(5, [(0,), (1, 2), (0, 3, 4)])
    info = s3.s3_format_inspect(hg.n, hg.edge_ptr, hg.members, rank=7, build_ccss=1)
    assert info["rank"] == 7 and info["max_edge"] == 3
    assert info["edges_per_size"][1:4] == [1, 1, 1]
    assert info["ccss_special_leaves"] == hg.nnz


def test_device_entry_points_fail_loudly_without_gpu(s3):
    import torch
    if torch.cuda.is_available():
        pytest.skip("GPU present")
    hg = s3synth.fig1_example()
    with pytest.raises(s3.S3Error) as ei:
        s3.s3_build_format(hg.n, hg.edge_ptr, hg.members)
    assert ei.value.status == 3  # S3_ECUDA


def test_product_does_not_import_oracle():
    pkg = os.path.join(ROOT, "paper_2311_08595_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cpp", ".h", ".cuh")):
                txt = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in txt and "from oracle" not in txt, f
                assert "aay_oracle" not in txt and "liboracle" not in txt, f
    for f in os.listdir(os.path.join(ROOT, "oracle")):
        if f.endswith((".py", ".c")):
            txt = open(os.path.join(ROOT, "oracle", f)).read()
            assert "paper_2311_08595_gb300" not in txt and "s3ttvc.h" not in txt, f
