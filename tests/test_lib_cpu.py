"""Host-side checks of the C ABI that need no GPU: the library loads, exports
every entry point declared in include/hm.h, builds the tree bit-exactly like the
oracle, and rejects bad arguments before touching a device."""
import ctypes as C
import os
import re

import numpy as np
import pytest

from conftest import ROOT
from oracle.tree import build_tree

hm = pytest.importorskip("paper_1503_07152_gb300")


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "hm.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(hm_[a-z0-9_]+)\s*\(", src)))


def test_exports_every_declared_symbol():
    names = declared_symbols()
    assert len(names) >= 20
    for name in names:
        assert hasattr(hm.lib, name), name
        assert C.cast(getattr(hm.lib, name), C.c_void_p).value


@pytest.mark.parametrize("N,m", [(1, 4), (7, 4), (400, 50), (1000, 64), (2112, 64), (65536, 256),
                                 (262144, 256)])
def test_tree_matches_oracle_bit_exact(N, m):
    t = hm.Tree(N, m)
    o = build_tree(N, m)
    assert t.levels == o.L
    for node in range(1, 2 ** (o.L + 1)):
        assert t.node(node) == (int(o.start[node]), int(o.size[node]))


def test_argument_errors_before_device_use():
    with pytest.raises(hm.HmError) as e:
        hm.Tree(0, 4)
    assert e.value.status == 1
    t = hm.Tree(100, 10)
    with pytest.raises(hm.HmError):
        t.node(0)
    with pytest.raises(hm.HmError):
        t.node(2 ** (t.levels + 1))
    # compress with mismatched operator size fails in argument checking
    op = hm.callback_operator(99, lambda *a: 0)
    with pytest.raises(hm.HmError) as e:
        hm.hm_compress_hodlr(op, t, k=4, p=2, stream=0)
    assert e.value.status == 1
    op = hm.callback_operator(100, lambda *a: 0)
    with pytest.raises(hm.HmError):
        hm.hm_compress_hodlr(op, t, tol=2.0, r=8, stream=0)
    assert hm.hm_version().startswith("hm")
    # the batch autotuner checks its candidates before running anything
    for cands in [(0,), (4, -1), ()]:
        with pytest.raises(hm.HmError) as e:
            hm.hm_tune_batched([op], [t], "hodlr", [dict(k=4, p=2)], candidates=cands, stream=0)
        assert e.value.status == 1


def test_load_rejects_garbage_without_a_device(tmp_path):
    """hm_load validates the header and checksum before any device call."""
    p = tmp_path / "junk.hm"
    p.write_bytes(bytes(range(256)) * 4)
    with pytest.raises(hm.HmError) as e:
        hm.hm_load(str(p), stream=0)
    assert e.value.status == 1
    with pytest.raises(hm.HmError) as e:
        hm.hm_load(str(tmp_path / "missing.hm"), stream=0)
    assert e.value.status == 1


def test_factored_and_operator_arguments_checked_before_device_use():
    """The factored applies and the operator constructors reject bad arguments
    (HM_EINVAL) before any device call, as include/hm.h states."""
    t = hm.Tree(1024, 64)
    for k in (0, 65):
        for fn in (hm.hm_hodlr_factored_apply, hm.hm_hodlr_factored_apply_noalloc):
            with pytest.raises(hm.HmError) as e:
                fn(t, k, None, None, None, None, None, stream=0)
            assert e.value.status == 1
    with pytest.raises(hm.HmError) as e:  # null factors
        hm.hm_hodlr_factored_apply(t, 8, None, None, None, None, None, stream=0)
    assert e.value.status == 1
    for n in (1, 524289):
        with pytest.raises(hm.HmError) as e:
            hm.hm_log_kernel_operator_create(n)
        assert e.value.status == 1
    assert hm.hm_compress_batched([], [], "hodlr", stream=0) == []
