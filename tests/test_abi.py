"""The C-ABI library builds, loads and exports every symbol include/*.h declares (no GPU needed)."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"\b(tw_[A-Za-z0-9_]+)\s*\(", text):
            names.add(m.group(1))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    from paper_2504_16344_gb300 import build, tw
    try:
        build.build()
    except RuntimeError as e:  # no toolkit on this machine
        pytest.skip(str(e))
    return ctypes.CDLL(tw.lib_path())


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("tw_create", "tw_set_block_column", "tw_p2o_apply", "tw_p2o_adjoint",
                     "tw_set_prior", "tw_destroy", "tw_last_error"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_signatures_cover_the_header():
    from paper_2504_16344_gb300 import tw
    assert set(declared_functions()) == set(tw.SIGNATURES)


def test_create_rejects_bad_sizes_without_touching_a_gpu(lib):
    from paper_2504_16344_gb300 import tw
    l = tw.load()
    h = ctypes.c_void_p()
    # argument validation happens before any CUDA call
    assert l.tw_create(ctypes.byref(h), 0, 1, 4, 4, 4, 1.0, 1.0, 1, 0) == tw.ERR_ARG
    assert l.tw_create(ctypes.byref(h), 4, 1, 4, 4, 4, 1.0, 1.0, 0, 0) == tw.ERR_ARG
    assert l.tw_create(ctypes.byref(h), 4, 1, 4, 4, 4, -1.0, 1.0, 1, 0) == tw.ERR_ARG


def test_autotune_selection_rule(lib):
    """The tile tuner keeps the smallest positive time; failed or missing
    measurements (<= 0, NaN) never win; ties keep the earlier candidate."""
    from paper_2504_16344_gb300 import tw
    assert tw.autotune_pick([3.0, 1.5, 2.0]) == 1
    assert tw.autotune_pick([-1.0, 4.0, 0.0, 5.0]) == 1
    assert tw.autotune_pick([2.0, 2.0, 3.0]) == 0
    assert tw.autotune_pick([float("nan"), 7.0]) == 1
    assert tw.autotune_pick([-1.0, 0.0]) == -1
    assert tw.autotune_pick([]) == -1
    tw.autotune_clear_cache()


def test_tile_struct_matches_header():
    """The binding's tw_tiles layout is the header's: three ints, three doubles, one int."""
    from paper_2504_16344_gb300 import tw
    names = [f for f, _ in tw.Tiles._fields_]
    text = open(os.path.join(ROOT, "include", "tw.h")).read()
    body = text[text.index("typedef struct {\n  int adj_tile"):text.index("} tw_tiles;")]
    order = re.findall(r"\b(adj_tile|adj_rw|fwd_lanes|adj_tile_ms|adj_rw_ms|fwd_lanes_ms|tuned)\b", body)
    assert names == order
