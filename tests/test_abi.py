"""CPU-side checks of the C ABI library: it builds for sm_103a, loads, exports every
symbol the header declares, rejects bad arguments before touching the GPU, and its
launch planner (host-only) makes sane choices."""
import ctypes
import os
import re

import pytest

from paper_1504_03687_gb300 import _build, api

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    src = open(os.path.join(ROOT, "include", "nbgpu.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?[a-z_0-9]+\s*\*?\s*(nb_[a-z_]+)\s*\(", src, flags=re.M)))


def test_library_exports_every_declared_symbol():
    lib = api.load_library()
    names = _declared_functions()
    assert len(names) >= 12
    for name in names:
        assert hasattr(lib, name), name
    assert set(names) == set(api.EXPORTS)
    assert lib.nb_version() == 100


def test_library_is_built_for_sm_103a_only():
    assert "arch=compute_103a,code=sm_103a" in " ".join(_build.ARCH)
    assert os.path.exists(_build.LIB)


def test_null_arguments_are_rejected_without_gpu():
    lib = api.load_library()
    assert lib.nb_init(None, None) == api.NB_ERR_ARG
    h = ctypes.c_void_p()
    assert lib.nb_init(ctypes.byref(h), None) == api.NB_ERR_ARG
    bad = api._Config(n_max=0, precision=1, nb_cap=512, device=0, flags=0, stream=None)
    assert lib.nb_init(ctypes.byref(h), ctypes.byref(bad)) == api.NB_ERR_ARG
    bad = api._Config(n_max=10, precision=7, nb_cap=512, device=0, flags=0, stream=None)
    assert lib.nb_init(ctypes.byref(h), ctypes.byref(bad)) == api.NB_ERR_ARG
    bad = api._Config(n_max=10, precision=1, nb_cap=0, device=0, flags=0, stream=None)
    assert lib.nb_init(ctypes.byref(h), ctypes.byref(bad)) == api.NB_ERR_ARG
    assert lib.nb_free(None) == api.NB_OK
    assert lib.nb_sync(None) == api.NB_ERR_ARG
    assert lib.nb_set_source_range(None, 0, 256) == api.NB_ERR_ARG
    assert lib.nb_last_error(None) == b"null context"


OCC = [3, 4, 4, 1, 3, 4, 3, 2, 8, 12, 3, 4, 2, 8, 12, 3, 4, 2, 3, 2, 3]  # resident CTAs/SM: 20 mixed tiled variants, FP64 tiled


@pytest.mark.parametrize("n_i", [1, 2, 3, 8, 16, 17, 32, 33, 100, 1024, 16384, 131072, 1 << 20])
def test_planner_mixed(n_i):
    n = 1 << 20
    p = api.plan_for("mixed", 152, OCC, n, n_i)
    if n_i <= 32:
        assert p["kernel"] == 2 and p["tile"] == 0
        assert p["ctas"] >= 152  # small blocks still spread over every SM
        # one row a CTA up to 2 rows, two-row packed pairs up to 16, four-row above
        assert (p["variant"], p["i_per_cta"]) == ((0, 1) if n_i <= 2 else (3, 2) if n_i <= 16 else (1, 4))
    else:
        assert p["kernel"] == 1 and p["tile"] in (128, 256)
        tiles = ((n + 255) // 256 * 256) // p["tile"]
        assert 1 <= p["splits"] <= tiles // 2
        assert p["ctas"] == -(-n_i // p["i_per_cta"]) * p["splits"]
        # at least one full wave of work whenever the block is large enough
        if n_i >= 16384:
            assert p["ctas"] >= 152


def test_planner_fp64_and_tiny_n():
    p = api.plan_for("fp64", 152, OCC, 1024, 1024)
    assert p["kernel"] == 0 and p["i_per_cta"] == 128 and p["tile"] == 64
    assert p["splits"] <= 1024 // 64 // 2
    p = api.plan_for("fp64", 152, OCC, 5, 3)
    assert p["kernel"] == 3 and p["splits"] == 1
    p = api.plan_for("mixed", 152, OCC, 1, 1)
    assert p["kernel"] == 2 and p["splits"] == 1


def test_planner_fills_waves_for_full_block():
    # 2^20 active particles: the CTA count should be close to a whole number of waves
    p = api.plan_for("mixed", 152, OCC, 1 << 20, 1 << 20)
    occ = OCC[p["variant"]]
    waves = p["ctas"] / (152 * occ)
    assert waves - int(waves) == 0 or waves - int(waves) > 0.9 or waves > 20
