"""The C-ABI library loads and exports every function that include/*.h
declares; host-only entry points behave as documented (no GPU needed)."""
import ctypes as C
import glob
import os
import re

import pytest

import __graft_entry__
from paper_2601_04185_gb300 import imloc

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"\b(imloc_[a-z0-9_]+)\s*\(", src):
            names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def lib():
    __graft_entry__.build()
    return imloc.load()


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert "imloc_lift_async" in names and "imloc_ransac_pnp" in names
    for n in sorted(names):
        assert hasattr(lib, n), n
    assert names <= set(imloc.EXPORTS)


def test_struct_sizes_match_the_header_layout():
    assert C.sizeof(imloc.RansacOpts) == 80
    assert C.sizeof(imloc.Result) == 264
    assert C.sizeof(imloc.View) == 8 + 4 + 4 + 8 + 24 + 96 + 8
    assert C.sizeof(imloc.Corr) == 8 * 9
    assert C.sizeof(imloc.Segment) == 16
    assert C.sizeof(imloc.Rig) == 8 + 8 * 24 + 8 * 96


def test_default_options_are_the_papers_constants(lib):
    o = imloc.default_opts()
    assert o.max_score_corr == 10000   # uniform subsampling to at most 10K (Sec. 3.3)
    assert o.batch == 1024             # batches of 1K minimal sets (Sec. 3.3)
    assert o.max_iters == 100000       # stop after 100K iterations (Sec. 3.3)
    assert o.p_miss == 1e-4            # or P(missing the best model) < 1e-4 (Sec. 3.3)
    assert o.tau_px == 4.0 and o.p3p_fp64_polish == 1
    # precision options off by default: FP32 accumulation and solve, FP32 scoring coordinates
    assert o.lo_fp64_accumulate == 0 and o.lo_fp64_solve == 0 and o.score_bf16 == 0


def test_status_strings(lib):
    for code in (0, 1, -1, -2, -3, -4, -5, -6, -7, -8):
        assert lib.imloc_status_str(code).decode()
    assert lib.imloc_status_str(-7).decode().startswith("degenerate")


def test_null_arguments_are_rejected_without_a_device(lib):
    assert lib.imloc_create(None, 0, 0) == -1
    assert lib.imloc_lift_async(None, None, 0, None, None, None) == -1
    assert lib.imloc_ransac_pnp(None, None, None, None, None, None, None) == -1
    lib.imloc_destroy(None)
    assert lib.imloc_score_config(None, None, None, None) == -1
    assert lib.imloc_set_scoring(None, 0, -1) == -1
    assert lib.imloc_depth_encode_log8_async(None, 4, 4, 4, None, 4, None) == -1
    assert lib.imloc_depth_decode_log8_async(None, 4, 4, 4, None, 4, None) == -1
    assert lib.imloc_triangulate_depth_async(None, None, 4, 4, None, None, 1, None, None, None, 16, None, None,
                                             None, None) == -1
    assert lib.imloc_ransac_rig_batch(None, 1, None, None, None, None, None, None, None, None) == -1
    assert lib.imloc_testing_rig(None, None, None, None, None, None, None, None, None) == -1
    assert lib.imloc_testing_lift_stalled(None, None, 0, None, None, 1, 32, None) == -1
    assert lib.imloc_lift_noalloc_async(None, 0, None, None, None) == -1
    assert lib.imloc_depth_tile4_async(None, 4, 4, 4, None, 16, None) == -1
    assert lib.imloc_depth_halo_async(None, 4, 4, 4, None, 32, None) == -1


def test_blocked_layout_pitches_are_checked_on_the_host(lib):
    """The re-layout calls check their block-row pitch before any device
    work (the pointers are never dereferenced on these paths): 4x4 blocks need
    a multiple of 16 elements >= 16 ceil(W / 4); overlapping 8x4 blocks a
    multiple of 32 >= 32 ((W - 1) // 7 + 1), for W = 10 two blocks (64)."""
    fake = C.c_void_p(0x1000)
    assert lib.imloc_depth_tile4_async(fake, 10, 8, 10, fake, 40, None) == -1
    assert lib.imloc_depth_tile4_async(fake, 10, 8, 10, fake, 36, None) == -1
    assert lib.imloc_depth_tile4_async(fake, 10, 8, 9, fake, 48, None) == -1
    assert lib.imloc_depth_halo_async(fake, 10, 8, 10, fake, 48, None) == -1
    assert lib.imloc_depth_halo_async(fake, 10, 8, 10, fake, 32, None) == -1
    assert lib.imloc_depth_halo_async(fake, 10, 8, 9, fake, 64, None) == -1
    assert lib.imloc_depth_halo_async(fake, 0, 8, 10, fake, 64, None) == -1
    assert lib.imloc_depth_halo_async(fake, 10, 0, 10, fake, 64, None) == -1
    # 1024 columns: (1023 // 7 + 1) = 147 blocks of 32 elements
    assert lib.imloc_depth_halo_async(fake, 1024, 768, 1024, fake, 32 * 146, None) == -1


def test_triangulation_defaults_are_the_papers_constants(lib):
    o = imloc.triangulate_opts()
    assert o.angle_deg == 2.0            # 2-degree angular error threshold (Sec. 3.3)
    assert abs(o.conf_min - 0.05) < 1e-9 # matches with confidence >= 0.05 (Sec. 3.3)
    assert o.keep_more_than == 3         # keep depths with more than 3 inliers (Sec. 3.3)
    assert lib.imloc_retrieve_topk_async(None, None, 1, None, 1, 8, 1, None, None, None) == -1
