"""Failure detection on the GPU without a fault: a bounded device-side wait
that runs out.

The lift's stable compaction waits, per tile, for its predecessors to publish
their counts (decoupled look-back).  The test hook imloc_testing_lift_stalled
never runs the first tile, so its successors can only leave the wait by the
iteration limit, which the hook sets to a few dozen probes.  The kernel must
end, the context's error word must read IMLOC_ERR_TIMEOUT, and the context
must stay usable: a regular lift on it afterwards matches the oracle.
"""
import numpy as np
import pytest

import oracle
from paper_2601_04185_gb300 import imloc, synth

from gpu_helpers import lifted_to_host, matches_to_device, torch, views_to_device

pytestmark = pytest.mark.gpu

IMLOC_ERR_TIMEOUT = -4


def test_lookback_wait_gives_up_and_reports_a_timeout():
    t = torch()
    t.cuda.set_device(0)
    ctx = imloc.Context(0, 256 << 20)
    q = synth.localization_query(np.random.default_rng(61), n_views=3, matches_per_pair=3001, width=320, height=240,
                                 f=260.0)
    views, m = views_to_device(q["views"]), matches_to_device(q["matches"])
    n = int(q["matches"]["seg_off"][-1])
    assert n > 4 * 1024  # several tiles behind the one that is never run
    assert ctx.device_error() == 0
    out = imloc.alloc_corr(n)
    rc = ctx.testing_lift_stalled(views, m, out, skip_tiles=1, spin_limit=32)
    assert rc == 0, imloc.load().imloc_status_str(rc)
    t.cuda.synchronize()  # the kernel ends by its own limit
    assert ctx.device_error() == IMLOC_ERR_TIMEOUT
    # the written count rests on the missing tile: at most the number of matches
    assert 0 <= int(out["count"].item()) <= n
    # the context still works: a regular lift on it equals the oracle's
    good = ctx.lift(views, m)
    t.cuda.synchronize()
    g = lifted_to_host(good)
    ref = oracle.lift(q["views"], q["matches"])
    assert g["n"] == len(ref["src"]) > 0
    np.testing.assert_array_equal(g["src"].astype(np.int64), ref["src"])
    ctx.close()


def test_stalled_hook_rejects_bad_arguments():
    t = torch()
    ctx = imloc.Context(0, 64 << 20)
    q = synth.localization_query(np.random.default_rng(62), n_views=1, matches_per_pair=500, width=320, height=240,
                                 f=260.0)
    views, m = views_to_device(q["views"]), matches_to_device(q["matches"])
    out = imloc.alloc_corr(500)
    # one tile only: nothing would be left to run
    assert ctx.testing_lift_stalled(views, m, out, skip_tiles=1, spin_limit=32) == -1
    assert ctx.testing_lift_stalled(views, m, out, skip_tiles=0, spin_limit=32) == -1
    assert ctx.testing_lift_stalled(views, m, out, skip_tiles=1, spin_limit=0) == -1
    t.cuda.synchronize()
    assert ctx.device_error() == 0
    ctx.close()
