"""Retrieval nearest-neighbour search (ImLoc Sec. 3.1, Sec. 4.4 "Runtime")
through the C ABI against the FP64 oracle.

The tensor cores accumulate the bf16 products (exact in FP32) in FP32 in an
unspecified order, so scores differ from the FP64 oracle by at most
delta = D * 2^-23 * sum_d |q_d db_d| (<= D * 2^-23 for unit descriptors).
Bar: every returned score within delta of the oracle's score of the same
database row; the list sorted (descending, ties by index); the returned set
equal to the oracle's up to rows whose oracle scores lie within 2 delta of
the k-th best (near-ties whose order FP32 cannot decide).
"""
import numpy as np
import pytest

import oracle
from paper_2601_04185_gb300 import imloc, synth

from gpu_helpers import torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    c = imloc.Context(0, 1 << 30)
    yield c
    c.close()


def as_float(bits):
    return (bits.astype(np.uint32) << 16).view(np.float32).astype(np.float64)


def check(gs, gi, q, db, k):
    t = torch()
    Q, D = q.shape
    N = db.shape[0]
    qf, dbf = as_float(q), as_float(db)
    delta = D * 2.0 ** -23 * (np.abs(qf) @ np.abs(dbf).T).max(axis=1)
    osc, oix = oracle.retrieve_topk(q, db, k)
    kk = min(k, N)
    for i in range(Q):
        idx = gi[i, :kk].astype(np.int64)
        assert (idx >= 0).all() and (idx < N).all()
        assert len(set(idx.tolist())) == kk
        exact = dbf[idx] @ qf[i]
        assert np.all(np.abs(gs[i, :kk] - exact) <= delta[i]), i
        # sorted by the returned scores, ties by index
        assert all((gs[i, j] > gs[i, j + 1]) or (gs[i, j] == gs[i, j + 1] and idx[j] < idx[j + 1])
                   for j in range(kk - 1)), i
        kth = osc[i, kk - 1]
        sure = set(oix[i, :kk][osc[i, :kk] > kth + 2 * delta[i]].tolist())
        assert sure <= set(idx.tolist()), i
        assert np.all(exact >= kth - 2 * delta[i]), i
        if k > N:
            assert (gi[i, N:] == -1).all() and np.isneginf(gs[i, N:]).all()


def run(ctx, q, db, k):
    t = torch()
    qd = t.from_numpy(q.view(np.int16)).cuda()
    dd = t.from_numpy(db.view(np.int16)).cuda()
    s, i = ctx.retrieve_topk(qd, dd, k)
    t.cuda.synchronize()
    assert ctx.device_error() == 0
    return s.cpu().numpy().astype(np.float64), i.cpu().numpy()


@pytest.mark.parametrize("seed,Q,N,D,k", [(0, 33, 5000, 768, 50), (1, 1, 1000, 64, 10), (2, 300, 3000, 256, 10),
                                           (3, 17, 20, 128, 50), (4, 256, 1029, 4096, 128),
                                           # one or two queries: the matrix-vector kernel, rows of D / 8
                                           # 16-byte words not a multiple of the warp, k > N
                                           (5, 2, 777, 296, 7), (6, 1, 3, 8, 5), (7, 2, 20, 200, 50),
                                           (8, 1, 4099, 2056, 128)])
def test_against_the_oracle(ctx, seed, Q, N, D, k):
    db, q, _ = synth.retrieval_set(np.random.default_rng(seed), N, Q, D)
    gs, gi = run(ctx, q, db, k)
    check(gs, gi, q, db, k)


def test_megaloc_sized_single_query(ctx):
    """one query against 70,001 descriptors of 8,448 dims (several selection chunks and a merge level)"""
    db, q, _ = synth.retrieval_set(np.random.default_rng(7), 70001, 1, 8448)
    gs, gi = run(ctx, q, db, 100)
    check(gs, gi, q, db, 100)


def test_exact_ties_go_to_the_lower_index(ctx):
    db, q, _ = synth.retrieval_set(np.random.default_rng(8), 600, 5, 192)
    db[100] = db[400] = db[599] = q[3]
    db[250] = q[1]
    gs, gi = run(ctx, q, db, 5)
    assert list(gi[3, :3]) == [100, 400, 599]
    assert gs[3, 0] == gs[3, 1] == gs[3, 2]
    assert gi[1, 0] == 250


def test_thousands_of_equal_scores(ctx):
    """more equal top scores than the histogram's candidate buffer holds (within a
    first-level chunk, and at the merge level): the exact radix path, still lowest
    indices first"""
    db, q, _ = synth.retrieval_set(np.random.default_rng(9), 20000, 256, 128)
    db[3000:9000] = q[0]
    gs, gi = run(ctx, q[:2], db, 64)  # two queries: chunks of 1,024, 1,280 keys merged by one block
    assert list(gi[0]) == list(range(3000, 3064))
    assert (gs[0] == gs[0, 0]).all()
    check(gs[1:], gi[1:], q[1:2], db, 64)
    same = np.repeat(db[:1], 20000, axis=0)  # every row equal: one bin, all tied
    gs, gi = run(ctx, q, same, 64)  # 256 queries: chunks of 4,096
    assert (gi == np.arange(64)[None, :]).all()
    assert (gs == gs[:, :1]).all()


def test_invalid_arguments_are_rejected(ctx):
    t = torch()
    q = t.zeros((2, 64), dtype=t.int16, device="cuda")
    db = t.zeros((10, 64), dtype=t.int16, device="cuda")
    for bad in (dict(k=0), dict(k=129)):
        with pytest.raises(imloc.ImlocError):
            ctx.retrieve_topk(q, db, bad["k"])
    with pytest.raises(imloc.ImlocError):  # dim not a multiple of 8
        ctx.retrieve_topk(t.zeros((2, 60), dtype=t.int16, device="cuda"), t.zeros((10, 60), dtype=t.int16, device="cuda"), 5)
    assert ctx.device_error() == 0
