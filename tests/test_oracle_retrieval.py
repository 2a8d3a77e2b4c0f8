"""Pins of the oracle's retrieval nearest-neighbour search (ImLoc Sec. 3.1:
precomputed global retrieval features; Sec. 4.4 "Runtime": nearest-neighbour
search of the retrieval features).  Reading: top-K database images by the dot
product of L2-normalised descriptors (cosine similarity), descending, ties to
the lower database index; descriptors stored as bfloat16."""
import numpy as np

import oracle
from paper_2601_04185_gb300 import synth


def test_bf16_decoding():
    assert oracle.bf16_to_double(0x3F80) == 1.0
    assert oracle.bf16_to_double(0xC000) == -2.0
    assert oracle.bf16_to_double(0x0000) == 0.0
    assert oracle.bf16_to_double(0x3E80) == 0.25
    assert oracle.bf16_to_double(0x0001) == 2.0 ** -133  # smallest subnormal
    assert oracle.bf16_to_double(0x7F7F) == (2 - 2 ** -7) * 2.0 ** 127


def test_rounding_to_bf16_is_nearest_even():
    x = np.array([1.0, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -8, 1.0 + 2 ** -7 + 2 ** -9, -0.0], np.float32)
    b = synth.to_bf16_bits(x)
    got = [oracle.bf16_to_double(v) for v in b]
    assert got == [1.0, 1.0, 1.0 + 2 ** -6, 1.0 + 2 ** -7, 0.0]


def test_scores_and_selection_against_numpy():
    rng = np.random.default_rng(0)
    db, q, _ = synth.retrieval_set(rng, 700, 9, 96)
    sc, ix = oracle.retrieve_topk(q, db, 25)
    dbf = (db.astype(np.uint32) << 16).view(np.float32).astype(np.float64)
    qf = (q.astype(np.uint32) << 16).view(np.float32).astype(np.float64)
    full = qf @ dbf.T
    for i in range(9):
        order = np.lexsort((np.arange(700), -full[i]))[:25]  # descending score, then index
        np.testing.assert_array_equal(ix[i], order)
        np.testing.assert_allclose(sc[i], full[i, order], rtol=0, atol=1e-15)


def test_ties_go_to_the_lower_index_and_k_equals_n():
    base = synth.to_bf16_bits(np.array([[0.5, 0.5, 0.0, 0.0]], np.float32))
    db = np.repeat(base, 5, axis=0)
    db[2] = synth.to_bf16_bits(np.array([0.0, 0.0, 1.0, 0.0], np.float32))
    q = synth.to_bf16_bits(np.array([[1.0, 1.0, 0.0, 0.0]], np.float32))
    sc, ix = oracle.retrieve_topk(q, db, 5)
    assert list(ix[0]) == [0, 1, 3, 4, 2]
    assert list(sc[0]) == [1.0, 1.0, 1.0, 1.0, 0.0]


def test_a_database_copy_of_the_query_ranks_first():
    rng = np.random.default_rng(1)
    db, q, _ = synth.retrieval_set(rng, 300, 4, 256)
    db[137] = q[2]
    sc, ix = oracle.retrieve_topk(q[2:3], db, 3)
    assert ix[0, 0] == 137
    assert abs(sc[0, 0] - 1.0) < 1e-2  # unit norm up to bfloat16 rounding
