"""abfs_relabel_order, the host-side numbering behind abfs_graph_relabel,
against the rule restated here with numpy: classes of whole equal-length groups
taken from the longest columns down (at most n/64 vertices, then at most n/8
with the first class), the other non-empty columns, the empty ones; input order
inside a class.  No GPU: the call only reads the column pointers."""
import numpy as np
import pytest

import paper_1906_03113_gb300 as abfs


def _expected(lengths: np.ndarray) -> np.ndarray:
    n = lengths.size
    cls = np.where(lengths > 0, 2, 3)
    vals, counts = np.unique(lengths[lengths > 0], return_counts=True)
    order = np.argsort(-vals)
    acc, g = 0, 0
    for c, cap in enumerate((n // 64, n // 8)):
        while g < order.size and acc + counts[order[g]] <= cap:
            acc += counts[order[g]]
            cls[lengths == vals[order[g]]] = c
            g += 1
    return np.argsort(cls, kind="stable").astype(np.uint32)


def _colptr(lengths) -> np.ndarray:
    return np.concatenate([[0], np.cumsum(np.asarray(lengths, dtype=np.uint64))]).astype(np.uint32)


def _check(lengths):
    lengths = np.asarray(lengths, dtype=np.uint32)
    lab, pos = abfs.relabel_order(_colptr(lengths))
    n = lengths.size
    assert np.array_equal(np.sort(lab), np.arange(n, dtype=np.uint32))
    assert np.array_equal(pos[lab], np.arange(n, dtype=np.uint32))
    assert np.array_equal(lab, _expected(lengths))
    return lab


def test_skewed_and_uniform_degree_sequences():
    rng = np.random.default_rng(11)
    for n in (1, 7, 63, 64, 65, 1000, 4096, 1 << 15):
        _check(np.minimum(rng.zipf(1.8, n), 50_000))          # power law, many ties
        _check(rng.integers(0, 6, n))                         # few lengths, large groups
        _check(np.full(n, 4))                                 # regular: the input order
        _check(np.zeros(n, dtype=np.uint32))                  # no edges at all
    lab = _check(np.full(500, 3))
    assert np.array_equal(lab, np.arange(500))


def test_whole_groups_at_the_caps():
    # n = 128: at most 2 vertices in class 0, at most 16 in classes 0-1
    base = [1] * 100 + [0] * 12
    lab = _check([100, 100] + [50] * 14 + base)  # both groups fit exactly
    assert list(lab[:16]) == list(range(16))
    lab = _check([100, 100, 100] + [50] * 13 + base)  # 3 > 2: the hubs move to class 1
    assert list(lab[:3]) == [0, 1, 2]
    # n = 64, k = 9: a group of 9 equal lengths fills the selected prefix and is
    # too large for n/8 = 8; a group of 8 fits
    lengths = [1] * 55 + [5] * 9
    lab = _check(lengths)
    assert list(lab[:3]) == [0, 1, 2]                     # input order, one class
    lab = _check([1] * 56 + [5] * 8)
    assert list(lab[:8]) == list(range(56, 64))
    # empty columns always go last, in input order
    lab = _check([0, 3, 0, 2, 0, 1] * 20)
    assert all(i % 2 == 0 for i in lab[-60:])


def test_invalid_arguments():
    assert abfs.load().abfs_relabel_order(None, 5, None, None) == 1
    with pytest.raises(abfs.AbfsError):
        abfs.relabel_order(np.array([0, 3, 2, 4], dtype=np.uint32))  # decreasing
    lab, pos = abfs.relabel_order(np.array([0], dtype=np.uint32))  # n = 0
    assert lab.size == 0 and pos.size == 0
