"""Pins for oracle.mj: the multi-jagged split rule checked by brute force."""

import numpy as np
import pytest

import oracle as O
import workloads as W


def brute_mj(coords, w, K):
    """Independent level-by-level implementation: every section scans all
    split positions explicitly with Python sorting and Python integers."""
    n, dims = coords.shape
    sections = [(list(range(n)), 0, K)]
    parts = [0] * n
    level = 0
    while sections:
        nxt = []
        for verts, lo, k in sections:
            if k == 1:
                for v in verts:
                    parts[v] = lo
                continue
            dim = level % dims
            kl = -(-k // 2)
            vs = sorted(verts, key=lambda v: (float(coords[v, dim]) + 0.0, v))
            tot = sum(int(w[v]) for v in vs)
            best, bestp, acc = None, 0, 0
            for p in range(len(vs) + 1):
                if p > 0:
                    acc += int(w[vs[p - 1]])
                val = abs(k * acc - kl * tot)
                if best is None or val < best:
                    best, bestp = val, p
            nxt.append((vs[:bestp], lo, kl))
            nxt.append((vs[bestp:], lo + kl, k - kl))
        sections = nxt
        level += 1
    return np.array(parts, dtype=np.int32)


@pytest.mark.parametrize("K", [2, 3, 5, 8, 13, 16])
@pytest.mark.parametrize("ties", [False, True])
def test_mj_against_brute_force(K, ties):
    n = 700
    dims = max(1, K.bit_length() - 1)
    c = W.random_coords(n, dims, seed=K, ties=ties)
    w = W.random_vertex_weights(n, 1, 7, seed=K + 100)
    assert np.array_equal(O.multijagged(c, w, K), brute_mj(c, w, K))
    ones = np.ones(n, dtype=np.int64)
    assert np.array_equal(O.multijagged(c, None, K), brute_mj(c, ones, K))


def test_mj_float32_coordinates_and_signed_zero():
    c = np.array([[0.0], [-0.0], [0.0], [-1.0], [2.0], [-0.0]], dtype=np.float32)
    parts = O.multijagged(c, None, 2)
    # order by (value, id): -1(3), 0(0), -0(1), 0(2), -0(5), 2(4): first 3 go left
    assert list(parts) == [0, 0, 1, 0, 1, 1]


def test_mj_unit_weight_part_sizes():
    n, K = 1000, 8
    c = W.random_coords(n, 3, seed=4)
    sizes = np.bincount(O.multijagged(c, None, K), minlength=K)
    assert list(sizes) == [125] * 8
    sizes = np.bincount(O.multijagged(W.random_coords(1001, 2, seed=5), None, 3), minlength=3)
    # k=3: left gets 2 parts: p* = argmin |3p - 2*1001| = 667, then 667 -> 333/334
    assert sorted(sizes) == [333, 334, 334] and sizes[2] == 334


def test_mj_uses_each_dimension_once_for_power_of_two():
    n, K = 512, 8
    c = W.random_coords(n, 3, seed=9)
    parts = O.multijagged(c, None, K)
    for bit, dim in ((2, 0), (1, 1), (0, 2)):
        # within each section of the previous levels, the split along ``dim``
        # separates by coordinate order
        for sec in range(K >> (bit + 1)):
            sel = (parts >> (bit + 1)) == sec
            left = sel & (((parts >> bit) & 1) == 0)
            right = sel & (((parts >> bit) & 1) == 1)
            assert c[left, dim].max() <= c[right, dim].min()


def test_mj_relabelling_invariance_for_distinct_coordinates():
    n, K = 300, 6
    c = W.random_coords(n, 2, seed=3)
    perm = np.random.default_rng(0).permutation(n)
    p1 = O.multijagged(c, None, K)
    p2 = O.multijagged(c[perm], None, K)
    assert np.array_equal(p1[perm], p2)


def test_mj_rejects_nan_and_nonpositive_weights():
    c = np.array([[0.0], [np.nan]])
    with pytest.raises(ValueError):
        O.multijagged(c, None, 2)
    with pytest.raises(ValueError):
        O.multijagged(np.zeros((2, 1)), np.array([1, 0]), 2)


def test_mj_more_parts_than_points():
    c = np.array([[0.3], [0.1]])
    parts = O.multijagged(c, None, 4)
    assert list(parts) == list(brute_mj(c, np.ones(2, dtype=np.int64), 4))
