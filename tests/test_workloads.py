"""Pins for the seeded input generator (workloads/), CPU only."""
import math

import numpy as np
import pytest

import workloads as W
from conftest import make_matrix


def _splitmix64_reference(state, count):
    """SplitMix64 (Steele, Lea and Flood, 2014), sequential form, written out."""
    out = []
    mask = (1 << 64) - 1
    for _ in range(count):
        state = (state + 0x9E3779B97F4A7C15) & mask
        z = state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & mask
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & mask
        out.append(z ^ (z >> 31))
    return out


def test_splitmix64_counter_form_matches_sequence():
    for seed in (0, 1, 1234567, 2**63 + 5):
        ref = _splitmix64_reference(seed, 6)
        got = [W.splitmix64_at(seed, i) for i in range(6)]
        assert got == ref


def test_portable_log_and_cos_match_libm():
    rng = np.random.Generator(np.random.PCG64(11))
    xs = np.concatenate([rng.random(2000), [2.0**-53, 1e-300, 0.5, 1.0, 0.7071067811865476]])
    for x in xs:
        if x <= 0:
            continue
        assert abs(W.portable_log(x) - math.log(x)) <= 4e-16 * max(1.0, abs(math.log(x)))
    for u in np.concatenate([rng.random(2000), [0.0, 0.125, 0.25, 0.5, 0.75, 0.999999]]):
        assert abs(W.portable_cos2pi(u) - math.cos(2 * math.pi * u)) <= 2e-15


def test_level_sizes_geometric():
    assert W.level_sizes_geometric(2_000_000, 7, 2.2) == [9660, 21253, 46757, 102864, 226302, 497864, 1095300]
    s9 = W.level_sizes_geometric(20_000_000, 9, 2.2)
    assert sum(s9) == 20_000_000 and s9[0] == 19896
    for a in range(1, 8):
        assert abs(s9[a] / s9[a - 1] - 2.2) < 1e-3


@pytest.mark.parametrize("name", ["small", "c1"])
def test_matrix_is_bit_symmetric_and_level_banded(name):
    w, rp, c, v = make_matrix(name)
    n = w.n
    assert rp[0] == 0 and rp[-1] == c.shape[0] and np.all(np.diff(rp) >= 1)
    assert c.min() >= 0 and c.max() < n
    rows = np.repeat(np.arange(n), np.diff(rp))
    # strictly increasing columns inside each row
    same = rows[1:] == rows[:-1]
    assert np.all(c[1:][same] > c[:-1][same])
    # bit-exact symmetry: sort the transpose's entries and compare the bytes
    key = rows.astype(np.int64) * n + c
    keyT = c.astype(np.int64) * n + rows
    oT = np.argsort(keyT, kind="stable")
    assert np.array_equal(key, keyT[oT])
    assert np.array_equal(v.view(np.uint64), v[oT].view(np.uint64))
    # only levels with |dN| <= 2 are coupled
    lvl = np.repeat(np.arange(len(w.level_sizes)), w.level_sizes)
    assert np.all(np.abs(lvl[rows] - lvl[c]) <= 2)


@pytest.mark.parametrize("name", ["small", "c1"])
def test_value_law(name):
    w, rp, c, v = make_matrix(name)
    n = w.n
    rows = np.repeat(np.arange(n), np.diff(rp))
    diag = rows == c
    assert diag.sum() == n
    lvl = np.repeat(np.arange(len(w.level_sizes)), w.level_sizes)
    dv = np.empty(n)
    dv[rows[diag]] = v[diag]
    u = dv - 10.0 * lvl
    assert u.min() >= -2.0 and u.max() < 2.0
    assert abs(u.mean()) < 0.06 and abs(u.std() - 4 / math.sqrt(12)) < 0.03
    off = v[~diag]
    # merged duplicates are rare; the law is N(0, 0.5^2)
    assert abs(off.mean()) < 0.01
    assert abs(off.std() - w.sigma) < 0.01 * w.sigma + 0.005


@pytest.mark.parametrize("name", ["small", "c1"])
def test_nonzeros_per_level_follow_the_draw_law(name):
    """Mean stored entries per row of level a = 1 + d + expected mirrored draws,
    minus the rare merged duplicates (< 2%)."""
    w, rp, c, v = make_matrix(name)
    L = w.level_sizes
    off = w.level_offsets
    d = w.draws_per_row
    nl = len(L)
    win = [off[min(b + 2, nl - 1) + 1] - off[max(b - 2, 0)] - 1 for b in range(nl)]
    for a in range(nl):
        inc = 0.0
        for b in range(max(a - 2, 0), min(a + 2, nl - 1) + 1):
            rows_b = L[b] - (1 if b == a else 0)
            inc += rows_b * d / win[b]
        expect = 1 + d + inc
        got = (rp[off[a + 1]] - rp[off[a]]) / L[a]
        assert expect * 0.97 < got <= expect * 1.001, (a, got, expect)


def test_generator_is_deterministic_and_seeded():
    w = W.config("small")
    a = W.generate(w)
    b = W.generate(w)
    for x, y in zip(a, b):
        assert np.array_equal(x, y)
    w2 = W.Workload("s2", w.level_sizes, w.nnz_per_row, w.k, seed=w.seed + 1)
    c = W.generate(w2)
    assert not (a[1].shape == c[1].shape and np.array_equal(a[1], c[1]))


def test_random_block_seeded():
    x = W.random_block(100, 8, 5)
    y = W.random_block(100, 8, 5)
    assert np.array_equal(x, y) and x.shape == (100, 8)
