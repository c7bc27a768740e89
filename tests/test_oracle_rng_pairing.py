"""Pins for the oracle's random numbers, binning and Takizuka-Abe pairing (CPU only).

Philox-4x32-10 is checked against the published known-answer values of its authors' reference distribution
(Random123); binning against numpy's stable sort; pairing against brute-force structure rules of the order-N
method [Sec. 3.2, Fig. TApairing] and a chi-square test that every intra-species pairing is equally likely.
"""
import math
import os

import numpy as np
import pytest

import oracle as O


GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _load_kat():
    rows = []
    with open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            x = [int(t, 16) for t in line.split()]
            rows.append((tuple(x[0:4]), tuple(x[4:6]), tuple(x[6:10])))
    return rows


# Philox-4x32-10 known-answer vectors: (counter, key) -> output, as published with the generator.
PHILOX_KAT = _load_kat()


@pytest.mark.parametrize("ctr,key,expect", PHILOX_KAT)
def test_philox_known_answers(ctr, key, expect):
    assert tuple(int(x) for x in O.philox4x32_10(ctr, key)) == expect


def test_philox_uniform_bits():
    # 4096 blocks over consecutive counters: each output bit is set with probability 1/2
    words = np.array([O.philox4x32_10((i, 7, 3, 0x301), (11, 13)) for i in range(4096)], dtype=np.uint64)
    bits = ((words[..., None] >> np.arange(32, dtype=np.uint64)) & 1).reshape(-1, 32)
    frac = bits.mean(axis=0)
    assert np.all(np.abs(frac - 0.5) < 5 * 0.5 / math.sqrt(bits.shape[0]))


def test_bin_equals_stable_sort():
    rng = np.random.default_rng(5)
    n, C, S = 5000, 37, 3
    cell = rng.integers(0, C, n).astype(np.int32)
    sp = rng.integers(0, S, n).astype(np.int32)
    perm, off = O.bin_particles(cell, sp, C, S)
    key = cell.astype(np.int64) * S + sp
    np.testing.assert_array_equal(perm, np.argsort(key, kind="stable"))
    np.testing.assert_array_equal(off, np.concatenate([[0], np.cumsum(np.bincount(key, minlength=C * S))]))


def test_bin_weighted_equals_lexicographic_sort():
    """Each segment ordered by descending weight truncated to 32 fraction bits (frexp: same exponent and the same
    floor of the fraction times 2^32 tie), ties by increasing particle index; segments as in the plain cell sort."""
    rng = np.random.default_rng(6)
    n, C, S = 6000, 29, 3
    cell = rng.integers(0, C, n).astype(np.int32)
    sp = rng.integers(0, S, n).astype(np.int32)
    base = 10.0 ** rng.uniform(0, 4, n)
    pick = rng.integers(0, 4, n)
    ref = base[rng.integers(0, n, n)]
    # exact ties, ties below the key width (2^-40), distinct just above it (2^-30), and free weights
    w = np.where(pick == 0, ref, np.where(pick == 1, ref * (1 + 2.0 ** -40), np.where(pick == 2,
                 ref * (1 + 2.0 ** -30), base)))
    w[:50] = 1.0
    perm, off = O.bin_particles_weighted(cell, sp, w, C, S)
    mant, ex = np.frexp(w)
    frac = np.floor((2.0 * mant - 1.0) * 2.0 ** 32)
    seg = cell.astype(np.int64) * S + sp
    want = np.lexsort((np.arange(n), -frac, -ex, seg))
    np.testing.assert_array_equal(perm, want)
    p0, off0 = O.bin_particles(cell, sp, C, S)
    np.testing.assert_array_equal(off, off0)


def test_bin_rejects_out_of_range():
    with pytest.raises(ValueError):
        O.bin_particles(np.array([0, 5], np.int32), np.array([0, 0], np.int32), 3, 1)


@pytest.mark.parametrize("n", [0, 1, 2, 3, 7, 64, 1000])
def test_permutation_is_permutation(n):
    p = O.permutation(n, seed=3, step=9, cell=4, inter=1, side=0)
    assert sorted(p.tolist()) == list(range(n))


def test_permutation_depends_on_every_counter_field():
    base = O.permutation(50, 3, 9, 4, 1, 0)
    for args in [(4, 9, 4, 1, 0), (3, 10, 4, 1, 0), (3, 9, 5, 1, 0), (3, 9, 4, 2, 0), (3, 9, 4, 1, 1)]:
        assert not np.array_equal(base, O.permutation(50, *args))


def test_permutation_uniform_chi2():
    # n = 4: all 24 orders equally likely over many steps
    n, trials = 4, 24 * 400
    counts = {}
    for t in range(trials):
        key = tuple(O.permutation(n, 17, t, 0, 0, 0).tolist())
        counts[key] = counts.get(key, 0) + 1
    assert len(counts) == 24
    obs = np.array(list(counts.values()), float)
    chi2 = ((obs - trials / 24) ** 2 / (trials / 24)).sum()
    assert chi2 < 49.7  # 23 dof, p = 0.001


def _cell_pairs(na, nb, intra, seed=1, step=0, inter=0):
    S = 1 if intra else 2
    off = np.array([0, na] if intra else [0, na, na + nb], dtype=np.int64)
    pi, pj, fl = O.pairs(off, 1, S, 0, 0 if intra else 1, inter, seed, step)
    ntot = na if intra else na + nb
    if intra:
        npairs = 0 if na < 2 else (na // 2 if na % 2 == 0 else (na + 3) // 2)
    else:
        npairs = 0 if (na == 0 or nb == 0) else max(na, nb)
    assert npairs <= ntot
    return pi[:npairs], pj[:npairs], fl[:npairs]


@pytest.mark.parametrize("n", [2, 3, 4, 5, 6, 7, 8])
def test_intra_pairing_structure(n):
    for step in range(20):
        pi, pj, fl = _cell_pairs(n, 0, True, step=step)
        if n % 2 == 0:
            assert len(pi) == n // 2 and not fl.any()
            assert sorted(np.concatenate([pi, pj]).tolist()) == list(range(n))
        else:
            assert len(pi) == (n + 3) // 2
            assert fl[:3].tolist() == [1, 1, 1] and not fl[3:].any()
            a, b, c = pi[0], pj[0], pj[1]
            # triplet (p0,p1),(p1,p2),(p2,p0): every particle of the triplet in exactly two of its pairs
            assert (pi[1], pi[2], pj[2]) == (b, c, a)
            rest = np.concatenate([pi[3:], pj[3:]]).tolist()
            assert sorted(rest + [a, b, c]) == list(range(n))


@pytest.mark.parametrize("na,nb", [(5, 2), (2, 5), (3, 3), (8, 3), (1, 4), (4, 1), (7, 7)])
def test_inter_pairing_structure(na, nb):
    for step in range(20):
        pi, pj, fl = _cell_pairs(na, nb, False, step=step)
        nmax, nmin = max(na, nb), min(na, nb)
        assert len(pi) == nmax and not fl.any()
        big, small = (pi, pj - na) if na >= nb else (pj - na, pi)
        assert sorted(big.tolist()) == list(range(nmax))           # larger population: exactly once
        cnt = np.bincount(small, minlength=nmin)
        assert cnt.min() >= nmax // nmin and cnt.max() <= -(-nmax // nmin)
        # rounds of N_min consecutive pairs touch distinct particles of the smaller population
        for r in range(0, nmax, nmin):
            blk = small[r:r + nmin]
            assert len(set(blk.tolist())) == len(blk)


def test_inter_pairing_empty_side():
    for na, nb in [(0, 3), (3, 0), (0, 0)]:
        pi, _, _ = _cell_pairs(na, nb, False)
        assert len(pi) == 0


@pytest.mark.parametrize("n", [4, 6])
def test_intra_pairings_uniform_chi2(n):
    # each of the (n-1)!! perfect matchings appears equally often
    n_match = math.prod(range(n - 1, 0, -2))
    trials = n_match * 300
    counts = {}
    for t in range(trials):
        pi, pj, _ = _cell_pairs(n, 0, True, seed=23, step=t)
        key = tuple(sorted(tuple(sorted(p)) for p in zip(pi.tolist(), pj.tolist())))
        counts[key] = counts.get(key, 0) + 1
    assert len(counts) == n_match
    obs = np.array(list(counts.values()), float)
    chi2 = ((obs - trials / n_match) ** 2 / (trials / n_match)).sum()
    # p = 0.001 critical values: 2 dof -> 13.8, 14 dof -> 36.1
    assert chi2 < {3: 13.8, 15: 36.1}[n_match]


def test_inter_pairing_partner_uniform():
    # every (i, j) partner combination equally likely for equal population sizes
    na = nb = 3
    trials = 3000
    counts = np.zeros((na, nb))
    for t in range(trials):
        pi, pj, _ = _cell_pairs(na, nb, False, seed=5, step=t)
        for i, j in zip(pi, pj):
            counts[i, j - na] += 1
    expect = trials / 3
    chi2 = ((counts - expect) ** 2 / expect).sum()
    assert chi2 < 27.9  # 9 cells, generous bound at p = 0.001


def test_pair_slots_are_cell_offsets():
    counts = np.array([[3, 2], [0, 4], [5, 5], [1, 0]])
    off = np.concatenate([[0], np.cumsum(counts.reshape(-1))]).astype(np.int64)
    pi, pj, fl = O.pairs(off, 4, 2, 0, 1, 1, 9, 2)
    for c in range(4):
        slot = off[2 * c]
        na, nb = counts[c]
        n = max(na, nb) if na and nb else 0
        assert np.all((pi[slot:slot + n] >= off[2 * c]) & (pi[slot:slot + n] < off[2 * c + 1]))
        assert np.all((pj[slot:slot + n] >= off[2 * c + 1]) & (pj[slot:slot + n] < off[2 * c + 2]))
