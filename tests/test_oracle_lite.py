"""Pins for the Lite oracle (Section 6.1 Fig. 7): the Fig. 6 worked example,
Theorem 1's bounds, Lemma 1 (stage 1 is best-processor-fit), Lemma 2 (no
stage-2 slice fits a gap), and the Section 3/4 framework example metrics."""
import numpy as np
import pytest

from oracle import lite_oracle as LO
from tests.conftest import read_golden


def _zipf_counts(rng, L, nnz, s):
    p = np.arange(1, L + 1, dtype=float) ** (-s)
    p /= p.sum()
    return np.bincount(rng.choice(L, size=nnz, p=p), minlength=L)


def test_fig6_worked_example_golden():
    g = read_golden("fig6_lite.txt")
    d = dict(g)
    P = int(d["P"][0])
    cnt = np.array([int(x) for x in d["sizes"]])
    res = LO.lite_pieces(cnt, P)
    assert res["limit"] == 20
    assert res["t_hat"] == int(d["t_hat"][0])
    bins = [r for k, r in g if k == "bin"]
    for b in bins:
        p = int(b[0])
        want = [(int(x.split(":")[0]), int(x.split(":")[1])) for x in b[1:]]
        got = [(s, c) for (s, _, c) in res["pieces"][p]]
        assert got == want, (p, got, want)
    m = LO.metrics(res["pieces"])
    assert m["E_max"] == int(d["E_max"][0])
    assert m["R_sum"] == int(d["R_sum"][0])
    assert m["R_max"] == int(d["R_max"][0])
    assert m["E"] == [20] * 5
    # slice 9 (S9 of the caption): head is bin 1, tail bins 2-3
    owners = [p for p in range(P) for (s, _, c) in res["pieces"][p] if s == 8]
    assert owners == [1, 2, 3]


def _check_theorem1(cnt, P):
    res = LO.lite_pieces(cnt, P)
    nnz = int(np.sum(cnt))
    Ln = int(np.count_nonzero(cnt))
    m = LO.metrics(res["pieces"])
    assert m["E_max"] <= -(-nnz // P)
    assert m["R_sum"] <= Ln + P
    assert m["R_max"] <= -(-Ln // P) + 2
    # every element assigned exactly once, each slice's pieces tile its ranks in order
    seen = {}
    for p in range(P):
        for (s, j0, c) in res["pieces"][p]:
            seen.setdefault(s, []).append((p, j0, c))
    for s, ps in seen.items():
        j = 0
        for (_, j0, c) in ps:
            assert j0 == j
            j += c
        assert j == cnt[s]
        bins = [p for (p, _, _) in ps]
        assert bins == sorted(bins)  # contiguous processors, in order
    assert set(seen) == set(np.flatnonzero(cnt).tolist())
    bad = [s for s, ps in seen.items() if len(ps) > 1]
    assert len(bad) <= P
    # each bin heads at most one and tails at most one split slice
    for p in range(P):
        heads = sum(1 for (s, j0, c) in res["pieces"][p] if s in bad and j0 == 0)
        tails = sum(1 for (s, j0, c) in res["pieces"][p] if s in bad and j0 > 0)
        assert heads <= 1 and tails <= 1
    return res


@pytest.mark.parametrize("seed", range(6))
@pytest.mark.parametrize("P", [1, 2, 3, 7, 16, 64])
def test_theorem1_random_sizes(seed, P):
    rng = np.random.default_rng(seed)
    L = int(rng.integers(1, 300))
    cnt = rng.integers(0, 50, size=L)
    if cnt.sum() == 0:
        cnt[0] = 1
    _check_theorem1(cnt, P)


@pytest.mark.parametrize("s", [0.8, 1.1, 1.3, 2.0])
@pytest.mark.parametrize("P", [5, 32, 100, 1000])
def test_theorem1_zipf_sizes(s, P):
    rng = np.random.default_rng(int(s * 10) + P)
    cnt = _zipf_counts(rng, 2000, 30000, s)
    _check_theorem1(cnt, P)


@pytest.mark.parametrize("seed", range(5))
def test_lemma1_stage1_is_best_processor_fit(seed):
    """In stage 1 the slice S_t goes to a bin with the least load (Lemma 1)."""
    rng = np.random.default_rng(seed)
    cnt = rng.integers(1, 30, size=200)
    P = int(rng.integers(2, 20))
    res = LO.lite_pieces(cnt, P)
    load = [0] * P
    for t in range(res["t_hat"]):
        s = res["order"][t]
        p = t % P
        assert load[p] == min(load)
        assert res["pieces"][p][t // P][0] == s
        load[p] += int(cnt[s])


@pytest.mark.parametrize("seed", range(5))
def test_lemma2_no_stage2_slice_fits_a_gap(seed):
    rng = np.random.default_rng(100 + seed)
    cnt = _zipf_counts(rng, 500, 8000, 1.2)
    P = 40
    res = LO.lite_pieces(cnt, P)
    limit = res["limit"]
    h = [0] * P
    for t in range(res["t_hat"]):
        h[t % P] += int(cnt[res["order"][t]])
    for t in range(res["t_hat"], len(res["order"])):
        s = res["order"][t]
        assert all(cnt[s] > limit - h[p] for p in range(P))


def test_framework_example_metrics():
    """Section 3 / Section 4.1 example: slices {e1,e3,e6},{e2,e7},{e4,e5,e8}
    split lexicographically over three processors gives R^p = 2 and R_sum = 6."""
    slice_of = np.array([0, 1, 0, 2, 2, 0, 1, 2])
    owner = np.array([0, 0, 0, 1, 1, 1, 2, 2])
    m = LO.metrics_from_assignment(owner, slice_of)
    assert m["R"] == [2, 2, 2]
    assert m["R_sum"] == 6
    assert m["E_max"] == 3


def test_assignment_lists_elements_in_listing_order():
    """Pieces tile each slice's elements in listing order: by the popularity
    rank of the fiber-mode coordinate (mode 2 here, the shortest other mode:
    its largest slice first, ties by lower id), then original position --
    checked against an order built by brute force from the definition."""
    rng = np.random.default_rng(7)
    L = (30, 12, 5)
    idx = np.stack([rng.integers(0, l, size=500) for l in L])
    assert LO.fiber_mode(L, 0) == 2 and LO.fiber_mode(L, 2) == 1 and LO.fiber_mode((4, 3, 3), 0) == 1
    cnt2 = np.bincount(idx[2], minlength=5)
    by_pop = sorted(range(5), key=lambda l: (-cnt2[l], l))
    bin_ptr, perm, info = LO.lite_assignment(idx, L, 0, 9)
    assert sorted(perm.tolist()) == list(range(500))
    for p in range(9):
        seg = perm[bin_ptr[p]: bin_ptr[p + 1]]
        assert len(seg) <= info["limit"]
        for (s, j0, c) in info["pieces"][p]:
            mem = [e for l2 in by_pop for e in range(500) if idx[0][e] == s and idx[2][e] == l2]
            assert np.array_equal(seg[:c], np.array(mem[j0: j0 + c]))
            seg = seg[c:]


def test_popularity_rank_definition():
    idx = np.array([3, 1, 3, 0, 1, 3, 4])
    # sizes: 0:1, 1:2, 2:0, 3:3, 4:1 -> order 3, 1, 0, 4, 2
    np.testing.assert_array_equal(LO.popularity_rank(idx, 5), [2, 1, 4, 0, 3])
