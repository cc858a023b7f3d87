"""Pins of the comparator schemes' oracle (Section 5: CoarseG, MediumG) and of
the Section 4.1 metrics: hand-worked examples, the paper's example grid, and
the structural bounds each scheme's definition implies."""
import numpy as np
import pytest

from oracle import lite_oracle as LO
from oracle import partition_schemes as PS
from paper_1804_09494_gb300 import synth


def _slices(sizes):
    """mode-n coordinates of a tensor whose slice l holds sizes[l] elements"""
    return np.repeat(np.arange(len(sizes)), sizes)


def test_coarseg_hand_worked_example():
    # slice sizes 5, 1, 1, 3 (|E| = 10), P = 2
    idx_n = _slices([5, 1, 1, 3])
    # identity order: H = 0, 5, 6, 7 -> processors floor(2 H / 10) = 0, 1, 1, 1
    own = PS.coarseg_owner(idx_n, 4, 2, [0, 1, 2, 3])
    m = PS.metrics(own, idx_n, 2)
    assert m["E"].tolist() == [5, 5] and m["R"].tolist() == [1, 3]
    assert (m["E_max"], m["R_sum"], m["R_max"]) == (5, 4, 3)
    # slice 0 last: order 1, 2, 3, 0 with H = 0, 1, 2, 5 -> 0, 0, 0, 1
    own = PS.coarseg_owner(idx_n, 4, 2, [3, 0, 1, 2])
    m = PS.metrics(own, idx_n, 2)
    assert m["E"].tolist() == [5, 5] and m["R"].tolist() == [3, 1]


@pytest.mark.parametrize("seed,P", [(0, 7), (1, 32), (2, 100)])
def test_coarseg_blocks_are_whole_contiguous_and_bounded(seed, P):
    rng = np.random.default_rng(seed)
    L = 300
    sizes = rng.zipf(1.5, size=L).clip(max=500) * (rng.random(L) < 0.8)
    idx_n = _slices(sizes)
    pos = rng.permutation(L)
    own = PS.coarseg_owner(idx_n, L, P, pos)
    m = PS.metrics(own, idx_n, P)
    # every slice whole on one processor: R_sum = number of non-empty slices
    assert m["R_sum"] == int((sizes > 0).sum())
    # blocks follow the order: the processor never decreases along it
    order = np.argsort(pos)
    proc_of_slice = {int(l): int(p) for l, p in zip(idx_n, own)}
    seq = [proc_of_slice[int(l)] for l in order if sizes[l] > 0]
    assert all(a <= b for a, b in zip(seq, seq[1:]))
    # a block starts below (p+1)|E|/P, so it exceeds |E|/P by less than one slice
    assert m["E_max"] < len(idx_n) / P + sizes.max()


def test_mediumg_grid_rule():
    # the paper's example grid for P = 16 (4 x 2 x 2), for lengths in ratio 2:1:1
    assert PS.mediumg_grid([200, 100, 100], 16) == [4, 2, 2]
    # 12 = 3 * 2 * 2, largest factor first, ties to the lowest mode
    assert PS.mediumg_grid([100, 100, 100], 12) == [3, 2, 2]
    assert PS.mediumg_grid([5, 1000, 10], 8) == [1, 8, 1]
    assert PS.mediumg_grid([10, 20], 1) == [1, 1]
    for L, P in [([2_000_000, 1_000_000, 50_000], 512), ([1000, 500, 20, 2], 96)]:
        assert int(np.prod(PS.mediumg_grid(L, P))) == P


@pytest.mark.parametrize("P", [8, 24, 64])
def test_mediumg_cells_and_sharing_bounds(P):
    L = (90, 70, 40)
    idx, _ = synth.coo(L, 6000, (1.2, None, 1.1), "uniform", 3)
    rng = np.random.default_rng(4)
    pos = [rng.permutation(l) for l in L]
    q = PS.mediumg_grid(L, P)
    own = PS.mediumg_owner(idx, L, P, pos)
    assert own.min() >= 0 and own.max() < P
    # decode the cell again and check each coordinate lies in its range
    rest = own.copy()
    for m in range(3):
        b = rest % q[m]
        rest //= q[m]
        x = pos[m][idx[m]]
        assert np.all(b * L[m] <= x * q[m]) and np.all(x * q[m] < (b + 1) * L[m])
    for n in range(3):
        m = PS.metrics(own, idx[n], P)
        # a processor holds slices of one range of ceil(L_n / q_n) indices at most
        assert m["R_max"] <= -(-L[n] // q[n])
        # a slice is shared by at most P / q_n processors
        R_n = len(np.unique(idx[n]))
        assert R_n <= m["R_sum"] <= R_n * (P // q[n])
        # uni-policy: the element counts do not depend on the mode
        assert m["E"].tolist() == PS.metrics(own, idx[0], P)["E"].tolist()


def test_metrics_agree_with_the_lite_module_definition():
    rng = np.random.default_rng(5)
    owner = rng.integers(0, 9, 500)
    owner[:9] = np.arange(9)  # every processor non-empty
    slice_of = rng.integers(0, 40, 500)
    a = PS.metrics(owner, slice_of, 9)
    b = LO.metrics_from_assignment(owner, slice_of)
    assert (a["E_max"], a["R_sum"], a["R_max"]) == (b["E_max"], b["R_sum"], b["R_max"])


def test_paper_comparison_holds_on_a_zipf_tensor():
    """Section 5 / Section 6: CoarseG is optimal on R_sum but pays in E_max
    (a slice far above |E|/P); Lite keeps E_max <= ceil(|E|/P) with R_sum <=
    R_n + P (Theorem 1); MediumG balances elements but shares slices."""
    L = (3000, 2000, 400)
    idx, _ = synth.coo(L, 60_000, (1.1, 1.1, 1.1), "uniform", 6)
    P = 64
    rng = np.random.default_rng(7)
    pos = [rng.permutation(l) for l in L]
    for n in range(3):
        R_n = len(np.unique(idx[n]))
        cg = PS.metrics(PS.coarseg_owner(idx[n], L[n], P, pos[n]), idx[n], P)
        mg = PS.metrics(PS.mediumg_owner(idx, L, P, pos), idx[n], P)
        lite = LO.metrics(LO.lite_pieces(np.bincount(idx[n], minlength=L[n]), P)["pieces"])
        assert cg["R_sum"] == R_n
        assert cg["E_max"] >= np.bincount(idx[n]).max() > -(-60_000 // P)
        assert lite["E_max"] <= -(-60_000 // P) and lite["R_sum"] <= R_n + P
        assert mg["R_sum"] > lite["R_sum"]
