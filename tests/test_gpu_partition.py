"""The device Lite partition (Section 6.1, Fig. 7) is bit-exact against the
literal CPU execution of the pseudocode, and its Section 4.1 metrics match."""
import numpy as np
import pytest
import torch

from oracle import lite_oracle as LO
from tests.gpu_cases import case, make

pytestmark = pytest.mark.gpu

PCASES = [
    ("uniform", (200, 150, 100), 20_000, None, (8, 8, 8), 0),
    ("zipf-auto", (3000, 2000, 500), 200_000, (1.1, 1.1, 1.1), (10, 10, 10), 0),
    ("zipf-P32", (3000, 2000, 500), 200_000, (1.1, 1.1, 1.1), (10, 10, 10), 32),
    ("zipf-P160", (5000, 400, 50), 150_000, (1.3, 1.3, 1.3), (4, 4, 4), 160),
    ("zipf-P77", (5000, 400, 50), 150_000, (1.3, 1.3, 1.3), (4, 4, 4), 77),
    ("zipf-4d", (400, 300, 60, 20), 100_000, (1.2, 1.2, None, None), (10, 10, 10, 10), 0),
    ("tiny", (7, 5, 3), 40, None, (2, 2, 2), 32),
]


@pytest.mark.parametrize("name,L,nnz,zipf,K,P", PCASES, ids=[c[0] for c in PCASES])
def test_partition_bit_exact(name, L, nnz, zipf, K, P):
    c = case(L, nnz, zipf, "uniform", seed=21)
    tk = make(c, K, "fp32", P_bins=P)
    for n in range(len(L)):
        st = tk.stats(n)
        bin_ptr, perm = tk.partition(n)
        torch.cuda.synchronize()
        ob, operm, info = LO.lite_assignment(c["idx"], L, n, st["P"])
        assert np.array_equal(bin_ptr.cpu().numpy(), ob), (n, "bin sizes")
        assert np.array_equal(perm.cpu().numpy().astype(np.int64), operm), (n, "element assignment")
        m = LO.metrics(info["pieces"])
        assert (st["E_max"], st["R_sum"], st["R_max"]) == (m["E_max"], m["R_sum"], m["R_max"])
        assert st["R_n"] == int(np.count_nonzero(np.bincount(c["idx"][n], minlength=L[n])))
        # Theorem 1 on the device result
        Ln = st["R_n"]
        assert st["E_max"] <= -(-nnz // st["P"])
        assert st["R_sum"] <= Ln + st["P"]
        assert st["R_max"] <= -(-Ln // st["P"]) + 2
    tk.close()


def test_partition_fig6_worked_example():
    """The Fig. 6 example itself (|E| = 100, P = 5, sizes 5x7, 18, 22, 25) on
    the device partitioner, against the hand-traced golden bins."""
    from tests.conftest import read_golden
    g = read_golden("fig6_lite.txt")
    d = dict(g)
    sizes = [int(x) for x in d["sizes"]]
    P = int(d["P"][0])
    idx0 = np.random.default_rng(0).permutation(np.repeat(np.arange(len(sizes)), sizes))
    nnz = len(idx0)
    idx = np.stack([idx0, np.arange(nnz) % 7, np.arange(nnz) % 11]).astype(np.int32)
    c = dict(L=(len(sizes), 7, 11), idx=idx, vals=np.ones(nnz, dtype=np.float32))
    tk = make(c, (1, 1, 1), "fp32", P_bins=P)
    bin_ptr, perm = tk.partition(0)
    bin_ptr = bin_ptr.cpu().numpy()
    perm = perm.cpu().numpy()
    for b in [r for k, r in g if k == "bin"]:
        p = int(b[0])
        got = idx0[perm[bin_ptr[p]:bin_ptr[p + 1]]]
        want = np.concatenate([np.full(int(x.split(":")[1]), int(x.split(":")[0])) for x in b[1:]])
        assert np.array_equal(got, want), (p, got, want)
    st = tk.stats(0)
    assert (st["E_max"], st["R_sum"], st["R_max"]) == (int(d["E_max"][0]), int(d["R_sum"][0]), int(d["R_max"][0]))
    ob, operm, _ = LO.lite_assignment(idx, c["L"], 0, P)
    assert np.array_equal(bin_ptr, ob) and np.array_equal(perm.astype(np.int64), operm)
    tk.close()
