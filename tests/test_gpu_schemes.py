"""GPU parity of the comparator schemes' metrics (Section 5: CoarseG, MediumG;
Section 4.1 metrics), computed on the device from a context's copies, against
the oracle: bit-exact per-processor element and slice counts."""
import numpy as np
import pytest
import torch

from oracle import partition_schemes as PS
from tests.gpu_cases import case, make

pytestmark = pytest.mark.gpu

CASES = [
    ("zipf-3d", (3000, 2000, 400), 60_000, (1.1, 1.1, 1.1), (8, 8, 8)),
    ("uniform-3d", (500, 400, 300), 40_000, None, (6, 6, 6)),
    ("zipf-4d", (400, 300, 60, 20), 50_000, (1.2, 1.2, None, None), (4, 4, 4, 4)),
]


@pytest.mark.parametrize("P", [1, 16, 96, 1000])
@pytest.mark.parametrize("name,L,nnz,zipf,K", CASES, ids=[c[0] for c in CASES])
def test_scheme_metrics_match_oracle(name, L, nnz, zipf, K, P):
    c = case(L, nnz, zipf, "uniform", seed=61)
    tk = make(c, K, "fp32")
    rng = np.random.default_rng(62)
    pos = [rng.permutation(l).astype(np.int32) for l in L]
    dpos = [torch.from_numpy(p).cuda() for p in pos]
    for n in range(len(L)):
        cg = tk.scheme_metrics(n, "coarseg", P, dpos)
        o = PS.metrics(PS.coarseg_owner(c["idx"][n], L[n], P, pos[n]), c["idx"][n], P)
        assert (cg["E_max"], cg["R_sum"], cg["R_max"]) == (o["E_max"], o["R_sum"], o["R_max"]), (n, "coarseg")
        assert cg["E"].cpu().numpy().tolist() == o["E"].tolist()
        assert cg["R"].cpu().numpy().tolist() == o["R"].tolist()
        mg = tk.scheme_metrics(n, "mediumg", P, dpos)
        o = PS.metrics(PS.mediumg_owner(c["idx"], L, P, pos), c["idx"][n], P)
        assert (mg["E_max"], mg["R_sum"], mg["R_max"]) == (o["E_max"], o["R_sum"], o["R_max"]), (n, "mediumg")
        assert mg["E"].cpu().numpy().tolist() == o["E"].tolist()
        assert mg["R"].cpu().numpy().tolist() == o["R"].tolist()
    tk.close()


def test_scheme_metrics_reject_bad_permutations():
    c = case((50, 40, 30), 2000, None, "uniform", seed=63)
    tk = make(c, (3, 3, 3), "fp32")
    pos = [torch.arange(l, dtype=torch.int32, device="cuda") for l in c["L"]]
    bad = [p.clone() for p in pos]
    bad[0][5] = 50  # out of [0, L_0)
    with pytest.raises(Exception):
        tk.scheme_metrics(0, "coarseg", 8, bad)
    dup = [p.clone() for p in pos]
    dup[0][5] = 6  # position 6 given twice
    with pytest.raises(Exception):
        tk.scheme_metrics(0, "coarseg", 8, dup)
    # the context stays usable
    ok = tk.scheme_metrics(0, "coarseg", 8, pos)
    assert ok["R_sum"] == len(np.unique(c["idx"][0]))
    tk.close()
