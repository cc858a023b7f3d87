"""GPU parity at the full size of the 3-mode benchmark workload
(2M x 1M x 50K, 100M nonzeros, Zipf 1.1, lognormal values, core 10^3), in the
launch configuration the benchmark times (FP32, one Lite bin per resident
thread).  The oracle cannot form whole 2M-row penultimate matrices quickly, so
the TTM-chain (eq. (1)) is checked on sampled rows -- the heaviest slices,
which Lite splits over many bins, the lightest and random ones -- each
computed by the oracle from that slice's elements alone; the factor update
(Fig. 1 "SVD") is checked against the oracle's SVD of the same Z."""
import numpy as np
import pytest
import torch

from oracle import tucker_oracle as O
from paper_1804_09494_gb300 import synth
from paper_1804_09494_gb300.tucker import Tucker
from tests.gpu_cases import ROW_TOL, TTM_TOL, rel_err, row_rel_err

pytestmark = pytest.mark.gpu

WORKLOAD = "zipf1.1-2Mx1Mx50K-nnz100M-k10"
PROJ_FP32 = 1e-4


@pytest.fixture(scope="module")
def full():
    w = synth.workload(WORKLOAD)
    L, K = w["L"], w["K"]
    F = synth.random_orthonormal_factors(L, K, seed=1234)
    Fo = [f.astype(np.float32).astype(np.float64) for f in F]
    Fd = [torch.from_numpy(f).float().cuda() for f in Fo]
    tk = Tucker(torch.from_numpy(w["idx"]).cuda(), torch.from_numpy(w["vals"]).cuda(), L, K, prec="fp32")
    yield dict(w=w, L=L, K=K, Fo=Fo, Fd=Fd, tk=tk)
    tk.close()


def sample_slices(cnt, E_max, rng):
    """Slices to check: the heaviest slice (millions of elements, split over
    thousands of bins and many fix-up chunks), the largest below 1.5M elements,
    the largest below 100K, two just longer than one bin, the six lightest and
    twelve random ones."""
    nz = np.flatnonzero(cnt > 0)
    by_size = nz[np.argsort(cnt[nz], kind="stable")]
    c = cnt[by_size]
    pick = [by_size[:6], by_size[-1:], rng.choice(nz, size=12, replace=False)]
    for cap in (1_500_000, 100_000):
        j = np.searchsorted(c, cap, side="right") - 1
        if j >= 0:
            pick.append(by_size[j:j + 1])
    j = np.searchsorted(c, E_max, side="right")
    pick.append(by_size[j:j + 2])
    return np.unique(np.concatenate(pick))


def oracle_rows(w, Fo, n, ids):
    """Oracle Z rows of the slices `ids` of mode n from their elements only
    (slice ids renumbered 0..len(ids)-1)."""
    idx = w["idx"]
    sel = np.isin(idx[n], ids)
    sub = idx[:, sel].copy()
    sub[n] = np.searchsorted(ids, sub[n])
    L = list(w["L"])
    L[n] = len(ids)
    return O.ttm_chain(tuple(L), sub, w["vals"][sel].astype(np.float64), Fo, n)


@pytest.mark.parametrize("n", [0, 1, 2])
def test_fullsize_ttm_chain_sampled_rows(full, n):
    w, tk = full["w"], full["tk"]
    Z, rid = tk.ttm_chain(n, full["Fd"])
    torch.cuda.synchronize()
    rid = rid.cpu().numpy()
    cnt = np.bincount(w["idx"][n], minlength=w["L"][n])
    assert np.array_equal(rid, np.flatnonzero(cnt > 0)), "row ids differ from the non-empty slices"
    ids = sample_slices(cnt, tk.stats(n)["E_max"], np.random.default_rng(100 + n))
    rows = np.searchsorted(rid, ids)
    Zg = Z[torch.from_numpy(rows).cuda()].double().cpu().numpy()
    Zo = oracle_rows(w, full["Fo"], n, ids)
    assert rel_err(Zg, Zo) <= TTM_TOL["fp32"], (n, rel_err(Zg, Zo))
    assert row_rel_err(Zg, Zo) <= ROW_TOL["fp32"], (n, "row", row_rel_err(Zg, Zo))
    # the heaviest slice alone (the most split pieces)
    h = int(np.argmax(cnt[ids]))
    assert cnt[ids[h]] == cnt.max() and cnt[ids[h]] > 100 * tk.stats(n)["E_max"]
    assert rel_err(Zg[h], Zo[h]) <= TTM_TOL["fp32"], (n, int(ids[h]), int(cnt[ids[h]]))


@pytest.mark.parametrize("n", [2, 0])
def test_fullsize_factor_update(full, n):
    tk, K = full["tk"], full["K"]
    Z, rid = tk.ttm_chain(n, full["Fd"])
    F, sigma = tk.factor_update(n, Z)
    torch.cuda.synchronize()
    Zc = Z.double().cpu().numpy()
    Uo, so = O.leading_left_singular_vectors(Zc, K[n])
    Fg = F.double().cpu().numpy()
    rid = rid.cpu().numpy()
    assert O.projector_distance(Fg[rid], Uo) <= PROJ_FP32
    assert rel_err(sigma.cpu().numpy(), so) <= 1e-5
    assert np.abs(Fg.T @ Fg - np.eye(K[n])).max() <= 1e-5
    empty = np.ones(Fg.shape[0], dtype=bool)
    empty[rid] = False
    assert not np.any(Fg[empty])


def test_hooi_invocation_20M_matches_oracle():
    """One HOOI invocation (Fig. 1) plus core and fit on the benchmark recipe
    at 20M nonzeros, in the launch configuration the benchmark times, against
    the FP64 oracle's: factor subspaces within projector distance 1e-4, fit
    within 1e-6."""
    w = synth.workload(WORKLOAD, nnz=20_000_000)
    L, K = w["L"], w["K"]
    F0 = synth.random_orthonormal_factors(L, K, seed=1234)
    Fr = [f.astype(np.float32).astype(np.float64) for f in F0]
    tk = Tucker(torch.from_numpy(w["idx"]).cuda(), torch.from_numpy(w["vals"]).cuda(), L, K, prec="fp32")
    try:
        F = [torch.from_numpy(f).float().cuda() for f in Fr]
        G, fit = tk.hooi_iter(F)
        torch.cuda.synchronize()
        idx = w["idx"].astype(np.int64)
        v = w["vals"].astype(np.float64)
        Fo = O.hooi_invocation(L, idx, v, Fr)
        fo = O.fit(v, O.core(L, idx, v, Fo))
        for m in range(3):
            assert O.projector_distance(F[m].double().cpu().numpy(), Fo[m]) <= PROJ_FP32, m
        assert abs(fit - fo) <= 1e-6, (fit, fo)
    finally:
        tk.close()
