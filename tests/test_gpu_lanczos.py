"""GPU parity of the paper's SVD route for the factor update (Section 3 "SVD
component"; Section 7: a Lanczos bidiagonalisation with 2K iterations)
against the oracle's ``lanczos_factor``: the same start vector and step
count on the same compact Z, then whole HOOI invocations on that route."""
import numpy as np
import pytest
import torch

from oracle import tucker_oracle as O
from tests.gpu_cases import DT, NP, case, factors, make, rel_err

pytestmark = pytest.mark.gpu

PROJ = {"fp32": 1e-4, "fp64": 1e-8}
SIG = {"fp32": 1e-5, "fp64": 1e-10}


def to_np(t):
    return t.detach().double().cpu().numpy()


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("L,nnz,zipf,K", [((300, 200, 100), 30_000, (1.1, 1.1, 1.1), (8, 6, 5)),
                                          ((2000, 1500, 300), 60_000, (1.1, 1.1, 1.1), (10, 10, 10)),
                                          ((400, 300, 60, 20), 100_000, (1.2, 1.2, None, None), (6, 5, 4, 3))])
def test_lanczos_factor_update_matches_oracle(L, nnz, zipf, K, prec):
    c = case(L, nnz, zipf, "lognormal", seed=71)
    tk = make(c, K, prec, svd="lanczos")
    _, Fo = factors(L, K, 7, prec)
    for n in range(len(L)):
        Zo = O.ttm_chain(L, c["idx"], c["vals"].astype(np.float64), Fo, n)
        rid = np.flatnonzero(np.bincount(c["idx"][n], minlength=L[n]) > 0)
        Zc = Zo[rid].astype(NP[prec]).astype(np.float64)
        Zfull = np.zeros_like(Zo)
        Zfull[rid] = Zc
        F, sigma = tk.factor_update(n, torch.from_numpy(Zc).to(DT[prec]).cuda())
        torch.cuda.synchronize()
        Uo, so = O.lanczos_factor(Zfull, K[n])
        Fg = to_np(F)
        assert O.projector_distance(Fg, Uo) <= PROJ[prec], n
        assert rel_err(sigma.cpu().numpy(), so) <= SIG[prec], n
        assert np.abs(Fg.T @ Fg - np.eye(K[n])).max() <= (1e-12 if prec == "fp64" else 1e-5)
        assert not np.any(Fg[np.setdiff1d(np.arange(L[n]), rid)])
        for k in range(K[n]):
            assert Fg[np.argmax(np.abs(Fg[:, k])), k] > 0
    tk.close()


def test_lanczos_route_differs_from_the_exact_route_only_by_the_truncated_iteration():
    """With 2K steps the route approximates the leading subspace: close to the
    exact factor on a tensor with a clear spectral gap, and exactly equal to
    the oracle's Lanczos result, not to the exact one, where they differ."""
    c = case((300, 200, 100), 30_000, (1.1, 1.1, 1.1), "lognormal", seed=72)
    K = (8, 6, 5)
    tk = make(c, K, "fp64", svd="lanczos")
    _, Fo = factors(c["L"], K, 8, "fp64")
    Zo = O.ttm_chain(c["L"], c["idx"], c["vals"].astype(np.float64), Fo, 0)
    rid = np.flatnonzero(np.bincount(c["idx"][0], minlength=c["L"][0]) > 0)
    F, _ = tk.factor_update(0, torch.from_numpy(Zo[rid]).cuda())
    Fg = to_np(F)
    Ul, _ = O.lanczos_factor(Zo, K[0])
    Ue, _ = O.leading_left_singular_vectors(Zo, K[0])
    d_l, d_e = O.projector_distance(Fg, Ul), O.projector_distance(Fg, Ue)
    assert d_l <= 1e-8
    assert d_l < 1e-3 * max(d_e, 1e-300) or d_e <= 1e-8
    tk.close()


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_hooi_on_the_lanczos_route_matches_oracle(prec):
    c = case((300, 200, 100), 30_000, (1.1, 1.1, 1.1), "lognormal", seed=73)
    K = (6, 5, 4)
    _, F0 = factors(c["L"], K, 9, prec)
    tk = make(c, K, prec, svd="lanczos")
    F = [torch.from_numpy(np.ascontiguousarray(f, dtype=NP[prec])).cuda() for f in F0]
    for _ in range(3):
        _, fit = tk.hooi_iter(F)
    Fg = [to_np(f) for f in F]
    tk.close()
    Fo, _, fito = O.hooi(c["L"], c["idx"], c["vals"].astype(np.float64), F0, iters=3, svd="lanczos")
    for m in range(3):
        assert O.projector_distance(Fg[m], Fo[m]) <= (1e-8 if prec == "fp64" else 2e-4), m
    assert abs(fit - fito) <= (1e-10 if prec == "fp64" else 1e-6)
