"""GPU parity of the TTM-chain (eq. (1)), its split-slice fix-up and its
adjoint, through the C ABI, against the FP64 oracle."""
import numpy as np
import pytest
import torch

from oracle import tucker_oracle as O
from tests.gpu_cases import DT, TTM_TOL, case, check_ttm, factors, make, rel_err

pytestmark = pytest.mark.gpu

CASES = [
    # (name, L, nnz, zipf, values, K)
    ("uniform-3d-k8", (200, 150, 100), 20_000, None, "uniform", (8, 8, 8)),
    ("zipf-3d-k10", (3000, 2000, 500), 200_000, (1.1, 1.1, 1.1), "lognormal", (10, 10, 10)),
    ("zipf-3d-k16", (2000, 1500, 300), 60_000, (1.1, 1.1, 1.1), "uniform", (16, 16, 16)),
    ("zipf-4d-k10", (400, 300, 60, 20), 100_000, (1.2, 1.2, None, None), "uniform", (10, 10, 10, 10)),
    ("zipf-4d-k8", (500, 500, 80, 30), 80_000, (1.3, 1.3, 1.3, 1.3), "uniform", (8, 8, 8, 8)),
    ("generic-3d", (300, 200, 100), 30_000, (1.1, None, None), "uniform", (12, 6, 9)),
    ("matrix-2d", (500, 400), 20_000, (1.1, 1.1), "uniform", (6, 6)),
    ("five-mode", (30, 25, 20, 15, 10), 20_000, None, "uniform", (3, 2, 4, 2, 3)),
]


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("name,L,nnz,zipf,values,K", CASES, ids=[c[0] for c in CASES])
def test_ttm_chain_matches_oracle(name, L, nnz, zipf, values, K, prec):
    c = case(L, nnz, zipf, values, seed=11)
    tk = make(c, K, prec)
    Fd, Fo = factors(L, K, 5, prec)
    for n in range(len(L)):
        check_ttm(tk, c, Fd, Fo, n, prec)
    tk.close()


@pytest.mark.parametrize("P", [32, 64, 96, 1024])
def test_ttm_chain_small_bin_counts(P):
    """Few bins: most heavy slices split over many bins (several fix-up chunks,
    ragged last bins)."""
    c = case((5000, 3000, 400), 300_000, (1.1, 1.1, 1.1), "lognormal", seed=3)
    tk = make(c, (10, 10, 10), "fp32", P_bins=P)
    Fd, Fo = factors(c["L"], (10, 10, 10), 1, "fp32")
    for n in range(3):
        check_ttm(tk, c, Fd, Fo, n, "fp32")
    st = tk.stats(0)
    assert st["P"] == P
    tk.close()


def test_ttm_chain_is_deterministic():
    c = case((3000, 2000, 500), 200_000, (1.1, 1.1, 1.1), "lognormal", seed=4)
    tk = make(c, (10, 10, 10), "fp32", P_bins=256)
    Fd, _ = factors(c["L"], (10, 10, 10), 2, "fp32")
    for n in range(3):
        Z1, _ = tk.ttm_chain(n, Fd)
        Z2, _ = tk.ttm_chain(n, Fd)
        assert torch.equal(Z1, Z2)
    tk.close()


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_ttm_chain_value_override(prec):
    c = case((400, 300, 200), 30_000, (1.1, 1.1, 1.1), "uniform", seed=5)
    K = (8, 8, 8)
    tk = make(c, K, prec)
    Fd, Fo = factors(c["L"], K, 3, prec)
    v = np.random.default_rng(0).standard_normal(len(c["vals"])).astype(np.float32).astype(np.float64)
    vd = torch.from_numpy(v).to(DT[prec]).cuda()
    for n in range(3):
        check_ttm(tk, c, Fd, Fo, n, prec, vals=vd, vals_np=v)
    tk.close()


def test_ttm_chain_degenerate_shapes():
    # a single element; a mode of length one (every element in one slice)
    c = case((7, 5, 3), 1, None, "uniform", seed=6)
    tk = make(c, (1, 1, 1), "fp64")
    Fd, Fo = factors(c["L"], (1, 1, 1), 0, "fp64")
    for n in range(3):
        check_ttm(tk, c, Fd, Fo, n, "fp64")
    tk.close()
    c = case((1, 300, 200), 5_000, None, "uniform", seed=7)
    tk = make(c, (1, 5, 5), "fp32", P_bins=64)
    Fd, Fo = factors(c["L"], (1, 5, 5), 0, "fp32")
    for n in range(3):
        check_ttm(tk, c, Fd, Fo, n, "fp32")
    tk.close()


# ---------------------------------------------------------------- adjoint
ADJ = [("uniform-3d-k16", (50, 40, 30), 2_000, None, (16, 16, 16)),
       ("zipf-3d-k10", (600, 500, 100), 40_000, (1.1, 1.1, 1.1), (10, 10, 10)),
       ("zipf-4d-k8", (200, 150, 40, 20), 30_000, (1.3, 1.3, None, None), (8, 8, 8, 8)),
       ("generic-3d", (300, 200, 100), 20_000, None, (12, 6, 9))]


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("name,L,nnz,zipf,K", ADJ, ids=[a[0] for a in ADJ])
def test_adjoint_matches_oracle(name, L, nnz, zipf, K, prec):
    c = case(L, nnz, zipf, "uniform", seed=8)
    tk = make(c, K, prec)
    Fd, Fo = factors(L, K, 9, prec)
    rng = np.random.default_rng(1)
    v = c["vals"].astype(np.float64)
    tol = 1e-4 if prec == "fp32" else 1e-11
    for n in range(len(L)):
        R = tk.R[n]
        dZc = rng.standard_normal((R, O.khat(K, n))).astype(np.float32).astype(np.float64)
        rid = np.flatnonzero(np.bincount(c["idx"][n], minlength=L[n]) > 0)
        dZ = np.zeros((L[n], O.khat(K, n)))
        dZ[rid] = dZc
        dF, dval = tk.ttm_chain_backward(n, Fd, torch.from_numpy(dZc).to(DT[prec]).cuda())
        torch.cuda.synchronize()
        dval_o, dF_o = O.ttm_chain_adjoint(L, c["idx"], v, Fo, n, dZ)
        assert rel_err(dval.double().cpu().numpy(), dval_o) <= tol
        for m in range(len(L)):
            if m == n:
                continue
            assert rel_err(dF[m].double().cpu().numpy(), dF_o[m]) <= tol, (n, m)
    tk.close()


def test_adjoint_central_differences_fp64():
    """dL/dF_m and dL/dvals of L = <ttm_chain(vals, F), W> on the 50x40x30,
    2,000-element instance against FP64 central differences of the GPU forward."""
    c = case((50, 40, 30), 2_000, None, "uniform", seed=3)
    K = (16, 16, 16)
    tk = make(c, K, "fp64")
    Fd, Fo = factors(c["L"], K, 4, "fp64")
    rng = np.random.default_rng(2)
    for n in range(3):
        W = torch.from_numpy(rng.standard_normal((tk.R[n], O.khat(K, n)))).cuda()
        dF, dval = tk.ttm_chain_backward(n, Fd, W)

        def loss(F=Fd, vals=None):
            Z, _ = tk.ttm_chain(n, F, vals=vals, row_id=False)
            return float((Z * W).sum())

        for m in range(3):
            if m == n:
                continue
            i = int(c["idx"][m][17])
            for k in (0, 7, 15):
                x = float(Fd[m][i, k])
                h = 1e-6 * max(1.0, abs(x))
                Fp = [f.clone() for f in Fd]
                Fm = [f.clone() for f in Fd]
                Fp[m][i, k] = x + h
                Fm[m][i, k] = x - h
                fd = (loss(Fp) - loss(Fm)) / (2 * h)
                assert abs(fd - float(dF[m][i, k])) <= 1e-4 * max(1.0, abs(fd))
        vals = torch.from_numpy(c["vals"].astype(np.float64)).cuda()
        for e in (0, 999, 1999):
            vp, vm = vals.clone(), vals.clone()
            vp[e] += 1e-6
            vm[e] -= 1e-6
            fd = (loss(vals=vp) - loss(vals=vm)) / 2e-6
            assert abs(fd - float(dval[e])) <= 1e-4 * max(1.0, abs(fd))
    tk.close()


def test_autograd_functions_gradcheck_fp64():
    """TTMChain and KronGather (torch.autograd.Function wrappers of the two C
    entry points) pass torch.autograd.gradcheck in FP64 on a tiny tensor."""
    from paper_1804_09494_gb300.tucker import KronGather, TTMChain
    c = case((6, 5, 4), 30, None, "uniform", seed=9)
    K = (2, 3, 2)
    tk = make(c, K, "fp64")
    Fd, _ = factors(c["L"], K, 1, "fp64")
    vals = torch.from_numpy(c["vals"].astype(np.float64)).cuda().requires_grad_(True)
    Fg = [f.clone().requires_grad_(True) for f in Fd]
    for n in range(3):
        fF = [f if m != n else f.detach() for m, f in enumerate(Fg)]
        assert torch.autograd.gradcheck(lambda v, *F: TTMChain.apply(tk, n, v, *F), (vals, *fF), eps=1e-6, atol=1e-8)
        W = torch.randn(tk.R[n], O.khat(K, n), dtype=torch.float64, device="cuda", requires_grad=True)
        assert torch.autograd.gradcheck(lambda w, *F: KronGather.apply(tk, n, w, *F), (W, *fF), eps=1e-6, atol=1e-8)
    tk.close()


def test_invalid_inputs_are_rejected():
    from paper_1804_09494_gb300.tucker import TuckerError
    c = case((20, 10, 5), 100, None, "uniform", seed=1)
    bad = c["idx"].copy()
    bad[1, 7] = 10  # == L_1
    with pytest.raises(TuckerError) as ei:
        make(dict(c, idx=bad), (2, 2, 2), "fp32")
    assert ei.value.status == "ERR_INDEX"
    with pytest.raises(TuckerError) as ei:
        make(c, (2, 11, 2), "fp32")  # K_1 > L_1
    assert ei.value.status == "ERR_ARG"
    with pytest.raises(TuckerError) as ei:
        make(c, (2, 2, 2), "fp32", P_bins=-1)
    assert ei.value.status == "ERR_ARG"


FIBER_CASES = [
    # 3-mode, exact tiles (K_a x K_b = 8 x 8, 10 x 10, 16 x 16); in every mode the
    # fiber mode (the other mode with fewer slices) is the second remaining mode
    ("uniform-3d-k8", (200, 150, 100), 20_000, None, "uniform", (8, 8, 8)),
    ("zipf-3d-k10", (3000, 2000, 500), 200_000, (1.1, 1.1, 1.1), "lognormal", (10, 10, 10)),
    ("zipf-3d-k16", (2000, 1500, 300), 60_000, (1.1, 1.1, 1.1), "uniform", (16, 16, 16)),
]


@pytest.mark.parametrize("P", [0, 64])
@pytest.mark.parametrize("name,L,nnz,zipf,values,K", FIBER_CASES, ids=[c[0] for c in FIBER_CASES])
def test_fiber_factored_ttm_chain_matches_oracle(name, L, nnz, zipf, values, K, P):
    """The fiber-factored form (sum over a fiber of val F_a, expanded with the
    fiber's F_b row once) against the oracle, with the default bin count and
    with few bins (most heavy slices split)."""
    c = case(L, nnz, zipf, values, seed=12)
    tk = make(c, K, "fp32", ttm_path="fiber", P_bins=P)
    Fd, Fo = factors(L, K, 6, "fp32")
    for n in range(3):
        check_ttm(tk, c, Fd, Fo, n, "fp32")
    tk.close()


def test_fiber_factored_ttm_chain_value_override():
    c = case((400, 300, 200), 30_000, (1.1, 1.1, 1.1), "uniform", seed=13)
    K = (10, 10, 10)
    tk = make(c, K, "fp32", ttm_path="fiber")
    Fd, Fo = factors(c["L"], K, 3, "fp32")
    v = np.random.default_rng(2).standard_normal(len(c["vals"])).astype(np.float32).astype(np.float64)
    vd = torch.from_numpy(v).to(DT["fp32"]).cuda()
    for n in range(3):
        check_ttm(tk, c, Fd, Fo, n, "fp32", vals=vd, vals_np=v)
    tk.close()
