"""GPU parity of the tensor-core TTM-chain (eq. (1) as per-slice MMAs over
8-element blocks, 3xTF32 in two MMAs) against the FP64 oracle, and against the CUDA-core
form of the same context options: 4-mode FP32 tensors with K_a K_b in
[32, 128], K_c <= 48 and Khat >= 256 (N = 16 and N = 32 accumulator widths)."""
import numpy as np
import pytest
import torch

from tests.gpu_cases import DT, case, check_ttm, factors, make, rel_err

pytestmark = pytest.mark.gpu

CASES = [
    # (name, L, nnz, zipf, K): every mode, or only some, on the tensor cores
    ("k10-all-modes", (400, 300, 60, 20), 100_000, (1.2, 1.2, None, None), (10, 10, 10, 10)),
    ("k8-all-modes", (500, 500, 80, 30), 80_000, (1.3, 1.3, 1.3, 1.3), (8, 8, 8, 8)),
    ("mixed-eligibility", (300, 250, 200, 150), 60_000, (1.1, 1.1, 1.1, 1.1), (6, 8, 6, 7)),
    ("n-side-32", (200, 150, 120, 400), 50_000, (1.1, None, 1.1, None), (4, 8, 8, 20)),
]


def _expected_tc(K, n):
    o = [m for m in range(4) if m != n]
    Mu, Nu = K[o[0]] * K[o[1]], K[o[2]]
    return 32 <= Mu <= 128 and Nu <= 48 and Mu * Nu >= 256


@pytest.mark.parametrize("name,L,nnz,zipf,K", CASES, ids=[c[0] for c in CASES])
def test_tensor_core_ttm_chain_matches_oracle(name, L, nnz, zipf, K):
    c = case(L, nnz, zipf, "uniform", seed=21)
    tk = make(c, K, "fp32")
    Fd, Fo = factors(L, K, 7, "fp32")
    for n in range(4):
        form = tk.ttm_form(n)
        assert form["tensor_cores"] == _expected_tc(K, n), (n, form)
        if form["tensor_cores"]:
            # padded copy: at least nnz / 8 blocks, at most one partial block per segment more
            st = tk.stats(n)
            assert nnz <= 8 * form["blocks"] <= nnz + 7 * st["R_sum"]
        check_ttm(tk, c, Fd, Fo, n, "fp32")
    tk.close()


@pytest.mark.parametrize("P", [32, 96, 512])
def test_tensor_core_ttm_chain_split_slices(P):
    """Few bins: the Zipf heads split over many bins, so most segments are
    head / tail pieces whose partials the fix-up adds in bin order."""
    c = case((2000, 1500, 100, 40), 400_000, (1.2, 1.2, None, None), "lognormal", seed=22)
    K = (10, 10, 10, 10)
    tk = make(c, K, "fp32", P_bins=P)
    Fd, Fo = factors(c["L"], K, 8, "fp32")
    for n in range(4):
        assert tk.ttm_form(n)["tensor_cores"]
        check_ttm(tk, c, Fd, Fo, n, "fp32")
    tk.close()


def test_tensor_core_and_cuda_core_forms_agree():
    c = case((800, 600, 100, 50), 200_000, (1.2, 1.2, None, None), "uniform", seed=23)
    K = (10, 10, 10, 10)
    tk = make(c, K, "fp32")
    tc = make(c, K, "fp32", ttm_path="cuda_cores")
    Fd, _ = factors(c["L"], K, 9, "fp32")
    for n in range(4):
        assert tk.ttm_form(n)["tensor_cores"] and not tc.ttm_form(n)["tensor_cores"]
        Z1, r1 = tk.ttm_chain(n, Fd)
        Z2, r2 = tc.ttm_chain(n, Fd)
        assert torch.equal(r1, r2)
        assert rel_err(Z1.double().cpu().numpy(), Z2.double().cpu().numpy()) <= 4e-6
    tk.close()
    tc.close()


def test_tensor_core_ttm_chain_is_deterministic():
    c = case((800, 600, 100, 50), 200_000, (1.2, 1.2, None, None), "uniform", seed=24)
    K = (8, 8, 8, 8)
    tk = make(c, K, "fp32", P_bins=128)
    Fd, _ = factors(c["L"], K, 10, "fp32")
    for n in range(4):
        Z1, _ = tk.ttm_chain(n, Fd)
        Z2, _ = tk.ttm_chain(n, Fd)
        assert torch.equal(Z1, Z2)
    tk.close()


def test_tensor_core_ttm_chain_value_override():
    c = case((300, 200, 80, 40), 40_000, (1.1, 1.1, None, None), "uniform", seed=25)
    K = (10, 10, 10, 10)
    tk = make(c, K, "fp32")
    Fd, Fo = factors(c["L"], K, 11, "fp32")
    v = np.random.default_rng(1).standard_normal(len(c["vals"])).astype(np.float32).astype(np.float64)
    vd = torch.from_numpy(v).to(DT["fp32"]).cuda()
    for n in range(4):
        assert tk.ttm_form(n)["tensor_cores"]
        check_ttm(tk, c, Fd, Fo, n, "fp32", vals=vd, vals_np=v)
    tk.close()


def test_tensor_core_ttm_chain_sparse_and_ragged():
    """Very few elements: most bins empty, most CTAs with an empty range, every
    slice a handful of elements (one padded block each)."""
    c = case((40, 40, 40, 40), 300, None, "uniform", seed=26)
    K = (8, 8, 8, 8)
    tk = make(c, K, "fp32")
    Fd, Fo = factors(c["L"], K, 12, "fp32")
    for n in range(4):
        assert tk.ttm_form(n)["tensor_cores"]
        check_ttm(tk, c, Fd, Fo, n, "fp32")
    tk.close()


def test_tensor_core_ttm_chain_forced_wait_cap_reports_timeout():
    """wait_cap = -1 makes every mbarrier wait give up at once, including the
    tensor-core TTM-chain's (its MMA issuer's single-thread waits too): a whole
    invocation on a 4-mode context whose every mode takes the tensor cores
    reports TUCKER_ERR_TIMEOUT at its synchronising end, and a context without
    the cap then matches the oracle on the same GPU."""
    from paper_1804_09494_gb300.tucker import TuckerError
    c = case((400, 300, 60, 20), 60_000, (1.2, 1.2, None, None), "uniform", seed=25)
    K = (10, 10, 10, 10)
    Fd, Fo = factors(c["L"], K, 9, "fp32")
    tk = make(c, K, "fp32", wait_cap=-1)
    assert all(tk.ttm_form(n)["tensor_cores"] for n in range(4))
    with pytest.raises(TuckerError) as e:
        tk.hooi_iter([f.clone() for f in Fd], want_fit=True)
    assert e.value.status == "ERR_TIMEOUT", str(e.value)
    tk.close()
    tk = make(c, K, "fp32")
    for n in range(4):
        check_ttm(tk, c, Fd, Fo, n, "fp32")
    tk.close()
