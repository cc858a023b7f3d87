"""GPU parity at the full sizes of the other workloads, in the launch
configuration of the library's defaults:
  * 4-mode 1M x 500K x 20K x 2K, 500M nonzeros (Zipf 1.2 on modes 1-2, uniform
    on 3-4), core 10^4 -- TTM-chain rows of every mode (Khat = 1000, ten
    column groups per element);
  * 3-mode 500K x 500K x 10K, 20M nonzeros (Zipf 1.1), core 16^3 -- TTM-chain
    rows and the adjoint (FP32 and FP64 contexts).
The oracle computes sampled rows of eq. (1) from the sampled slices' elements
alone (a bounded number of elements per mode).  The adjoint is checked element
by element on sampled entries: dval(e) for sampled elements (including a
heavy slice's) and whole rows dF_m[l] for sampled slices l of every other mode
(the heaviest below a budget, the lightest, random ones), each computed by the
oracle's adjoint from exactly the elements it depends on."""
import numpy as np
import pytest
import torch

from oracle import tucker_oracle as O
from paper_1804_09494_gb300 import synth
from paper_1804_09494_gb300.tucker import Tucker
from tests.gpu_cases import ROW_TOL, TTM_TOL, rel_err, row_rel_err

pytestmark = pytest.mark.gpu


def budget_slices(cnt, E_max, rng, budget):
    """Slices to check, within `budget` elements in total: first split slices
    (longer than one bin; the largest below budget/2, then two just longer
    than one bin), then the lightest slices, then random ones."""
    nz = np.flatnonzero(cnt > 0)
    by_size = nz[np.argsort(cnt[nz], kind="stable")]
    c = cnt[by_size]
    cand = []
    j = np.searchsorted(c, budget // 2, side="right") - 1
    if j >= 0 and c[j] > E_max:
        cand.append(by_size[j])
    j = np.searchsorted(c, E_max, side="right")
    cand += list(by_size[j:j + 2])
    cand += list(by_size[:6])
    cand += list(rng.choice(nz, size=min(24, nz.size), replace=False))
    pick, used = [], 0
    for s in cand:
        if s in pick:
            continue
        if used + cnt[s] > budget and pick:
            continue
        pick.append(s)
        used += int(cnt[s])
    return np.unique(np.array(pick, dtype=np.int64))


def oracle_rows(L, idx, vals, Fo, n, ids):
    sel = np.isin(idx[n], ids)
    sub = idx[:, sel].copy()
    sub[n] = np.searchsorted(ids, sub[n])
    Ls = list(L)
    Ls[n] = len(ids)
    return O.ttm_chain(tuple(Ls), sub, vals[sel].astype(np.float64), Fo, n)


def check_sampled_rows(tk, w, Fd, Fo, n, budget, seed):
    Z, rid = tk.ttm_chain(n, Fd)
    torch.cuda.synchronize()
    rid = rid.cpu().numpy()
    cnt = np.bincount(w["idx"][n], minlength=w["L"][n])
    assert np.array_equal(rid, np.flatnonzero(cnt > 0)), "row ids differ from the non-empty slices"
    ids = budget_slices(cnt, tk.stats(n)["E_max"], np.random.default_rng(seed), budget)
    rows = np.searchsorted(rid, ids)
    Zg = Z[torch.from_numpy(rows).cuda()].double().cpu().numpy()
    Zo = oracle_rows(w["L"], w["idx"], w["vals"], Fo, n, ids)
    assert rel_err(Zg, Zo) <= TTM_TOL["fp32"], (n, rel_err(Zg, Zo))
    assert row_rel_err(Zg, Zo) <= ROW_TOL["fp32"], (n, "row", row_rel_err(Zg, Zo))
    h = int(np.argmax(cnt[ids]))
    assert rel_err(Zg[h], Zo[h]) <= TTM_TOL["fp32"], (n, int(ids[h]), int(cnt[ids[h]]))


def load(name):
    w = synth.workload(name)
    F = synth.random_orthonormal_factors(w["L"], w["K"], seed=77)
    Fo = [f.astype(np.float32).astype(np.float64) for f in F]
    Fd = [torch.from_numpy(f).float().cuda() for f in Fo]
    tk = Tucker(torch.from_numpy(w["idx"]).cuda(), torch.from_numpy(w["vals"]).cuda(), w["L"], w["K"], prec="fp32")
    return w, Fo, Fd, tk


def test_fullsize_4mode_500M_ttm_chain_sampled_rows():
    w, Fo, Fd, tk = load("zipf1.2-1Mx500Kx20Kx2K-nnz500M-k10")
    try:
        for n in range(4):
            check_sampled_rows(tk, w, Fd, Fo, n, budget=600_000, seed=300 + n)
    finally:
        tk.close()


ADJ_TOL = {torch.float32: 1e-4, torch.float64: 1e-11}


def _sub_adjoint(L, idx, vals, Fo, n, W, rid, sel, m=None, ids_m=None):
    """Oracle adjoint of eq. (1) over the elements `sel` only: mode n's
    coordinates are renumbered to the distinct slices among them (their rows of
    W are the cotangent), and, for a dF_m check, mode m's to the sampled slices
    ids_m.  Returns (dval over sel, dF_m rows of ids_m or None)."""
    sub = idx[:, sel].astype(np.int64)
    ln = np.unique(sub[n])
    rows = np.searchsorted(rid, ln)
    assert np.array_equal(rid[rows], ln)
    sub[n] = np.searchsorted(ln, sub[n])
    Ls = list(L)
    Ls[n] = len(ln)
    F = list(Fo)
    F[n] = np.zeros((len(ln), Fo[n].shape[1]))
    if m is not None:
        sub[m] = np.searchsorted(ids_m, sub[m])
        Ls[m] = len(ids_m)
        F[m] = Fo[m][ids_m]
    dv, dF = O.ttm_chain_adjoint(tuple(Ls), sub, vals[sel].astype(np.float64), F, n, W[rows])
    return dv, sub, F, (dF[m] if m is not None else None)


def _adjoint_sampled(tk, w, Fd, Fo, n, g, dtype, seed, budget):
    """Element-wise parity of the adjoint: dval(e) within ADJ_TOL of the sum of
    |terms| of its dot product (an error bound of the dot product itself), and
    every sampled dF_m row within ADJ_TOL of the oracle row (relative)."""
    L, idx, vals = w["L"], w["idx"], w["vals"]
    tol = ADJ_TOL[dtype]
    R, kh = tk.R[n], tk.khat(n)
    Wd = torch.randn(R, kh, device="cuda", generator=g, dtype=torch.float64).to(dtype)
    W = Wd.double().cpu().numpy()
    dF, dval = tk.ttm_chain_backward(n, Fd, Wd)
    torch.cuda.synchronize()
    cnt_n = np.bincount(idx[n], minlength=L[n])
    rid = np.flatnonzero(cnt_n > 0)
    rng = np.random.default_rng(seed)
    # dval on random elements plus part of the heaviest slice of mode n
    heavy = int(np.argmax(cnt_n))
    hel = np.flatnonzero(idx[n] == heavy)
    sel = np.unique(np.concatenate([rng.choice(len(vals), 3000, replace=False), hel[:: max(1, len(hel) // 3000)]]))
    dv_o, sub, F, _ = _sub_adjoint(L, idx, vals, Fo, n, W, rid, sel)
    terms = np.abs(W[np.searchsorted(rid, idx[n][sel])]) * np.abs(O.kron_n(F, sub, n))
    scale = terms.sum(axis=1)
    err = np.abs(dval.double().cpu().numpy()[sel] - dv_o)
    assert np.all(err <= tol * scale), (n, "dval", float(np.max(err / scale)))
    for m in range(len(L)):
        if m == n:
            continue
        cnt_m = np.bincount(idx[m], minlength=L[m])
        ids = budget_slices(cnt_m, 0, rng, budget)
        selm = np.flatnonzero(np.isin(idx[m], ids))
        _, _, _, dFo = _sub_adjoint(L, idx, vals, Fo, n, W, rid, selm, m=m, ids_m=ids)
        dFg = dF[m][torch.from_numpy(ids).cuda()].double().cpu().numpy()
        assert row_rel_err(dFg, dFo) <= tol, (n, m, row_rel_err(dFg, dFo))


def test_fullsize_differentiable_20M_k16_rows_and_adjoint():
    """FP32 context: sampled TTM-chain rows against the oracle, and the adjoint
    element by element within 1e-4 (dF sums run in a fixed order, per bin in
    FP32 and across bins in FP64).  FP64 context on the same tensor: the
    adjoint within 1e-11."""
    w, Fo, Fd, tk = load("zipf1.1-500Kx500Kx10K-nnz20M-k16")
    try:
        g = torch.Generator(device="cuda").manual_seed(5)
        for n in range(3):
            check_sampled_rows(tk, w, Fd, Fo, n, budget=1_000_000, seed=400 + n)
            _adjoint_sampled(tk, w, Fd, Fo, n, g, torch.float32, seed=500 + n, budget=300_000)
    finally:
        tk.close()
    tk = Tucker(torch.from_numpy(w["idx"]).cuda(), torch.from_numpy(w["vals"]).double().cuda(), w["L"], w["K"],
                prec="fp64")
    try:
        g = torch.Generator(device="cuda").manual_seed(6)
        Fd64 = [torch.from_numpy(f).cuda() for f in Fo]
        for n in range(3):
            _adjoint_sampled(tk, w, Fd64, Fo, n, g, torch.float64, seed=600 + n, budget=200_000)
    finally:
        tk.close()


def test_fullsize_adjoint_is_deterministic():
    """The adjoint's sums run in a fixed order: two calls agree bit for bit."""
    w, Fo, Fd, tk = load("zipf1.1-500Kx500Kx10K-nnz20M-k16")
    try:
        g = torch.Generator(device="cuda").manual_seed(7)
        W = torch.randn(tk.R[0], tk.khat(0), device="cuda", generator=g)
        dF1, dv1 = tk.ttm_chain_backward(0, Fd, W)
        dF2, dv2 = tk.ttm_chain_backward(0, Fd, W)
        torch.cuda.synchronize()
        assert torch.equal(dv1, dv2)
        for m in (1, 2):
            assert torch.equal(dF1[m], dF2[m])
    finally:
        tk.close()
