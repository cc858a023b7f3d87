"""Helpers shared by the GPU parity tests: seeded inputs (from the synthetic
input module) moved to the device, and comparisons against the oracle."""
import numpy as np
import torch

from oracle import tucker_oracle as O
from paper_1804_09494_gb300 import synth
from paper_1804_09494_gb300.tucker import Tucker

DT = {"fp32": torch.float32, "bf16x3": torch.float32, "fp64": torch.float64}
NP = {"fp32": np.float32, "bf16x3": np.float32, "fp64": np.float64}
# relative Frobenius tolerance of the TTM-chain: FP32 per the method's
# acceptance bound; FP64 from ~1e3 rounding steps of 1.1e-16
TTM_TOL = {"fp32": 1e-5, "fp64": 1e-12}
# per-row bound: max over rows of ||Z_r - Zo_r|| / ||Zo_r||.  A row sums at most
# one bin's worth of elements (<= ceil(nnz/P)) sequentially in the working
# precision, a relative rounding error of about eps * sqrt(n/2) (2e-6 in FP32
# at n = 2,600); dropping or doubling one element of a row of n elements moves
# it by about 1/sqrt(n) (2e-3 at n = 2e5), far above both bounds.
ROW_TOL = {"fp32": 5e-5, "fp64": 1e-11}


def case(L, nnz, zipf=None, values="uniform", seed=0):
    idx, vals = synth.coo(L, nnz, zipf, values, seed)
    return dict(L=tuple(L), idx=idx, vals=vals)


def make(c, K, prec, **kw):
    idx = torch.from_numpy(c["idx"]).cuda()
    vals = torch.from_numpy(c["vals"].astype(np.float64)).to(DT[prec]).cuda()
    return Tucker(idx, vals, c["L"], K, prec=prec, **kw)


def factors(L, K, seed, prec):
    """Seeded orthonormal factors rounded to the working precision, returned as
    (device tensors, float64 copies of the very same values for the oracle)."""
    F = synth.random_orthonormal_factors(L, K, seed)
    Fr = [f.astype(NP[prec]).astype(np.float64) for f in F]
    return [torch.from_numpy(f).to(DT[prec]).cuda() for f in Fr], Fr


def rel_err(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def row_rel_err(a, b):
    """max over rows of ||a_r - b_r|| / ||b_r|| (rows of b that are exactly zero
    must be exactly zero in a)."""
    na = np.linalg.norm(a - b, axis=1)
    nb = np.linalg.norm(b, axis=1)
    zero = nb == 0
    assert not np.any(na[zero] > 0), "a row that must be zero is not"
    return float(np.max(na[~zero] / nb[~zero])) if np.any(~zero) else 0.0


def check_ttm(tk, c, Fd, Fo, n, prec, vals=None, vals_np=None):
    Z, rid = tk.ttm_chain(n, Fd, vals=vals)
    torch.cuda.synchronize()
    v = c["vals"].astype(np.float64) if vals_np is None else vals_np
    Zo = O.ttm_chain(c["L"], c["idx"], v, Fo, n)
    cnt = np.bincount(c["idx"][n], minlength=c["L"][n])
    rid = rid.cpu().numpy()
    assert np.array_equal(rid, np.flatnonzero(cnt > 0)), "row ids differ from the non-empty slices"
    Zg = Z.double().cpu().numpy()
    err = rel_err(Zg, Zo[rid])
    assert err <= TTM_TOL[prec], (n, err)
    rerr = row_rel_err(Zg, Zo[rid])
    assert rerr <= ROW_TOL[prec], (n, "row", rerr)
    return Z, rid, Zo, err
