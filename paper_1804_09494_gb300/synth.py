"""Seeded synthetic inputs for the sparse-Tucker hot path.

This module only *draws inputs*: COO tensors shaped like the paper's FROSTT
workloads (Section 7, dataset table) and initial factor matrices.  It holds
none of the method's arithmetic, and both the CUDA path's tests/bench and the
CPU oracle receive the very same arrays from it.

Recipe (every workload):
* coordinates per mode are either uniform on [0, L_m) or Zipf(s): rank k in
  1..L_m drawn with probability proportional to k^-s by inverse CDF, then
  mapped through a seeded random permutation of [0, L_m) so that the heavy
  slices sit at random positions;
* duplicate coordinates are removed (first draw wins, draw order kept) and the
  tensor is topped up with fresh draws until it holds exactly ``nnz`` distinct
  elements;
* values are drawn as float64 and rounded to float32, so the FP32 and FP64
  forms of the method see the identical tensor;
* every random stream is a numpy PCG64 generator seeded from (seed, purpose).
"""
from __future__ import annotations

import numpy as np

# Named workloads.  Sizes follow the configurations the method is measured on.
WORKLOADS = {
    # 3-mode 200x150x100, 20,000 uniform distinct nonzeros, U(0,1) values, core 8^3.
    "uniform-200x150x100-nnz20k-k8": dict(
        L=(200, 150, 100), nnz=20_000, zipf=(None, None, None), values="uniform", K=(8, 8, 8), seed=0),
    # 3-mode 2M x 1M x 50K, 100M nonzeros, Zipf s=1.1 per mode, lognormal(0,1) values, core 10^3.
    "zipf1.1-2Mx1Mx50K-nnz100M-k10": dict(
        L=(2_000_000, 1_000_000, 50_000), nnz=100_000_000, zipf=(1.1, 1.1, 1.1), values="lognormal",
        K=(10, 10, 10), seed=1),
    # 4-mode 1M x 500K x 20K x 2K, 500M nonzeros, Zipf 1.2 on modes 1-2, uniform on 3-4, core 10^4.
    "zipf1.2-1Mx500Kx20Kx2K-nnz500M-k10": dict(
        L=(1_000_000, 500_000, 20_000, 2_000), nnz=500_000_000, zipf=(1.2, 1.2, None, None),
        values="uniform", K=(10, 10, 10, 10), seed=2),
    # 3-mode 500K x 500K x 10K, 20M nonzeros, Zipf 1.1, core 16^3 (differentiable TTM-chain).
    "zipf1.1-500Kx500Kx10K-nnz20M-k16": dict(
        L=(500_000, 500_000, 10_000), nnz=20_000_000, zipf=(1.1, 1.1, 1.1), values="uniform",
        K=(16, 16, 16), seed=3),
    # finite-difference instance: 50x40x30, 2,000 uniform nonzeros.
    "uniform-50x40x30-nnz2000-k16": dict(
        L=(50, 40, 30), nnz=2_000, zipf=(None, None, None), values="uniform", K=(16, 16, 16), seed=3),
    # 4-mode 4M x 4M x 100K x 1K, 1.5B nonzeros, Zipf 1.3, core 8^4.
    "zipf1.3-4Mx4Mx100Kx1K-nnz1500M-k8": dict(
        L=(4_000_000, 4_000_000, 100_000, 1_000), nnz=1_500_000_000, zipf=(1.3, 1.3, 1.3, 1.3),
        values="uniform", K=(8, 8, 8, 8), seed=4),
}


def _rng(seed, *purpose):
    return np.random.Generator(np.random.PCG64(np.random.SeedSequence([int(seed), *[int(p) for p in purpose]])))


class ZipfSampler:
    """Inverse-CDF sampler of Zipf(s) ranks on 1..L followed by a seeded
    permutation of the index space."""

    def __init__(self, L, s, seed, mode):
        import torch
        self.L = int(L)
        w = np.arange(1, self.L + 1, dtype=np.float64) ** (-float(s))
        cdf = np.cumsum(w)
        self.cdf = torch.from_numpy(cdf / cdf[-1])
        self.perm = torch.from_numpy(_rng(seed, 1000 + mode).permutation(self.L).astype(np.int32))

    def draw(self, u):
        import torch
        k = torch.searchsorted(self.cdf, torch.from_numpy(u), right=True)
        k.clamp_(max=self.L - 1)
        return self.perm[k].numpy()


def _draw_coords(L, zipf, samplers, rng, n):
    out = np.empty((len(L), n), dtype=np.int32)
    for m, (Lm, s) in enumerate(zip(L, zipf)):
        if s is None:
            out[m] = rng.integers(0, Lm, size=n, dtype=np.int64).astype(np.int32)
        else:
            out[m] = samplers[m].draw(rng.random(n))
    return out


def _keys(L, idx):
    key = np.zeros(idx.shape[1], dtype=np.int64)
    for m in reversed(range(len(L))):
        key *= np.int64(L[m])
        key += idx[m].astype(np.int64)
    return key


def _first_occurrences(keys):
    """Positions of the first occurrence of every distinct key, in draw order."""
    import torch
    k = torch.from_numpy(keys)
    sk, perm = torch.sort(k, stable=True)
    first = torch.ones(len(sk), dtype=torch.bool)
    first[1:] = sk[1:] != sk[:-1]
    return torch.sort(perm[first]).values.numpy()


def coo(L, nnz, zipf=None, values="uniform", seed=0):
    """Distinct-coordinate COO tensor: returns (idx int32 (N, nnz), vals float32 (nnz,))."""
    L = tuple(int(x) for x in L)
    N = len(L)
    if zipf is None:
        zipf = (None,) * N
    total = 1
    for x in L:
        total *= x
    if nnz > total:
        raise ValueError("more nonzeros than cells")
    samplers = [ZipfSampler(L[m], zipf[m], seed, m) if zipf[m] is not None else None for m in range(N)]
    rng = _rng(seed, 1)
    idx = np.zeros((N, 0), dtype=np.int32)
    keys = np.zeros(0, dtype=np.int64)
    rounds = 0
    frac_new = 1.0  # fraction of the last round's draws that were new distinct cells
    while keys.size < nnz:
        extra = int((nnz - keys.size) / max(frac_new, 0.02) * 1.1) + 1024
        new = _draw_coords(L, zipf, samplers, rng, extra)
        allk = np.concatenate([keys, _keys(L, new)])
        first = _first_occurrences(allk)
        frac_new = (len(first) - keys.size) / extra
        first = first[:nnz]
        idx = np.concatenate([idx, new], axis=1)[:, first]
        keys = allk[first]
        rounds += 1
        if rounds > 64:
            raise RuntimeError("could not draw enough distinct coordinates")
    vrng = _rng(seed, 2)
    if values == "uniform":
        vals = vrng.random(nnz)
    elif values == "lognormal":
        vals = vrng.lognormal(0.0, 1.0, nnz)
    else:
        raise ValueError(values)
    return np.ascontiguousarray(idx), vals.astype(np.float32)


def workload(name, nnz=None):
    """Draw a named workload (optionally with fewer nonzeros, same recipe).
    Returns dict(L, K, idx, vals, name)."""
    w = WORKLOADS[name]
    n = w["nnz"] if nnz is None else int(nnz)
    idx, vals = coo(w["L"], n, w["zipf"], w["values"], w["seed"])
    return dict(name=name, L=tuple(w["L"]), K=tuple(w["K"]), idx=idx, vals=vals)


def random_orthonormal_factors(L, K, seed, dtype=np.float64):
    """Seeded Gaussian L_m x K_m matrices, orthonormalised by QR (random
    bootstrap of Section 2.2).  Column signs fixed so that R has a positive
    diagonal."""
    F = []
    for m, (Lm, Km) in enumerate(zip(L, K)):
        A = _rng(seed, 3000 + m).standard_normal((int(Lm), int(Km)))
        Q, R = np.linalg.qr(A)
        Q = Q * np.sign(np.where(np.diag(R) == 0, 1.0, np.diag(R)))[None, :]
        F.append(Q.astype(dtype))
    return F
