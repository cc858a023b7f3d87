"""Differentiation end to end: the Tucker loss on the nonzeros,
    loss(G, F) = sum_e (val_e - xhat_e)^2,  xhat_e = <F_n[l_n] G_(n), Kron_n(e)>,
optimised by gradient steps through the library's autograd functions
(KronGather's forward is the adjoint of the TTM-chain in the values, its
backward the TTM-chain with the residual as values plus the adjoint in the
factors).  The values are those of a planted Tucker model on a sparse
support, so the loss can fall to rounding level."""
import numpy as np
import pytest
import torch

from paper_1804_09494_gb300 import synth
from paper_1804_09494_gb300.tucker import KronGather
from tests.gpu_cases import make

pytestmark = pytest.mark.gpu


def _unfold_core(G, n):
    """G_(n): K_n x prod_{m != n} K_m, the first remaining mode fastest."""
    N = G.dim()
    others = [m for m in range(N) if m != n]
    # column index c_{o0} + K_{o0} c_{o1} + ...: reversed order of the other modes, row-major
    return G.permute(n, *reversed(others)).reshape(G.shape[n], -1)


def _planted(L, K, nnz, seed):
    c = synth.coo(L, nnz, None, "uniform", seed)
    idx = c[0]
    F = synth.random_orthonormal_factors(L, K, seed + 1)
    G = np.random.default_rng(seed + 2).standard_normal(K)
    x = np.einsum("abc,ea,eb,ec->e", G, F[0][idx[0]], F[1][idx[1]], F[2][idx[2]])
    return dict(L=tuple(L), idx=idx, vals=x), F, G


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_gradient_steps_reduce_the_nonzero_loss(prec):
    L, K = (60, 50, 40), (4, 3, 5)
    c, F_true, G_true = _planted(L, K, 8000, seed=40)
    tk = make(c, K, prec)
    dt = torch.float64 if prec == "fp64" else torch.float32
    vals = torch.from_numpy(c["vals"]).to(dt).cuda()
    rng = np.random.default_rng(41)
    # start near the planted model (the loss is not convex in (G, F))
    F = [torch.tensor(f + 0.05 * rng.standard_normal(f.shape), dtype=dt, device="cuda", requires_grad=True)
         for f in F_true]
    G = torch.tensor(G_true + 0.2 * rng.standard_normal(K), dtype=dt, device="cuda", requires_grad=True)
    _, rid = tk.ttm_chain(0, [f.detach() for f in F])
    rid = rid.long()
    opt = torch.optim.Adam(F + [G], lr=0.01)
    losses = []
    for step in range(150):
        opt.zero_grad()
        W = F[0][rid] @ _unfold_core(G, 0)
        xhat = KronGather.apply(tk, 0, W, *F)
        loss = ((vals - xhat) ** 2).sum()
        loss.backward()
        opt.step()
        losses.append(float(loss.detach()))
    tk.close()
    assert all(np.isfinite(losses))
    assert losses[-1] < 1e-4 * losses[0], (losses[0], losses[-1])
    # steadily downhill: every window of 30 steps ends below where it started
    for s in range(0, 120, 30):
        assert losses[s + 30] < losses[s], (s, losses[s], losses[s + 30])


def test_kron_gather_gradient_matches_dense_autograd():
    """The gradient of the loss through KronGather equals the one torch
    computes for the same loss written with dense einsums (FP64)."""
    L, K = (30, 25, 20), (3, 4, 2)
    c, F_true, G_true = _planted(L, K, 1500, seed=50)
    tk = make(c, K, "fp64")
    vals = torch.from_numpy(c["vals"]).cuda()
    rng = np.random.default_rng(51)
    F0 = [f + 0.1 * rng.standard_normal(f.shape) for f in F_true]
    G0 = G_true + 0.3 * rng.standard_normal(K)
    idx = [torch.from_numpy(i.astype(np.int64)).cuda() for i in c["idx"]]

    def grads(use_lib):
        F = [torch.tensor(f, device="cuda", requires_grad=True) for f in F0]
        G = torch.tensor(G0, device="cuda", requires_grad=True)
        if use_lib:
            _, rid = tk.ttm_chain(0, [f.detach() for f in F])
            W = F[0][rid.long()] @ _unfold_core(G, 0)
            xhat = KronGather.apply(tk, 0, W, *F)
        else:
            xhat = torch.einsum("abc,ea,eb,ec->e", G, F[0][idx[0]], F[1][idx[1]], F[2][idx[2]])
        loss = ((vals - xhat) ** 2).sum()
        loss.backward()
        return [f.grad.cpu().numpy() for f in F] + [G.grad.cpu().numpy()], float(loss)

    g_lib, l_lib = grads(True)
    g_ref, l_ref = grads(False)
    tk.close()
    assert abs(l_lib - l_ref) <= 1e-10 * max(1.0, abs(l_ref))
    for a, b in zip(g_lib, g_ref):
        assert np.linalg.norm(a - b) <= 1e-9 * max(1.0, np.linalg.norm(b))
