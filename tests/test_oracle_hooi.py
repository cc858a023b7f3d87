"""Pins for the oracle's SVD step, HOOI (Fig. 1), core, fit and HOSVD bootstrap.

Independent checks: planted subspaces, Eckart-Young, exact recovery of tensors
of exact multilinear rank, the Pythagoras identity with a dense residual, and a
dense brute-force HOOI that goes through dense unfoldings instead of eq. (1)."""
import numpy as np
import pytest

from oracle import tucker_oracle as O


def _rand_coo(rng, L, nnz):
    flat = rng.choice(int(np.prod(L)), size=nnz, replace=False)
    idx = np.array(np.unravel_index(flat, L, order="F"), dtype=np.int64)
    return idx, rng.random(nnz)


def _dense(L, idx, vals):
    T = np.zeros(L)
    T[tuple(idx)] = vals
    return T


def _orth(rng, n, k):
    Q, _ = np.linalg.qr(rng.standard_normal((n, k)))
    return Q


def test_planted_subspace_recovered():
    rng = np.random.default_rng(0)
    A = _orth(rng, 40, 12)
    B = _orth(rng, 12, 12)
    s = np.linspace(10, 1, 12)
    Z = A @ np.diag(s) @ B.T
    U, sig = O.leading_left_singular_vectors(Z, 4)
    assert O.projector_distance(U, A[:, :4]) < 1e-12
    np.testing.assert_allclose(sig, s[:4], rtol=1e-12)
    np.testing.assert_allclose(U.T @ U, np.eye(4), atol=1e-13)


def test_eckart_young_residual():
    rng = np.random.default_rng(1)
    Z = rng.standard_normal((30, 9))
    U, _ = O.leading_left_singular_vectors(Z, 3)
    lam = np.sort(np.linalg.eigvalsh(Z.T @ Z))[::-1]
    res = np.linalg.norm(Z - U @ (U.T @ Z)) ** 2
    assert abs(res - lam[3:].sum()) < 1e-10 * lam.sum()


def test_sign_rule():
    U = np.array([[0.6, -0.8], [-0.8, -0.6]])
    S = O.sign_normalise(U)
    np.testing.assert_array_equal(S, np.array([[-0.6, 0.8], [0.8, 0.6]]))
    T = O.sign_normalise(np.array([[-0.5], [0.5]]))  # tie: lowest row decides
    np.testing.assert_array_equal(T, np.array([[0.5], [-0.5]]))


def test_projector_distance_properties():
    rng = np.random.default_rng(2)
    A = _orth(rng, 10, 3)
    R = _orth(rng, 3, 3)
    assert O.projector_distance(A, A @ R) < 1e-14
    E = np.eye(6)
    assert abs(O.projector_distance(E[:, :2], E[:, 2:4]) - 1.0) < 1e-15
    th = 1e-3
    B = np.array([[np.cos(th)], [np.sin(th)], [0.0]])
    assert abs(O.projector_distance(np.eye(3)[:, :1], B) - np.sin(th)) < 1e-15
    assert abs(O.projector_distance(A, B if False else A) ) < 1e-15
    P1 = A @ A.T
    C = _orth(rng, 10, 3)
    assert abs(np.linalg.norm(P1 - C @ C.T, 2) - O.projector_distance(A, C)) < 1e-12


def _exact_rank_tensor(rng, L, K, live):
    """Sparse tensor of exact multilinear rank K: factors with only ``live[m]``
    nonzero rows, so T = [[C; A_1..A_N]] is nonzero only on a small block."""
    A = []
    for l, k, r in zip(L, K, live):
        M = np.zeros((l, k))
        rows = rng.choice(l, size=r, replace=False)
        M[rows] = rng.standard_normal((r, k))
        A.append(M)
    C = rng.standard_normal(K)
    T = C
    for m in range(len(L)):
        T = np.moveaxis(np.tensordot(T, A[m], axes=([m], [1])), -1, m)
    idx = np.array(np.nonzero(T))
    return idx, T[tuple(idx)], A


@pytest.mark.parametrize("L,K,live", [((30, 25, 20), (3, 4, 2), (6, 7, 5)),
                                      ((12, 10, 9, 8), (2, 2, 3, 2), (4, 3, 5, 4))])
def test_exact_multilinear_rank_recovered(L, K, live):
    rng = np.random.default_rng(4)
    idx, vals, A = _exact_rank_tensor(rng, L, K, live)
    assert len(vals) < np.prod(L) // 10  # genuinely sparse
    F0 = [_orth(rng, l, k) for l, k in zip(L, K)]
    F, G, fit = O.hooi(L, idx, vals, F0, iters=2)
    # ||T||^2 - ||G||^2 cancels to rounding here, so the fit identity is only
    # sqrt(eps)-accurate near 1; the dense residual pins exact recovery.
    assert abs(fit - 1.0) < 1e-6
    T = _dense(L, idx, vals)
    R = G.reshape(K, order="F")
    for m in range(len(L)):
        R = np.moveaxis(np.tensordot(R, F[m], axes=([m], [1])), -1, m)
    assert np.linalg.norm(T - R) < 1e-12 * np.linalg.norm(T)
    for m in range(len(L)):
        Q, _ = np.linalg.qr(A[m])
        assert O.projector_distance(F[m], Q) < 1e-10
        np.testing.assert_allclose(F[m].T @ F[m], np.eye(K[m]), atol=1e-12)


def test_pythagoras_with_dense_residual():
    rng = np.random.default_rng(5)
    L = (7, 6, 5)
    idx, vals = _rand_coo(rng, L, 60)
    F0 = [_orth(rng, l, 3) for l in L]
    F, G, fit = O.hooi(L, idx, vals, F0, iters=1)
    T = _dense(L, idx, vals)
    R = G.reshape((3, 3, 3), order="F")
    for m in range(3):
        R = np.moveaxis(np.tensordot(R, F[m], axes=([m], [1])), -1, m)
    t2 = np.sum(T * T)
    assert abs(t2 - (G @ G + np.sum((T - R) ** 2))) < 1e-12 * t2
    assert abs(fit - (1 - np.linalg.norm(T - R) / np.linalg.norm(T))) < 1e-12


def _dense_hooi(T, F0, iters, in_place=False):
    """HOOI on the dense tensor: TTM by tensordot, SVD of the dense unfolding.
    ``in_place`` = textbook (Gauss-Seidel) HOOI: mode n's TTM sees the factors
    already replaced earlier in the same sweep."""
    N = T.ndim
    F = [f.copy() for f in F0]
    for _ in range(iters):
        new = [f.copy() for f in F]
        for n in range(N):
            src = new if in_place else F
            Z = T
            for m in range(N):
                if m != n:
                    Z = np.moveaxis(np.tensordot(Z, src[m], axes=([m], [0])), -1, m)
            U, _, _ = np.linalg.svd(np.moveaxis(Z, n, 0).reshape(T.shape[n], -1), full_matrices=False)
            new[n] = U[:, : F[n].shape[1]]
        F = new
    G = T
    for m in range(N):
        G = np.moveaxis(np.tensordot(G, F[m], axes=([m], [0])), -1, m)
    return F, G


@pytest.mark.parametrize("L,K", [((9, 8, 7), (3, 2, 3)), ((6, 5, 4, 5), (2, 3, 2, 2))])
def test_hooi_matches_dense_bruteforce(L, K):
    rng = np.random.default_rng(6)
    idx, vals = _rand_coo(rng, L, int(np.prod(L)) // 3)
    F0 = [_orth(rng, l, k) for l, k in zip(L, K)]
    F, G, fit = O.hooi(L, idx, vals, F0, iters=3)
    Fd, Gd = _dense_hooi(_dense(L, idx, vals), F0, 3)
    for m in range(len(L)):
        assert O.projector_distance(F[m], Fd[m]) < 1e-9
    # align the dense factors' column signs to the oracle's, then compare the cores
    for m in range(len(L)):
        sgn = np.sign(np.sum(F[m] * Fd[m], axis=0))
        Gd = np.moveaxis(np.moveaxis(Gd, m, -1) * sgn, -1, m)
    np.testing.assert_allclose(G, Gd.reshape(-1, order="F"), rtol=1e-8, atol=1e-9)
    T = _dense(L, idx, vals)
    assert abs(fit - (1 - np.sqrt(np.sum(T * T) - np.sum(Gd * Gd)) / np.linalg.norm(T))) < 1e-10


@pytest.mark.parametrize("L,K", [((9, 8, 7), (3, 2, 3)), ((6, 5, 4, 5), (2, 3, 2, 2))])
def test_gauss_seidel_matches_dense_bruteforce(L, K):
    """The Gauss-Seidel variant against a dense HOOI that replaces each factor
    in place within the sweep; the Jacobi dense HOOI must land elsewhere, so a
    variant that silently kept the input factors fails here."""
    rng = np.random.default_rng(16)
    idx, vals = _rand_coo(rng, L, int(np.prod(L)) // 3)
    F0 = [_orth(rng, l, k) for l, k in zip(L, K)]
    F, G, fit = O.hooi(L, idx, vals, F0, iters=2, variant="gauss_seidel")
    T = _dense(L, idx, vals)
    Fd, Gd = _dense_hooi(T, F0, 2, in_place=True)
    Fj, _ = _dense_hooi(T, F0, 2, in_place=False)
    for m in range(len(L)):
        assert O.projector_distance(F[m], Fd[m]) < 1e-9
    assert max(O.projector_distance(F[m], Fj[m]) for m in range(1, len(L))) > 1e-6
    assert abs(fit - (1 - np.sqrt(np.sum(T * T) - np.sum(Gd * Gd)) / np.linalg.norm(T))) < 1e-10


def test_jacobi_invocation_uses_input_factors():
    """Fig. 1 writes every TTM-chain with the input factors: the new F_n of the
    Jacobi reading does not depend on the order in which modes are visited."""
    rng = np.random.default_rng(8)
    L = (8, 7, 6)
    idx, vals = _rand_coo(rng, L, 80)
    F0 = [_orth(rng, l, 2) for l in L]
    F = O.hooi_invocation(L, idx, vals, F0)
    for n in range(3):
        U, _ = O.leading_left_singular_vectors(O.ttm_chain(L, idx, vals, F0, n), 2)
        np.testing.assert_allclose(F[n], U, atol=1e-13)


def test_gauss_seidel_fit_nondecreasing():
    """Textbook (Gauss-Seidel) HOOI never decreases the fit: each step maximises ||G||."""
    rng = np.random.default_rng(9)
    L = (10, 9, 8)
    idx, vals = _rand_coo(rng, L, 150)
    F = [_orth(rng, l, 3) for l in L]
    prev = -np.inf
    for _ in range(5):
        F = O.hooi_invocation(L, idx, vals, F, variant="gauss_seidel")
        f = O.fit(vals, O.core(L, idx, vals, F))
        assert f >= prev - 1e-12
        prev = f


def test_hosvd_matches_dense_unfolding():
    rng = np.random.default_rng(10)
    L = (8, 7, 6)
    idx, vals = _rand_coo(rng, L, 90)
    T = _dense(L, idx, vals)
    F = O.hosvd_init(L, idx, vals, (3, 3, 2))
    for n in range(3):
        U, _, _ = np.linalg.svd(np.moveaxis(T, n, 0).reshape(L[n], -1), full_matrices=False)
        assert O.projector_distance(F[n], U[:, : F[n].shape[1]]) < 1e-10
