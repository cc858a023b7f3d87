"""Pins of the oracle's Lanczos bidiagonalisation route (Section 3 "SVD
component", Section 7: 2K iterations): the Lanczos relations, exactness when
the Krylov space is the whole row space, Ritz values bounded by the singular
values, and recovery of a planted rank-K matrix in 2K steps."""
import numpy as np
import pytest

from oracle import tucker_oracle as O


def _decaying(R, kh, seed, decay=0.8):
    rng = np.random.default_rng(seed)
    A, _ = np.linalg.qr(rng.standard_normal((R, kh)))
    B, _ = np.linalg.qr(rng.standard_normal((kh, kh)))
    return (A * decay ** np.arange(kh)) @ B.T


def test_lanczos_relations_hold():
    Z = _decaying(300, 40, 1)
    U, V, a, b = O.lanczos_bidiagonalization(Z, 12, np.ones(40))
    m = len(a)
    B = np.diag(a) + np.diag(b[: m - 1], 1)
    assert np.linalg.norm(Z @ V - U @ B) <= 1e-12 * np.linalg.norm(Z)
    assert np.linalg.norm(U.T @ U - np.eye(m)) <= 1e-12
    assert np.linalg.norm(V.T @ V - np.eye(m)) <= 1e-12


def test_full_iteration_gives_the_exact_svd():
    Z = _decaying(200, 30, 2, decay=0.9)
    U, V, a, b = O.lanczos_bidiagonalization(Z, 30, np.ones(30))
    B = np.diag(a) + np.diag(b[:29], 1)
    s_lanczos = np.linalg.svd(B, compute_uv=False)
    s_exact = np.linalg.svd(Z, compute_uv=False)
    assert np.allclose(s_lanczos, s_exact, rtol=1e-11, atol=1e-13)
    F, s = O.lanczos_factor(Z, 6, m=30)
    E, se = O.leading_left_singular_vectors(Z, 6)
    assert O.projector_distance(F, E) <= 1e-9 and np.allclose(s, se, rtol=1e-11)


def test_ritz_values_are_bounded_by_the_singular_values():
    Z = _decaying(400, 60, 3)
    _, _, a, b = O.lanczos_bidiagonalization(Z, 10, np.ones(60))
    B = np.diag(a) + np.diag(b[:9], 1)
    s_ritz = np.linalg.svd(B, compute_uv=False)
    s_exact = np.linalg.svd(Z, compute_uv=False)
    assert np.all(s_ritz <= s_exact[:10] * (1 + 1e-12))
    # the largest converges first
    assert s_ritz[0] >= 0.99 * s_exact[0]


@pytest.mark.parametrize("K", [3, 5])
def test_planted_rank_K_is_recovered_in_2K_steps(K):
    rng = np.random.default_rng(K)
    A, _ = np.linalg.qr(rng.standard_normal((250, K)))
    B, _ = np.linalg.qr(rng.standard_normal((50, K)))
    Z = A @ np.diag(np.linspace(3, 1, K)) @ B.T
    F, s = O.lanczos_factor(Z, K)
    assert O.projector_distance(F, A) <= 1e-10
    assert np.allclose(s, np.linspace(3, 1, K), rtol=1e-10)


def test_empty_rows_stay_zero():
    Z = _decaying(100, 20, 4)
    Z[[3, 50, 77]] = 0.0
    F, _ = O.lanczos_factor(Z, 4)
    assert np.all(F[[3, 50, 77]] == 0.0)
    assert np.linalg.norm(F.T @ F - np.eye(4)) <= 1e-12
