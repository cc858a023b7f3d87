"""Pins for the oracle's TTM-chain (eq. (1), Appendix A, Section 2.1).

Each test checks the oracle against something other than itself: a
hand-worked example, the dense mode-by-mode definition of TTM, or the
unfolding's column numbering written in Section 2.1."""
import numpy as np
import pytest

from oracle import tucker_oracle as O
from tests.conftest import read_golden


def _rand_coo(rng, L, nnz):
    total = int(np.prod(L))
    flat = rng.choice(total, size=nnz, replace=False)
    idx = np.array(np.unravel_index(flat, L, order="F"), dtype=np.int64)
    vals = rng.standard_normal(nnz)
    return idx, vals


def _dense(L, idx, vals):
    T = np.zeros(L)
    T[tuple(idx)] = vals
    return T


def _dense_ttm_chain(T, F, n):
    """T x_{m != n} F_m^T by mode products (Section 2.1 TTM: A x T_(m) refolded),
    then the mode-n unfolding with the first remaining mode fastest."""
    Z = T
    for m in range(T.ndim):
        if m == n:
            continue
        Z = np.moveaxis(np.tensordot(Z, F[m], axes=([m], [0])), -1, m)
    Y = np.moveaxis(Z, n, 0)
    return Y.reshape(Y.shape[0], -1, order="F")


def test_kron_appendix_a_golden():
    g = dict(read_golden("appA_kron.txt"))
    u1 = np.array(g["u1"], dtype=float)[None, :]
    u2 = np.array(g["u2"], dtype=float)[None, :]
    np.testing.assert_array_equal(O.kron_row([u1, u2])[0], np.array(g["kron"], dtype=float))


def test_ttm_hand_example_golden():
    rows = read_golden("ttm_hand_example.txt")
    L = tuple(int(x) for x in dict(rows)["L"])
    elems = [r for k, r in rows if k == "elem"]
    idx = np.array([[int(e[m]) for e in elems] for m in range(3)])
    vals = np.array([float(e[3]) for e in elems])
    F = []
    for key in ("F1", "F2", "F3"):
        t = dict(rows)[key]
        F.append(np.array(t[2:], dtype=float).reshape(int(t[0]), int(t[1])))
    t = dict(rows)["Z0"]
    Zexp = np.array(t[2:], dtype=float).reshape(int(t[0]), int(t[1]))
    np.testing.assert_array_equal(O.ttm_chain(L, idx, vals, F, 0), Zexp)


@pytest.mark.parametrize("L,K", [((5, 4), (2, 3)), ((4, 3, 5), (2, 3, 2)), ((3, 4, 2, 3), (2, 2, 2, 3)),
                                 ((3, 2, 4, 2, 3), (2, 1, 3, 2, 2))])
def test_ttm_chain_matches_dense_mode_products(L, K):
    rng = np.random.default_rng(7)
    nnz = int(np.prod(L)) // 2
    idx, vals = _rand_coo(rng, L, nnz)
    F = [rng.standard_normal((l, k)) for l, k in zip(L, K)]
    T = _dense(L, idx, vals)
    for n in range(len(L)):
        Z = O.ttm_chain(L, idx, vals, F, n)
        np.testing.assert_allclose(Z, _dense_ttm_chain(T, F, n), rtol=1e-13, atol=1e-13)


def test_unfolding_column_numbering_section_2_1():
    """With identity factors Z_(n) is the unfolding T_(n); its column for the
    fiber <l_j, j != n> must be sum_{j != n} l_j prod_{i != n, i < j} L_i."""
    rng = np.random.default_rng(3)
    L = (3, 4, 5, 2)
    idx, vals = _rand_coo(rng, L, 40)
    F = [np.eye(l) for l in L]
    for n in range(4):
        expect = np.zeros((L[n], int(np.prod(L)) // L[n]))
        for e in range(len(vals)):
            col = 0
            for j in range(4):
                if j == n:
                    continue
                stride = 1
                for i in range(j):
                    if i != n:
                        stride *= L[i]
                col += idx[j, e] * stride
            expect[idx[n, e], col] += vals[e]
        np.testing.assert_array_equal(O.ttm_chain(L, idx, vals, F, n), expect)


def test_slice_row_depends_only_on_its_slice():
    """Section 3: row Z_(n)[l,:] is determined by the elements of Slice_n^l only."""
    rng = np.random.default_rng(5)
    L = (6, 5, 4)
    idx, vals = _rand_coo(rng, L, 60)
    F = [rng.standard_normal((l, 3)) for l in L]
    Z = O.ttm_chain(L, idx, vals, F, 1)
    for l in range(L[1]):
        keep = idx[1] == l
        Zl = O.ttm_chain(L, idx[:, keep], vals[keep], F, 1)
        np.testing.assert_allclose(Zl[l], Z[l], rtol=1e-14, atol=1e-14)
        assert not np.any(np.delete(Zl, l, axis=0))


def test_core_definition_matches_dense():
    rng = np.random.default_rng(11)
    L = (5, 4, 3)
    idx, vals = _rand_coo(rng, L, 30)
    F = [rng.standard_normal((l, k)) for l, k in zip(L, (2, 3, 2))]
    T = _dense(L, idx, vals)
    G = T
    for m in range(3):
        G = np.moveaxis(np.tensordot(G, F[m], axes=([m], [0])), -1, m)
    np.testing.assert_allclose(O.core(L, idx, vals, F), G.reshape(-1, order="F"), rtol=1e-13, atol=1e-13)


def test_core_equals_projection_of_penultimate_matrix():
    """G_(n) = F_n^T Z_(n) for every n (the TTM-chain is order independent, Section 2.1)."""
    rng = np.random.default_rng(12)
    L = (5, 6, 4, 3)
    K = (2, 3, 2, 2)
    idx, vals = _rand_coo(rng, L, 70)
    F = [rng.standard_normal((l, k)) for l, k in zip(L, K)]
    G = O.core(L, idx, vals, F).reshape(K, order="F")
    for n in range(4):
        Gn = F[n].T @ O.ttm_chain(L, idx, vals, F, n)
        Y = np.moveaxis(G, n, 0).reshape(K[n], -1, order="F")
        np.testing.assert_allclose(Gn, Y, rtol=1e-12, atol=1e-12)
