"""Plain FP64 CPU oracle for the sparse-Tucker HOOI hot path.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import or run
anything in this package.  The product path (the CUDA library and its Python
binding) never calls it and shares no code with it.

Every function is written from the paper's definitions, in its notation
(Chakaravarthy et al., "On Optimizing Distributed Tucker Decomposition for
Sparse Tensors", arXiv:1804.09494), in float64, with no blocking or fusion
beyond chunking the element loop to bound memory:

* ``kron_row``            -- Appendix A (Kronecker vectorisation, first vector fastest)
* ``ttm_chain``           -- Section 3, eq. (1): Z_(n)[l,:] = sum_{e in Slice_n^l} val(e) Kron_n(e)
* ``leading_left_singular_vectors`` -- Section 2.2 / Fig. 1 "SVD" step
* ``lanczos_bidiagonalization``, ``lanczos_factor`` -- the paper's SVD route
                            (Section 3 "SVD component", Section 7: 2K iterations)
* ``hooi_invocation``     -- Fig. 1 (Jacobi reading: every mode uses the input factors)
* ``core``                -- Fig. 1 "New core": G = T x_1 F_1^T ... x_N F_N^T
* ``fit``                 -- Kolda-Bader fit via ||T - [[G;F]]||^2 = ||T||^2 - ||G||^2
* ``hosvd_init``          -- Section 2.2 bootstrap (HOSVD)
* ``ttm_chain_adjoint``   -- adjoint of eq. (1) w.r.t. the values and every F_m
* Lite partition          -- see ``oracle/lite_oracle.py`` (Section 6.1, Fig. 7)

Conventions: indices are 0-based (the paper is 1-based); a COO tensor is
``(L, idx, vals)`` with ``L`` the N mode lengths, ``idx`` an (N, nnz) integer
array and ``vals`` an (nnz,) float array.  Pins for every function live in
``tests/test_oracle_*.py``.
"""
from __future__ import annotations

import numpy as np

_CHUNK = 1 << 16  # elements per chunk of the element loop (memory bound only)


def khat(K, n):
    """K-hat_n = prod_{m != n} K_m (Section 2.2): the row length of Z_(n)."""
    out = 1
    for m, k in enumerate(K):
        if m != n:
            out *= int(k)
    return out


def kron_row(rows):
    """Kronecker product of vectors u_1..u_r, vectorised as in Appendix A.

    ``rows`` is a list of arrays of shape (e, s_j) (one row per element).  The
    entry with coordinate (c_1..c_r) lands at position sum_j c_j prod_{i<j} s_i,
    i.e. the first vector varies fastest.  Returns shape (e, prod s_j).
    """
    e = rows[0].shape[0]
    out = np.ones((e, 1), dtype=np.float64)
    for u in rows:
        # the new vector becomes the slower axis: position = c_new * len(out) + c_old
        out = (u[:, :, None] * out[:, None, :]).reshape(e, -1)
    return out


def kron_n(F, idx, n, sl=slice(None)):
    """Kron_n(e) of Appendix A for the elements ``sl``: rows F_m[l_m(e), :] for
    every m != n, in increasing m."""
    N = len(F)
    return kron_row([np.asarray(F[m], dtype=np.float64)[idx[m][sl]] for m in range(N) if m != n])


def ttm_chain(L, idx, vals, F, n):
    """Penultimate matrix Z_(n) = T x_{m != n} F_m^T via eq. (1).

    Z_(n)[l, :] = sum over elements e with l_n(e) = l of val(e) * Kron_n(e).
    Returns the full L_n x K-hat_n matrix (rows of empty slices are zero).
    """
    N = len(F)
    K = [np.asarray(F[m]).shape[1] for m in range(N)]
    Z = np.zeros((int(L[n]), khat(K, n)), dtype=np.float64)
    nnz = len(vals)
    for s in range(0, nnz, _CHUNK):
        sl = slice(s, min(nnz, s + _CHUNK))
        contr = np.asarray(vals[sl], dtype=np.float64)[:, None] * kron_n(F, idx, n, sl)
        np.add.at(Z, np.asarray(idx[n][sl]), contr)
    return Z


def sign_normalise(U):
    """Flip each column so that its entry of largest magnitude (lowest row on a
    tie) is positive.  The paper is silent on the sign of singular vectors;
    this is the reading both sides use so that cores can be compared."""
    U = np.array(U, dtype=np.float64, copy=True)
    for k in range(U.shape[1]):
        i = int(np.argmax(np.abs(U[:, k])))  # argmax returns the lowest index on ties
        if U[i, k] < 0:
            U[:, k] = -U[:, k]
    return U


def leading_left_singular_vectors(Z, K):
    """F~_n <- leading K left singular vectors of Z_(n) (Fig. 1, SVD step).

    Uses the library SVD as the step; columns ordered by descending singular
    value and sign-normalised.  Rows of empty slices are zero (Section 3: the
    truncated copy omits them) and the SVD of [A; 0] is [U_A; 0], so the SVD
    is taken over the non-empty rows only.  Returns (U, sigma)."""
    Z = np.asarray(Z, dtype=np.float64)
    nz = np.flatnonzero(np.any(Z != 0.0, axis=1))
    if len(nz) < K:
        nz = np.arange(Z.shape[0])
    Uc, s, _ = np.linalg.svd(Z[nz], full_matrices=False)
    U = np.zeros((Z.shape[0], K))
    U[nz] = Uc[:, :K]
    return sign_normalise(U), s[:K].copy()


def lanczos_bidiagonalization(Z, m, v0):
    """Golub-Kahan-Lanczos bidiagonalisation of Z (R x Khat), m steps from the
    start vector v0 -- the matrix-free iteration of Section 3 ("SVD
    component"), in which every step asks for one product Z x and one product
    y Z.  Both bases are re-orthogonalised in full (classical Gram-Schmidt,
    twice).  Returns (U, V, alpha, beta): U is R x m, V is Khat x m, both with
    orthonormal columns, and Z V = U B with B upper bidiagonal, alpha on its
    diagonal and beta[:m-1] above it (beta[m-1] is the residual norm of the
    last step).  Stops early at an invariant subspace (a zero alpha or beta)."""
    Z = np.asarray(Z, dtype=np.float64)
    R, kh = Z.shape
    U = np.zeros((R, m))
    V = np.zeros((kh, m + 1))
    alpha = np.zeros(m)
    beta = np.zeros(m)
    V[:, 0] = np.asarray(v0, dtype=np.float64) / np.linalg.norm(v0)
    done = m
    for j in range(m):
        p = Z @ V[:, j]
        if j > 0:
            p -= beta[j - 1] * U[:, j - 1]
        for _ in range(2):
            p -= U[:, :j] @ (U[:, :j].T @ p)
        alpha[j] = np.linalg.norm(p)
        if alpha[j] == 0.0:
            done = j
            break
        U[:, j] = p / alpha[j]
        r = Z.T @ U[:, j] - alpha[j] * V[:, j]
        for _ in range(2):
            r -= V[:, : j + 1] @ (V[:, : j + 1].T @ r)
        beta[j] = np.linalg.norm(r)
        if beta[j] == 0.0:
            done = j + 1
            break
        V[:, j + 1] = r / beta[j]
    return U[:, :done], V[:, :done], alpha[:done], beta[:done]


def lanczos_factor(Z, K, m=None, v0=None):
    """F~_n by the paper's SVD route (Section 3 "SVD component"; Section 7: a
    Lanczos bidiagonalisation with m = 2K iterations).  The K leading singular
    triplets of the m x m bidiagonal B give the right vectors V_K = V Q_K and
    sigma_K; then U = Z V_K diag(1/sigma_K), orthonormalised (QR with a positive
    diagonal) and sign-normalised -- the same back-projection as the exact
    route.  Readings: v0 = the all-ones vector (the paper's library starts
    from a random vector; a fixed one keeps both sides on the same Krylov
    space); m = min(2K, Khat, non-empty rows).  As in
    ``leading_left_singular_vectors`` the iteration runs over the non-empty
    rows.  Returns (U, sigma)."""
    Z = np.asarray(Z, dtype=np.float64)
    nz = np.flatnonzero(np.any(Z != 0.0, axis=1))
    Zc = Z[nz]
    R, kh = Zc.shape
    m = min(2 * K if m is None else m, kh, R)
    v0 = np.ones(kh) if v0 is None else v0
    U, V, alpha, beta = lanczos_bidiagonalization(Zc, m, v0)
    mm = len(alpha)
    B = np.diag(alpha) + np.diag(beta[: mm - 1], 1)
    _, s, Qt = np.linalg.svd(B)
    VK = V @ Qt[:K].T
    Uc = Zc @ VK / s[:K]
    Q, Rr = np.linalg.qr(Uc)
    Q = Q * np.sign(np.diag(Rr))
    out = np.zeros((Z.shape[0], K))
    out[nz] = Q
    return sign_normalise(out), s[:K].copy()


def hooi_invocation(L, idx, vals, F, K=None, variant="jacobi", svd="exact"):
    """One invocation of the HOOI procedure of Fig. 1 (without the core).

    For each mode n: Z <- T x_{m != n} F_m^T (TTM-chain), F~_n <- leading K_n
    left singular vectors of Z_(n).  ``variant="jacobi"`` takes every TTM-chain
    from the input factors (Fig. 1 as printed); ``"gauss_seidel"`` uses the
    factors already refined in this invocation (textbook HOOI).  ``svd="lanczos"``
    takes the factor by the paper's Lanczos route (``lanczos_factor``)."""
    N = len(F)
    if K is None:
        K = [np.asarray(f).shape[1] for f in F]
    new = [np.asarray(f, dtype=np.float64) for f in F]
    for n in range(N):
        src = F if variant == "jacobi" else new
        Z = ttm_chain(L, idx, vals, src, n)
        if svd == "lanczos":
            new[n], _ = lanczos_factor(Z, K[n])
        else:
            new[n], _ = leading_left_singular_vectors(Z, K[n])
    return new


def core(L, idx, vals, F):
    """New core G = T x_1 F_1^T x_2 ... x_N F_N^T (Fig. 1).

    Written out from the definition: G[k_1..k_N] = sum_e val(e) prod_m F_m[l_m(e), k_m],
    i.e. the Kronecker vector of all N rows scaled by val(e), summed over all
    elements.  Returned flat with the first mode fastest (length prod K_m)."""
    N = len(F)
    K = [np.asarray(F[m]).shape[1] for m in range(N)]
    G = np.zeros(int(np.prod(K)), dtype=np.float64)
    nnz = len(vals)
    for s in range(0, nnz, _CHUNK):
        sl = slice(s, min(nnz, s + _CHUNK))
        rows = [np.asarray(F[m], dtype=np.float64)[idx[m][sl]] for m in range(N)]
        G += np.asarray(vals[sl], dtype=np.float64) @ kron_row(rows)
    return G


def tensor_norm2(vals):
    """||T||_F^2 = sum of squared values of the (duplicate-free) COO tensor."""
    v = np.asarray(vals, dtype=np.float64)
    return float(v @ v)


def fit(vals, G):
    """fit = 1 - ||T - [[G;F]]||_F / ||T||_F, evaluated (orthonormal F,
    G = T x F^T) as 1 - sqrt(max(0, ||T||^2 - ||G||^2)) / ||T||.
    The paper does not define a fit; this is the Kolda-Bader reading."""
    t2 = tensor_norm2(vals)
    g2 = float(np.dot(G, G))
    return 1.0 - np.sqrt(max(0.0, t2 - g2)) / np.sqrt(t2)


def hooi(L, idx, vals, F0, iters, variant="jacobi", svd="exact"):
    """``iters`` invocations of Fig. 1 followed by the core, computed once after
    all invocations (Section 2.2).  Returns (F, G, fit)."""
    F = [np.asarray(f, dtype=np.float64) for f in F0]
    for _ in range(iters):
        F = hooi_invocation(L, idx, vals, F, variant=variant, svd=svd)
    G = core(L, idx, vals, F)
    return F, G, fit(vals, G)


def unfolding_gram(L, idx, vals, n):
    """T_(n) T_(n)^T (L_n x L_n) for the HOSVD bootstrap.

    Two elements contribute val*val' to entry (l_n, l_n') when they lie on the
    same mode-n fiber, i.e. agree on every coordinate except n (Section 2.1)."""
    N = len(L)
    others = [m for m in range(N) if m != n]
    # group elements by fiber: lexicographic key over the other coordinates
    keys = np.zeros(len(vals), dtype=np.int64)
    for m in reversed(others):
        keys = keys * int(L[m]) + np.asarray(idx[m], dtype=np.int64)
    order = np.argsort(keys, kind="stable")
    ks = keys[order]
    M = np.zeros((int(L[n]), int(L[n])), dtype=np.float64)
    starts = np.flatnonzero(np.r_[True, ks[1:] != ks[:-1]])
    ends = np.r_[starts[1:], len(ks)]
    ln = np.asarray(idx[n])[order]
    v = np.asarray(vals, dtype=np.float64)[order]
    for a, b in zip(starts, ends):
        rows = ln[a:b]
        w = v[a:b]
        M[np.ix_(rows, rows)] += np.outer(w, w)
    return M


def hosvd_init(L, idx, vals, K):
    """HOSVD bootstrap (Section 2.2): F_n^0 = leading K_n left singular vectors
    of the unfolding T_(n), i.e. the leading eigenvectors of T_(n) T_(n)^T."""
    F = []
    for n in range(len(L)):
        M = unfolding_gram(L, idx, vals, n)
        w, V = np.linalg.eigh(M)
        sel = np.argsort(-w, kind="stable")[: K[n]]
        F.append(sign_normalise(V[:, sel]))
    return F


def ttm_chain_adjoint(L, idx, vals, F, n, dZ):
    """Adjoint of eq. (1) for a cotangent dZ (L_n x K-hat_n, full rows).

    dval(e)      = < dZ[l_n(e), :], Kron_n(e) >
    dF_m[i, k]   = sum_{e: l_m(e) = i} val(e) * < dZ[l_n(e), :], Kron_n(e) with row m replaced by unit vector e_k >
    Returns (dval, [dF_m or None for m == n])."""
    N = len(F)
    K = [np.asarray(F[m]).shape[1] for m in range(N)]
    nnz = len(vals)
    dval = np.zeros(nnz, dtype=np.float64)
    dF = [None if m == n else np.zeros((int(L[m]), K[m]), dtype=np.float64) for m in range(N)]
    for s in range(0, nnz, _CHUNK):
        sl = slice(s, min(nnz, s + _CHUNK))
        D = np.asarray(dZ, dtype=np.float64)[np.asarray(idx[n][sl])]
        v = np.asarray(vals[sl], dtype=np.float64)
        dval[sl] = np.sum(D * kron_n(F, idx, n, sl), axis=1)
        for m in range(N):
            if m == n:
                continue
            for k in range(K[m]):
                unit = np.zeros((1, K[m]))
                unit[0, k] = 1.0
                rows = []
                for mm in range(N):
                    if mm == n:
                        continue
                    if mm == m:
                        rows.append(np.repeat(unit, sl.stop - sl.start, axis=0))
                    else:
                        rows.append(np.asarray(F[mm], dtype=np.float64)[idx[mm][sl]])
                g = v * np.sum(D * kron_row(rows), axis=1)
                np.add.at(dF[m][:, k], np.asarray(idx[m][sl]), g)
    return dval, dF


def projector_distance(A, B):
    """|| A A^T - B B^T ||_2 for matrices with orthonormal columns (sign- and
    rotation-invariant comparison of the spanned subspaces)."""
    A = np.asarray(A, dtype=np.float64)
    B = np.asarray(B, dtype=np.float64)
    # For orthonormal A, B of equal rank, ||AA^T - BB^T||_2 = sin(largest principal
    # angle) = ||(I - AA^T) B||_2; the residual form stays accurate for tiny angles.
    return float(np.linalg.norm(B - A @ (A.T @ B), 2)) if B.size else 0.0
