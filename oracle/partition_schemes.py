"""Prior distribution schemes the paper compares Lite with (Section 5),
restated from their descriptions, plus the Section 4.1 metrics of any
element-to-processor policy.  TEST INFRASTRUCTURE ONLY (see
``oracle/tucker_oracle.py``): plain numpy, no blocking or reordering.

CoarseG (Section 5, coarse-grained schemes; multi-policy): along mode n every
slice goes whole to one processor; the slices, arranged in a random order,
are allocated to the processors in contiguous blocks.  Readings:
* the random order is an input: ``pos[l]`` = position of slice l in it (a
  permutation of [0, L_n));
* blocks balance elements: the slice at position t, preceded in the order by
  slices holding H_t elements, goes to processor floor(P * H_t / |E|).

MediumG (Section 5, medium-grained scheme; uni-policy): P = q_1 x ... x q_N,
a processor grid overlaid on the tensor after every mode's indices are
randomly permuted; each sub-tensor (grid cell) goes to one processor.
Readings:
* the permutations are inputs: ``pos[m][l]`` = permuted position of index l;
* "q_n in proportion to L_n": the prime factors of P, largest first, each
  multiply the q_m of the mode with the largest L_m / q_m so far (the lowest
  m on a tie);
* mode m's permuted positions are cut into q_m contiguous ranges, position x
  falling in range floor(x q_m / L_m);
* the processor of cell (b_1, ..., b_N) is b_1 + q_1 (b_2 + q_2 (b_3 + ...)).
"""
from __future__ import annotations

import numpy as np


def metrics(owner, slice_of, P):
    """Section 4.1 metrics of a policy along mode n: element e -> processor
    owner[e]; slice_of[e] = the element's mode-n coordinate.
    E_max = max_p |E^p|, R_sum = sum_p R^p, R_max = max_p R^p, R^p = number of
    distinct mode-n slices processor p holds elements of."""
    owner = np.asarray(owner, dtype=np.int64)
    slice_of = np.asarray(slice_of, dtype=np.int64)
    E = np.bincount(owner, minlength=P)
    R = np.zeros(P, dtype=np.int64)
    for p in range(P):
        R[p] = len(set(slice_of[owner == p].tolist()))
    return {"E_max": int(E.max()), "R_sum": int(R.sum()), "R_max": int(R.max()), "E": E, "R": R}


def coarseg_owner(idx_n, L_n, P, pos):
    """Processor of every element under CoarseG along mode n."""
    idx_n = np.asarray(idx_n, dtype=np.int64)
    nnz = len(idx_n)
    cnt = np.bincount(idx_n, minlength=L_n)
    order = np.empty(L_n, dtype=np.int64)
    order[np.asarray(pos, dtype=np.int64)] = np.arange(L_n)  # order[t] = slice at position t
    proc = np.zeros(L_n, dtype=np.int64)
    H = 0
    for t in range(L_n):
        s = int(order[t])
        proc[s] = (P * H) // nnz
        H += int(cnt[s])
    return proc[idx_n]


def prime_factors_desc(P):
    f, d, x = [], 2, int(P)
    while d * d <= x:
        while x % d == 0:
            f.append(d)
            x //= d
        d += 1
    if x > 1:
        f.append(x)
    return sorted(f, reverse=True)


def mediumg_grid(L, P):
    """The grid q_1 x ... x q_N of MediumG for mode lengths L and P processors."""
    q = [1] * len(L)
    for f in prime_factors_desc(P):
        best = 0
        for m in range(1, len(L)):
            # L_m / q_m > L_best / q_best, compared exactly
            if L[m] * q[best] > L[best] * q[m]:
                best = m
        q[best] *= f
    return q


def mediumg_owner(idx, L, P, pos):
    """Processor of every element under MediumG (the same for every mode)."""
    q = mediumg_grid(L, P)
    owner = np.zeros(len(idx[0]), dtype=np.int64)
    stride = 1
    for m in range(len(L)):
        x = np.asarray(pos[m], dtype=np.int64)[np.asarray(idx[m], dtype=np.int64)]
        b = (x * q[m]) // int(L[m])
        owner += b * stride
        stride *= q[m]
    return owner
