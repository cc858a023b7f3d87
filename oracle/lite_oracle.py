"""Lite distribution scheme along one mode (Section 6.1, Fig. 7), executed
literally on the CPU.  TEST INFRASTRUCTURE ONLY (see ``oracle/tucker_oracle.py``).

Readings of points the paper leaves open:

* empty slices are dropped before sorting -- they own no element and are
  shared by no bin;
* slices are sorted by (cardinality, slice id) ascending (the paper only says
  "increasing order of cardinality");
* "Select any g elements" takes the first g remaining elements of the slice in
  its *listing order*: the slice's elements ordered by the popularity rank of
  their coordinate along the fiber mode f(n) -- the other mode with the fewest
  slices (smallest L_m, lowest m on a tie); rank 0 is that mode's largest slice,
  ties by lower slice id -- and then by original COO position.  The paper leaves
  the choice free; this order lists each mode-n fiber's elements together and
  every bin's elements from the most to the least frequent fiber coordinate;
* both stages stop when the slices run out (the printed loops have no bound on
  t); stage 2 always finishes because P * ceil(|E|/P) >= |E|;
* the bin index follows the pseudocode's counter (p starts at 0, advances
  modulo P), which matches the Fig. 6 caption.

A bin's contents are kept as a list of *pieces* (slice id, first rank j0 within
the slice, count) in the order the pseudocode assigns them; the elements of a
piece are the slice's elements of listing-order rank j0 .. j0+count-1.
"""
from __future__ import annotations

import numpy as np


def lite_pieces(cnt, P):
    """Run Fig. 7 on slice cardinalities ``cnt`` (length L_n) with P bins.

    Returns a dict with
      pieces : list (per bin) of [(slice, j0, count), ...] in assignment order
      t_hat  : 0-based position (in sorted order) of the first stage-2 slice
      order  : the sorted non-empty slice ids (S_1, S_2, ... of Fig. 7)
      limit  : ceil(|E| / P)
    """
    cnt = np.asarray(cnt, dtype=np.int64)
    nnz = int(cnt.sum())
    limit = -(-nnz // P)  # ceil(|E|/P)
    nonempty = [int(l) for l in np.flatnonzero(cnt > 0)]
    order = sorted(nonempty, key=lambda l: (int(cnt[l]), l))
    pieces = [[] for _ in range(P)]
    load = [0] * P

    # Stage 1: round robin in increasing order of cardinality while the limit holds.
    p = 0
    t = 0
    while t < len(order):
        s = order[t]
        if load[p] + int(cnt[s]) > limit:
            break  # GOTO stage 2
        pieces[p].append((s, 0, int(cnt[s])))
        load[p] += int(cnt[s])
        p = (p + 1) % P
        t += 1
    t_hat = t

    # Stage 2: fill each bin to the limit, splitting slices over contiguous bins.
    p = 0
    taken = 0  # elements of order[t] already assigned
    while p < P and t < len(order):
        s = order[t]
        g = limit - load[p]
        rem = int(cnt[s]) - taken
        if rem <= g:
            if rem > 0:
                pieces[p].append((s, taken, rem))
            load[p] += rem
            t += 1
            taken = 0
        else:
            if g > 0:
                pieces[p].append((s, taken, g))
            load[p] += g
            taken += g
            p += 1
    assert t == len(order), "stage 2 ran out of bins (impossible when P*limit >= |E|)"
    return {"pieces": pieces, "t_hat": t_hat, "order": order, "limit": limit}


def fiber_mode(L, n):
    """f(n): the mode other than n with the fewest slices (smallest L_m,
    lowest m on a tie)."""
    return min((m for m in range(len(L)) if m != n), key=lambda m: (int(L[m]), m))


def popularity_rank(idx_m, L_m):
    """rank[l] = position of slice l of a mode when its slices are listed by
    decreasing cardinality, ties by increasing slice id (empty slices last)."""
    cnt = np.bincount(np.asarray(idx_m, dtype=np.int64), minlength=int(L_m))
    order = sorted(range(int(L_m)), key=lambda l: (-int(cnt[l]), l))
    rank = np.empty(int(L_m), dtype=np.int64)
    rank[np.array(order, dtype=np.int64)] = np.arange(int(L_m))
    return rank


def slice_members(idx, L, n):
    """Elements of every mode-n slice in listing order (popularity rank of the
    fiber-mode coordinate, then original position): returns (elems, start)
    such that slice l's elements are elems[start[l]:start[l+1]]."""
    idx = [np.asarray(x, dtype=np.int64) for x in idx]
    f = fiber_mode(L, n)
    key = popularity_rank(idx[f], L[f])[idx[f]]
    nnz = len(idx[n])
    elems = np.lexsort((np.arange(nnz), key, idx[n]))
    cnt = np.bincount(idx[n], minlength=int(L[n]))
    start = np.zeros(int(L[n]) + 1, dtype=np.int64)
    np.cumsum(cnt, out=start[1:])
    return elems, start


def lite_assignment(idx, L, n, P):
    """Element-level Lite partition along mode n of a COO tensor with
    coordinates ``idx`` (N arrays) and mode lengths ``L``.

    Returns (bin_ptr, perm, info): bin p owns the original element ids
    perm[bin_ptr[p]:bin_ptr[p+1]], listed piece by piece in assignment order and,
    within a piece, in listing order.  ``info`` is the dict of ``lite_pieces``.
    """
    cnt = np.bincount(np.asarray(idx[n], dtype=np.int64), minlength=int(L[n]))
    info = lite_pieces(cnt, P)
    elems, start = slice_members(idx, L, n)
    bin_ptr = np.zeros(P + 1, dtype=np.int64)
    out = []
    for p in range(P):
        n_p = 0
        for (s, j0, c) in info["pieces"][p]:
            out.append(elems[start[s] + j0 : start[s] + j0 + c])
            n_p += c
        bin_ptr[p + 1] = bin_ptr[p] + n_p
    perm = np.concatenate(out) if out else np.zeros(0, dtype=np.int64)
    return bin_ptr, perm, info


def metrics(pieces, L_n=None):
    """Section 4.1 metrics of a partition given as per-bin piece lists:
    E_max = max_p |E_n^p|, R_sum = sum_p R_n^p, R_max = max_p R_n^p, where
    R_n^p counts the distinct slices bin p shares (owns >= 1 element of)."""
    E = [sum(c for (_, _, c) in bp) for bp in pieces]
    R = [len({s for (s, _, c) in bp if c > 0}) for bp in pieces]
    return {"E_max": max(E), "R_sum": sum(R), "R_max": max(R), "E": E, "R": R}


def metrics_from_assignment(owner, slice_of):
    """Same three metrics for an arbitrary policy pi: element e -> bin owner[e]
    (Section 4.1).  ``slice_of[e]`` is the element's mode-n coordinate."""
    owner = np.asarray(owner)
    slice_of = np.asarray(slice_of)
    P = int(owner.max()) + 1 if len(owner) else 0
    E = np.bincount(owner, minlength=P)
    R = [len(set(slice_of[owner == p].tolist())) for p in range(P)]
    return {"E_max": int(E.max()), "R_sum": int(sum(R)), "R_max": int(max(R)), "E": E.tolist(), "R": R}
