"""VR overlap graph, non-orthogonal sets and the orthogonal set F.

* Lemma 1: users whose VRs do not overlap have orthogonal channels, so the
  corresponding rows of B = [H, sqrt(xi) I] are orthogonal.
* Sec. IV-B: X_k is the set of users whose VR overlaps user k's VR; k itself
  is included (its own residual changes when row k is projected).
* Sec. V-B, eq. (max_set): F is a maximum independent set of the overlap
  graph (the text's "|M_i n M_j| > 0" for F is read as "= 0"), V the rest.

VRs are half-open contiguous intervals [o, o + L); intervals that only touch
do not overlap.  Contiguous VRs make the overlap graph an interval graph, on
which the earliest-end greedy rule (activity selection) is an exact maximum
independent set; ``mis_bruteforce`` enumerates subsets for small K.
"""
from itertools import combinations

import numpy as np


def overlaps(o1, l1, o2, l2) -> bool:
    return (o1 < o2 + l2) and (o2 < o1 + l1)


def adjacency(vr_offset, vr_len) -> np.ndarray:
    K = len(vr_len)
    A = np.zeros((K, K), dtype=bool)
    for i in range(K):
        for j in range(K):
            if i != j and overlaps(int(vr_offset[i]), int(vr_len[i]), int(vr_offset[j]), int(vr_len[j])):
                A[i, j] = True
    return A


def x_sets(vr_offset, vr_len):
    """X_k (including k) for every user, as sorted lists."""
    A = adjacency(vr_offset, vr_len)
    return [sorted(set(np.nonzero(A[k])[0].tolist()) | {k}) for k in range(len(vr_len))]


def mis_interval(vr_offset, vr_len):
    """Earliest-end greedy; ties broken by later start, then lower index."""
    K = len(vr_len)
    ends = [int(vr_offset[k]) + int(vr_len[k]) for k in range(K)]
    order = sorted(range(K), key=lambda k: (ends[k], -int(vr_offset[k]), k))
    F, last_end = [], None
    for k in order:
        if last_end is None or int(vr_offset[k]) >= last_end:
            F.append(k)
            last_end = ends[k]
    return sorted(F)


def is_independent(F, vr_offset, vr_len) -> bool:
    A = adjacency(vr_offset, vr_len)
    return not any(A[i, j] for i in F for j in F if i != j)


def mis_bruteforce(vr_offset, vr_len) -> int:
    """Size of a maximum independent set by subset enumeration (small K only)."""
    K = len(vr_len)
    A = adjacency(vr_offset, vr_len)
    for size in range(K, 0, -1):
        for sub in combinations(range(K), size):
            if not any(A[i, j] for i in sub for j in sub if i < j):
                return size
    return 0


def split_fv(vr_offset, vr_len):
    F = mis_interval(vr_offset, vr_len)
    fs = set(F)
    V = [k for k in range(len(vr_len)) if k not in fs]
    return F, V


# ---------------------------------------------------------------------------
# Subarray VRs (Sec. II eq. (5), Sec. VII): user k sees the subarrays M_k.
# Two users' rows are orthogonal when they share no subarray (Lemma 1), so the
# overlap graph joins users with a common subarray; it is a general graph, and
# F is found by a near-maximum independent-set heuristic (the paper cites a
# linear-time near-MIS method): repeatedly take a vertex of least degree in
# the remaining graph and delete it with its neighbours.


def subarray_adjacency(M):
    K = len(M)
    sets = [set(m) for m in M]
    A = np.zeros((K, K), dtype=bool)
    for i in range(K):
        for j in range(K):
            if i != j and sets[i] & sets[j]:
                A[i, j] = True
    return A


def x_sets_graph(A):
    """X_k (k included) from an adjacency matrix."""
    return [sorted(set(np.nonzero(A[k])[0].tolist()) | {k}) for k in range(A.shape[0])]


def mis_min_degree(A):
    """Near-maximum independent set: least remaining degree first (ties: lower index)."""
    alive = set(range(A.shape[0]))
    F = []
    while alive:
        k = min(alive, key=lambda v: (sum(1 for u in alive if A[v, u]), v))
        F.append(k)
        alive -= {k} | {u for u in alive if A[k, u]}
    return sorted(F)


def mis_bruteforce_graph(A) -> int:
    K = A.shape[0]
    for size in range(K, 0, -1):
        for sub in combinations(range(K), size):
            if not any(A[i, j] for i in sub for j in sub if i < j):
                return size
    return 0


def is_independent_graph(F, A) -> bool:
    return not any(A[i, j] for i in F for j in F if i != j)


def is_maximal_graph(F, A) -> bool:
    fs = set(F)
    return all(any(A[v, u] for u in fs) for v in range(A.shape[0]) if v not in fs)
