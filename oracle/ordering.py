"""Reverse Cuthill-McKee ordering, bandwidth and profile (oracle; test
infrastructure only).

Section "Direct factorization": the ordering is computed on the structure of
the symmetrised matrix A + A^T. Cuthill-McKee is a breadth-first search that
starts from a node of lowest degree (degree = number of stored entries in the
node's row of A + A^T) and, within each level, visits the unvisited
neighbours of a node from lowest to highest degree; it is repeated for each
connected component; reversing the resulting order gives RCM.

Tie-breaking, which the paper leaves open, is fixed as follows:
  * start node: among the unvisited nodes of minimum degree, the one with the
    highest index;
  * neighbours of a node: ascending (degree, index);
  * the next component starts by the same rule over the remaining nodes;
  * the degree counts the diagonal entry when it is stored.

Bandwidth and profile follow the definitions of the same section:
ub = max (j - i), lb = max (i - j), B = ub + lb + 1;
up = sum over rows i of max_j (j - i), lp = sum over columns j of max_i (i - j),
P = up + lp, with each max taken over stored entries and floored at zero.
"""
from __future__ import annotations

from typing import List, Tuple

import numpy as np
import scipy.sparse as sp


def symmetric_pattern(A) -> List[List[int]]:
    """Adjacency lists (sorted, self excluded) and the pattern of A + A^T."""
    A = sp.csr_matrix(A)
    n = A.shape[0]
    nbrs = [set() for _ in range(n)]
    indptr, indices = A.indptr, A.indices
    for i in range(n):
        for t in range(indptr[i], indptr[i + 1]):
            j = int(indices[t])
            nbrs[i].add(j)
            nbrs[j].add(i)
    return [sorted(s) for s in nbrs]


def rcm_order(A) -> np.ndarray:
    """perm with perm[new] = old, the reverse Cuthill-McKee order of A + A^T."""
    adj = symmetric_pattern(A)
    n = len(adj)
    degree = [len(a) for a in adj]            # the diagonal, when stored, is in adj
    nodes_by_start = sorted(range(n), key=lambda v: (degree[v], -v))
    visited = [False] * n
    order: List[int] = []
    cursor = 0
    while len(order) < n:
        while visited[nodes_by_start[cursor]]:
            cursor += 1
        start = nodes_by_start[cursor]
        visited[start] = True
        queue = [start]
        head = 0
        while head < len(queue):
            u = queue[head]
            head += 1
            fresh = [v for v in adj[u] if v != u and not visited[v]]
            fresh.sort(key=lambda v: (degree[v], v))
            for v in fresh:
                visited[v] = True
                queue.append(v)
        order.extend(queue)
    order.reverse()
    return np.asarray(order, dtype=np.int64)


def permute_symmetric(A, perm: np.ndarray) -> sp.csr_matrix:
    """P A P^T with (P A P^T)[r, c] = A[perm[r], perm[c]]."""
    A = sp.csr_matrix(A)
    B = A[perm, :][:, perm]
    B = sp.csr_matrix(B)
    B.sort_indices()
    return B


def bandwidth_profile(A) -> Tuple[int, int, int, int, int, int]:
    """(B, P, ub, lb, up, lp) of the stored pattern of A."""
    A = sp.coo_matrix(A)
    n = A.shape[0]
    r = A.row.astype(np.int64)
    c = A.col.astype(np.int64)
    ub = int(max(0, (c - r).max())) if r.size else 0
    lb = int(max(0, (r - c).max())) if r.size else 0
    row_up = np.zeros(n, dtype=np.int64)
    np.maximum.at(row_up, r, c - r)
    col_lp = np.zeros(n, dtype=np.int64)
    np.maximum.at(col_lp, c, r - c)
    up = int(row_up.sum())
    lp = int(col_lp.sum())
    return ub + lb + 1, up + lp, ub, lb, up, lp
