"""Weighted maximum bipartite matching for a zero-free diagonal (oracle; test
infrastructure only).

Section "Direct factorization": the modified Liouvillian L~ may have zeros on
its diagonal; a non-symmetric row permutation makes the diagonal zero-free
and, being weighted, tries to put large entries there. The paper's variant
of maximum bipartite matching takes the columns one at a time, beginning
with the column that holds the largest |entry|, and searches breadth-first
for an augmenting path, trying the rows of each column in descending order
of |entry|.

Readings fixed here (the paper does not spell them out):
  * weight of an entry: |a_ij|^2 = re^2 + im^2 (the same order as |a_ij|);
  * columns are processed in descending order of their largest weight, ties
    by ascending column index; an empty column is left unmatched;
  * the search from column c is a breadth-first search over alternating
    paths: the rows of a dequeued column are tried in descending weight
    (ties by ascending row index); an unvisited row that is unmatched ends
    the search and the path is flipped; a matched one is marked visited and
    its column is queued;
  * a column with no augmenting path stays unmatched (A is structurally
    singular). Searching every column once this way gives a matching of
    maximum cardinality.

Result: match[j] = the row matched to column j (or -1), so that
B = A[match, :] has a zero-free diagonal when A is structurally nonsingular.
"""
from __future__ import annotations

from collections import deque

import numpy as np
import scipy.sparse as sp


def weighted_mbm(A):
    """(match, matched): match[j] = row assigned to column j (-1 if none),
    matched = number of matched columns."""
    A = sp.csc_matrix(A)
    A.sum_duplicates()
    A.sort_indices()
    n = A.shape[0]
    col_rows = []
    col_best = np.full(n, -1.0)
    for j in range(n):
        rows = A.indices[A.indptr[j]:A.indptr[j + 1]]
        vals = A.data[A.indptr[j]:A.indptr[j + 1]]
        wts = vals.real * vals.real + vals.imag * vals.imag
        order = sorted(range(len(rows)), key=lambda t: (-wts[t], rows[t]))
        col_rows.append([int(rows[t]) for t in order])
        if len(rows):
            col_best[j] = wts[order[0]]
    columns = sorted((j for j in range(n) if col_rows[j]), key=lambda j: (-col_best[j], j))
    match = [-1] * n          # column -> row
    row_of = [-1] * n         # row -> column
    for c in columns:
        parent = {}            # row -> column it was reached from
        queue = deque([c])
        end = -1
        while queue and end < 0:
            col = queue.popleft()
            for r in col_rows[col]:
                if r in parent:
                    continue
                parent[r] = col
                if row_of[r] < 0:
                    end = r
                    break
                queue.append(row_of[r])
        if end < 0:
            continue
        r = end
        while True:             # flip the alternating path back to c
            col = parent[r]
            prev = match[col]
            match[col] = r
            row_of[r] = col
            if col == c:
                break
            r = prev
    matched = sum(1 for m in match if m >= 0)
    return np.asarray(match, dtype=np.int64), matched
