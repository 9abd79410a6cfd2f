// Host-side ordering and level analysis.
//
// Reverse Cuthill-McKee (section "Direct factorization"): the structure of
// A + A^T is read as an undirected graph, degree(v) = stored entries of row v
// of A + A^T (the diagonal included when stored).  Cuthill-McKee is a
// breadth-first search from an unvisited node of minimum degree -- the one
// with the highest index among ties -- that appends the unvisited neighbours
// of each dequeued node in ascending (degree, index); it restarts the same
// way for every connected component.  Reversing the sequence gives RCM.
#include <algorithm>
#include <numeric>
#include <vector>

#include "host_algos.h"

void rcm_host(int64_t n, const int32_t* row_ptr, const int32_t* col, int32_t* perm) {
    // symmetrised adjacency: counts, then fill, then sort + unique per node
    std::vector<int64_t> cnt(n + 1, 0);
    for (int64_t i = 0; i < n; ++i)
        for (int32_t t = row_ptr[i]; t < row_ptr[i + 1]; ++t) {
            ++cnt[i + 1];
            if (col[t] != i) ++cnt[(int64_t)col[t] + 1];
        }
    for (int64_t i = 0; i < n; ++i) cnt[i + 1] += cnt[i];
    std::vector<int32_t> adj(cnt[n]);
    std::vector<int64_t> fill(cnt.begin(), cnt.end() - 1);
    for (int64_t i = 0; i < n; ++i)
        for (int32_t t = row_ptr[i]; t < row_ptr[i + 1]; ++t) {
            int32_t j = col[t];
            adj[fill[i]++] = j;
            if (j != i) adj[fill[j]++] = (int32_t)i;
        }
    std::vector<int32_t> deg(n);
    std::vector<int64_t> beg(n), end(n);
    for (int64_t v = 0; v < n; ++v) {
        auto b = adj.begin() + cnt[v], e = adj.begin() + fill[v];
        std::sort(b, e);
        e = std::unique(b, e);
        beg[v] = cnt[v];
        end[v] = e - adj.begin();
        deg[v] = (int32_t)(end[v] - beg[v]);            // includes v itself when stored
    }
    // neighbour lists ordered by (degree, index), self removed
    for (int64_t v = 0; v < n; ++v) {
        auto b = adj.begin() + beg[v], e = adj.begin() + end[v];
        e = std::remove(b, e, (int32_t)v);
        end[v] = e - adj.begin();
        std::sort(b, e, [&](int32_t a, int32_t c) { return deg[a] != deg[c] ? deg[a] < deg[c] : a < c; });
    }
    // start candidates: ascending degree, descending index
    std::vector<int32_t> starts(n);
    std::iota(starts.begin(), starts.end(), 0);
    std::sort(starts.begin(), starts.end(),
              [&](int32_t a, int32_t c) { return deg[a] != deg[c] ? deg[a] < deg[c] : a > c; });
    std::vector<char> seen(n, 0);
    std::vector<int32_t> order;
    order.reserve(n);
    int64_t cursor = 0;
    while ((int64_t)order.size() < n) {
        while (seen[starts[cursor]]) ++cursor;
        int32_t s = starts[cursor];
        seen[s] = 1;
        size_t head = order.size();
        order.push_back(s);
        while (head < order.size()) {
            int32_t u = order[head++];
            for (int64_t t = beg[u]; t < end[u]; ++t) {
                int32_t v = adj[t];
                if (!seen[v]) {
                    seen[v] = 1;
                    order.push_back(v);
                }
            }
        }
    }
    for (int64_t r = 0; r < n; ++r) perm[r] = order[n - 1 - r];
}

int32_t level_sets_host(int64_t n, const int32_t* row_ptr, const int32_t* col, bool lower,
                        std::vector<int32_t>& order, std::vector<int32_t>& level_ptr) {
    std::vector<int32_t> level(n, 0);
    int32_t nlev = 0;
    if (lower) {
        for (int64_t i = 0; i < n; ++i) {
            int32_t l = 0;
            for (int32_t t = row_ptr[i]; t < row_ptr[i + 1] && col[t] < i; ++t) l = std::max(l, level[col[t]] + 1);
            level[i] = l;
            nlev = std::max(nlev, l + 1);
        }
    } else {
        for (int64_t i = n - 1; i >= 0; --i) {
            int32_t l = 0;
            for (int32_t t = row_ptr[i + 1] - 1; t >= row_ptr[i] && col[t] > i; --t)
                l = std::max(l, level[col[t]] + 1);
            level[i] = l;
            nlev = std::max(nlev, l + 1);
        }
    }
    // counting sort by level, rows ascending inside a level
    std::vector<int64_t> start(nlev + 1, 0);
    for (int64_t i = 0; i < n; ++i) ++start[level[i] + 1];
    for (int32_t l = 0; l < nlev; ++l) start[l + 1] += start[l];
    level_ptr.assign(start.begin(), start.end());
    order.assign(n, 0);
    for (int64_t i = 0; i < n; ++i) order[start[level[i]]++] = (int32_t)i;
    return nlev;
}

void level_units_host(const std::vector<int32_t>& order, const std::vector<int32_t>& level_ptr, int R,
                      std::vector<int32_t>& units) {
    units.clear();
    for (size_t l = 0; l + 1 < level_ptr.size(); ++l) {
        for (int32_t a = level_ptr[l]; a < level_ptr[l + 1]; a += R)
            for (int g = 0; g < R; ++g) units.push_back(a + g < level_ptr[l + 1] ? order[a + g] : -1);
    }
}

// iLU(0) elimination schedule (section "Iterative solvers": incomplete LU
// without fill): for every pivot position t of row i, the entries of row i
// after t that the pivot row's upper part also holds.  Columns are sorted,
// so each match is a binary search in row i's remaining columns.
void ilu0_schedule_host(int64_t n, const int32_t* row_ptr, const int32_t* col, const int32_t* dpos,
                        std::vector<int32_t>& ptr, std::vector<int32_t>& tgt, std::vector<int32_t>& src) {
    const int32_t nnz = n > 0 ? row_ptr[n] : 0;
    ptr.assign((size_t)nnz + 1, 0);
    tgt.clear();
    src.clear();
    for (int64_t i = 0; i < n; ++i) {
        const int32_t rb = row_ptr[i], re = row_ptr[i + 1];
        for (int32_t t = rb; t < re; ++t) {
            ptr[t] = (int32_t)tgt.size();
            if (t >= dpos[i]) continue;
            const int32_t k = col[t];
            for (int32_t u = dpos[k] + 1; u < row_ptr[k + 1]; ++u) {
                const int32_t* it = std::lower_bound(col + t + 1, col + re, col[u]);
                if (it != col + re && *it == col[u]) {
                    tgt.push_back((int32_t)(it - col) - rb);
                    src.push_back(u);
                }
            }
        }
    }
    ptr[nnz] = (int32_t)tgt.size();
}
