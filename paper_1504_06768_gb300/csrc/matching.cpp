// Weighted maximum bipartite matching for a zero-free diagonal (section
// "Direct factorization").  Columns are taken in descending order of their
// largest weight |a_ij|^2 (ties: ascending column); each runs a
// breadth-first search over alternating paths that tries the rows of a
// column in descending weight (ties: ascending row) and stops at the first
// unmatched row, whose path is then flipped.  A column without an augmenting
// path stays unmatched; one search per column gives a maximum matching.
#include <algorithm>
#include <vector>

#include "host_algos.h"

int64_t mbm_host(int64_t n, const int32_t* row_ptr, const int32_t* col, const double* val, int32_t* match) {
    // columns of A with their rows sorted by (weight desc, row asc)
    std::vector<int64_t> cptr(n + 1, 0);
    for (int64_t i = 0; i < n; ++i)
        for (int32_t t = row_ptr[i]; t < row_ptr[i + 1]; ++t) ++cptr[(int64_t)col[t] + 1];
    for (int64_t j = 0; j < n; ++j) cptr[j + 1] += cptr[j];
    std::vector<int32_t> crow(cptr[n]);
    std::vector<double> cw(cptr[n]);
    {
        std::vector<int64_t> fill(cptr.begin(), cptr.end() - 1);
        for (int64_t i = 0; i < n; ++i)
            for (int32_t t = row_ptr[i]; t < row_ptr[i + 1]; ++t) {
                const double re = val[2 * (int64_t)t], im = val[2 * (int64_t)t + 1];
                const int64_t p = fill[col[t]]++;
                crow[p] = (int32_t)i;
                cw[p] = re * re + im * im;
            }
    }
    std::vector<double> best(n, -1.0);
    std::vector<int32_t> idx;
    for (int64_t j = 0; j < n; ++j) {
        const int64_t b = cptr[j], e = cptr[j + 1];
        idx.resize(e - b);
        for (int64_t t = 0; t < e - b; ++t) idx[t] = (int32_t)t;
        std::sort(idx.begin(), idx.end(), [&](int32_t x, int32_t y) {
            if (cw[b + x] != cw[b + y]) return cw[b + x] > cw[b + y];
            return crow[b + x] < crow[b + y];
        });
        std::vector<int32_t> r2(e - b);
        std::vector<double> w2(e - b);
        for (int64_t t = 0; t < e - b; ++t) {
            r2[t] = crow[b + idx[t]];
            w2[t] = cw[b + idx[t]];
        }
        std::copy(r2.begin(), r2.end(), crow.begin() + b);
        std::copy(w2.begin(), w2.end(), cw.begin() + b);
        if (e > b) best[j] = cw[b];
    }
    std::vector<int32_t> cols;
    for (int64_t j = 0; j < n; ++j)
        if (cptr[j + 1] > cptr[j]) cols.push_back((int32_t)j);
    std::sort(cols.begin(), cols.end(), [&](int32_t x, int32_t y) {
        if (best[x] != best[y]) return best[x] > best[y];
        return x < y;
    });
    std::vector<int32_t> row_of(n, -1), parent(n, -1), queue;
    std::vector<int64_t> seen(n, -1);               // search stamp per row
    for (int64_t j = 0; j < n; ++j) match[j] = -1;
    int64_t stamp = 0;
    for (int32_t c : cols) {
        ++stamp;
        queue.assign(1, c);
        int32_t end = -1;
        for (size_t head = 0; head < queue.size() && end < 0; ++head) {
            const int32_t cc = queue[head];
            for (int64_t t = cptr[cc]; t < cptr[cc + 1]; ++t) {
                const int32_t r = crow[t];
                if (seen[r] == stamp) continue;
                seen[r] = stamp;
                parent[r] = cc;
                if (row_of[r] < 0) {
                    end = r;
                    break;
                }
                queue.push_back(row_of[r]);
            }
        }
        if (end < 0) continue;
        for (int32_t r = end;;) {                   // flip the path back to c
            const int32_t cc = parent[r];
            const int32_t prev = match[cc];
            match[cc] = r;
            row_of[r] = cc;
            if (cc == c) break;
            r = prev;
        }
    }
    int64_t matched = 0;
    for (int64_t j = 0; j < n; ++j) matched += match[j] >= 0;
    return matched;
}
