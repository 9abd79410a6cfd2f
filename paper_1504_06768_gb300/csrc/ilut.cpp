// Dual-threshold incomplete LU (ILUT) on the host, section "Iterative
// solvers": in row i, entries below drop_tol * ||a_i||_inf (infinity norm of
// the original row) are dropped, both when a multiplier l_ik is formed and
// after the row is eliminated; each of the strict lower and strict upper
// parts then keeps at most ceil(fill_factor * nnz(a_i) / 2) entries of largest
// modulus (ties: lower column first); the diagonal is always kept.  No
// pivoting.  Rows are eliminated in the IKJ order with a dense work row and
// a min-heap of pending lower columns.
#include <algorithm>
#include <cmath>
#include <functional>
#include <queue>
#include <vector>

#include "host_algos.h"

namespace {

struct Cx {
    double re, im;
};
inline Cx mul(Cx a, Cx b) { return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re}; }
inline double mag(Cx a) { return std::hypot(a.re, a.im); }
// Smith's algorithm for a / b (R. L. Smith, CACM 1962).
inline Cx div(Cx a, Cx b) {
    if (std::fabs(b.re) >= std::fabs(b.im)) {
        double r = b.im / b.re, den = b.re + b.im * r;
        return {(a.re + a.im * r) / den, (a.im - a.re * r) / den};
    }
    double r = b.re / b.im, den = b.im + b.re * r;
    return {(a.re * r + a.im) / den, (a.im * r - a.re) / den};
}

}  // namespace

int64_t ilut_host(int64_t n, const int32_t* row_ptr, const int32_t* col, const double* val,
                  double drop_tol, double fill_factor, std::vector<int32_t>& f_row_ptr,
                  std::vector<int32_t>& f_col, std::vector<double>& f_val) {
    f_row_ptr.assign(n + 1, 0);
    f_col.clear();
    f_val.clear();
    std::vector<int64_t> udiag(n, -1);              // position of u_ii in the output
    std::vector<Cx> w(n, Cx{0.0, 0.0});
    std::vector<char> used(n, 0);
    std::vector<int32_t> touched;
    std::priority_queue<int32_t, std::vector<int32_t>, std::greater<int32_t>> pending;
    std::vector<std::pair<int32_t, Cx>> lower, upper;

    for (int64_t i = 0; i < n; ++i) {
        double rnorm = 0.0;
        int32_t a = row_ptr[i], b = row_ptr[i + 1];
        for (int32_t t = a; t < b; ++t) rnorm = std::max(rnorm, mag(Cx{val[2 * t], val[2 * t + 1]}));
        const double tau = drop_tol * rnorm;
        const int64_t lfil = (int64_t)std::ceil(fill_factor * (double)(b - a) / 2.0);
        touched.clear();
        for (int32_t t = a; t < b; ++t) {
            int32_t j = col[t];
            w[j] = Cx{val[2 * t], val[2 * t + 1]};
            used[j] = 1;
            touched.push_back(j);
            if (j < i) pending.push(j);
        }
        while (!pending.empty()) {
            int32_t k = pending.top();
            pending.pop();
            if (!used[k]) continue;
            Cx wk = div(w[k], Cx{f_val[2 * udiag[k]], f_val[2 * udiag[k] + 1]});
            if (mag(wk) < tau) {                    // drop the multiplier
                used[k] = 0;
                w[k] = Cx{0.0, 0.0};
                continue;
            }
            w[k] = wk;
            for (int64_t t = udiag[k] + 1; t < f_row_ptr[k + 1]; ++t) {   // strict upper part of row k
                int32_t j = f_col[t];
                Cx p = mul(wk, Cx{f_val[2 * t], f_val[2 * t + 1]});
                if (used[j]) {
                    w[j] = Cx{w[j].re - p.re, w[j].im - p.im};
                } else {
                    w[j] = Cx{-p.re, -p.im};
                    used[j] = 1;
                    touched.push_back(j);
                    if (j < i) pending.push(j);
                }
            }
        }
        if (!used[i] || (w[i].re == 0.0 && w[i].im == 0.0)) {
            for (int32_t j : touched) { used[j] = 0; w[j] = Cx{0.0, 0.0}; }
            return i + 1;
        }
        lower.clear();
        upper.clear();
        for (int32_t j : touched) {
            if (!used[j] || j == i) continue;
            Cx v = w[j];
            if ((v.re == 0.0 && v.im == 0.0) || mag(v) < tau) continue;
            (j < i ? lower : upper).push_back({j, v});
        }
        auto by_size = [](const std::pair<int32_t, Cx>& x, const std::pair<int32_t, Cx>& y) {
            double mx = mag(x.second), my = mag(y.second);
            return mx != my ? mx > my : x.first < y.first;
        };
        auto by_col = [](const std::pair<int32_t, Cx>& x, const std::pair<int32_t, Cx>& y) { return x.first < y.first; };
        std::sort(lower.begin(), lower.end(), by_size);
        std::sort(upper.begin(), upper.end(), by_size);
        if ((int64_t)lower.size() > lfil) lower.resize(lfil);
        if ((int64_t)upper.size() > lfil) upper.resize(lfil);
        std::sort(lower.begin(), lower.end(), by_col);
        std::sort(upper.begin(), upper.end(), by_col);
        for (auto& e : lower) {
            f_col.push_back(e.first);
            f_val.push_back(e.second.re);
            f_val.push_back(e.second.im);
        }
        udiag[i] = (int64_t)f_col.size();
        f_col.push_back((int32_t)i);
        f_val.push_back(w[i].re);
        f_val.push_back(w[i].im);
        for (auto& e : upper) {
            f_col.push_back(e.first);
            f_val.push_back(e.second.re);
            f_val.push_back(e.second.im);
        }
        f_row_ptr[i + 1] = (int32_t)f_col.size();
        for (int32_t j : touched) { used[j] = 0; w[j] = Cx{0.0, 0.0}; }
    }
    return 0;
}
