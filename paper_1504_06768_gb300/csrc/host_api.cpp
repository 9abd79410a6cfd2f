// Host-side steps of the path as C entry points that need no GPU: the RCM
// ordering of rcm_permute, the level sets of the triangular solves, the ILUT
// of ilu_factor (the same functions the device path calls) and the weighted
// bipartite matching for a zero-free diagonal.
#include <cstring>
#include <vector>

#include "host_algos.h"
#include "lindblad_ss.h"

namespace {

// A well-formed n x n CSR pattern: row_ptr[0] = 0, non-decreasing, columns
// in [0, n) and strictly ascending inside each row.
bool csr_ok(int64_t n, const int32_t* rp, const int32_t* col) {
    if (n < 0 || !rp || (n > 0 && rp[n] > 0 && !col) || rp[0] != 0) return false;
    for (int64_t i = 0; i < n; ++i) {
        if (rp[i + 1] < rp[i]) return false;
        for (int32_t t = rp[i]; t < rp[i + 1]; ++t) {
            if (col[t] < 0 || col[t] >= n) return false;
            if (t > rp[i] && col[t] <= col[t - 1]) return false;
        }
    }
    return true;
}

}  // namespace

extern "C" ss_status ss_rcm_order_host(int64_t n, const int32_t* row_ptr, const int32_t* col, int32_t* perm_out) {
    if (!perm_out || !csr_ok(n, row_ptr, col)) return SS_ERR_INVALID;
    rcm_host(n, row_ptr, col, perm_out);
    return SS_OK;
}

extern "C" ss_status ss_level_sets_host(int64_t n, const int32_t* row_ptr, const int32_t* col, int lower,
                                        int32_t* order_out, int32_t* level_ptr_out, int32_t* n_levels_out) {
    if (!order_out || !level_ptr_out || !n_levels_out || !csr_ok(n, row_ptr, col)) return SS_ERR_INVALID;
    std::vector<int32_t> order, ptr;
    const int32_t nl = level_sets_host(n, row_ptr, col, lower != 0, order, ptr);
    if (n > 0) std::memcpy(order_out, order.data(), sizeof(int32_t) * (size_t)n);
    std::memcpy(level_ptr_out, ptr.data(), sizeof(int32_t) * ptr.size());
    *n_levels_out = nl;
    return SS_OK;
}

extern "C" ss_status ss_ilu0_schedule_host(int64_t n, const int32_t* row_ptr, const int32_t* col, int64_t capacity,
                                           int32_t* ptr_out, int32_t* tgt_out, int32_t* src_out, int64_t* count_out) {
    if (!count_out || !csr_ok(n, row_ptr, col)) return SS_ERR_INVALID;
    std::vector<int32_t> dpos((size_t)n, -1);
    for (int64_t i = 0; i < n; ++i)
        for (int32_t t = row_ptr[i]; t < row_ptr[i + 1]; ++t)
            if (col[t] == i) dpos[i] = t;
    for (int64_t i = 0; i < n; ++i)
        if (dpos[i] < 0) return SS_ZERO_PIVOT;
    std::vector<int32_t> ptr, tgt, src;
    ilu0_schedule_host(n, row_ptr, col, dpos.data(), ptr, tgt, src);
    const int64_t count = (int64_t)tgt.size();
    *count_out = count;
    if (capacity < count || !ptr_out || (count > 0 && (!tgt_out || !src_out))) return SS_ERR_INVALID;
    std::memcpy(ptr_out, ptr.data(), sizeof(int32_t) * ptr.size());
    if (count > 0) {
        std::memcpy(tgt_out, tgt.data(), sizeof(int32_t) * (size_t)count);
        std::memcpy(src_out, src.data(), sizeof(int32_t) * (size_t)count);
    }
    return SS_OK;
}

extern "C" ss_status ss_ilut_host(int64_t n, const int32_t* row_ptr, const int32_t* col, const double* val,
                                  double drop_tol, double fill_factor, int64_t capacity, int32_t* f_row_ptr,
                                  int32_t* f_col, double* f_val, int64_t* nnz_out, int64_t* zero_pivot_row) {
    if (!nnz_out || !zero_pivot_row || !csr_ok(n, row_ptr, col) || (n > 0 && row_ptr[n] > 0 && !val) ||
        !(drop_tol >= 0.0) || !(fill_factor > 0.0))
        return SS_ERR_INVALID;
    std::vector<int32_t> frp, fcol;
    std::vector<double> fval;
    const int64_t bad = ilut_host(n, row_ptr, col, val, drop_tol, fill_factor, frp, fcol, fval);
    *zero_pivot_row = bad ? bad - 1 : -1;
    if (bad) return SS_ZERO_PIVOT;
    const int64_t nnz = (int64_t)fcol.size();
    *nnz_out = nnz;
    if (capacity < nnz || !f_row_ptr || (nnz > 0 && (!f_col || !f_val))) return SS_ERR_INVALID;
    std::memcpy(f_row_ptr, frp.data(), sizeof(int32_t) * (size_t)(n + 1));
    if (nnz > 0) {
        std::memcpy(f_col, fcol.data(), sizeof(int32_t) * (size_t)nnz);
        std::memcpy(f_val, fval.data(), sizeof(double) * 2 * (size_t)nnz);
    }
    return SS_OK;
}

extern "C" ss_status ss_mbm_host(int64_t n, const int32_t* row_ptr, const int32_t* col, const double* val,
                                 int32_t* match_out, int64_t* matched_out) {
    if (!match_out || !matched_out || !csr_ok(n, row_ptr, col) || (n > 0 && row_ptr[n] > 0 && !val))
        return SS_ERR_INVALID;
    *matched_out = mbm_host(n, row_ptr, col, val, match_out);
    return SS_OK;
}

namespace {
double table_cost(const TuneChoice& c, void* user) {
    const double* t = static_cast<const double*>(user);
    const int span = TUNE_SHIFT_MAX - TUNE_SHIFT_MIN + 1;
    return t[(((c.lo - TUNE_SHIFT_MIN) * span + (c.up - TUNE_SHIFT_MIN)) * span + (c.a - TUNE_SHIFT_MIN)) * 2 + c.stage];
}
}  // namespace

extern "C" ss_status ss_tune_search_host(const double* cost_table, int32_t max_probes, int32_t* best_out,
                                         int32_t* probes_out) {
    if (!cost_table || !best_out || max_probes < 1) return SS_ERR_INVALID;
    TuneChoice best{}, start{0, 0, 0, 0};
    const int probes = tune_search(start, table_cost, const_cast<double*>(cost_table), max_probes, &best, nullptr);
    best_out[0] = best.lo;
    best_out[1] = best.up;
    best_out[2] = best.a;
    best_out[3] = best.stage;
    if (probes_out) *probes_out = probes;
    return SS_OK;
}
