// Setup of a batch of systems for the persistent solver with a fixed number
// of launches per batch, whatever the number of systems:
//   * the operators H and C_k of all systems are stacked block-diagonally, so
//     that one transpose and one C^+C product serve every system;
//   * the rows of every Liouvillian (Eq. lindblad) are built by one pair of
//     launches with the arithmetic of the single-system assembly;
//   * the trace weight w = mean |L_ii| of each system, the trace row of
//     Eq. (linear) and the compaction to one CSR per system take one launch
//     each;
//   * a hash of each system's pattern lets the host find the systems that
//     share an RCM ordering and a level schedule without downloading them;
//   * one gather puts every system's values in its pattern's RCM order.
#include <algorithm>
#include <cmath>
#include <vector>

#include "batched.cuh"
#include "common.cuh"

namespace {

inline unsigned grid_for(int64_t n, int b) { return (unsigned)std::max<int64_t>(1, (n + b - 1) / b); }

__device__ __forceinline__ int64_t system_of(const int64_t* __restrict__ row_off, int64_t ns, int64_t p) {
    int64_t lo = 0, hi = ns - 1;
    while (lo < hi) {
        int64_t mid = (lo + hi + 1) >> 1;
        if (row_off[mid] <= p) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// ------------------------------------------------------------ stacking

struct StackEntry {        // one device view placed in a block-diagonal stack
    const int32_t* rp;
    const int32_t* col;
    const double* val;     // interleaved (re, im); only 8-byte alignment is assumed
    int64_t d, nnz, doff, nzoff;
};

__global__ void stack_views(const StackEntry* __restrict__ tab, int32_t* __restrict__ rp, int32_t* __restrict__ col,
                            double2* __restrict__ val) {
    const StackEntry e = tab[blockIdx.y];
    const int64_t span = e.d > e.nnz ? e.d : e.nnz;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < span; t += (int64_t)gridDim.x * blockDim.x) {
        if (t < e.d) rp[e.doff + t] = (int32_t)(e.nzoff + e.rp[t]);
        if (t < e.nnz) {
            col[e.nzoff + t] = (int32_t)(e.col[t] + e.doff);
            val[e.nzoff + t] = make_double2(e.val[2 * t], e.val[2 * t + 1]);
        }
    }
}

// ---------------------------------------------------- trace weight w

// |L_rr| of row p (local row r), 0 when the row has no diagonal entry.
__device__ __forceinline__ double diag_abs(const BatchRows& R, int64_t p, int64_t r) {
    int32_t lo = R.off[p], hi = R.off[p] + R.cnt[p] - 1;
    while (lo <= hi) {
        const int32_t mid = (lo + hi) >> 1;
        const long long c = (long long)R.key[mid];
        if (c == r) return hypot(R.val[mid].x, R.val[mid].y);
        if (c < r) lo = mid + 1; else hi = mid - 1;
    }
    return 0.0;
}

// Sum of 256 values held 8 per lane (value of thread t = lane + 32 k in v[k]),
// added in the order of a shared-memory tree of 256 threads that halves the
// active range each step (t < o: s[t] += s[t + o], o = 128 ... 1).
__device__ __forceinline__ double tree256(double (&v)[8]) {
#pragma unroll
    for (int k = 0; k < 4; ++k) v[k] += v[k + 4];
    v[0] += v[2];
    v[1] += v[3];
    v[0] += v[1];
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) v[0] += __shfl_down_sync(0xffffffffu, v[0], o);
    return v[0];
}

// w = mean_i |L_ii| per system, summed in the order of the single-system
// reduction (256 blocks x 256 threads striding over the rows, a tree in each
// block, then a tree over the 256 block sums), so that a system's weight is
// the same alone, in any batch, and through add_trace_row.  w_in > 0 is used
// as given; an all-zero diagonal gives w = 1.
__global__ void __launch_bounds__(256) trace_weight_b(BatchRows R, const int64_t* __restrict__ row_off, double w_in,
                                                     double* __restrict__ w_out) {
    __shared__ double part[256];
    const int64_t s = blockIdx.x, p0 = row_off[s], n = row_off[s + 1] - p0;
    if (w_in > 0.0) {
        if (threadIdx.x == 0) w_out[s] = w_in;
        return;
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    constexpr int64_t STRIDE = 256 * 256;
    for (int vb = warp; vb < 256; vb += 8) {
        double v[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            double acc = 0.0;
            for (int64_t r = (int64_t)vb * 256 + lane + 32 * k; r < n; r += STRIDE) acc += diag_abs(R, p0 + r, r);
            v[k] = acc;
        }
        const double b = tree256(v);
        if (lane == 0) part[vb] = b;
    }
    __syncthreads();
    if (warp == 0) {
        double v[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) v[k] = 0.0 + part[lane + 32 * k];
        const double tot = tree256(v);
        if (lane == 0) {
            double w = tot * (1.0 / (double)n);
            w_out[s] = (w == 0.0) ? 1.0 : w;
        }
    }
}

// ------------------------------------------------------- trace row

// Row 0 of each system merged with w at the columns i (d + 1), i < d
// (Eq. linear: T has ones where the diagonal elements of rho sit), in place:
// the merge runs from the largest column down into the d spare slots after
// the row, then the result moves to the front.  Sums that are exactly zero
// are not stored, as in the single-system trace row.
__global__ void trace_merge_b(BatchRows R, const int64_t* __restrict__ row_off, const int64_t* __restrict__ doff,
                              const double* __restrict__ wv, int64_t ns) {
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= ns) return;
    const int64_t p = row_off[s], d = doff[s + 1] - doff[s];
    const int32_t base = R.off[p], m = R.cnt[p];
    const double w = wv[s];
    int64_t a = m - 1, ti = d - 1, out = m + d;
    while (a >= 0 || ti >= 0) {
        const long long tc = ti >= 0 ? (long long)(ti * (d + 1)) : -1;
        const long long lc = a >= 0 ? (long long)R.key[base + a] : -1;
        long long c;
        double2 v;
        if (lc > tc) { c = lc; v = R.val[base + a]; --a; }
        else if (tc > lc) { c = tc; v = make_double2(w, 0.0); --ti; }
        else { c = lc; v = make_double2(__dadd_rn(R.val[base + a].x, w), R.val[base + a].y); --a; --ti; }
        if (v.x != 0.0 || v.y != 0.0) {
            --out;
            R.key[base + out] = (unsigned long long)c;
            R.val[base + out] = v;
        }
    }
    const int32_t len = (int32_t)(m + d - out);
    for (int32_t t = 0; t < len; ++t) {
        R.key[base + t] = R.key[base + out + t];
        R.val[base + t] = R.val[base + out + t];
    }
    R.cnt[p] = len;
}

// ------------------------------------------------------- compaction

// Stored entries to the concatenated CSR: global positions from rpg (scan of
// the counts), system s's local row pointers at rp[row_off[s] + s ...].
__global__ void compact_b(BatchRows R, const int32_t* __restrict__ rpg, const int64_t* __restrict__ row_off, int64_t ns,
                          int32_t* __restrict__ rp, int32_t* __restrict__ col, double2* __restrict__ val) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= row_off[ns]) return;
    const int64_t s = system_of(row_off, ns, p), pl = p - row_off[s], n = row_off[s + 1] - row_off[s];
    const int32_t src = R.off[p], dst = rpg[p], m = rpg[p + 1] - dst, nz0 = rpg[row_off[s]];
    for (int32_t t = 0; t < m; ++t) {
        col[dst + t] = (int32_t)R.key[src + t];
        val[dst + t] = R.val[src + t];
    }
    rp[row_off[s] + s + pl] = dst - nz0;
    if (pl == n - 1) rp[row_off[s] + s + n] = rpg[p + 1] - nz0;
}

// ------------------------------------------------------ pattern hash

// SplitMix64 output function (G. Steele, D. Lea, C. Flood, "Fast splittable
// pseudorandom number generators", OOPSLA 2014) as a 64-bit mixer.
__device__ __forceinline__ unsigned long long mix64(unsigned long long z) {
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    return z ^ (z >> 31);
}

// Per system: offset and count of its entries and an order-free hash of its
// pattern (sum of mixed (row, column) pairs, with n and nnz).
__global__ void __launch_bounds__(256) pattern_meta_b(const int32_t* __restrict__ rpg, const int32_t* __restrict__ rp,
                                                     const int32_t* __restrict__ col,
                                                     const int64_t* __restrict__ row_off, BatchMeta* __restrict__ meta) {
    __shared__ unsigned long long red[8];
    const int64_t s = blockIdx.x, n = row_off[s + 1] - row_off[s];
    const int32_t nz0 = rpg[row_off[s]], nnz = rpg[row_off[s + 1]] - nz0;
    const int32_t* lrp = rp + row_off[s] + s;
    unsigned long long h = 0;
    for (int64_t r = threadIdx.x; r < n; r += blockDim.x)
        for (int32_t t = lrp[r]; t < lrp[r + 1]; ++t)
            h += mix64(((unsigned long long)r << 32) | (unsigned long long)(uint32_t)col[nz0 + t]);
    for (int o = 16; o >= 1; o >>= 1) h += __shfl_down_sync(0xffffffffu, h, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = h;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long t = 0;
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) t += red[k];
        meta[s].nz_off = nz0;
        meta[s].nnz = nnz;
        meta[s].hash = mix64(t ^ mix64((unsigned long long)n * 0x9e3779b97f4a7c15ull + (unsigned long long)nnz));
    }
}

// Members whose pattern hash equals their representative's: exact check.
__global__ void pattern_verify_b(const int2* __restrict__ pairs, const int32_t* __restrict__ rp,
                                 const int32_t* __restrict__ col, const int64_t* __restrict__ row_off,
                                 const BatchMeta* __restrict__ meta, int* __restrict__ mismatch) {
    const int2 pr = pairs[blockIdx.y];
    const int64_t a = pr.x, b = pr.y;
    const int64_t n = row_off[a + 1] - row_off[a];
    const int32_t* ra = rp + row_off[a] + a;
    const int32_t* rb = rp + row_off[b] + b;
    const int32_t* ca = col + meta[a].nz_off;
    const int32_t* cb = col + meta[b].nz_off;
    const int64_t nnz = meta[a].nnz;
    bool bad = false;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n + 1 || t < nnz;
         t += (int64_t)gridDim.x * blockDim.x) {
        if (t < n + 1 && ra[t] != rb[t]) bad = true;
        if (t < nnz && ca[t] != cb[t]) bad = true;
    }
    if (bad) atomicOr(&mismatch[blockIdx.y], 1);
}

// System s's pattern against a pattern held elsewhere on the device.
__global__ void pattern_compare(const int32_t* __restrict__ ra, const int32_t* __restrict__ ca,
                                const int32_t* __restrict__ rb, const int32_t* __restrict__ cb, int64_t n,
                                int64_t nnz, int* __restrict__ mismatch) {
    bool bad = false;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n + 1 || t < nnz;
         t += (int64_t)gridDim.x * blockDim.x) {
        if (t < n + 1 && ra[t] != rb[t]) bad = true;
        if (t < nnz && ca[t] != cb[t]) bad = true;
    }
    if (bad) atomicOr(mismatch, 1);
}

// --------------------------------------------------------- gather

__global__ void gather_values_b(const GatherEntry* __restrict__ tab, const double2* __restrict__ val) {
    const GatherEntry e = tab[blockIdx.y];
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < e.nnz; k += (int64_t)gridDim.x * blockDim.x)
        e.dst[k] = val[e.src_off + e.map[k]];
}

}  // namespace

void batch_lt_free(ss_ctx ctx, BatchLt& b) {
    dev_free(ctx, b.rp);
    dev_free(ctx, b.col);
    dev_free(ctx, b.val);
    dev_free(ctx, b.row_off_d);
    dev_free(ctx, b.meta_d);
    b = BatchLt();
}

ss_status batch_trace_systems(ss_ctx ctx, const std::vector<const ss_csr_view*>& H, const std::vector<int>& n_c,
                              const std::vector<const ss_csr_view*>& C, double w_in, BatchLt& out) {
    out = BatchLt();
    const int64_t ns = (int64_t)H.size();
    if (ns == 0) return SS_OK;
    // shapes and host-view contents
    int nc_max = 0;
    for (int64_t s = 0; s < ns; ++s) {
        SS_TRY(check_csr_view(ctx, H[s]));
        const int64_t d = H[s]->n_rows;
        if (H[s]->n_cols != d || d <= 0) return set_error(ctx, SS_ERR_INVALID, "H must be square and non-empty");
        if (d * d > INT32_MAX) return set_error(ctx, SS_ERR_UNSUPPORTED, "Liouvillian dimension exceeds 2^31-1");
        if (n_c[s] < 0 || (n_c[s] > 0 && !C[s])) return set_error(ctx, SS_ERR_INVALID, "null collapse operators");
        for (int c = 0; c < n_c[s]; ++c) {
            SS_TRY(check_csr_view(ctx, &C[s][c]));
            if (C[s][c].n_rows != d || C[s][c].n_cols != d)
                return set_error(ctx, SS_ERR_INVALID, "collapse operator " + std::to_string(c) + " is not d x d");
        }
        nc_max = std::max(nc_max, n_c[s]);
    }
    std::vector<int64_t> doff(ns + 1, 0), row_off(ns + 1, 0);
    for (int64_t s = 0; s < ns; ++s) {
        const int64_t d = H[s]->n_rows;
        doff[s + 1] = doff[s] + d;
        row_off[s + 1] = row_off[s] + d * d;
    }
    const int64_t D = doff[ns], P = row_off[ns];
    if (D > INT32_MAX || P + ns > INT32_MAX) return set_error(ctx, SS_ERR_UNSUPPORTED, "batch too large: split it");
    out.ns = ns;
    out.d.resize(ns);
    out.n.resize(ns);
    for (int64_t s = 0; s < ns; ++s) {
        out.d[s] = doff[s + 1] - doff[s];
        out.n[s] = row_off[s + 1] - row_off[s];
    }
    out.row_off = row_off;

    // block-diagonal stacks: slot 0 = H, slot 1 + c = C_c (empty blocks where absent)
    std::vector<DeviceCSR> stk(1 + nc_max);
    int64_t* doff_d = nullptr;
    BatchRows R;
    int32_t* rpg = nullptr;
    double* w_d = nullptr;
    auto fail = [&](ss_status e) {
        for (auto& m : stk) free_csr(ctx, m);
        dev_free(ctx, doff_d);
        dev_free(ctx, rpg);
        dev_free(ctx, w_d);
        batch_rows_free(ctx, R);
        batch_lt_free(ctx, out);
        return e;
    };
    ss_status st;
    if ((st = dev_alloc_n(ctx, &out.row_off_d, (size_t)ns + 1)) != SS_OK) return fail(st);
    if ((st = dev_alloc_n(ctx, &doff_d, (size_t)ns + 1)) != SS_OK) return fail(st);
    cudaError_t ce = cudaMemcpyAsync(out.row_off_d, row_off.data(), sizeof(int64_t) * (ns + 1), cudaMemcpyHostToDevice,
                                     ctx->stream);
    if (ce == cudaSuccess)
        ce = cudaMemcpyAsync(doff_d, doff.data(), sizeof(int64_t) * (ns + 1), cudaMemcpyHostToDevice, ctx->stream);
    if (ce != cudaSuccess) return fail(cuda_check(ctx, ce, "batch tables"));
    // host staging of every slot stays alive until the stream is synchronised below
    std::vector<std::vector<StackEntry>> tabs(1 + nc_max);
    std::vector<std::vector<int32_t>> rp_hs(1 + nc_max), col_hs(1 + nc_max);
    std::vector<std::vector<double2>> val_hs(1 + nc_max);
    for (int slot = 0; slot <= nc_max; ++slot) {
        auto view = [&](int64_t s) -> const ss_csr_view* {
            if (slot == 0) return H[s];
            return slot - 1 < n_c[s] ? &C[s][slot - 1] : nullptr;
        };
        std::vector<int64_t> nzoff(ns + 1, 0);
        bool any_host = false;
        for (int64_t s = 0; s < ns; ++s) {
            const ss_csr_view* v = view(s);
            nzoff[s + 1] = nzoff[s] + (v ? v->nnz : 0);
            any_host = any_host || (v && !v->on_device && v->nnz > 0);
        }
        const int64_t T = nzoff[ns];
        if (T > INT32_MAX) return fail(set_error(ctx, SS_ERR_UNSUPPORTED, "batch too large: split it"));
        DeviceCSR& m = stk[slot];
        m.n_rows = m.n_cols = D;
        m.nnz = T;
        if ((st = dev_alloc_n(ctx, &m.row_ptr, (size_t)D + 1)) != SS_OK) return fail(st);
        if ((st = dev_alloc_n(ctx, &m.col, (size_t)T)) != SS_OK) return fail(st);
        if ((st = dev_alloc_n(ctx, &m.val, (size_t)T)) != SS_OK) return fail(st);
        std::vector<int32_t>& rp_h = rp_hs[slot];
        std::vector<int32_t>& col_h = col_hs[slot];
        std::vector<double2>& val_h = val_hs[slot];
        rp_h.resize(D + 1);
        col_h.resize(any_host ? T : 0);
        val_h.resize(any_host ? T : 0);
        std::vector<StackEntry>& tab = tabs[slot];
        for (int64_t s = 0; s < ns; ++s) {
            const ss_csr_view* v = view(s);
            const int64_t d = out.d[s], o = doff[s];
            if (!v) {
                for (int64_t i = 0; i < d; ++i) rp_h[o + i] = (int32_t)nzoff[s];
            } else if (v->on_device) {
                if ((reinterpret_cast<uintptr_t>(v->row_ptr) & 3) || (reinterpret_cast<uintptr_t>(v->col) & 3) ||
                    (reinterpret_cast<uintptr_t>(v->val) & 7))
                    return fail(set_error(ctx, SS_ERR_INVALID, "misaligned device CSR view"));
                tab.push_back(StackEntry{v->row_ptr, v->col, v->val, d, v->nnz, o, nzoff[s]});
            } else {
                for (int64_t i = 0; i < d; ++i) rp_h[o + i] = (int32_t)(nzoff[s] + v->row_ptr[i]);
                for (int64_t t = 0; t < v->nnz; ++t) {
                    col_h[nzoff[s] + t] = (int32_t)(v->col[t] + o);
                    val_h[nzoff[s] + t] = make_double2(v->val[2 * t], v->val[2 * t + 1]);
                }
            }
        }
        rp_h[D] = (int32_t)T;
        ce = cudaMemcpyAsync(m.row_ptr, rp_h.data(), sizeof(int32_t) * (D + 1), cudaMemcpyHostToDevice, ctx->stream);
        if (ce == cudaSuccess && any_host)
            ce = cudaMemcpyAsync(m.col, col_h.data(), sizeof(int32_t) * T, cudaMemcpyHostToDevice, ctx->stream);
        if (ce == cudaSuccess && any_host)
            ce = cudaMemcpyAsync(m.val, val_h.data(), sizeof(double2) * T, cudaMemcpyHostToDevice, ctx->stream);
        if (ce != cudaSuccess) return fail(cuda_check(ctx, ce, "operator stack upload"));
        if (!tab.empty()) {
            // the table goes through its own small buffer per slot (the copy must not be overwritten in flight)
            StackEntry* td = nullptr;
            if ((st = dev_alloc_n(ctx, &td, tab.size())) != SS_OK) return fail(st);
            ce = cudaMemcpyAsync(td, tab.data(), sizeof(StackEntry) * tab.size(), cudaMemcpyHostToDevice, ctx->stream);
            if (ce == cudaSuccess) {
                int64_t span = 1;
                for (const auto& e : tab) span = std::max(span, std::max(e.d, e.nnz));
                for (size_t k0 = 0; ce == cudaSuccess && k0 < tab.size(); k0 += 65535) {
                    dim3 grid(std::min<unsigned>(grid_for(span, 256), 64u),
                              (unsigned)std::min<size_t>(65535, tab.size() - k0));
                    stack_views<<<(ss_count_launch(), grid), 256, 0, ctx->stream>>>(td + k0, m.row_ptr, m.col, m.val);
                    ce = cudaGetLastError();
                }
            }
            dev_free(ctx, td);
            if (ce != cudaSuccess) return fail(cuda_check(ctx, ce, "operator stack"));
        }
    }

    // rows of every Liouvillian, with d spare slots on each row 0 for the trace row
    std::vector<DeviceCSR> Cs(stk.begin() + 1, stk.end());
    if ((st = batch_lrows(ctx, stk[0], Cs, out.row_off_d, doff_d, ns, P, 1, R)) != SS_OK) return fail(st);
    for (auto& m : stk) free_csr(ctx, m);
    if ((st = dev_alloc_n(ctx, &w_d, (size_t)ns)) != SS_OK) return fail(st);
    trace_weight_b<<<(ss_count_launch(), (unsigned)ns), 256, 0, ctx->stream>>>(R, out.row_off_d, w_in, w_d);
    trace_merge_b<<<(ss_count_launch(), grid_for(ns, 128)), 128, 0, ctx->stream>>>(R, out.row_off_d, doff_d, w_d, ns);
    if ((ce = cudaGetLastError()) != cudaSuccess) return fail(cuda_check(ctx, ce, "trace row"));
    if ((st = dev_alloc_n(ctx, &rpg, (size_t)P + 1)) != SS_OK) return fail(st);
    int64_t nnz_tot = 0;
    if ((st = exclusive_scan_i32(ctx, R.cnt, rpg, P, &nnz_tot)) != SS_OK) return fail(st);
    if ((st = dev_alloc_n(ctx, &out.rp, (size_t)(P + ns))) != SS_OK) return fail(st);
    if ((st = dev_alloc_n(ctx, &out.col, (size_t)nnz_tot)) != SS_OK) return fail(st);
    if ((st = dev_alloc_n(ctx, &out.val, (size_t)nnz_tot)) != SS_OK) return fail(st);
    if ((st = dev_alloc_n(ctx, &out.meta_d, (size_t)ns)) != SS_OK) return fail(st);
    compact_b<<<(ss_count_launch(), grid_for(P, 256)), 256, 0, ctx->stream>>>(R, rpg, out.row_off_d, ns, out.rp, out.col,
                                                                              out.val);
    pattern_meta_b<<<(ss_count_launch(), (unsigned)ns), 256, 0, ctx->stream>>>(rpg, out.rp, out.col, out.row_off_d,
                                                                               out.meta_d);
    if ((ce = cudaGetLastError()) != cudaSuccess) return fail(cuda_check(ctx, ce, "compaction"));
    out.meta.resize(ns);
    out.w.resize(ns);
    ce = cudaMemcpyAsync(out.meta.data(), out.meta_d, sizeof(BatchMeta) * ns, cudaMemcpyDeviceToHost, ctx->stream);
    if (ce == cudaSuccess)
        ce = cudaMemcpyAsync(out.w.data(), w_d, sizeof(double) * ns, cudaMemcpyDeviceToHost, ctx->stream);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(ctx->stream);
    if (ce != cudaSuccess) return fail(cuda_check(ctx, ce, "batched setup"));
    batch_rows_free(ctx, R);
    dev_free(ctx, rpg);
    dev_free(ctx, w_d);
    dev_free(ctx, doff_d);
    rpg = nullptr;
    w_d = nullptr;
    doff_d = nullptr;
    for (int64_t s = 0; s < ns; ++s)
        if (!(out.w[s] > 0.0) || !std::isfinite(out.w[s]))
            return fail(set_error(ctx, SS_ERR_INVALID, "weight w must be positive and finite"));
    return SS_OK;
}

ss_status batch_verify_patterns(ss_ctx ctx, const BatchLt& b, const std::vector<std::pair<int, int>>& pairs,
                                std::vector<int>& mismatch) {
    mismatch.assign(pairs.size(), 0);
    if (pairs.empty()) return SS_OK;
    std::vector<int2> hp(pairs.size());
    int64_t span = 1;
    for (size_t k = 0; k < pairs.size(); ++k) {
        hp[k] = make_int2(pairs[k].first, pairs[k].second);
        span = std::max(span, std::max(b.n[pairs[k].first] + 1, b.meta[pairs[k].first].nnz));
    }
    int2* pd = nullptr;
    int* md = nullptr;
    SS_TRY(dev_alloc_n(ctx, &pd, hp.size()));
    ss_status st = dev_alloc_n(ctx, &md, hp.size());
    if (st != SS_OK) { dev_free(ctx, pd); return st; }
    cudaError_t ce = cudaMemcpyAsync(pd, hp.data(), sizeof(int2) * hp.size(), cudaMemcpyHostToDevice, ctx->stream);
    if (ce == cudaSuccess) ce = cudaMemsetAsync(md, 0, sizeof(int) * hp.size(), ctx->stream);
    if (ce == cudaSuccess) {
        for (size_t k0 = 0; k0 < hp.size(); k0 += 65535) {
            const unsigned ny = (unsigned)std::min<size_t>(65535, hp.size() - k0);
            dim3 grid(std::min<unsigned>(grid_for(span, 256), 64u), ny);
            pattern_verify_b<<<(ss_count_launch(), grid), 256, 0, ctx->stream>>>(pd + k0, b.rp, b.col, b.row_off_d,
                                                                                  b.meta_d, md + k0);
        }
        ce = cudaGetLastError();
    }
    if (ce == cudaSuccess)
        ce = cudaMemcpyAsync(mismatch.data(), md, sizeof(int) * hp.size(), cudaMemcpyDeviceToHost, ctx->stream);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(ctx->stream);
    dev_free(ctx, pd);
    dev_free(ctx, md);
    if (ce != cudaSuccess) return cuda_check(ctx, ce, "pattern verification");
    return SS_OK;
}

ss_status batch_download_pattern(ss_ctx ctx, const BatchLt& b, int s, std::vector<int32_t>& rp,
                                 std::vector<int32_t>& col) {
    rp.resize(b.n[s] + 1);
    col.resize(b.meta[s].nnz);
    SS_CUDA(ctx, cudaMemcpyAsync(rp.data(), b.rp + b.row_off[s] + s, sizeof(int32_t) * rp.size(),
                                 cudaMemcpyDeviceToHost, ctx->stream));
    if (!col.empty())
        SS_CUDA(ctx, cudaMemcpyAsync(col.data(), b.col + b.meta[s].nz_off, sizeof(int32_t) * col.size(),
                                     cudaMemcpyDeviceToHost, ctx->stream));
    return SS_OK;
}

ss_status batch_gather_values(ss_ctx ctx, const BatchLt& b, const std::vector<GatherEntry>& tab) {
    if (tab.empty()) return SS_OK;
    GatherEntry* td = nullptr;
    SS_TRY(dev_alloc_n(ctx, &td, tab.size()));
    int64_t span = 1;
    for (const auto& e : tab) span = std::max(span, e.nnz);
    cudaError_t ce = cudaMemcpyAsync(td, tab.data(), sizeof(GatherEntry) * tab.size(), cudaMemcpyHostToDevice,
                                     ctx->stream);
    for (size_t k0 = 0; ce == cudaSuccess && k0 < tab.size(); k0 += 65535) {
        const unsigned ny = (unsigned)std::min<size_t>(65535, tab.size() - k0);
        dim3 grid(std::min<unsigned>(grid_for(span, 256), 64u), ny);
        gather_values_b<<<(ss_count_launch(), grid), 256, 0, ctx->stream>>>(td + k0, b.val);
        ce = cudaGetLastError();
    }
    dev_free(ctx, td);
    if (ce != cudaSuccess) return cuda_check(ctx, ce, "value gather");
    return SS_OK;
}

ss_status batch_verify_against(ss_ctx ctx, const BatchLt& b, int s, const int32_t* rp_d, const int32_t* col_d,
                               int* mismatch) {
    *mismatch = 1;
    int* md = nullptr;
    SS_TRY(dev_alloc_n(ctx, &md, 1));
    const int64_t n = b.n[s], nnz = b.meta[s].nnz;
    cudaError_t ce = cudaMemsetAsync(md, 0, sizeof(int), ctx->stream);
    if (ce == cudaSuccess) {
        pattern_compare<<<(ss_count_launch(), std::min<unsigned>(grid_for(std::max(n + 1, nnz), 256), 128u)), 256, 0,
                           ctx->stream>>>(b.rp + b.row_off[s] + s, b.col + b.meta[s].nz_off, rp_d, col_d, n, nnz, md);
        ce = cudaGetLastError();
    }
    if (ce == cudaSuccess) ce = cudaMemcpyAsync(mismatch, md, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(ctx->stream);
    dev_free(ctx, md);
    if (ce != cudaSuccess) return cuda_check(ctx, ce, "pattern verification");
    return SS_OK;
}

// ------------------------------------------------------- cost estimate

namespace {

// Per system: the squared Frobenius norms of the diagonal and of the
// off-diagonal entries of L~ (one block per system, fixed-order sums).
__global__ void diag_offdiag_b(const int32_t* __restrict__ rp, const int32_t* __restrict__ col,
                               const double2* __restrict__ val, const int64_t* __restrict__ row_off,
                               const BatchMeta* __restrict__ meta, double2* __restrict__ out) {
    const int64_t s = blockIdx.x;
    const int64_t n = row_off[s + 1] - row_off[s];
    const int32_t* lrp = rp + row_off[s] + s;
    const int32_t* lcol = col + meta[s].nz_off;
    const double2* lval = val + meta[s].nz_off;
    double dg = 0.0, off = 0.0;
    for (int64_t r = threadIdx.x; r < n; r += blockDim.x)
        for (int32_t t = lrp[r]; t < lrp[r + 1]; ++t) {
            const double m2 = lval[t].x * lval[t].x + lval[t].y * lval[t].y;
            if (lcol[t] == r) dg += m2; else off += m2;
        }
    __shared__ double sd[256], so[256];
    sd[threadIdx.x] = dg;
    so[threadIdx.x] = off;
    __syncthreads();
    for (int h = blockDim.x / 2; h > 0; h >>= 1) {
        if ((int)threadIdx.x < h) {
            sd[threadIdx.x] += sd[threadIdx.x + h];
            so[threadIdx.x] += so[threadIdx.x + h];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) out[s] = make_double2(sd[0], so[0]);
}

}  // namespace

ss_status batch_cost_order(ss_ctx ctx, const BatchLt& b, std::vector<int32_t>& order, std::vector<double2>* fp) {
    const int64_t ns = b.ns;
    order.resize(ns);
    for (int64_t s = 0; s < ns; ++s) order[s] = (int32_t)s;
    if (ns == 0) return SS_OK;
    double2* nd = nullptr;
    SS_TRY(dev_alloc_n(ctx, &nd, (size_t)ns));
    std::vector<double2> h(ns);
    diag_offdiag_b<<<(ss_count_launch(), (unsigned)ns), 256, 0, ctx->stream>>>(b.rp, b.col, b.val, b.row_off_d,
                                                                             b.meta_d, nd);
    cudaError_t ce = cudaGetLastError();
    if (ce == cudaSuccess) ce = cudaMemcpyAsync(h.data(), nd, sizeof(double2) * ns, cudaMemcpyDeviceToHost, ctx->stream);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(ctx->stream);
    dev_free(ctx, nd);
    if (ce != cudaSuccess) return cuda_check(ctx, ce, "cost estimate");
    if (fp) fp->assign(h.begin(), h.end());
    std::vector<double> cost(ns);
    for (int64_t s = 0; s < ns; ++s) {
        const double ratio = h[s].x > 0.0 ? std::sqrt(h[s].y / h[s].x) : 1.0;
        cost[s] = (double)b.meta[s].nnz * (1.0 + ratio);
    }
    std::stable_sort(order.begin(), order.end(), [&](int32_t a, int32_t c) { return cost[a] > cost[c]; });
    return SS_OK;
}
