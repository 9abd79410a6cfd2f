// On-device assembly of the Lindblad Liouvillian (Eq. lindblad, vectorised by
// column stacking as in Eq. eigval):
//
//   L = -i (I kron H - H^T kron I)
//       + sum_k ( conj(C_k) kron C_k - 1/2 I kron C_k^+C_k - 1/2 (C_k^+C_k)^T kron I ).
//
// Row p = i + d j of L is the equation for d rho_ij / dt; column q = k + d l
// multiplies rho_kl.  Its entries come from
//   H-term      : l = j, k in row i of H         (+H_ik)
//                 k = i, l in column j of H      (-H_lj)      then times -i
//   per C       : l in row j of C, k in row i of C   (+conj(C_jl) C_ik)
//                 l = j, k in row i of C^+C          (-1/2 (C^+C)_ik)
//                 k = i, l in column j of C^+C       (-1/2 (C^+C)_lj)
// Every row is built as a list of (column, term) candidates that is sorted
// and then summed term by term in the order the sum above is written:
// val = -i (H_ik - H_lj), then for each operator in turn
// val = ((val + conj(C_jl) C_ik) - (C^+C)_ik / 2) - (C^+C)_lj / 2.
// Entries whose sum is exactly zero are not stored.  All products and sums use
// explicit round-to-nearest intrinsics so the compiler contracts nothing.
#include <vector>

#include "common.cuh"

namespace {

__device__ __forceinline__ double2 mul_rn(double2 a, double2 b) {
    return make_double2(__dsub_rn(__dmul_rn(a.x, b.x), __dmul_rn(a.y, b.y)),
                        __dadd_rn(__dmul_rn(a.x, b.y), __dmul_rn(a.y, b.x)));
}
__device__ __forceinline__ double2 add_rn(double2 a, double2 b) {
    return make_double2(__dadd_rn(a.x, b.x), __dadd_rn(a.y, b.y));
}
__device__ __forceinline__ double2 sub_rn(double2 a, double2 b) {
    return make_double2(__dsub_rn(a.x, b.x), __dsub_rn(a.y, b.y));
}

struct CsrRef {
    const int32_t* rp;
    const int32_t* col;
    const double2* val;
};

// ---------------------------------------------------------------- transpose

__global__ void count_cols(const int32_t* __restrict__ col, int64_t nnz, int32_t* __restrict__ cnt) {
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < nnz) atomicAdd(&cnt[col[t]], 1);
}

__global__ void scatter_transpose(CsrRef a, int64_t n_rows, int32_t* __restrict__ cursor,
                                  int32_t* __restrict__ tcol, double2* __restrict__ tval) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_rows) return;
    for (int32_t t = a.rp[i]; t < a.rp[i + 1]; ++t) {
        int32_t pos = atomicAdd(&cursor[a.col[t]], 1);
        tcol[pos] = (int32_t)i;
        tval[pos] = a.val[t];
    }
}

// Insertion sort of each row segment by column index (rows are short).
__global__ void sort_rows(const int32_t* __restrict__ rp, int64_t n_rows, int32_t* __restrict__ col,
                          double2* __restrict__ val) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_rows) return;
    int32_t a = rp[i], b = rp[i + 1];
    for (int32_t t = a + 1; t < b; ++t) {
        int32_t c = col[t];
        double2 v = val[t];
        int32_t u = t - 1;
        while (u >= a && col[u] > c) {
            col[u + 1] = col[u];
            val[u + 1] = val[u];
            --u;
        }
        col[u + 1] = c;
        val[u + 1] = v;
    }
}

// --------------------------------------------------------------- C^+ C
// Row k of C^+C = sum over i in column k of C of conj(C_ik) * (row i of C),
// contributions to one column summed in ascending i.

__global__ void ctc_count(CsrRef ct, CsrRef c, int64_t d, int32_t* __restrict__ cnt) {
    int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= d) return;
    int32_t s = 0;
    for (int32_t t = ct.rp[k]; t < ct.rp[k + 1]; ++t) {
        int32_t i = ct.col[t];
        s += c.rp[i + 1] - c.rp[i];
    }
    cnt[k] = s;
}

__global__ void ctc_fill(CsrRef ct, CsrRef c, int64_t d, const int32_t* __restrict__ off,
                         int32_t* __restrict__ kcol, double2* __restrict__ kval, int32_t* __restrict__ outcnt) {
    int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= d) return;
    int32_t base = off[k], m = 0;
    for (int32_t t = ct.rp[k]; t < ct.rp[k + 1]; ++t) {
        int32_t i = ct.col[t];
        double2 v = cconj(ct.val[t]);                       // conj(C_ik)
        for (int32_t u = c.rp[i]; u < c.rp[i + 1]; ++u) {
            kcol[base + m] = c.col[u];
            kval[base + m] = mul_rn(v, c.val[u]);
            ++m;
        }
    }
    // stable insertion sort by column, then sum equal columns in order
    for (int32_t t = 1; t < m; ++t) {
        int32_t cc = kcol[base + t];
        double2 vv = kval[base + t];
        int32_t u = t - 1;
        while (u >= 0 && kcol[base + u] > cc) {
            kcol[base + u + 1] = kcol[base + u];
            kval[base + u + 1] = kval[base + u];
            --u;
        }
        kcol[base + u + 1] = cc;
        kval[base + u + 1] = vv;
    }
    int32_t w = 0;
    for (int32_t t = 0; t < m;) {
        int32_t cc = kcol[base + t];
        double2 acc = make_double2(0.0, 0.0);
        while (t < m && kcol[base + t] == cc) {
            acc = add_rn(acc, kval[base + t]);
            ++t;
        }
        if (acc.x != 0.0 || acc.y != 0.0) {
            kcol[base + w] = cc;
            kval[base + w] = acc;
            ++w;
        }
    }
    outcnt[k] = w;
}

__global__ void compact_rows(const int32_t* __restrict__ src_off, const int32_t* __restrict__ dst_off, int64_t n,
                             const int32_t* __restrict__ scol, const double2* __restrict__ sval,
                             int32_t* __restrict__ dcol, double2* __restrict__ dval) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int32_t s = src_off[i], d0 = dst_off[i], m = dst_off[i + 1] - d0;
    for (int32_t t = 0; t < m; ++t) {
        dcol[d0 + t] = scol[s + t];
        dval[d0 + t] = sval[s + t];
    }
}

// ------------------------------------------------------------ Kronecker rows

struct OpSet {            // per collapse operator: C, C^+C, (C^+C)^T
    CsrRef c, ctc, ctct;
};

// Number of candidates of row (i, j) of L.  gi = row i and gj = row j of the
// operators, which may be blocks of a block-diagonal stack (see row_build).
__device__ __forceinline__ int64_t row_count(const CsrRef& h, const CsrRef& ht, const OpSet* __restrict__ ops, int n_c,
                                             int64_t gi, int64_t gj) {
    int64_t s = (h.rp[gi + 1] - h.rp[gi]) + (ht.rp[gj + 1] - ht.rp[gj]);
    for (int c = 0; c < n_c; ++c) {
        const OpSet& o = ops[c];
        s += (int64_t)(o.c.rp[gj + 1] - o.c.rp[gj]) * (o.c.rp[gi + 1] - o.c.rp[gi]);
        s += o.ctc.rp[gi + 1] - o.ctc.rp[gi];
        s += o.ctct.rp[gj + 1] - o.ctct.rp[gj];
    }
    return s;
}

// Candidates of row p = i + d j of L, written from key/val[base], sorted and
// summed in place; returns the number of stored (non-zero) entries, whose keys
// are then the column indices.  The operators' rows and columns are offset by
// doff (a system inside a block-diagonal stack; 0 for a single system).
// Candidate key = column * T + term, T = 2 + 3 n_c.  Terms: 0 (+H_ik),
// 1 (H_lj, subtracted), 2 + 3c + {0: conj(C_jl) C_ik, 1: (C^+C)_ik, 2: (C^+C)_lj}.
__device__ int32_t row_build(const CsrRef& h, const CsrRef& ht, const OpSet* __restrict__ ops, int n_c, int64_t d,
                             int64_t doff, int64_t i, int64_t j, int32_t base, unsigned long long* __restrict__ key,
                             double2* __restrict__ val) {
    const unsigned long long T = 2ull + 3ull * (unsigned long long)n_c;
    const int64_t gi = doff + i, gj = doff + j;
    int32_t m = 0;
    for (int32_t t = h.rp[gi]; t < h.rp[gi + 1]; ++t) {         // l = j, k = col
        unsigned long long q = (unsigned long long)(h.col[t] - doff + d * j);
        key[base + m] = q * T + 0;
        val[base + m] = h.val[t];
        ++m;
    }
    for (int32_t t = ht.rp[gj]; t < ht.rp[gj + 1]; ++t) {       // k = i, l = row of H
        unsigned long long q = (unsigned long long)(i + d * (ht.col[t] - doff));
        key[base + m] = q * T + 1;
        val[base + m] = ht.val[t];
        ++m;
    }
    for (int c = 0; c < n_c; ++c) {
        const OpSet& o = ops[c];
        unsigned long long tb = 2ull + 3ull * c;
        for (int32_t a = o.c.rp[gj]; a < o.c.rp[gj + 1]; ++a) {
            int64_t l = o.c.col[a] - doff;
            double2 cj = cconj(o.c.val[a]);                      // conj(C_jl)
            for (int32_t b = o.c.rp[gi]; b < o.c.rp[gi + 1]; ++b) {
                unsigned long long q = (unsigned long long)(o.c.col[b] - doff + d * l);
                key[base + m] = q * T + tb;
                val[base + m] = mul_rn(cj, o.c.val[b]);
                ++m;
            }
        }
        for (int32_t t = o.ctc.rp[gi]; t < o.ctc.rp[gi + 1]; ++t) {
            unsigned long long q = (unsigned long long)(o.ctc.col[t] - doff + d * j);
            key[base + m] = q * T + tb + 1;
            val[base + m] = o.ctc.val[t];
            ++m;
        }
        for (int32_t t = o.ctct.rp[gj]; t < o.ctct.rp[gj + 1]; ++t) {
            unsigned long long q = (unsigned long long)(i + d * (o.ctct.col[t] - doff));
            key[base + m] = q * T + tb + 2;
            val[base + m] = o.ctct.val[t];
            ++m;
        }
    }
    // insertion sort by key (terms of one column end up in term order)
    for (int32_t t = 1; t < m; ++t) {
        unsigned long long kk = key[base + t];
        double2 vv = val[base + t];
        int32_t u = t - 1;
        while (u >= 0 && key[base + u] > kk) {
            key[base + u + 1] = key[base + u];
            val[base + u + 1] = val[base + u];
            --u;
        }
        key[base + u + 1] = kk;
        val[base + u + 1] = vv;
    }
    // merge: evaluate each column's sum in the written order
    int32_t w = 0;
    for (int32_t t = 0; t < m;) {
        unsigned long long q = key[base + t] / T;
        double2 acc = make_double2(0.0, 0.0);
        bool has_h = false;
        double2 hv = make_double2(0.0, 0.0);
        while (t < m && key[base + t] / T == q) {
            unsigned long long term = key[base + t] % T;
            double2 v = val[base + t];
            if (term == 0) {
                hv = v;
                has_h = true;
            } else if (term == 1) {
                hv = has_h ? sub_rn(hv, v) : make_double2(-v.x, -v.y);
                has_h = true;
            } else {
                if (has_h) {                                   // close the H group: times -i
                    acc = make_double2(hv.y, -hv.x);
                    has_h = false;
                }
                unsigned long long r = (term - 2) % 3;
                if (r == 0) {
                    acc = add_rn(acc, v);
                } else {
                    acc = sub_rn(acc, make_double2(__dmul_rn(0.5, v.x), __dmul_rn(0.5, v.y)));
                }
            }
            ++t;
        }
        if (has_h) acc = make_double2(hv.y, -hv.x);
        if (acc.x != 0.0 || acc.y != 0.0) {
            key[base + w] = q;
            val[base + w] = acc;
            ++w;
        }
    }
    return w;
}

__global__ void lrow_count(CsrRef h, CsrRef ht, const OpSet* __restrict__ ops, int n_c, int64_t d,
                           int32_t* __restrict__ cnt) {
    int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= d * d) return;
    cnt[p] = (int32_t)row_count(h, ht, ops, n_c, p % d, p / d);
}

__global__ void lrow_build(CsrRef h, CsrRef ht, const OpSet* __restrict__ ops, int n_c, int64_t d,
                           const int32_t* __restrict__ off, unsigned long long* __restrict__ key,
                           double2* __restrict__ val, int32_t* __restrict__ outcnt) {
    int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= d * d) return;
    outcnt[p] = row_build(h, ht, ops, n_c, d, 0, p % d, p / d, off[p], key, val);
}

// Batched forms: the operators of several systems stacked block-diagonally;
// system s owns operator rows [doff[s], doff[s+1]) and rows
// [row_off[s], row_off[s+1]) of the concatenated Liouvillians.
__device__ __forceinline__ int64_t find_system(const int64_t* __restrict__ row_off, int64_t nsys, int64_t p) {
    int64_t lo = 0, hi = nsys - 1;
    while (lo < hi) {                      // last s with row_off[s] <= p
        int64_t mid = (lo + hi + 1) >> 1;
        if (row_off[mid] <= p) lo = mid; else hi = mid - 1;
    }
    return lo;
}

__global__ void lrow_count_b(CsrRef h, CsrRef ht, const OpSet* __restrict__ ops, int n_c,
                             const int64_t* __restrict__ row_off, const int64_t* __restrict__ doff, int64_t nsys,
                             int32_t reserve_row0, int32_t* __restrict__ cnt) {
    int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= row_off[nsys]) return;
    const int64_t s = find_system(row_off, nsys, p), pl = p - row_off[s];
    const int64_t d = doff[s + 1] - doff[s];
    int64_t c = row_count(h, ht, ops, n_c, doff[s] + pl % d, doff[s] + pl / d);
    if (pl == 0) c += reserve_row0 ? d : 0;
    cnt[p] = (int32_t)c;
}

__global__ void lrow_build_b(CsrRef h, CsrRef ht, const OpSet* __restrict__ ops, int n_c,
                             const int64_t* __restrict__ row_off, const int64_t* __restrict__ doff, int64_t nsys,
                             const int32_t* __restrict__ off, unsigned long long* __restrict__ key,
                             double2* __restrict__ val, int32_t* __restrict__ outcnt) {
    int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= row_off[nsys]) return;
    const int64_t s = find_system(row_off, nsys, p), pl = p - row_off[s];
    const int64_t d = doff[s + 1] - doff[s];
    outcnt[p] = row_build(h, ht, ops, n_c, d, doff[s], pl % d, pl / d, off[p], key, val);
}

__global__ void lrow_compact(const int32_t* __restrict__ src_off, const int32_t* __restrict__ dst_off, int64_t n,
                             const unsigned long long* __restrict__ key, const double2* __restrict__ sval,
                             int32_t* __restrict__ dcol, double2* __restrict__ dval) {
    int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    int32_t s = src_off[p], d0 = dst_off[p], m = dst_off[p + 1] - d0;
    for (int32_t t = 0; t < m; ++t) {
        dcol[d0 + t] = (int32_t)key[s + t];
        dval[d0 + t] = sval[s + t];
    }
}

inline unsigned grid_for(int64_t n, int b) { return (unsigned)((n + b - 1) / b); }

ss_status transpose_csr(ss_ctx ctx, const DeviceCSR& a, DeviceCSR& t) {
    t = DeviceCSR();
    t.n_rows = a.n_cols;
    t.n_cols = a.n_rows;
    t.nnz = a.nnz;
    int32_t* cnt = nullptr;
    SS_TRY(dev_alloc_n(ctx, &cnt, (size_t)a.n_cols + 1));
    SS_TRY(dev_alloc_n(ctx, &t.row_ptr, (size_t)a.n_cols + 1));
    SS_TRY(dev_alloc_n(ctx, &t.col, (size_t)a.nnz));
    SS_TRY(dev_alloc_n(ctx, &t.val, (size_t)a.nnz));
    SS_CUDA(ctx, cudaMemsetAsync(cnt, 0, sizeof(int32_t) * (a.n_cols + 1), ctx->stream));
    if (a.nnz > 0) count_cols<<<(ss_count_launch(), grid_for(a.nnz, 256)), 256, 0, ctx->stream>>>(a.col, a.nnz, cnt);
    SS_TRY(exclusive_scan_i32(ctx, cnt, t.row_ptr, a.n_cols, nullptr));
    SS_CUDA(ctx, cudaMemcpyAsync(cnt, t.row_ptr, sizeof(int32_t) * (a.n_cols + 1), cudaMemcpyDeviceToDevice,
                                 ctx->stream));
    if (a.n_rows > 0)
        scatter_transpose<<<(ss_count_launch(), grid_for(a.n_rows, 128)), 128, 0, ctx->stream>>>(CsrRef{a.row_ptr, a.col, a.val}, a.n_rows,
                                                                            cnt, t.col, t.val);
    if (t.n_rows > 0) sort_rows<<<(ss_count_launch(), grid_for(t.n_rows, 128)), 128, 0, ctx->stream>>>(t.row_ptr, t.n_rows, t.col, t.val);
    SS_CUDA(ctx, cudaGetLastError());
    dev_free(ctx, cnt);
    return SS_OK;
}

// C^+ C for one operator (d x d)
ss_status ctc_csr(ss_ctx ctx, const DeviceCSR& c, const DeviceCSR& ct, DeviceCSR& out) {
    int64_t d = c.n_rows;
    out = DeviceCSR();
    out.n_rows = out.n_cols = d;
    int32_t *cnt = nullptr, *off = nullptr, *cnt2 = nullptr, *kcol = nullptr;
    double2* kval = nullptr;
    SS_TRY(dev_alloc_n(ctx, &cnt, (size_t)d + 1));
    SS_TRY(dev_alloc_n(ctx, &off, (size_t)d + 1));
    SS_TRY(dev_alloc_n(ctx, &cnt2, (size_t)d + 1));
    ctc_count<<<(ss_count_launch(), grid_for(d, 128)), 128, 0, ctx->stream>>>(CsrRef{ct.row_ptr, ct.col, ct.val},
                                                          CsrRef{c.row_ptr, c.col, c.val}, d, cnt);
    int64_t total = 0;
    SS_TRY(exclusive_scan_i32(ctx, cnt, off, d, &total));
    SS_TRY(dev_alloc_n(ctx, &kcol, (size_t)total));
    SS_TRY(dev_alloc_n(ctx, &kval, (size_t)total));
    ctc_fill<<<(ss_count_launch(), grid_for(d, 128)), 128, 0, ctx->stream>>>(CsrRef{ct.row_ptr, ct.col, ct.val},
                                                         CsrRef{c.row_ptr, c.col, c.val}, d, off, kcol, kval, cnt2);
    SS_TRY(dev_alloc_n(ctx, &out.row_ptr, (size_t)d + 1));
    int64_t nnz = 0;
    SS_TRY(exclusive_scan_i32(ctx, cnt2, out.row_ptr, d, &nnz));
    out.nnz = nnz;
    SS_TRY(dev_alloc_n(ctx, &out.col, (size_t)nnz));
    SS_TRY(dev_alloc_n(ctx, &out.val, (size_t)nnz));
    compact_rows<<<(ss_count_launch(), grid_for(d, 128)), 128, 0, ctx->stream>>>(off, out.row_ptr, d, kcol, kval, out.col, out.val);
    SS_CUDA(ctx, cudaGetLastError());
    dev_free(ctx, cnt);
    dev_free(ctx, off);
    dev_free(ctx, cnt2);
    dev_free(ctx, kcol);
    dev_free(ctx, kval);
    return SS_OK;
}

}  // namespace

namespace {

struct OpPrep {                       // H^T and, per collapse operator, C^T, C^+C, (C^+C)^T
    DeviceCSR Ht;
    std::vector<DeviceCSR> Ct, CtC, CtCt;
    std::vector<OpSet> hops;          // host copy of the table (kept until the copy has run)
    OpSet* dops = nullptr;            // device table of the operator triples
};

void free_ops(ss_ctx ctx, OpPrep& o) {
    dev_free(ctx, o.dops);
    o.dops = nullptr;
    free_csr(ctx, o.Ht);
    for (size_t c = 0; c < o.Ct.size(); ++c) {
        free_csr(ctx, o.Ct[c]);
        free_csr(ctx, o.CtC[c]);
        free_csr(ctx, o.CtCt[c]);
    }
}

ss_status prep_ops(ss_ctx ctx, const DeviceCSR& H, const std::vector<DeviceCSR>& C, OpPrep& o) {
    const int n_c = (int)C.size();
    SS_TRY(transpose_csr(ctx, H, o.Ht));
    o.Ct.resize(n_c);
    o.CtC.resize(n_c);
    o.CtCt.resize(n_c);
    std::vector<OpSet>& hops = o.hops;
    hops.resize(n_c);
    for (int c = 0; c < n_c; ++c) {
        SS_TRY(transpose_csr(ctx, C[c], o.Ct[c]));
        SS_TRY(ctc_csr(ctx, C[c], o.Ct[c], o.CtC[c]));
        SS_TRY(transpose_csr(ctx, o.CtC[c], o.CtCt[c]));
        hops[c].c = CsrRef{C[c].row_ptr, C[c].col, C[c].val};
        hops[c].ctc = CsrRef{o.CtC[c].row_ptr, o.CtC[c].col, o.CtC[c].val};
        hops[c].ctct = CsrRef{o.CtCt[c].row_ptr, o.CtCt[c].col, o.CtCt[c].val};
    }
    SS_TRY(dev_alloc_n(ctx, &o.dops, (size_t)(n_c > 0 ? n_c : 1)));
    if (n_c > 0)
        SS_CUDA(ctx, cudaMemcpyAsync(o.dops, hops.data(), sizeof(OpSet) * n_c, cudaMemcpyHostToDevice, ctx->stream));
    return SS_OK;
}

}  // namespace

ss_status assemble_impl(ss_ctx ctx, const DeviceCSR& H, const std::vector<DeviceCSR>& C, DeviceCSR& L) {
    L = DeviceCSR();
    const int64_t d = H.n_rows;
    const int64_t n = d * d;
    if (n > INT32_MAX) return set_error(ctx, SS_ERR_UNSUPPORTED, "Liouvillian dimension exceeds 2^31-1");
    const int n_c = (int)C.size();
    OpPrep o;
    ss_status st = prep_ops(ctx, H, C, o);
    if (st != SS_OK) { free_ops(ctx, o); return st; }
    OpSet* dops = o.dops;
    const DeviceCSR& Ht = o.Ht;

    int32_t *cnt = nullptr, *off = nullptr, *cnt2 = nullptr;
    SS_TRY(dev_alloc_n(ctx, &cnt, (size_t)n + 1));
    SS_TRY(dev_alloc_n(ctx, &off, (size_t)n + 1));
    SS_TRY(dev_alloc_n(ctx, &cnt2, (size_t)n + 1));
    CsrRef h{H.row_ptr, H.col, H.val}, ht{Ht.row_ptr, Ht.col, Ht.val};
    lrow_count<<<(ss_count_launch(), grid_for(n, 256)), 256, 0, ctx->stream>>>(h, ht, dops, n_c, d, cnt);
    int64_t total = 0;
    SS_TRY(exclusive_scan_i32(ctx, cnt, off, n, &total));
    unsigned long long* key = nullptr;
    double2* val = nullptr;
    SS_TRY(dev_alloc_n(ctx, &key, (size_t)total));
    SS_TRY(dev_alloc_n(ctx, &val, (size_t)total));
    lrow_build<<<(ss_count_launch(), grid_for(n, 128)), 128, 0, ctx->stream>>>(h, ht, dops, n_c, d, off, key, val, cnt2);
    L.n_rows = L.n_cols = n;
    SS_TRY(dev_alloc_n(ctx, &L.row_ptr, (size_t)n + 1));
    int64_t nnz = 0;
    SS_TRY(exclusive_scan_i32(ctx, cnt2, L.row_ptr, n, &nnz));
    L.nnz = nnz;
    SS_TRY(dev_alloc_n(ctx, &L.col, (size_t)nnz));
    SS_TRY(dev_alloc_n(ctx, &L.val, (size_t)nnz));
    lrow_compact<<<(ss_count_launch(), grid_for(n, 256)), 256, 0, ctx->stream>>>(off, L.row_ptr, n, key, val, L.col, L.val);
    SS_CUDA(ctx, cudaGetLastError());

    dev_free(ctx, key);
    dev_free(ctx, val);
    dev_free(ctx, cnt);
    dev_free(ctx, off);
    dev_free(ctx, cnt2);
    free_ops(ctx, o);
    return SS_OK;
}

ss_status batch_lrows(ss_ctx ctx, const DeviceCSR& H, const std::vector<DeviceCSR>& C, const int64_t* row_off_d,
                      const int64_t* doff_d, int64_t nsys, int64_t P, int32_t reserve_row0, BatchRows& out) {
    out = BatchRows();
    const int n_c = (int)C.size();
    OpPrep o;
    ss_status st = prep_ops(ctx, H, C, o);
    if (st != SS_OK) { free_ops(ctx, o); return st; }
    CsrRef h{H.row_ptr, H.col, H.val}, ht{o.Ht.row_ptr, o.Ht.col, o.Ht.val};
    int32_t* cnt = nullptr;
    auto fail = [&](ss_status e) { dev_free(ctx, cnt); free_ops(ctx, o); batch_rows_free(ctx, out); return e; };
    if ((st = dev_alloc_n(ctx, &cnt, (size_t)P + 1)) != SS_OK) return fail(st);
    if ((st = dev_alloc_n(ctx, &out.off, (size_t)P + 1)) != SS_OK) return fail(st);
    if ((st = dev_alloc_n(ctx, &out.cnt, (size_t)P + 1)) != SS_OK) return fail(st);
    if (P > 0)
        lrow_count_b<<<(ss_count_launch(), grid_for(P, 256)), 256, 0, ctx->stream>>>(h, ht, o.dops, n_c, row_off_d,
                                                                                      doff_d, nsys, reserve_row0, cnt);
    if ((st = exclusive_scan_i32(ctx, cnt, out.off, P, &out.total)) != SS_OK) return fail(st);
    if ((st = dev_alloc_n(ctx, &out.key, (size_t)out.total)) != SS_OK) return fail(st);
    if ((st = dev_alloc_n(ctx, &out.val, (size_t)out.total)) != SS_OK) return fail(st);
    if (P > 0)
        lrow_build_b<<<(ss_count_launch(), grid_for(P, 128)), 128, 0, ctx->stream>>>(
            h, ht, o.dops, n_c, row_off_d, doff_d, nsys, out.off, out.key, out.val, out.cnt);
    cudaError_t e = cudaGetLastError();
    dev_free(ctx, cnt);
    cnt = nullptr;
    free_ops(ctx, o);
    if (e != cudaSuccess) {
        batch_rows_free(ctx, out);
        return cuda_check(ctx, e, "batched Liouvillian rows");
    }
    return SS_OK;
}

void batch_rows_free(ss_ctx ctx, BatchRows& r) {
    dev_free(ctx, r.off);
    dev_free(ctx, r.cnt);
    dev_free(ctx, r.key);
    dev_free(ctx, r.val);
    r = BatchRows();
}
