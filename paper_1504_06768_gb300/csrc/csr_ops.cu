// Structural CSR kernels: the trace row of Eq. (linear), the shift of
// Eq. (inverse), the symmetric permutation P A P^T, and the bandwidth /
// profile of the section "Direct factorization".
#include <vector>

#include "common.cuh"

namespace {

inline unsigned grid_for(int64_t n, int b) { return (unsigned)((n + b - 1) / b); }

// --------------------------------------------------------- mean |L_ii|

__global__ void abs_diag_partial(const int32_t* __restrict__ rp, const int32_t* __restrict__ col,
                                 const double2* __restrict__ val, int64_t n, double* __restrict__ part) {
    __shared__ double sh[256];
    double s = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        for (int32_t t = rp[i]; t < rp[i + 1]; ++t)
            if (col[t] == i) { s += hypot(val[t].x, val[t].y); break; }
    }
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
}

__global__ void sum_partials(const double* __restrict__ part, int np, double scale, double* __restrict__ out) {
    __shared__ double sh[256];
    double s = 0.0;
    for (int t = threadIdx.x; t < np; t += blockDim.x) s += part[t];
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = sh[0] * scale;
}

// ----------------------------------------------------------- trace row

// One thread merges row 0 of L with w at the columns i (d + 1).
__global__ void trace_row0(const int32_t* __restrict__ rp, const int32_t* __restrict__ col,
                           const double2* __restrict__ val, int64_t d, double w, int32_t* __restrict__ ocol,
                           double2* __restrict__ oval, int32_t* __restrict__ olen) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    int32_t a = rp[0], b = rp[1], m = 0;
    int64_t i = 0;
    while (a < b || i < d) {
        int64_t tc = (i < d) ? i * (d + 1) : INT64_MAX;
        int64_t lc = (a < b) ? col[a] : INT64_MAX;
        double2 v;
        int64_t c;
        if (lc < tc) { c = lc; v = val[a++]; }
        else if (tc < lc) { c = tc; v = make_double2(w, 0.0); ++i; }
        else { c = lc; v = make_double2(__dadd_rn(val[a].x, w), val[a].y); ++a; ++i; }
        if (v.x != 0.0 || v.y != 0.0) {
            ocol[m] = (int32_t)c;
            oval[m] = v;
            ++m;
        }
    }
    *olen = m;
}

__global__ void shift_rows(const int32_t* __restrict__ rp, int64_t n, const int32_t* __restrict__ row0len,
                           int32_t* __restrict__ orp) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i > n) return;
    int32_t delta = *row0len - (rp[1] - rp[0]);
    orp[i] = (i == 0) ? 0 : rp[i] + delta;
}

__global__ void copy_tail(const int32_t* __restrict__ rp, const int32_t* __restrict__ col,
                          const double2* __restrict__ val, int64_t nnz, const int32_t* __restrict__ orp,
                          int32_t* __restrict__ ocol, double2* __restrict__ oval) {
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int32_t start = rp[1];
    if (t + start >= nnz) return;
    int32_t dst = orp[1] + (int32_t)t;
    ocol[dst] = col[start + t];
    oval[dst] = val[start + t];
}

// -------------------------------------------------------------- shift

__global__ void shift_count(const int32_t* __restrict__ rp, const int32_t* __restrict__ diag_pos, int64_t n,
                            int32_t* __restrict__ cnt) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    cnt[i] = rp[i + 1] - rp[i] + (diag_pos[i] < 0 ? 1 : 0);
}

__global__ void shift_fill(const int32_t* __restrict__ rp, const int32_t* __restrict__ col,
                           const double2* __restrict__ val, int64_t n, double sigma,
                           const int32_t* __restrict__ orp, int32_t* __restrict__ ocol, double2* __restrict__ oval) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int32_t o = orp[i];
    bool placed = false;
    for (int32_t t = rp[i]; t < rp[i + 1]; ++t) {
        int32_t c = col[t];
        if (!placed && c > i) {
            ocol[o] = (int32_t)i;
            oval[o] = make_double2(-sigma, 0.0);
            ++o;
            placed = true;
        }
        double2 v = val[t];
        if (c == i) {
            v.x = __dsub_rn(v.x, sigma);
            placed = true;
        }
        ocol[o] = c;
        oval[o] = v;
        ++o;
    }
    if (!placed) {
        ocol[o] = (int32_t)i;
        oval[o] = make_double2(-sigma, 0.0);
    }
}

// ------------------------------------------------------------ permute

__global__ void perm_count(const int32_t* __restrict__ rp, const int32_t* __restrict__ perm, int64_t n,
                           int32_t* __restrict__ cnt) {
    int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n) return;
    int32_t i = perm[r];
    cnt[r] = rp[i + 1] - rp[i];
}

__global__ void perm_fill(const int32_t* __restrict__ rp, const int32_t* __restrict__ col,
                          const double2* __restrict__ val, const int32_t* __restrict__ perm,
                          const int32_t* __restrict__ iperm, int64_t n, const int32_t* __restrict__ orp,
                          int32_t* __restrict__ ocol, double2* __restrict__ oval) {
    int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n) return;
    int32_t i = perm[r];
    int32_t a = rp[i], b = rp[i + 1], o = orp[r];
    for (int32_t t = a; t < b; ++t) {           // insertion into the sorted output segment
        int32_t c = iperm[col[t]];
        double2 v = val[t];
        int32_t u = o + (t - a) - 1;
        while (u >= o && ocol[u] > c) {
            ocol[u + 1] = ocol[u];
            oval[u + 1] = oval[u];
            --u;
        }
        ocol[u + 1] = c;
        oval[u + 1] = v;
    }
}

__global__ void invert_perm(const int32_t* __restrict__ perm, int64_t n, int32_t* __restrict__ iperm) {
    int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r < n) iperm[perm[r]] = (int32_t)r;
}

// -------------------------------------------------- bandwidth / profile

__global__ void bw_rows(const int32_t* __restrict__ rp, const int32_t* __restrict__ col, int64_t n,
                        unsigned long long* __restrict__ acc /* [ub, lb, up] */, int32_t* __restrict__ colmax) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int32_t a = rp[i], b = rp[i + 1];
    if (a == b) return;
    long long up = (long long)col[b - 1] - i;       // columns sorted: last one is the row maximum
    long long lo = (long long)i - col[a];
    if (up > 0) {
        atomicMax(&acc[0], (unsigned long long)up);
        atomicAdd(&acc[2], (unsigned long long)up);
    }
    if (lo > 0) atomicMax(&acc[1], (unsigned long long)lo);
    for (int32_t t = a; t < b; ++t) {
        int32_t c = col[t];
        if (c < i) atomicMax(&colmax[c], (int32_t)(i - c));
    }
}

__global__ void sum_colmax(const int32_t* __restrict__ colmax, int64_t n, unsigned long long* __restrict__ acc) {
    int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j < n && colmax[j] > 0) atomicAdd(&acc[3], (unsigned long long)colmax[j]);
}

}  // namespace

ss_status mean_abs_diag(ss_ctx ctx, const DeviceCSR& L, double* w) {
    const int nb = 256;
    double* part = nullptr;
    SS_TRY(dev_alloc_n(ctx, &part, nb + 1));
    abs_diag_partial<<<(ss_count_launch(), nb), 256, 0, ctx->stream>>>(L.row_ptr, L.col, L.val, L.n_rows, part);
    sum_partials<<<(ss_count_launch(), 1), 256, 0, ctx->stream>>>(part, nb, 1.0 / (double)L.n_rows, part + nb);
    SS_CUDA(ctx, cudaMemcpyAsync(w, part + nb, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    SS_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    dev_free(ctx, part);
    return SS_OK;
}

ss_status add_trace_row_impl(ss_ctx ctx, const DeviceCSR& L, int64_t d, double w, DeviceCSR& out) {
    out = DeviceCSR();
    const int64_t n = L.n_rows;
    int32_t h_rp[2];
    SS_CUDA(ctx, cudaMemcpyAsync(h_rp, L.row_ptr, sizeof(int32_t) * 2, cudaMemcpyDeviceToHost, ctx->stream));
    SS_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    const int64_t cap = (h_rp[1] - h_rp[0]) + d;
    int32_t *tcol = nullptr, *tlen = nullptr;
    double2* tval = nullptr;
    SS_TRY(dev_alloc_n(ctx, &tcol, (size_t)cap));
    SS_TRY(dev_alloc_n(ctx, &tval, (size_t)cap));
    SS_TRY(dev_alloc_n(ctx, &tlen, 1));
    trace_row0<<<(ss_count_launch(), 1), 32, 0, ctx->stream>>>(L.row_ptr, L.col, L.val, d, w, tcol, tval, tlen);
    int32_t len0 = 0;
    SS_CUDA(ctx, cudaMemcpyAsync(&len0, tlen, sizeof(int32_t), cudaMemcpyDeviceToHost, ctx->stream));
    SS_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    out.n_rows = out.n_cols = n;
    out.nnz = L.nnz + (len0 - (h_rp[1] - h_rp[0]));
    if (out.nnz > INT32_MAX) return set_error(ctx, SS_ERR_UNSUPPORTED, "more than 2^31-1 stored entries");
    SS_TRY(dev_alloc_n(ctx, &out.row_ptr, (size_t)n + 1));
    SS_TRY(dev_alloc_n(ctx, &out.col, (size_t)out.nnz));
    SS_TRY(dev_alloc_n(ctx, &out.val, (size_t)out.nnz));
    shift_rows<<<(ss_count_launch(), grid_for(n + 1, 256)), 256, 0, ctx->stream>>>(L.row_ptr, n, tlen, out.row_ptr);
    int64_t tail = L.nnz - h_rp[1];
    if (tail > 0)
        copy_tail<<<(ss_count_launch(), grid_for(tail, 256)), 256, 0, ctx->stream>>>(L.row_ptr, L.col, L.val, L.nnz, out.row_ptr,
                                                                out.col, out.val);
    SS_CUDA(ctx, cudaMemcpyAsync(out.col, tcol, sizeof(int32_t) * len0, cudaMemcpyDeviceToDevice, ctx->stream));
    SS_CUDA(ctx, cudaMemcpyAsync(out.val, tval, sizeof(double2) * len0, cudaMemcpyDeviceToDevice, ctx->stream));
    SS_CUDA(ctx, cudaGetLastError());
    dev_free(ctx, tcol);
    dev_free(ctx, tval);
    dev_free(ctx, tlen);
    return SS_OK;
}

ss_status add_shift_impl(ss_ctx ctx, const DeviceCSR& L, double sigma, DeviceCSR& out) {
    out = DeviceCSR();
    const int64_t n = L.n_rows;
    int32_t *dpos = nullptr, *cnt = nullptr;
    SS_TRY(dev_alloc_n(ctx, &dpos, (size_t)n));
    SS_TRY(dev_alloc_n(ctx, &cnt, (size_t)n + 1));
    SS_TRY(find_diag(ctx, L, dpos));
    shift_count<<<(ss_count_launch(), grid_for(n, 256)), 256, 0, ctx->stream>>>(L.row_ptr, dpos, n, cnt);
    out.n_rows = out.n_cols = n;
    SS_TRY(dev_alloc_n(ctx, &out.row_ptr, (size_t)n + 1));
    int64_t nnz = 0;
    SS_TRY(exclusive_scan_i32(ctx, cnt, out.row_ptr, n, &nnz));
    out.nnz = nnz;
    SS_TRY(dev_alloc_n(ctx, &out.col, (size_t)nnz));
    SS_TRY(dev_alloc_n(ctx, &out.val, (size_t)nnz));
    shift_fill<<<(ss_count_launch(), grid_for(n, 256)), 256, 0, ctx->stream>>>(L.row_ptr, L.col, L.val, n, sigma, out.row_ptr, out.col,
                                                          out.val);
    SS_CUDA(ctx, cudaGetLastError());
    dev_free(ctx, dpos);
    dev_free(ctx, cnt);
    return SS_OK;
}

ss_status permute_impl(ss_ctx ctx, const DeviceCSR& A, const int32_t* perm_host, DeviceCSR& out) {
    out = DeviceCSR();
    const int64_t n = A.n_rows;
    int32_t *perm = nullptr, *iperm = nullptr, *cnt = nullptr;
    SS_TRY(dev_alloc_n(ctx, &perm, (size_t)n));
    SS_TRY(dev_alloc_n(ctx, &iperm, (size_t)n));
    SS_TRY(dev_alloc_n(ctx, &cnt, (size_t)n + 1));
    SS_CUDA(ctx, cudaMemcpyAsync(perm, perm_host, sizeof(int32_t) * n, cudaMemcpyHostToDevice, ctx->stream));
    invert_perm<<<(ss_count_launch(), grid_for(n, 256)), 256, 0, ctx->stream>>>(perm, n, iperm);
    perm_count<<<(ss_count_launch(), grid_for(n, 256)), 256, 0, ctx->stream>>>(A.row_ptr, perm, n, cnt);
    out.n_rows = out.n_cols = n;
    out.nnz = A.nnz;
    SS_TRY(dev_alloc_n(ctx, &out.row_ptr, (size_t)n + 1));
    SS_TRY(exclusive_scan_i32(ctx, cnt, out.row_ptr, n, nullptr));
    SS_TRY(dev_alloc_n(ctx, &out.col, (size_t)A.nnz));
    SS_TRY(dev_alloc_n(ctx, &out.val, (size_t)A.nnz));
    perm_fill<<<(ss_count_launch(), grid_for(n, 128)), 128, 0, ctx->stream>>>(A.row_ptr, A.col, A.val, perm, iperm, n, out.row_ptr,
                                                         out.col, out.val);
    SS_CUDA(ctx, cudaGetLastError());
    dev_free(ctx, perm);
    dev_free(ctx, iperm);
    dev_free(ctx, cnt);
    return SS_OK;
}

ss_status bandwidth_profile_impl(ss_ctx ctx, const DeviceCSR& A, int64_t* bw, int64_t* prof) {
    const int64_t n = A.n_rows;
    unsigned long long* acc = nullptr;
    int32_t* colmax = nullptr;
    SS_TRY(dev_alloc_n(ctx, &acc, 4));
    SS_TRY(dev_alloc_n(ctx, &colmax, (size_t)n));
    SS_CUDA(ctx, cudaMemsetAsync(acc, 0, sizeof(unsigned long long) * 4, ctx->stream));
    SS_CUDA(ctx, cudaMemsetAsync(colmax, 0, sizeof(int32_t) * n, ctx->stream));
    bw_rows<<<(ss_count_launch(), grid_for(n, 256)), 256, 0, ctx->stream>>>(A.row_ptr, A.col, n, acc, colmax);
    sum_colmax<<<(ss_count_launch(), grid_for(n, 256)), 256, 0, ctx->stream>>>(colmax, n, acc);
    unsigned long long h[4];
    SS_CUDA(ctx, cudaMemcpyAsync(h, acc, sizeof(h), cudaMemcpyDeviceToHost, ctx->stream));
    SS_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    if (bw) *bw = (int64_t)(h[0] + h[1] + 1);
    if (prof) *prof = (int64_t)(h[2] + h[3]);
    dev_free(ctx, acc);
    dev_free(ctx, colmax);
    return SS_OK;
}
