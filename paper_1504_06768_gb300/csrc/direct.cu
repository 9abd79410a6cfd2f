// method=direct: LU factorisation with partial pivoting of the RCM-ordered
// trace-row system L~ held as a band (section "Direct factorization": the
// reverse Cuthill-McKee ordering keeps the nonzeros, and the fill of the
// factors, inside a narrow band around the diagonal), then the two banded
// triangular solves.  Everything runs on the device in FP64.
//
// Storage follows the usual band layout: entry (i, k) of the matrix sits at
// ab[(kl + ku + i - k) + k * ldab], ldab = 2 kl + ku + 1, so the row
// interchanges of partial pivoting (which widen the upper band to kl + ku)
// stay inside the array.  Column j is factorised by one launch in which every
// block finds the pivot of column j and its multipliers on its own (the column
// is only read), then swaps and updates its share of the trailing columns;
// the multipliers and the pivots go to separate arrays, so no block writes
// what another block of the same launch reads.
#include <algorithm>
#include <vector>

#include "common.cuh"
#include "direct.cuh"

namespace {

inline unsigned grid_for(int64_t n, int b) { return (unsigned)std::max<int64_t>(1, (n + b - 1) / b); }

constexpr int LU_THREADS = 256;
constexpr int LU_COLS = 4;            // trailing columns per block
constexpr int LU_MAX_KL = 2048;       // rows of a column kept in shared memory

__global__ void band_extent(const int32_t* __restrict__ rp, const int32_t* __restrict__ col, int64_t n,
                            int* __restrict__ ext) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int lo = 0, hi = 0;
    for (int32_t t = rp[i]; t < rp[i + 1]; ++t) {
        const int64_t dlt = (int64_t)col[t] - i;
        if (dlt < 0) lo = max(lo, (int)(-dlt));
        else hi = max(hi, (int)dlt);
    }
    atomicMax(&ext[0], lo);
    atomicMax(&ext[1], hi);
}

__global__ void band_scatter(const int32_t* __restrict__ rp, const int32_t* __restrict__ col,
                             const double2* __restrict__ val, int64_t n, int64_t kl, int64_t ku, int64_t ldab,
                             double2* __restrict__ ab) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    for (int32_t t = rp[i]; t < rp[i + 1]; ++t) {
        const int64_t k = col[t];
        ab[(kl + ku + i - k) + k * ldab] = val[t];
    }
}

__device__ __forceinline__ double cabs1(double2 a) { return hypot(a.x, a.y); }

// Column j: pivot, multipliers, interchange and update of the trailing
// columns j+1 .. min(n-1, j+kl+ku), LU_COLS of them per block.
__global__ void __launch_bounds__(LU_THREADS) lu_column(int64_t j, int64_t n, int64_t kl, int64_t ku, int64_t ldab,
                                                        double2* __restrict__ ab, double2* __restrict__ lmul,
                                                        double2* __restrict__ udiag, int32_t* __restrict__ ipiv,
                                                        int* __restrict__ singular) {
    __shared__ double2 c[LU_MAX_KL + 1];      // column j, rows j .. j+m-1, pivot row moved to the top
    __shared__ double wabs[LU_THREADS / 32];
    __shared__ int widx[LU_THREADS / 32];
    __shared__ int piv;
    const int m = (int)(kl + 1 < n - j ? kl + 1 : n - j);
    const double2* colj = ab + (kl + ku) + j * ldab;     // &A(j, j); A(j + r, j) = colj[r]
    for (int r = threadIdx.x; r < m; r += blockDim.x) c[r] = colj[r];
    __syncthreads();
    // pivot: the largest modulus, the first such row on ties
    double best = -1.0;
    int bi = 0;
    for (int r = threadIdx.x; r < m; r += blockDim.x) {
        const double a = cabs1(c[r]);
        if (a > best) { best = a; bi = r; }
    }
    for (int o = 16; o > 0; o >>= 1) {
        const double ob = __shfl_down_sync(0xffffffffu, best, o);
        const int oi = __shfl_down_sync(0xffffffffu, bi, o);
        if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
    }
    if ((threadIdx.x & 31) == 0) { wabs[threadIdx.x >> 5] = best; widx[threadIdx.x >> 5] = bi; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double b = wabs[0];
        int ix = widx[0];
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w)
            if (wabs[w] > b || (wabs[w] == b && widx[w] < ix)) { b = wabs[w]; ix = widx[w]; }
        piv = ix;
    }
    __syncthreads();
    const int p = piv;                                    // pivot row j + p
    const double2 a_p = c[p];
    const bool zero = a_p.x == 0.0 && a_p.y == 0.0;
    const double2 inv = zero ? make_double2(0.0, 0.0) : cdiv(make_double2(1.0, 0.0), a_p);
    __syncthreads();
    if (threadIdx.x == 0 && p != 0) { const double2 t = c[0]; c[0] = c[p]; c[p] = t; }
    __syncthreads();
    // multipliers l_r = c[r] / a_p, r = 1 .. m-1
    for (int r = 1 + threadIdx.x; r < m; r += blockDim.x) c[r] = cmul(c[r], inv);
    __syncthreads();
    if (blockIdx.x == 0) {
        for (int r = 1 + threadIdx.x; r < m; r += blockDim.x) lmul[j * kl + (r - 1)] = c[r];
        if (threadIdx.x == 0) {
            udiag[j] = a_p;
            ipiv[j] = (int32_t)(j + p);
            if (zero) atomicExch(singular, 1);
        }
    }
    // trailing columns of this block
    const int64_t kend = (n - 1 < j + kl + ku) ? n - 1 : j + kl + ku;
    const int64_t k0 = j + 1 + (int64_t)blockIdx.x * LU_COLS;
    for (int64_t k = k0; k < k0 + LU_COLS && k <= kend; ++k) {
        double2* colk = ab + (kl + ku) + k * ldab;        // A(i, k) = colk[i - k]
        const int64_t off = j - k;                        // A(j + r, k) = colk[off + r]
        __shared__ double2 ujk;
        if (threadIdx.x == 0) {
            double2 u = colk[off];
            if (p != 0 && j + p <= k + kl) {              // interchange rows j and j + p in column k
                const double2 t = colk[off + p];
                colk[off + p] = u;
                u = t;
                colk[off] = u;
            }
            ujk = u;
        }
        __syncthreads();
        const double2 u = ujk;
        for (int r = 1 + threadIdx.x; r < m; r += blockDim.x) {
            if (j + r > k + kl) continue;                 // outside the band of column k (stays zero)
            double2 a = colk[off + r];
            const double2 l = c[r];
            a.x -= l.x * u.x - l.y * u.y;
            a.y -= l.x * u.y + l.y * u.x;
            colk[off + r] = a;
        }
        __syncthreads();
    }
}

// Forward (P then unit L) and backward (U) substitution in one block.
__global__ void __launch_bounds__(1024) lu_solve(int64_t n, int64_t kl, int64_t ku, int64_t ldab,
                                                 const double2* __restrict__ ab, const double2* __restrict__ lmul,
                                                 const double2* __restrict__ udiag, const int32_t* __restrict__ ipiv,
                                                 double2* __restrict__ y) {
    __shared__ double2 yj;
    for (int64_t j = 0; j < n; ++j) {
        if (threadIdx.x == 0) {
            const int64_t p = ipiv[j];
            double2 v = y[j];
            if (p != j) {
                const double2 t = y[p];
                y[p] = v;
                v = t;
                y[j] = v;
            }
            yj = v;
        }
        __syncthreads();
        const double2 v = yj;
        const int64_t m = kl < n - 1 - j ? kl : n - 1 - j;
        for (int64_t r = threadIdx.x; r < m; r += blockDim.x) {
            const double2 l = lmul[j * kl + r];
            double2 a = y[j + 1 + r];
            a.x -= l.x * v.x - l.y * v.y;
            a.y -= l.x * v.y + l.y * v.x;
            y[j + 1 + r] = a;
        }
        __syncthreads();
    }
    for (int64_t j = n - 1; j >= 0; --j) {
        if (threadIdx.x == 0) {
            const double2 xj = cdiv(y[j], udiag[j]);
            y[j] = xj;
            yj = xj;
        }
        __syncthreads();
        const double2 v = yj;
        const int64_t top = j - (kl + ku) > 0 ? j - (kl + ku) : 0;
        const double2* colj = ab + (kl + ku) + j * ldab;  // U(i, j) = colj[i - j], i < j
        for (int64_t i = top + threadIdx.x; i < j; i += blockDim.x) {
            const double2 u = colj[i - j];
            double2 a = y[i];
            a.x -= u.x * v.x - u.y * v.y;
            a.y -= u.x * v.y + u.y * v.x;
            y[i] = a;
        }
        __syncthreads();
    }
}

}  // namespace

ss_status band_lu_solve(ss_ctx ctx, const DeviceCSR& A, const double2* b, double2* x, BandInfo* info) {
    const int64_t n = A.n_rows;
    if (n <= 0) return set_error(ctx, SS_ERR_INVALID, "empty matrix");
    int* ext = nullptr;
    SS_TRY(dev_alloc_n(ctx, &ext, 3));
    SS_CUDA(ctx, cudaMemsetAsync(ext, 0, sizeof(int) * 3, ctx->stream));
    band_extent<<<(ss_count_launch(), grid_for(n, 256)), 256, 0, ctx->stream>>>(A.row_ptr, A.col, n, ext);
    int h_ext[2] = {0, 0};
    SS_CUDA(ctx, cudaMemcpyAsync(h_ext, ext, sizeof(int) * 2, cudaMemcpyDeviceToHost, ctx->stream));
    SS_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    const int64_t kl = h_ext[0], ku = h_ext[1], ldab = 2 * kl + ku + 1;
    if (info) { info->kl = kl; info->ku = ku; }
    if (kl > LU_MAX_KL) {
        dev_free(ctx, ext);
        return set_error(ctx, SS_ERR_UNSUPPORTED, "direct method: lower bandwidth " + std::to_string(kl) +
                                                      " beyond the banded LU's limit of " + std::to_string(LU_MAX_KL));
    }
    const double bytes = (double)n * (double)ldab * 16.0;
    if (bytes > 8.0e9) {
        dev_free(ctx, ext);
        return set_error(ctx, SS_ERR_UNSUPPORTED, "direct method: the band (" + std::to_string((long long)(bytes / 1e6)) +
                                                      " MB) is too large; use an iterative method");
    }
    double2 *ab = nullptr, *lmul = nullptr, *udiag = nullptr;
    int32_t* ipiv = nullptr;
    auto cleanup = [&]() {
        dev_free(ctx, ab);
        dev_free(ctx, lmul);
        dev_free(ctx, udiag);
        dev_free(ctx, ipiv);
        dev_free(ctx, ext);
    };
    ss_status st;
    if ((st = dev_alloc_n(ctx, &ab, (size_t)(n * ldab))) != SS_OK) { cleanup(); return st; }
    if ((st = dev_alloc_n(ctx, &lmul, (size_t)(n * std::max<int64_t>(kl, 1)))) != SS_OK) { cleanup(); return st; }
    if ((st = dev_alloc_n(ctx, &udiag, (size_t)n)) != SS_OK) { cleanup(); return st; }
    if ((st = dev_alloc_n(ctx, &ipiv, (size_t)n)) != SS_OK) { cleanup(); return st; }
    cudaError_t e = cudaMemsetAsync(ab, 0, sizeof(double2) * n * ldab, ctx->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(ext + 2, 0, sizeof(int), ctx->stream);
    if (e != cudaSuccess) { cleanup(); return cuda_check(ctx, e, "band storage"); }
    band_scatter<<<(ss_count_launch(), grid_for(n, 256)), 256, 0, ctx->stream>>>(A.row_ptr, A.col, A.val, n, kl, ku,
                                                                                ldab, ab);
    for (int64_t j = 0; j < n; ++j) {
        const int64_t trailing = std::min<int64_t>(n - 1, j + kl + ku) - j;
        lu_column<<<(ss_count_launch(), grid_for(std::max<int64_t>(trailing, 1), LU_COLS)), LU_THREADS, 0,
                     ctx->stream>>>(j, n, kl, ku, ldab, ab, lmul, udiag, ipiv, ext + 2);
    }
    if ((e = cudaGetLastError()) != cudaSuccess) { cleanup(); return cuda_check(ctx, e, "banded LU"); }
    e = cudaMemcpyAsync(x, b, sizeof(double2) * n, cudaMemcpyDeviceToDevice, ctx->stream);
    if (e == cudaSuccess) {
        lu_solve<<<(ss_count_launch(), 1), 1024, 0, ctx->stream>>>(n, kl, ku, ldab, ab, lmul, udiag, ipiv, x);
        e = cudaGetLastError();
    }
    int singular = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&singular, ext + 2, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    cleanup();
    if (e != cudaSuccess) return cuda_check(ctx, e, "banded LU");
    if (singular) return set_error(ctx, SS_ZERO_PIVOT, "direct method: the matrix is singular (zero pivot column)");
    return SS_OK;
}
