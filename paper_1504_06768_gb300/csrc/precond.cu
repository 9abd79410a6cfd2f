// Incomplete-LU preconditioner (section "Iterative solvers"): the iLU(0)
// numeric factorisation on the device, the level analysis that schedules it,
// and the triangular solves z = U^{-1} L^{-1} r that apply M^{-1}.
//
// Triangular solves are "sync-free": rows are grouped into level-aligned
// units, blocks take runs of units in level order from a ticket counter, and
// a row waits (bounded) until the values of the rows it depends on have been
// written -- the output vector is pre-marked with a NaN payload that no
// arithmetic produces, so the value doubles as its own completion flag.
#include <algorithm>
#include <vector>

#include "common.cuh"

namespace {

constexpr unsigned FULL = 0xffffffffu;

inline unsigned grid_for(int64_t n, int b) { return (unsigned)((n + b - 1) / b); }

template <class T> struct Cplx;
template <> struct Cplx<double2> {
    using R = double;
    __device__ static double2 zero() { return make_double2(0.0, 0.0); }
    __device__ static double2 fma_(double2 a, double2 b, double2 acc) {   // acc + a * b
        return make_double2(acc.x + a.x * b.x - a.y * b.y, acc.y + a.x * b.y + a.y * b.x);
    }
    __device__ static double2 sub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
    __device__ static double2 mul(double2 a, double2 b) { return cmul(a, b); }
    __device__ static double2 shfl_down(double2 v, int o) {
        return make_double2(__shfl_down_sync(FULL, v.x, o), __shfl_down_sync(FULL, v.y, o));
    }
    __device__ static double2 ldcg(const double2* p) { return __ldcg(p); }
};
template <> struct Cplx<float2> {
    using R = float;
    __device__ static float2 zero() { return make_float2(0.f, 0.f); }
    __device__ static float2 fma_(float2 a, float2 b, float2 acc) {
        return make_float2(acc.x + a.x * b.x - a.y * b.y, acc.y + a.x * b.y + a.y * b.x);
    }
    __device__ static float2 sub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
    __device__ static float2 mul(float2 a, float2 b) { return fcmul(a, b); }
    __device__ static float2 shfl_down(float2 v, int o) {
        return make_float2(__shfl_down_sync(FULL, v.x, o), __shfl_down_sync(FULL, v.y, o));
    }
    __device__ static float2 ldcg(const float2* p) { return __ldcg(p); }
};

__device__ __forceinline__ unsigned long long globaltimer_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
    return t;
}

constexpr unsigned long long WAIT_NS = 2000000000ull;   // a single wait gives up after 2 s

// "Not yet computed" marks: NaN bit patterns with a payload that arithmetic
// never produces (arithmetic NaNs carry the canonical payload).
constexpr unsigned long long PENDING64 = 0xFFFDEADBEEFDEAD1ull;
constexpr unsigned int PENDING32 = 0xFFBADBADu;

__device__ __forceinline__ bool ready(double2 v) {
    return __double_as_longlong(v.x) != (long long)PENDING64 && __double_as_longlong(v.y) != (long long)PENDING64;
}
__device__ __forceinline__ bool ready(float2 v) {
    return __float_as_uint(v.x) != PENDING32 && __float_as_uint(v.y) != PENDING32;
}
template <class T> __device__ __forceinline__ T pending();
template <> __device__ __forceinline__ double2 pending<double2>() {
    return make_double2(__longlong_as_double((long long)PENDING64), __longlong_as_double((long long)PENDING64));
}
template <> __device__ __forceinline__ float2 pending<float2>() {
    return make_float2(__uint_as_float(PENDING32), __uint_as_float(PENDING32));
}

// Sync-free triangular solve.  One warp handles one "unit": up to R = 32 / G
// rows of the same level, G lanes per row.  Blocks take consecutive runs of
// units in level order through a ticket counter (one atomic per block), so a
// row only ever waits for rows held by earlier, resident blocks.  The output
// vector starts filled with the PENDING mark; a row waits (bounded) until the
// values it depends on are no longer PENDING -- the value itself is the
// completion signal, so no flag or fence is needed.
//   LOWER: x_i = b_i - sum_{j<i} l_ij x_j (unit diagonal); also re-marks
//          `other[i]` (the upper solve's output) PENDING.
//   UPPER: x_i = (b_i - sum_{j>i} u_ij x_j) / u_ii; afterwards re-marks b_i
//          (the lower solve's output) PENDING for the next application.
// A row's range comes from a precomputed record {row, first, end, -} of its
// unit, and in FP32 each lane issues the column and value loads of its next
// SYNCFREE_K entries, then their x loads, before it waits on any of them, so a
// row costs three dependent memory round trips when its inputs are ready.
constexpr int SYNCFREE_K = 4;

template <bool LOWER, int G, class T>
__global__ void __launch_bounds__(256) sptrsv_syncfree(const int32_t* __restrict__ col, const T* __restrict__ val,
                                                       const T* __restrict__ inv_diag, const int4* __restrict__ meta,
                                                       int64_t n_units, T* b, T* x, T* other,
                                                       unsigned long long* __restrict__ ticket, int* __restrict__ err,
                                                       const int* __restrict__ halt) {
    using C = Cplx<T>;
    constexpr int R = 32 / G;
    constexpr int K = sizeof(T) == 16 ? 1 : SYNCFREE_K;   // FP64: registers of more in-flight entries cost more
    if (halt && *halt) return;      // uniform over the launch: no ticket is taken
    __shared__ unsigned long long s_ticket;
    if (threadIdx.x == 0) s_ticket = atomicAdd(ticket, 1ull);
    __syncthreads();
    const int64_t nblocks = gridDim.x;
    const int64_t wpb = blockDim.x >> 5;
    const int64_t u = (int64_t)(s_ticket % (unsigned long long)nblocks) * wpb + (threadIdx.x >> 5);
    if (u >= n_units) return;
    const int lane = threadIdx.x & 31;
    const int grp = lane / G, sub = lane % G;
    const int4 m = meta[u * R + grp];              // row -1 pads a unit at the end of a level
    const int32_t i = m.x, s = m.y, e = m.z;
    T dinv = C::zero();
    if (!LOWER && i >= 0 && sub == 0) dinv = inv_diag[i];
    T acc = C::zero();
    bool timed_out = false;
    for (int32_t base = s + sub; base < e; base += K * G) {
        int32_t c[K];
        T v[K], xj[K];
#pragma unroll
        for (int q = 0; q < K; ++q) {
            const int32_t k = base + q * G;
            c[q] = k < e ? col[k] : -1;
            v[q] = k < e ? val[k] : C::zero();
        }
#pragma unroll
        for (int q = 0; q < K; ++q) xj[q] = c[q] >= 0 ? __ldcv(&x[c[q]]) : C::zero();
#pragma unroll
        for (int q = 0; q < K; ++q) {
            if (c[q] >= 0 && !ready(xj[q])) {
                const T* xp = &x[c[q]];
                const unsigned long long t0 = globaltimer_ns();
                int spins = 0;
                while (true) {
                    if (++spins > 64) __nanosleep(64);
                    xj[q] = __ldcv(xp);
                    if (ready(xj[q])) break;
                    if ((spins & 63) == 0 && (*(volatile int*)err != 0 || globaltimer_ns() - t0 > WAIT_NS)) {
                        timed_out = true;
                        xj[q] = C::zero();
                        break;
                    }
                }
            }
            acc = C::fma_(v[q], xj[q], acc);
        }
    }
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) {
        T other_v = C::shfl_down(acc, o);
        acc.x += other_v.x;
        acc.y += other_v.y;
    }
    if (__any_sync(FULL, timed_out) && lane == 0) atomicExch(err, 1);
    if (i >= 0 && sub == 0) {
        T xi = C::sub(b[i], acc);
        if (!LOWER) xi = C::mul(xi, dinv);
        __stcg(&x[i], xi);
        if (LOWER) __stcg(&other[i], pending<T>());
        else __stcg(&b[i], pending<T>());
    }
}

template <class T>
__global__ void fill_pending(int64_t n, T* __restrict__ a) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        a[i] = pending<T>();
}

// ---------------------------------------------------------------- iLU(0)
// IKJ elimination restricted to the pattern, one warp per row of one level:
// for each stored k < i in ascending order, a_ik <- a_ik / a_kk, then every
// stored a_ij with j > k that also appears in row k gets a_ij -= a_ik a_kj.

__device__ __forceinline__ int32_t find_col(const int32_t* __restrict__ col, int32_t lo, int32_t hi, int32_t c) {
    hi -= 1;
    while (lo <= hi) {
        int32_t mid = (lo + hi) >> 1;
        int32_t v = col[mid];
        if (v == c) return mid;
        if (v < c) lo = mid + 1; else hi = mid - 1;
    }
    return -1;
}

__global__ void ilu0_level(const int32_t* __restrict__ rp, const int32_t* __restrict__ col, double2* __restrict__ val,
                           const int32_t* __restrict__ dpos, const int32_t* __restrict__ order, int32_t lvl_begin,
                           int32_t lvl_end, int* __restrict__ err) {
    const int32_t w = (int32_t)(((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    if (lvl_begin + w >= lvl_end) return;
    const int lane = threadIdx.x & 31;
    const int32_t i = order[lvl_begin + w];
    const int32_t rb = rp[i], re = rp[i + 1], di = dpos[i];
    for (int32_t t = rb; t < di; ++t) {
        const int32_t k = col[t];
        double2 f = make_double2(0.0, 0.0);
        if (lane == 0) {
            f = cdiv(val[t], val[dpos[k]]);
            val[t] = f;
        }
        f.x = __shfl_sync(FULL, f.x, 0);
        f.y = __shfl_sync(FULL, f.y, 0);
        for (int32_t u = dpos[k] + 1 + lane; u < rp[k + 1]; u += 32) {
            const int32_t pos = find_col(col, t + 1, re, col[u]);
            if (pos >= 0) val[pos] = csub(val[pos], cmul(f, val[u]));
        }
        __syncwarp();
    }
    if (lane == 0) {
        const double2 p = val[di];
        if (p.x == 0.0 && p.y == 0.0) atomicExch(err, 2);
    }
}

__global__ void make_inv_diag(const double2* __restrict__ val, const int32_t* __restrict__ dpos, int64_t n,
                              double2* __restrict__ inv, float2* __restrict__ inv32, int* __restrict__ err) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int32_t p = dpos[i];
    if (p < 0) { atomicExch(err, 2); inv[i] = make_double2(0.0, 0.0); return; }
    double2 d = val[p];
    if (d.x == 0.0 && d.y == 0.0) { atomicExch(err, 2); inv[i] = make_double2(0.0, 0.0); return; }
    double2 r = cdiv(make_double2(1.0, 0.0), d);
    inv[i] = r;
    if (inv32) inv32[i] = make_float2((float)r.x, (float)r.y);
}

__global__ void to_f32(const double2* __restrict__ a, int64_t n, float2* __restrict__ b) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) b[i] = make_float2((float)a[i].x, (float)a[i].y);
}

__global__ void check_missing_diag(const int32_t* __restrict__ dpos, int64_t n, int* __restrict__ err) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n && dpos[i] < 0) atomicExch(err, 2);
}

ss_status upload_levels(ss_ctx ctx, const std::vector<int32_t>& order, const std::vector<int32_t>& lptr,
                        double avg_row, TriLevels& L, int32_t nlev, bool lower, const std::vector<int32_t>& hrp,
                        const std::vector<int32_t>& hdpos) {
    L.n_levels = nlev;
    int g = 2;
    while (g < 32 && g < avg_row) g <<= 1;
    L.g = g;
    std::vector<int32_t> units;
    level_units_host(order, lptr, 32 / g, units);
    L.n_units = (int64_t)units.size() / (32 / g);
    // per unit row: {row, first entry, end} of the triangle's part of the row
    std::vector<int4> meta(units.size());
    for (size_t k = 0; k < units.size(); ++k) {
        const int32_t i = units[k];
        if (i < 0) meta[k] = make_int4(-1, 0, 0, 0);
        else if (hdpos[i] < 0) meta[k] = make_int4(i, 0, 0, 0);     // no diagonal: reported as a zero pivot
        else if (lower) meta[k] = make_int4(i, hrp[i], hdpos[i], 0);
        else meta[k] = make_int4(i, hdpos[i] + 1, hrp[i + 1], 0);
    }
    SS_TRY(dev_alloc_n(ctx, &L.meta, meta.size()));
    SS_CUDA(ctx, cudaMemcpyAsync(L.meta, meta.data(), sizeof(int4) * meta.size(), cudaMemcpyHostToDevice,
                                 ctx->stream));
    SS_TRY(dev_alloc_n(ctx, &L.order, order.size()));
    SS_TRY(dev_alloc_n(ctx, &L.units, units.size()));
    SS_CUDA(ctx, cudaMemcpyAsync(L.order, order.data(), sizeof(int32_t) * order.size(), cudaMemcpyHostToDevice,
                                 ctx->stream));
    SS_CUDA(ctx, cudaMemcpyAsync(L.units, units.data(), sizeof(int32_t) * units.size(), cudaMemcpyHostToDevice,
                                 ctx->stream));
    SS_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    return SS_OK;
}

}  // namespace

// Host level analysis of the factor pattern, device buffers of the solves.
static ss_status analyse(ss_ctx ctx, ss_prec M, const std::vector<int32_t>& hrp, const std::vector<int32_t>& hcol,
                         std::vector<int32_t>& lower_order, std::vector<int32_t>& lower_ptr) {
    const int64_t n = M->f.n_rows;
    std::vector<int32_t> upper_order, upper_ptr;
    int32_t nl = level_sets_host(n, hrp.data(), hcol.data(), true, lower_order, lower_ptr);
    int32_t nu = level_sets_host(n, hrp.data(), hcol.data(), false, upper_order, upper_ptr);
    int64_t nnz_lower = 0;
    for (int64_t i = 0; i < n; ++i)
        for (int32_t t = hrp[i]; t < hrp[i + 1] && hcol[t] < i; ++t) ++nnz_lower;
    const int64_t nnz_upper = (int64_t)hcol.size() - nnz_lower - n;
    std::vector<int32_t> hdpos(n, -1);
    for (int64_t i = 0; i < n; ++i)
        for (int32_t t = hrp[i]; t < hrp[i + 1]; ++t)
            if (hcol[t] == i) { hdpos[i] = t; break; }
    SS_TRY(upload_levels(ctx, lower_order, lower_ptr, n ? (double)nnz_lower / n : 1.0, M->lower, nl, true, hrp, hdpos));
    SS_TRY(upload_levels(ctx, upper_order, upper_ptr, n ? (double)nnz_upper / n : 1.0, M->upper, nu, false, hrp, hdpos));
    SS_TRY(dev_alloc_n(ctx, &M->tickets, 2));
    SS_TRY(dev_alloc_n(ctx, &M->err, 1));
    SS_TRY(dev_alloc_n(ctx, &M->tmp, (size_t)n));
    fill_pending<double2><<<(ss_count_launch(), 256), 256, 0, ctx->stream>>>(n, M->tmp);
    SS_CUDA(ctx, cudaMemsetAsync(M->tickets, 0, sizeof(unsigned long long) * 2, ctx->stream));
    SS_CUDA(ctx, cudaMemsetAsync(M->err, 0, sizeof(int), ctx->stream));
    return SS_OK;
}

ss_status ilu0_device(ss_ctx ctx, const DeviceCSR& A, ss_prec M) {
    const int64_t n = A.n_rows;
    M->f.n_rows = M->f.n_cols = n;
    M->f.nnz = A.nnz;
    SS_TRY(dev_alloc_n(ctx, &M->f.row_ptr, (size_t)n + 1));
    SS_TRY(dev_alloc_n(ctx, &M->f.col, (size_t)A.nnz));
    SS_TRY(dev_alloc_n(ctx, &M->f.val, (size_t)A.nnz));
    SS_CUDA(ctx, cudaMemcpyAsync(M->f.row_ptr, A.row_ptr, sizeof(int32_t) * (n + 1), cudaMemcpyDeviceToDevice, ctx->stream));
    SS_CUDA(ctx, cudaMemcpyAsync(M->f.col, A.col, sizeof(int32_t) * A.nnz, cudaMemcpyDeviceToDevice, ctx->stream));
    SS_CUDA(ctx, cudaMemcpyAsync(M->f.val, A.val, sizeof(double2) * A.nnz, cudaMemcpyDeviceToDevice, ctx->stream));
    SS_TRY(dev_alloc_n(ctx, &M->diag_pos, (size_t)n));
    SS_TRY(find_diag(ctx, M->f, M->diag_pos));
    std::vector<int32_t> hrp(n + 1), hcol(A.nnz);
    SS_CUDA(ctx, cudaMemcpyAsync(hrp.data(), A.row_ptr, sizeof(int32_t) * (n + 1), cudaMemcpyDeviceToHost, ctx->stream));
    SS_CUDA(ctx, cudaMemcpyAsync(hcol.data(), A.col, sizeof(int32_t) * A.nnz, cudaMemcpyDeviceToHost, ctx->stream));
    SS_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    std::vector<int32_t> lorder, lptr;
    SS_TRY(analyse(ctx, M, hrp, hcol, lorder, lptr));
    check_missing_diag<<<(ss_count_launch(), grid_for(n, 256)), 256, 0, ctx->stream>>>(M->diag_pos, n, M->err);
    int herr = 0;
    SS_CUDA(ctx, cudaMemcpyAsync(&herr, M->err, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
    SS_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    if (herr) return set_error(ctx, SS_ZERO_PIVOT, "iLU(0): missing diagonal entry");
    for (int32_t l = 0; l < M->lower.n_levels; ++l) {
        int32_t rows = lptr[l + 1] - lptr[l];
        ilu0_level<<<(ss_count_launch(), grid_for((int64_t)rows * 32, 256)), 256, 0, ctx->stream>>>(
            M->f.row_ptr, M->f.col, M->f.val, M->diag_pos, M->lower.order, lptr[l], lptr[l + 1], M->err);
    }
    SS_CUDA(ctx, cudaGetLastError());
    return SS_OK;
}

// Upload host factors (ILUT) into M.
ss_status prec_from_host(ss_ctx ctx, ss_prec M, int64_t n, const std::vector<int32_t>& rp,
                         const std::vector<int32_t>& col, const std::vector<double>& val) {
    M->f.n_rows = M->f.n_cols = n;
    M->f.nnz = (int64_t)col.size();
    SS_TRY(dev_alloc_n(ctx, &M->f.row_ptr, (size_t)n + 1));
    SS_TRY(dev_alloc_n(ctx, &M->f.col, col.size()));
    SS_TRY(dev_alloc_n(ctx, &M->f.val, col.size()));
    SS_CUDA(ctx, cudaMemcpyAsync(M->f.row_ptr, rp.data(), sizeof(int32_t) * (n + 1), cudaMemcpyHostToDevice, ctx->stream));
    SS_CUDA(ctx, cudaMemcpyAsync(M->f.col, col.data(), sizeof(int32_t) * col.size(), cudaMemcpyHostToDevice, ctx->stream));
    SS_CUDA(ctx, cudaMemcpyAsync(M->f.val, val.data(), sizeof(double) * val.size(), cudaMemcpyHostToDevice, ctx->stream));
    SS_TRY(dev_alloc_n(ctx, &M->diag_pos, (size_t)n));
    SS_TRY(find_diag(ctx, M->f, M->diag_pos));
    std::vector<int32_t> lorder, lptr;
    SS_TRY(analyse(ctx, M, rp, col, lorder, lptr));
    return SS_OK;
}

ss_status prec_finish(ss_ctx ctx, ss_prec M, bool want_fp32) {
    const int64_t n = M->f.n_rows;
    SS_TRY(dev_alloc_n(ctx, &M->inv_diag, (size_t)n));
    if (want_fp32) {
        SS_TRY(dev_alloc_n(ctx, &M->val32, (size_t)M->f.nnz));
        SS_TRY(dev_alloc_n(ctx, &M->inv_diag32, (size_t)n));
        SS_TRY(dev_alloc_n(ctx, &M->tmp32, (size_t)n));
        fill_pending<float2><<<(ss_count_launch(), 256), 256, 0, ctx->stream>>>(n, M->tmp32);
    }
    make_inv_diag<<<(ss_count_launch(), grid_for(n, 256)), 256, 0, ctx->stream>>>(M->f.val, M->diag_pos, n, M->inv_diag, M->inv_diag32,
                                                             M->err);
    if (want_fp32 && M->f.nnz > 0)
        to_f32<<<(ss_count_launch(), grid_for(M->f.nnz, 256)), 256, 0, ctx->stream>>>(M->f.val, M->f.nnz, M->val32);
    SS_CUDA(ctx, cudaGetLastError());
    int herr = 0;
    SS_CUDA(ctx, cudaMemcpyAsync(&herr, M->err, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
    SS_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    if (herr == 2) return set_error(ctx, SS_ZERO_PIVOT, "incomplete LU met a zero pivot");
    if (herr) return set_error(ctx, SS_ERR_TIMEOUT, "device wait timed out");
    return SS_OK;
}

template <bool LOWER, class T>
static void launch_trsv(ss_ctx ctx, ss_prec M, const TriLevels& L, const T* vals, const T* inv, T* b, T* x, T* other,
                        unsigned long long* ticket, const int* halt) {
    const int threads = 256;
    const unsigned g = (unsigned)((L.n_units * 32 + threads - 1) / threads);
#define SS_TRSV_CASE(GG)                                                                                    \
    case GG:                                                                                                \
        sptrsv_syncfree<LOWER, GG, T><<<(ss_count_launch(), g), threads, 0, ctx->stream>>>(M->f.col, vals, inv, L.meta,  \
                                                                       L.n_units, b, x, other, ticket,       \
                                                                       M->err, halt);                        \
        break;
    switch (L.g) {
        SS_TRSV_CASE(2)
        SS_TRSV_CASE(4)
        SS_TRSV_CASE(8)
        SS_TRSV_CASE(16)
        default:
        SS_TRSV_CASE(32)
    }
#undef SS_TRSV_CASE
}

// z = U^{-1} L^{-1} r.  tmp (the lower solve's output) is all PENDING between
// applications; the lower solve marks z PENDING and the upper solve restores
// tmp.  r and z must not alias.
template <class T>
static ss_status apply_impl(ss_ctx ctx, ss_prec M, const T* vals, const T* inv, T* tmp, const T* r, T* z,
                            const int* halt) {
    const int64_t n = M->f.n_rows;
    if (n == 0) return SS_OK;
    {
        ProfScope ps(ctx, PROF_TRSV_LOWER);
        launch_trsv<true, T>(ctx, M, M->lower, vals, inv, const_cast<T*>(r), tmp, z, M->tickets, halt);
    }
    {
        ProfScope ps(ctx, PROF_TRSV_UPPER);
        launch_trsv<false, T>(ctx, M, M->upper, vals, inv, tmp, z, nullptr, M->tickets + 1, halt);
    }
    SS_CUDA(ctx, cudaGetLastError());
    return SS_OK;
}

ss_status prec_apply_dev(ss_ctx ctx, ss_prec M, const double2* r, double2* z, const int* halt) {
    return apply_impl<double2>(ctx, M, M->f.val, M->inv_diag, M->tmp, r, z, halt);
}

ss_status prec_apply_dev32(ss_ctx ctx, ss_prec M, const float2* r, float2* z, const int* halt) {
    if (!M->val32) return set_error(ctx, SS_ERR_INVALID, "preconditioner has no FP32 factors");
    return apply_impl<float2>(ctx, M, M->val32, M->inv_diag32, M->tmp32, r, z, halt);
}

ss_status prec_check_error(ss_ctx ctx, ss_prec M) {
    int herr = 0;
    SS_CUDA(ctx, cudaMemcpyAsync(&herr, M->err, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
    SS_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    if (herr == 1) return set_error(ctx, SS_ERR_TIMEOUT, "triangular solve wait timed out");
    return SS_OK;
}

void prec_destroy(ss_ctx ctx, ss_prec M) {
    free_csr(ctx, M->f);
    dev_free(ctx, M->diag_pos);
    dev_free(ctx, M->inv_diag);
    dev_free(ctx, M->val32);
    dev_free(ctx, M->inv_diag32);
    dev_free(ctx, M->lower.order);
    dev_free(ctx, M->upper.order);
    dev_free(ctx, M->lower.units);
    dev_free(ctx, M->upper.units);
    dev_free(ctx, M->lower.meta);
    dev_free(ctx, M->upper.meta);
    dev_free(ctx, M->flags);
    dev_free(ctx, M->tickets);
    dev_free(ctx, M->err);
    dev_free(ctx, M->tmp);
    dev_free(ctx, M->tmp32);
}
