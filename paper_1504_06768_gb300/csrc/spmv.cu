// Complex CSR SpMV y = A x (FP64 and FP32).  G consecutive lanes share a row
// (G = 2..32 chosen from the mean row length and the precision), so the
// column indices and values of neighbouring rows are read as one contiguous,
// coalesced stream.  On GB300 the FP64 form is bound by the FP64 pipe (4 DFMA
// per stored entry at about 1.26 TFLOP/s), the FP32 form by memory.
#include "common.cuh"
#include "spmv.cuh"

namespace {
inline unsigned grid_for(int64_t n, int b) { return (unsigned)((n + b - 1) / b); }
}

int spmv_group_size(int64_t n_rows, int64_t nnz, bool fp32) {
    const double avg = n_rows > 0 ? (double)nnz / (double)n_rows : 1.0;
    if (avg <= 3.0) return 2;
    if (fp32) {
        if (avg <= 8.0) return 4;
        if (avg <= 32.0) return 8;
    } else {
        if (avg <= 6.0) return 2;
        if (avg <= 24.0) return 4;
        if (avg <= 48.0) return 8;
    }
    return avg <= 96.0 ? 16 : 32;
}

namespace {
constexpr int SPMV_K = 2;   // entries per lane whose loads are in flight together
}

template <int G>
static void launch_f64(const DeviceCSR& A, const double2* x, double2* y, const int* halt, cudaStream_t s) {
    const int threads = 256;
    spmv_kernel<G, SPMV_K, double2, double2><<<(ss_count_launch(), grid_for(A.n_rows * G, threads)), threads, 0, s>>>(
        A.row_ptr, A.col, A.val, A.n_rows, x, y, halt);
}

template <int G>
static void launch_f32(const DeviceCSR& A, const float2* val32, const float2* x, float2* y, const int* halt,
                       cudaStream_t s) {
    const int threads = 256;
    spmv_kernel<G, SPMV_K, float2, float2><<<(ss_count_launch(), grid_for(A.n_rows * G, threads)), threads, 0, s>>>(
        A.row_ptr, A.col, val32, A.n_rows, x, y, halt);
}

int spmv_split_group_size(int64_t n_rows, int64_t parts) {
    const double avg = n_rows > 0 ? (double)parts / (double)n_rows : 1.0;
    return avg <= 4.0 ? 2 : 4;
}

constexpr int SPLIT_K = 2;   // parts per lane whose loads are in flight together in the FP64 split SpMV

template <int G>
static void launch_split(const DeviceCSR& A, const double2* x, double2* y, const int* halt, cudaStream_t s) {
    const int threads = 256;
    spmv_split_kernel<G, SPLIT_K><<<(ss_count_launch(), grid_for(A.n_rows * G, threads)), threads, 0, s>>>(
        A.s_row_ptr, A.s_mid, A.s_col, A.s_val, A.n_rows, x, y, halt);
}

void spmv_launch(const DeviceCSR& A, const double2* x, double2* y, const int* halt, cudaStream_t s) {
    if (A.n_rows == 0) return;
    if (A.s_state == 1) {
        switch (spmv_split_group_size(A.n_rows, A.s_nnz)) {
            case 1: launch_split<1>(A, x, y, halt, s); break;
            case 2: launch_split<2>(A, x, y, halt, s); break;
            case 4: launch_split<4>(A, x, y, halt, s); break;
            default: launch_split<8>(A, x, y, halt, s); break;
        }
        return;
    }
    switch (spmv_group_size(A.n_rows, A.nnz, false)) {
        case 2: launch_f64<2>(A, x, y, halt, s); break;
        case 4: launch_f64<4>(A, x, y, halt, s); break;
        case 8: launch_f64<8>(A, x, y, halt, s); break;
        case 16: launch_f64<16>(A, x, y, halt, s); break;
        default: launch_f64<32>(A, x, y, halt, s); break;
    }
}

void spmv_launch32(const DeviceCSR& A, const float2* val32, const float2* x, float2* y, const int* halt,
                   cudaStream_t s) {
    if (A.n_rows == 0) return;
    switch (spmv_group_size(A.n_rows, A.nnz, true)) {
        case 2: launch_f32<2>(A, val32, x, y, halt, s); break;
        case 4: launch_f32<4>(A, val32, x, y, halt, s); break;
        case 8: launch_f32<8>(A, val32, x, y, halt, s); break;
        case 16: launch_f32<16>(A, val32, x, y, halt, s); break;
        default: launch_f32<32>(A, val32, x, y, halt, s); break;
    }
}

ss_status spmv_dev(ss_ctx ctx, const DeviceCSR& A, const double2* x, double2* y) {
    { ProfScope ps_(ctx, PROF_SPMV); spmv_launch(A, x, y, nullptr, ctx->stream); }
    SS_CUDA(ctx, cudaGetLastError());
    return SS_OK;
}

ss_status spmv_dev32(ss_ctx ctx, const DeviceCSR& A, const float2* val32, const float2* x, float2* y) {
    spmv_launch32(A, val32, x, y, nullptr, ctx->stream);
    SS_CUDA(ctx, cudaGetLastError());
    return SS_OK;
}

// ------------------------------------------------------- part-split copy

namespace {

__global__ void split_count(const int32_t* __restrict__ rp, const double2* __restrict__ val, int64_t n,
                            int32_t* __restrict__ cnt) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int32_t c = 0;
    for (int32_t t = rp[i]; t < rp[i + 1]; ++t) c += (val[t].x != 0.0) + (val[t].y != 0.0);
    cnt[i] = c;
}

__global__ void split_fill(const int32_t* __restrict__ rp, const int32_t* __restrict__ col,
                           const double2* __restrict__ val, int64_t n, const int32_t* __restrict__ srp,
                           int32_t* __restrict__ smid, uint32_t* __restrict__ scol, double* __restrict__ sval) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int32_t k = srp[i];
    for (int32_t t = rp[i]; t < rp[i + 1]; ++t)          // real parts first
        if (val[t].x != 0.0) { scol[k] = (uint32_t)col[t]; sval[k] = val[t].x; ++k; }
    smid[i] = k;
    for (int32_t t = rp[i]; t < rp[i + 1]; ++t)          // then the imaginary parts
        if (val[t].y != 0.0) { scol[k] = (uint32_t)col[t]; sval[k] = val[t].y; ++k; }
}

}  // namespace

ss_status csr_split(ss_ctx ctx, DeviceCSR& A) {
    if (A.s_state != 0 || A.n_rows == 0) return SS_OK;
    const int64_t n = A.n_rows;
    int32_t* cnt = nullptr;
    SS_TRY(dev_alloc_n(ctx, &cnt, (size_t)n));
    split_count<<<(ss_count_launch(), grid_for(n, 256)), 256, 0, ctx->stream>>>(A.row_ptr, A.val, n, cnt);
    SS_TRY(dev_alloc_n(ctx, &A.s_row_ptr, (size_t)n + 1));
    int64_t total = 0;
    ss_status st = exclusive_scan_i32(ctx, cnt, A.s_row_ptr, n, &total);
    dev_free(ctx, cnt);
    if (st != SS_OK || (double)total > 1.6 * (double)A.nnz) {
        dev_free(ctx, A.s_row_ptr);
        A.s_row_ptr = nullptr;
        A.s_state = -1;
        return st == SS_ERR_UNSUPPORTED ? SS_OK : st;
    }
    A.s_nnz = total;
    SS_TRY(dev_alloc_n(ctx, &A.s_col, (size_t)total));
    SS_TRY(dev_alloc_n(ctx, &A.s_val, (size_t)total));
    SS_TRY(dev_alloc_n(ctx, &A.s_mid, (size_t)n));
    split_fill<<<(ss_count_launch(), grid_for(n, 256)), 256, 0, ctx->stream>>>(A.row_ptr, A.col, A.val, n,
                                                                               A.s_row_ptr, A.s_mid, A.s_col,
                                                                               A.s_val);
    SS_CUDA(ctx, cudaGetLastError());
    A.s_state = 1;
    return SS_OK;
}

void csr_split_free(ss_ctx ctx, DeviceCSR& A) {
    dev_free(ctx, A.s_mid);
    A.s_mid = nullptr;
    dev_free(ctx, A.s_row_ptr);
    dev_free(ctx, A.s_col);
    dev_free(ctx, A.s_val);
    A.s_row_ptr = nullptr;
    A.s_col = nullptr;
    A.s_val = nullptr;
    A.s_nnz = 0;
    A.s_state = 0;
}
