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

void spmv_launch(const DeviceCSR& A, const double2* x, double2* y, const int* halt, cudaStream_t s) {
    if (A.n_rows == 0) return;
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
