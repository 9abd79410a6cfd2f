// C ABI entry points (include/lindblad_ss.h) and the steady-state driver.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "common.cuh"
#include "krylov.cuh"
#include "solver_util.cuh"
#include "spmv.cuh"
#include "direct.cuh"

namespace {

double now_ms() {
    using namespace std::chrono;
    return duration<double, std::milli>(steady_clock::now().time_since_epoch()).count();
}

ss_mat wrap(ss_ctx ctx, DeviceCSR& m, int64_t d) {
    ss_mat h = new (std::nothrow) ss_mat_s();
    if (!h) return nullptr;
    h->m = m;
    h->d = d;
    (void)ctx;
    return h;
}

int64_t isqrt_exact(int64_t n) {
    int64_t r = (int64_t)std::llround(std::sqrt((double)n));
    while (r * r > n) --r;
    while ((r + 1) * (r + 1) <= n) ++r;
    return r * r == n ? r : -1;
}

ss_status check_ctx(ss_ctx ctx) {
    if (!ctx) return SS_ERR_INVALID;
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess) return cuda_check(ctx, e, "cudaSetDevice");
    return SS_OK;
}

// Download the pattern (row_ptr, col) of a device matrix.
ss_status download_pattern(ss_ctx ctx, const DeviceCSR& A, std::vector<int32_t>& rp, std::vector<int32_t>& col) {
    rp.resize(A.n_rows + 1);
    col.resize(A.nnz);
    SS_CUDA(ctx, cudaMemcpyAsync(rp.data(), A.row_ptr, sizeof(int32_t) * (A.n_rows + 1), cudaMemcpyDeviceToHost,
                                 ctx->stream));
    if (A.nnz)
        SS_CUDA(ctx, cudaMemcpyAsync(col.data(), A.col, sizeof(int32_t) * A.nnz, cudaMemcpyDeviceToHost, ctx->stream));
    SS_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    return SS_OK;
}

ss_status build_prec(ss_ctx ctx, const DeviceCSR& A, int kind, double drop_tol, double fill_factor, bool fp32,
                     ss_prec* out) {
    *out = nullptr;
    ss_prec M = new (std::nothrow) ss_prec_s();
    if (!M) return set_error(ctx, SS_ERR_OOM, "host allocation failed");
    ss_status st = SS_OK;
    if (kind == SS_PRECOND_ILU0) {
        st = ilu0_device(ctx, A, M);
    } else if (kind == SS_PRECOND_ILUT) {
        std::vector<int32_t> rp(A.n_rows + 1), col(A.nnz), frp, fcol;
        std::vector<double> val(2 * A.nnz), fval;
        cudaMemcpyAsync(rp.data(), A.row_ptr, sizeof(int32_t) * (A.n_rows + 1), cudaMemcpyDeviceToHost, ctx->stream);
        cudaMemcpyAsync(col.data(), A.col, sizeof(int32_t) * A.nnz, cudaMemcpyDeviceToHost, ctx->stream);
        cudaMemcpyAsync(val.data(), A.val, sizeof(double2) * A.nnz, cudaMemcpyDeviceToHost, ctx->stream);
        cudaError_t e = cudaStreamSynchronize(ctx->stream);
        if (e != cudaSuccess) st = cuda_check(ctx, e, "download for ILUT");
        if (st == SS_OK) {
            int64_t bad = ilut_host(A.n_rows, rp.data(), col.data(), val.data(), drop_tol, fill_factor, frp, fcol, fval);
            if (bad) st = set_error(ctx, SS_ZERO_PIVOT, "ILUT: zero pivot in row " + std::to_string(bad - 1));
            else if ((int64_t)fcol.size() > INT32_MAX) st = set_error(ctx, SS_ERR_UNSUPPORTED, "ILUT factors too large");
            else st = prec_from_host(ctx, M, A.n_rows, frp, fcol, fval);
        }
    } else {
        st = set_error(ctx, SS_ERR_INVALID, "unknown preconditioner kind");
    }
    if (st == SS_OK) st = prec_finish(ctx, M, fp32);
    if (st != SS_OK) {
        prec_destroy(ctx, M);
        delete M;
        return st;
    }
    *out = M;
    return SS_OK;
}

}  // namespace

// ------------------------------------------------------------------ context

extern "C" ss_status ss_ctx_create(int device, void* cuda_stream, ss_ctx* out) {
    if (!out) return SS_ERR_INVALID;
    *out = nullptr;
    int count = 0;
    if (cudaGetDeviceCount(&count) != cudaSuccess || device < 0 || device >= count) {
        cudaGetLastError();
        return SS_ERR_CUDA;
    }
    if (cudaSetDevice(device) != cudaSuccess) return SS_ERR_CUDA;
    ss_ctx c = new (std::nothrow) ss_ctx_s();
    if (!c) return SS_ERR_OOM;
    c->device = device;
    c->stream = reinterpret_cast<cudaStream_t>(cuda_stream);
    cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, device);
    c->pool = device_pool(device);
    // the allocation-free entry point's workspace is loaded here, not in its first call
    const ss_status st = noalloc_prepare(c);
    if (st != SS_OK) {
        delete c;
        return st;
    }
    *out = c;
    return SS_OK;
}

extern "C" ss_status ss_ctx_destroy(ss_ctx ctx) {
    if (!ctx) return SS_ERR_INVALID;
    cudaSetDevice(ctx->device);
    cudaStreamSynchronize(ctx->stream);
    if (ctx->host_stage) cudaFreeHost(ctx->host_stage);
    delete ctx;
    return SS_OK;
}

extern "C" ss_status ss_ctx_set_stream(ss_ctx ctx, void* cuda_stream) {
    if (!ctx) return SS_ERR_INVALID;
    ctx->stream = reinterpret_cast<cudaStream_t>(cuda_stream);
    return SS_OK;
}

extern "C" const char* ss_last_error(ss_ctx ctx) { return ctx ? ctx->last_error.c_str() : "null context"; }

extern "C" void ss_options_default(ss_options* o) {
    if (!o) return;
    o->method = SS_METHOD_ITER_BICGSTAB;
    o->precond = SS_PRECOND_ILU0;
    o->precision = SS_PREC_FP64;
    o->tol = 1e-10;
    o->maxiter = 1000;
    o->restart = 30;
    o->drop_tol = 1e-4;
    o->fill_factor = 10.0;
    o->w = 0.0;
    o->sigma = 1e-15;
    o->use_rcm = 1;
    o->seed = 0;
    o->inner_rtol = 1e-5;
    o->lgmres_k = 0;
    o->warm_start = 0;
    o->autotune = 0;
}

// ----------------------------------------------------------------- matrices

extern "C" ss_status assemble_liouvillian(ss_ctx ctx, const ss_csr_view* H, int n_c, const ss_csr_view* c_ops,
                                          ss_mat* L_out) {
    SS_TRY(check_ctx(ctx));
    if (!L_out || !H || n_c < 0 || (n_c > 0 && !c_ops)) return set_error(ctx, SS_ERR_INVALID, "null argument");
    *L_out = nullptr;
    const int64_t d = H->n_rows;
    if (H->n_cols != d || d <= 0) return set_error(ctx, SS_ERR_INVALID, "H must be square and non-empty");
    for (int c = 0; c < n_c; ++c)
        if (c_ops[c].n_rows != d || c_ops[c].n_cols != d)
            return set_error(ctx, SS_ERR_INVALID, "collapse operator " + std::to_string(c) + " is not d x d");
    DeviceCSR Hd;
    std::vector<DeviceCSR> C(n_c);
    ss_status st = upload_csr(ctx, H, Hd);
    for (int c = 0; c < n_c && st == SS_OK; ++c) st = upload_csr(ctx, &c_ops[c], C[c]);
    DeviceCSR L;
    if (st == SS_OK) st = assemble_impl(ctx, Hd, C, L);
    free_csr(ctx, Hd);
    for (auto& c : C) free_csr(ctx, c);
    if (st != SS_OK) { free_csr(ctx, L); return st; }
    cudaError_t e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) { free_csr(ctx, L); return cuda_check(ctx, e, "assemble_liouvillian"); }
    *L_out = wrap(ctx, L, d);
    return *L_out ? SS_OK : set_error(ctx, SS_ERR_OOM, "host allocation failed");
}

extern "C" ss_status add_trace_row(ss_ctx ctx, ss_mat L, double w, ss_mat* out, double* w_used) {
    SS_TRY(check_ctx(ctx));
    if (!L || !out) return set_error(ctx, SS_ERR_INVALID, "null argument");
    *out = nullptr;
    int64_t d = L->d > 0 ? L->d : isqrt_exact(L->m.n_rows);
    if (d <= 0) return set_error(ctx, SS_ERR_INVALID, "matrix size is not a square d^2");
    if (!(w > 0.0)) {
        SS_TRY(mean_abs_diag(ctx, L->m, &w));
        if (w == 0.0) w = 1.0;      // an all-zero diagonal: any positive weight will do
    }
    if (!(w > 0.0) || !std::isfinite(w)) return set_error(ctx, SS_ERR_INVALID, "weight w must be positive and finite");
    DeviceCSR o;
    ss_status st = add_trace_row_impl(ctx, L->m, d, w, o);
    if (st == SS_OK) {
        cudaError_t e = cudaStreamSynchronize(ctx->stream);
        if (e != cudaSuccess) st = cuda_check(ctx, e, "add_trace_row");
    }
    if (st != SS_OK) { free_csr(ctx, o); return st; }
    if (w_used) *w_used = w;
    *out = wrap(ctx, o, d);
    return SS_OK;
}

extern "C" ss_status add_shift(ss_ctx ctx, ss_mat L, double sigma, ss_mat* out) {
    SS_TRY(check_ctx(ctx));
    if (!L || !out) return set_error(ctx, SS_ERR_INVALID, "null argument");
    *out = nullptr;
    DeviceCSR o;
    ss_status st = add_shift_impl(ctx, L->m, sigma, o);
    if (st == SS_OK) {
        cudaError_t e = cudaStreamSynchronize(ctx->stream);
        if (e != cudaSuccess) st = cuda_check(ctx, e, "add_shift");
    }
    if (st != SS_OK) { free_csr(ctx, o); return st; }
    *out = wrap(ctx, o, L->d);
    return SS_OK;
}

extern "C" ss_status rcm_permute(ss_ctx ctx, ss_mat A, int32_t* perm_out, int64_t* bw_out, int64_t* profile_out) {
    SS_TRY(check_ctx(ctx));
    if (!A || !perm_out) return set_error(ctx, SS_ERR_INVALID, "null argument");
    if (A->m.n_rows != A->m.n_cols) return set_error(ctx, SS_ERR_INVALID, "matrix must be square");
    std::vector<int32_t> rp, col;
    SS_TRY(download_pattern(ctx, A->m, rp, col));
    rcm_host(A->m.n_rows, rp.data(), col.data(), perm_out);
    if (bw_out || profile_out) {
        DeviceCSR P;
        ss_status st = permute_impl(ctx, A->m, perm_out, P);
        if (st == SS_OK) st = bandwidth_profile_impl(ctx, P, bw_out, profile_out);
        free_csr(ctx, P);
        SS_TRY(st);
    }
    return SS_OK;
}

extern "C" ss_status permute(ss_ctx ctx, ss_mat A, const int32_t* perm, ss_mat* out) {
    SS_TRY(check_ctx(ctx));
    if (!A || !perm || !out) return set_error(ctx, SS_ERR_INVALID, "null argument");
    *out = nullptr;
    const int64_t n = A->m.n_rows;
    std::vector<char> seen(n, 0);
    for (int64_t r = 0; r < n; ++r) {
        if (perm[r] < 0 || perm[r] >= n || seen[perm[r]]) return set_error(ctx, SS_ERR_INVALID, "not a permutation");
        seen[perm[r]] = 1;
    }
    DeviceCSR o;
    ss_status st = permute_impl(ctx, A->m, perm, o);
    if (st == SS_OK) {
        cudaError_t e = cudaStreamSynchronize(ctx->stream);
        if (e != cudaSuccess) st = cuda_check(ctx, e, "permute");
    }
    if (st != SS_OK) { free_csr(ctx, o); return st; }
    *out = wrap(ctx, o, A->d);
    return SS_OK;
}

extern "C" ss_status bandwidth_profile(ss_ctx ctx, ss_mat A, int64_t* bw_out, int64_t* profile_out) {
    SS_TRY(check_ctx(ctx));
    if (!A) return set_error(ctx, SS_ERR_INVALID, "null argument");
    return bandwidth_profile_impl(ctx, A->m, bw_out, profile_out);
}

extern "C" ss_status ss_mat_shape(ss_mat A, int64_t* n_rows, int64_t* nnz) {
    if (!A) return SS_ERR_INVALID;
    if (n_rows) *n_rows = A->m.n_rows;
    if (nnz) *nnz = A->m.nnz;
    return SS_OK;
}

extern "C" ss_status ss_mat_export(ss_ctx ctx, ss_mat A, int32_t* row_ptr, int32_t* col, double* val) {
    SS_TRY(check_ctx(ctx));
    if (!A || !row_ptr) return set_error(ctx, SS_ERR_INVALID, "null argument");
    SS_CUDA(ctx, cudaMemcpyAsync(row_ptr, A->m.row_ptr, sizeof(int32_t) * (A->m.n_rows + 1), cudaMemcpyDeviceToHost,
                                 ctx->stream));
    if (A->m.nnz && col)
        SS_CUDA(ctx, cudaMemcpyAsync(col, A->m.col, sizeof(int32_t) * A->m.nnz, cudaMemcpyDeviceToHost, ctx->stream));
    if (A->m.nnz && val)
        SS_CUDA(ctx, cudaMemcpyAsync(val, A->m.val, sizeof(double2) * A->m.nnz, cudaMemcpyDeviceToHost, ctx->stream));
    SS_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    return SS_OK;
}

extern "C" ss_status ss_mat_import(ss_ctx ctx, const ss_csr_view* v, ss_mat* out) {
    SS_TRY(check_ctx(ctx));
    if (!out) return set_error(ctx, SS_ERR_INVALID, "null argument");
    *out = nullptr;
    DeviceCSR m;
    ss_status st = upload_csr(ctx, v, m);
    if (st == SS_OK) {
        cudaError_t e = cudaStreamSynchronize(ctx->stream);
        if (e != cudaSuccess) st = cuda_check(ctx, e, "ss_mat_import");
    }
    if (st != SS_OK) { free_csr(ctx, m); return st; }
    int64_t d = (m.n_rows == m.n_cols) ? isqrt_exact(m.n_rows) : -1;
    *out = wrap(ctx, m, d > 0 ? d : 0);
    return SS_OK;
}

extern "C" void ss_mat_free(ss_mat A) {
    if (!A) return;
    dev_free_nostream(A->m.row_ptr);
    dev_free_nostream(A->m.col);
    dev_free_nostream(A->m.val);
    dev_free_nostream(A->diag_pos);
    dev_free_nostream(A->val32);
    dev_free_nostream(A->m.s_row_ptr);
    dev_free_nostream(A->m.s_mid);
    dev_free_nostream(A->m.s_col);
    dev_free_nostream(A->m.s_val);
    cudaStreamSynchronize(0);
    delete A;
}

extern "C" ss_status spmv(ss_ctx ctx, ss_mat A, const double* x, double* y) {
    SS_TRY(check_ctx(ctx));
    if (!A || !x || !y) return set_error(ctx, SS_ERR_INVALID, "null argument");
    SS_TRY(csr_split(ctx, A->m));
    SS_TRY(spmv_dev(ctx, A->m, reinterpret_cast<const double2*>(x), reinterpret_cast<double2*>(y)));
    SS_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    return SS_OK;
}

__global__ static void to_f32_vals(const double2* __restrict__ a, int64_t n, float2* __restrict__ b) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) b[i] = make_float2((float)a[i].x, (float)a[i].y);
}

static ss_status ensure_f32(ss_ctx ctx, ss_mat A) {
    if (A->val32) return SS_OK;
    SS_TRY(dev_alloc_n(ctx, &A->val32, (size_t)A->m.nnz));
    if (A->m.nnz)
        to_f32_vals<<<(ss_count_launch(), (unsigned)((A->m.nnz + 255) / 256)), 256, 0, ctx->stream>>>(A->m.val, A->m.nnz, A->val32);
    SS_CUDA(ctx, cudaGetLastError());
    return SS_OK;
}

extern "C" ss_status spmv_f32(ss_ctx ctx, ss_mat A, const float* x, float* y) {
    SS_TRY(check_ctx(ctx));
    if (!A || !x || !y) return set_error(ctx, SS_ERR_INVALID, "null argument");
    SS_TRY(ensure_f32(ctx, A));
    SS_TRY(spmv_dev32(ctx, A->m, A->val32, reinterpret_cast<const float2*>(x), reinterpret_cast<float2*>(y)));
    SS_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    return SS_OK;
}

// ------------------------------------------------------------ preconditioner

extern "C" ss_status ilu_factor(ss_ctx ctx, ss_mat A, int kind, double drop_tol, double fill_factor, int precision,
                                ss_prec* out, double* condest_out) {
    SS_TRY(check_ctx(ctx));
    if (!A || !out) return set_error(ctx, SS_ERR_INVALID, "null argument");
    *out = nullptr;
    if (A->m.n_rows != A->m.n_cols) return set_error(ctx, SS_ERR_INVALID, "matrix must be square");
    if (kind == SS_PRECOND_ILUT && (!(drop_tol >= 0.0) || !(fill_factor > 0.0)))
        return set_error(ctx, SS_ERR_INVALID, "ILUT needs drop_tol >= 0 and fill_factor > 0");
    ss_prec M = nullptr;
    SS_TRY(build_prec(ctx, A->m, kind, drop_tol, fill_factor, precision == SS_PREC_MIXED, &M));
    if (condest_out) {
        const int64_t n = A->m.n_rows;
        double2* buf = nullptr;
        double* scr = nullptr;
        ss_status st = dev_alloc_n(ctx, &buf, (size_t)2 * n);
        if (st == SS_OK) st = dev_alloc_n(ctx, &scr, (size_t)su_scratch_doubles());
        if (st == SS_OK) st = su_condest(ctx, M, n, buf, buf + n, scr, condest_out);
        dev_free(ctx, buf);
        dev_free(ctx, scr);
        if (st != SS_OK) { prec_destroy(ctx, M); delete M; return st; }
    }
    *out = M;
    return SS_OK;
}

extern "C" ss_status precond_apply(ss_ctx ctx, ss_prec M, const double* r, double* z) {
    SS_TRY(check_ctx(ctx));
    if (!M || !r || !z) return set_error(ctx, SS_ERR_INVALID, "null argument");
    SS_TRY(prec_apply_dev(ctx, M, reinterpret_cast<const double2*>(r), reinterpret_cast<double2*>(z)));
    return prec_check_error(ctx, M);
}

extern "C" ss_status precond_apply_f32(ss_ctx ctx, ss_prec M, const float* r, float* z) {
    SS_TRY(check_ctx(ctx));
    if (!M || !r || !z) return set_error(ctx, SS_ERR_INVALID, "null argument");
    SS_TRY(prec_apply_dev32(ctx, M, reinterpret_cast<const float2*>(r), reinterpret_cast<float2*>(z)));
    return prec_check_error(ctx, M);
}

extern "C" ss_status ss_set_wait_limit(ss_ctx ctx, uint64_t limit_ns) {
    if (!ctx || limit_ns == 0) return SS_ERR_INVALID;
    ctx->wait_ns = limit_ns;
    return SS_OK;
}

extern "C" ss_status ss_diag_batched_stall(ss_ctx ctx, int64_t seq) {
    if (!ctx || seq < -1) return SS_ERR_INVALID;
    ctx->diag_stall_seq = seq;
    return SS_OK;
}

extern "C" ss_status ss_diag_prec_skip_row(ss_ctx ctx, ss_prec M, int64_t row, int restore) {
    SS_TRY(check_ctx(ctx));
    if (!M) return set_error(ctx, SS_ERR_INVALID, "null argument");
    return prec_skip_row(ctx, M, row, restore);
}

extern "C" ss_status ss_prec_info(ss_prec M, int64_t* nnz, int32_t* levels_lower, int32_t* levels_upper) {
    if (!M) return SS_ERR_INVALID;
    if (nnz) *nnz = M->f.nnz;
    if (levels_lower) *levels_lower = M->lower.n_levels;
    if (levels_upper) *levels_upper = M->upper.n_levels;
    return SS_OK;
}

extern "C" ss_status ss_prec_export(ss_ctx ctx, ss_prec M, int32_t* row_ptr, int32_t* col, double* val) {
    SS_TRY(check_ctx(ctx));
    if (!M || !row_ptr) return set_error(ctx, SS_ERR_INVALID, "null argument");
    SS_CUDA(ctx, cudaMemcpyAsync(row_ptr, M->f.row_ptr, sizeof(int32_t) * (M->f.n_rows + 1), cudaMemcpyDeviceToHost,
                                 ctx->stream));
    if (M->f.nnz && col)
        SS_CUDA(ctx, cudaMemcpyAsync(col, M->f.col, sizeof(int32_t) * M->f.nnz, cudaMemcpyDeviceToHost, ctx->stream));
    if (M->f.nnz && val)
        SS_CUDA(ctx, cudaMemcpyAsync(val, M->f.val, sizeof(double2) * M->f.nnz, cudaMemcpyDeviceToHost, ctx->stream));
    SS_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    return SS_OK;
}

extern "C" void ss_prec_free(ss_prec M) {
    if (!M) return;
    ss_ctx_s tmp;
    tmp.stream = 0;
    prec_destroy(&tmp, M);
    cudaStreamSynchronize(0);
    delete M;
}

// ------------------------------------------------------------------ solvers

extern "C" ss_status krylov_solve(ss_ctx ctx, ss_mat A, ss_prec M, int krylov, const double* b, double* x, double tol,
                                  int maxiter, int restart, int* iters_out, double* resid_out) {
    SS_TRY(check_ctx(ctx));
    if (!A || !M || !b || !x) return set_error(ctx, SS_ERR_INVALID, "null argument");
    if (M->f.n_rows != A->m.n_rows) return set_error(ctx, SS_ERR_INVALID, "preconditioner size mismatch");
    SS_TRY(csr_split(ctx, A->m));
    KrylovWork w;
    const int m = krylov == SS_KRYLOV_GMRES ? restart : 0;
    ss_status st = krylov_workspace(ctx, w, A->m.n_rows, krylov, m);
    KrylovResultHost res;
    if (st == SS_OK) {
        if (krylov == SS_KRYLOV_GMRES)
            st = gmres_dev(ctx, A->m, M, w, reinterpret_cast<const double2*>(b), reinterpret_cast<double2*>(x), tol,
                           maxiter, restart, &res);
        else
            st = bicgstab_dev(ctx, A->m, M, w, reinterpret_cast<const double2*>(b), reinterpret_cast<double2*>(x), tol,
                              maxiter, &res);
    }
    krylov_workspace_free(ctx, w);
    SS_TRY(st);
    if (iters_out) *iters_out = res.iters;
    if (resid_out) *resid_out = res.resid;
    if (res.status != SS_OK) {
        ctx->last_error = res.status == SS_BREAKDOWN ? "BiCGSTAB breakdown" : "iteration cap reached";
        return (ss_status)res.status;
    }
    return SS_OK;
}

extern "C" ss_status lgmres_solve(ss_ctx ctx, ss_mat A, ss_prec M, const double* b, double* x, double tol,
                                  int maxiter, int restart, int augment, int* iters_out, double* resid_out) {
    SS_TRY(check_ctx(ctx));
    if (!A || !M || !b || !x) return set_error(ctx, SS_ERR_INVALID, "null argument");
    if (M->f.n_rows != A->m.n_rows) return set_error(ctx, SS_ERR_INVALID, "preconditioner size mismatch");
    SS_TRY(csr_split(ctx, A->m));
    KrylovWork w;
    ss_status st = krylov_workspace(ctx, w, A->m.n_rows, SS_KRYLOV_GMRES, restart, augment);
    KrylovResultHost res;
    if (st == SS_OK)
        st = gmres_dev(ctx, A->m, M, w, reinterpret_cast<const double2*>(b), reinterpret_cast<double2*>(x), tol,
                       maxiter, restart, &res, nullptr, augment);
    krylov_workspace_free(ctx, w);
    SS_TRY(st);
    if (iters_out) *iters_out = res.iters;
    if (resid_out) *resid_out = res.resid;
    if (res.status != SS_OK) {
        ctx->last_error = "iteration cap reached";
        return (ss_status)res.status;
    }
    return SS_OK;
}

// Steady state of one system (all §-references are to the paper).
namespace {

// method=direct: x = L~^{-1} (w e_0) by the banded LU (direct.cu), acceptance
// test ||L rho||_2 <= tol on the trace-normalised rho, finalisation.  Takes
// ownership of Ap.
ss_status steady_state_direct(ss_ctx ctx, ss_mat Ap, const std::vector<int32_t>& perm, int64_t d, double w_used,
                              const ss_options& opt, double t0, ss_info inf, double* rho_out, int rho_on_device,
                              ss_info* info) {
    const int64_t n = Ap->m.n_rows;
    std::vector<int32_t> iperm(n), tidx(d);
    for (int64_t r = 0; r < n; ++r) iperm[perm[r]] = (int32_t)r;
    for (int64_t i = 0; i < d; ++i) tidx[i] = iperm[i * (d + 1)];
    const int64_t r0 = iperm[0];
    int32_t *perm_d = nullptr, *tidx_d = nullptr;
    double2 *b = nullptr, *x = nullptr, *y = nullptr, *rho = nullptr, *trace_d = nullptr;
    double* scr = nullptr;
    ss_status st = SS_OK;
    auto cleanup = [&]() {
        dev_free(ctx, perm_d); dev_free(ctx, tidx_d); dev_free(ctx, b); dev_free(ctx, x); dev_free(ctx, y);
        dev_free(ctx, rho); dev_free(ctx, trace_d); dev_free(ctx, scr);
        ss_mat_free(Ap);
    };
#define DSTEP(call) do { st = (call); if (st != SS_OK) { cleanup(); return st; } } while (0)
    DSTEP(dev_alloc_n(ctx, &perm_d, (size_t)n));
    DSTEP(dev_alloc_n(ctx, &tidx_d, (size_t)d));
    DSTEP(dev_alloc_n(ctx, &b, (size_t)n));
    DSTEP(dev_alloc_n(ctx, &x, (size_t)n));
    DSTEP(dev_alloc_n(ctx, &y, (size_t)n));
    DSTEP(dev_alloc_n(ctx, &rho, (size_t)n));
    DSTEP(dev_alloc_n(ctx, &trace_d, 1));
    DSTEP(dev_alloc_n(ctx, &scr, (size_t)su_scratch_doubles()));
    SS_CUDA(ctx, cudaMemcpyAsync(perm_d, perm.data(), sizeof(int32_t) * n, cudaMemcpyHostToDevice, ctx->stream));
    SS_CUDA(ctx, cudaMemcpyAsync(tidx_d, tidx.data(), sizeof(int32_t) * d, cudaMemcpyHostToDevice, ctx->stream));
    DSTEP(su_zero(ctx, n, b));
    const double2 wb = make_double2(w_used, 0.0);
    SS_CUDA(ctx, cudaMemcpyAsync(b + r0, &wb, sizeof(double2), cudaMemcpyHostToDevice, ctx->stream));
    const double t1 = now_ms();
    BandInfo bi;
    DSTEP(band_lu_solve(ctx, Ap->m, b, x, &bi));
    double lr = INFINITY;
    DSTEP(su_lrho(ctx, Ap->m, x, 0, w_used, r0, d, tidx_d, y, scr, trace_d, &lr, nullptr));
    DSTEP(su_trace(ctx, d, tidx_d, x, trace_d));
    DSTEP(su_finalise(ctx, n, perm_d, x, trace_d, rho));
    SS_CUDA(ctx, cudaMemcpyAsync(rho_out, rho, sizeof(double2) * n,
                                 rho_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, ctx->stream));
    SS_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    const int status = lr <= opt.tol ? SS_OK : SS_NOT_CONVERGED;
    inf.status = status;
    inf.iters = 0;
    inf.outer_iters = 1;
    inf.resid_Lrho = lr;
    inf.nnz_factors = n * (2 * bi.kl + bi.ku + 1);      // band entries of L and U
    inf.ms_setup = t1 - t0;
    inf.ms_solve = now_ms() - t1;
    if (info) *info = inf;
    cleanup();
#undef DSTEP
    if (status != SS_OK) ctx->last_error = "direct solve: ||L rho|| above tol (rounding of an ill-conditioned system)";
    return (ss_status)status;
}

}  // namespace

extern "C" ss_status steady_state(ss_ctx ctx, const ss_csr_view* H, int n_c, const ss_csr_view* c_ops,
                                  const ss_options* opt_in, double* rho_out, int rho_on_device, ss_info* info) {
    SS_TRY(check_ctx(ctx));
    ss_options opt;
    ss_options_default(&opt);
    if (opt_in) opt = *opt_in;
    if (!rho_out || !H) return set_error(ctx, SS_ERR_INVALID, "null argument");
    if (opt.method < SS_METHOD_DIRECT || opt.method > SS_METHOD_AUTO)
        return set_error(ctx, SS_ERR_INVALID, "unknown method");
    const bool mixed = opt.precision == SS_PREC_MIXED;
    const bool direct = opt.method == SS_METHOD_DIRECT;
    const bool automatic = opt.method == SS_METHOD_AUTO;
    if (mixed && opt.method != SS_METHOD_ITER_BICGSTAB)
        return set_error(ctx, SS_ERR_UNSUPPORTED, "mixed precision is built for iterative-bicgstab only");
    if (!(opt.tol > 0.0) || opt.maxiter < 1) return set_error(ctx, SS_ERR_INVALID, "tol must be > 0, maxiter >= 1");
    if ((opt.method == SS_METHOD_ITER_GMRES || automatic) &&
        (opt.restart < 1 || opt.lgmres_k < 0 || opt.restart + opt.lgmres_k > KRYLOV_MAX_M))
        return set_error(ctx, SS_ERR_INVALID, "GMRES needs restart >= 1, lgmres_k >= 0, restart + lgmres_k <= 64");
    bool power = opt.method == SS_METHOD_INVERSE_POWER;
    int krylov = opt.method == SS_METHOD_ITER_GMRES || automatic ? SS_KRYLOV_GMRES : SS_KRYLOV_BICGSTAB;
    const double t0 = now_ms();

    ss_mat L = nullptr, A = nullptr, Ap = nullptr;
    ss_prec M = nullptr;
    ss_status st = assemble_liouvillian(ctx, H, n_c, c_ops, &L);
    if (st != SS_OK) return st;
    const int64_t d = L->d, n = L->m.n_rows;
    double w_used = 0.0;
    std::vector<int32_t> perm(n);
    int64_t bw_mod = 0, bw_shift = 0;
    bool have_perm = false;
    if (automatic) {
        // sections "Results" and "Conclusion": compare the RCM bandwidths of
        // L~ and L - sigma I; inverse power when the trace row spoils the
        // reduction (1.5 separates the paper's printed pairs: 139/137 and
        // 239/229 for GMRES, 405/167 for inverse power)
        ss_mat Am = nullptr, As = nullptr;
        std::vector<int32_t> pm(n), ps(n);
        st = add_trace_row(ctx, L, opt.w, &Am, &w_used);
        if (st == SS_OK) st = add_shift(ctx, L, opt.sigma, &As);
        if (st == SS_OK) st = rcm_permute(ctx, Am, pm.data(), &bw_mod, nullptr);
        if (st == SS_OK) st = rcm_permute(ctx, As, ps.data(), &bw_shift, nullptr);
        if (st == SS_OK) {
            power = (double)bw_mod > 1.5 * (double)bw_shift;
            A = power ? As : Am;
            ss_mat_free(power ? Am : As);
            if (power) w_used = 0.0;
            perm.swap(power ? ps : pm);
            have_perm = opt.use_rcm != 0;
        } else {
            ss_mat_free(Am);
            ss_mat_free(As);
        }
    } else if (power) {
        st = add_shift(ctx, L, opt.sigma, &A);
    } else {
        st = add_trace_row(ctx, L, opt.w, &A, &w_used);
    }
    ss_mat_free(L);
    if (st != SS_OK) return st;

    if (!have_perm) {
        if (opt.use_rcm) st = rcm_permute(ctx, A, perm.data(), nullptr, nullptr);
        else for (int64_t i = 0; i < n; ++i) perm[i] = (int32_t)i;
    }
    if (st == SS_OK) st = permute(ctx, A, perm.data(), &Ap);
    ss_mat_free(A);
    if (st != SS_OK) return st;

    ss_info inf{};
    inf.method = automatic ? (power ? SS_METHOD_INVERSE_POWER : SS_METHOD_ITER_GMRES) : opt.method;
    inf.bw_modified = bw_mod;
    inf.bw_shifted = bw_shift;
    const int kaug = krylov == SS_KRYLOV_GMRES ? opt.lgmres_k : 0;
    inf.n = n;
    inf.nnz = Ap->m.nnz;
    inf.w_used = w_used;
    bandwidth_profile_impl(ctx, Ap->m, &inf.bandwidth, &inf.profile);
    if (direct) return steady_state_direct(ctx, Ap, perm, d, w_used, opt, t0, inf, rho_out, rho_on_device, info);
    st = build_prec(ctx, Ap->m, opt.precond, opt.drop_tol, opt.fill_factor, mixed, &M);
    if (st == SS_OK && mixed) st = ensure_f32(ctx, Ap);
    if (st == SS_OK) st = csr_split(ctx, Ap->m);
    if (st != SS_OK) { ss_mat_free(Ap); return st; }
    inf.nnz_factors = M->f.nnz;
    inf.levels_lower = M->lower.n_levels;
    inf.levels_upper = M->upper.n_levels;

    // device buffers: perm, trace index, b, x, y, rho, scratch
    std::vector<int32_t> iperm(n), tidx(d);
    for (int64_t r = 0; r < n; ++r) iperm[perm[r]] = (int32_t)r;
    for (int64_t i = 0; i < d; ++i) tidx[i] = iperm[i * (d + 1)];
    int32_t *perm_d = nullptr, *tidx_d = nullptr;
    double2 *b = nullptr, *x = nullptr, *y = nullptr, *rho = nullptr, *trace_d = nullptr;
    double* scr = nullptr;
    KrylovWork kw;
    auto cleanup = [&]() {
        dev_free(ctx, perm_d); dev_free(ctx, tidx_d); dev_free(ctx, b); dev_free(ctx, x); dev_free(ctx, y);
        dev_free(ctx, rho); dev_free(ctx, trace_d); dev_free(ctx, scr);
        krylov_workspace_free(ctx, kw);
        if (M) { prec_destroy(ctx, M); delete M; }
        ss_mat_free(Ap);
    };
#define STEP(call) do { st = (call); if (st != SS_OK) { cleanup(); return st; } } while (0)
    STEP(dev_alloc_n(ctx, &perm_d, (size_t)n));
    STEP(dev_alloc_n(ctx, &tidx_d, (size_t)d));
    STEP(dev_alloc_n(ctx, &b, (size_t)n));
    STEP(dev_alloc_n(ctx, &x, (size_t)n));
    STEP(dev_alloc_n(ctx, &y, (size_t)n));
    STEP(dev_alloc_n(ctx, &rho, (size_t)n));
    STEP(dev_alloc_n(ctx, &trace_d, 1));
    STEP(dev_alloc_n(ctx, &scr, (size_t)su_scratch_doubles()));
    SS_CUDA(ctx, cudaMemcpyAsync(perm_d, perm.data(), sizeof(int32_t) * n, cudaMemcpyHostToDevice, ctx->stream));
    SS_CUDA(ctx, cudaMemcpyAsync(tidx_d, tidx.data(), sizeof(int32_t) * d, cudaMemcpyHostToDevice, ctx->stream));
    STEP(su_condest(ctx, M, n, y, x, scr, &inf.condest));
    STEP(krylov_workspace(ctx, kw, n, krylov, krylov == SS_KRYLOV_GMRES ? opt.restart : 0, kaug));
    // warm start: the caller's guess (natural order, in rho_out) arrives in `rho`
    if (opt.warm_start)
        SS_CUDA(ctx, cudaMemcpyAsync(rho, rho_out, sizeof(double2) * n,
                                     rho_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, ctx->stream));
    auto initial = [&](double2* v) {
        return opt.warm_start ? su_warm_start(ctx, n, d, perm_d, rho, trace_d, v) : su_zero(ctx, n, v);
    };
    const double t1 = now_ms();

    double lr = INFINITY;
    int status = SS_NOT_CONVERGED, total = 0, outer = 0;
    bool fp64_fallback = false;
    const int64_t r0 = iperm[0];
    KrylovResultHost res;
    // FP64 BiCGSTAB/GMRES from the current x on the trace-row system until
    // ||L rho|| <= tol or the iteration budget is spent
    auto fp64_passes = [&]() -> ss_status {
        double inner = 0.5 * opt.tol;
        for (int pass = 0; pass < 8; ++pass) {
            int left = opt.maxiter - total;
            if (krylov == SS_KRYLOV_GMRES)
                SS_TRY(gmres_dev(ctx, Ap->m, M, kw, b, x, inner, left, opt.restart, &res, nullptr, kaug));
            else
                SS_TRY(bicgstab_dev(ctx, Ap->m, M, kw, b, x, inner, left, &res));
            total += res.iters;
            SS_TRY(su_lrho(ctx, Ap->m, x, 0, w_used, r0, d, tidx_d, y, scr, trace_d, &lr, nullptr));
            if (lr <= opt.tol) { status = SS_OK; break; }
            if (total >= opt.maxiter || res.status == SS_NOT_CONVERGED || (res.status == SS_BREAKDOWN && res.iters == 0)) {
                status = res.status == SS_OK ? SS_NOT_CONVERGED : res.status;
                break;
            }
            if (res.status == SS_OK) inner *= 0.1;
            // a breakdown after progress restarts from x with a fresh shadow residual
        }
        return SS_OK;
    };
    if (mixed) {
        // FP32 inner BiCGSTAB on r / ||r||, refined in FP64: x += ||r|| c
        STEP(su_zero(ctx, n, b));
        double2 wb = make_double2(w_used, 0.0);
        SS_CUDA(ctx, cudaMemcpyAsync(b + r0, &wb, sizeof(double2), cudaMemcpyHostToDevice, ctx->stream));
        STEP(initial(x));
        double2* r64 = nullptr;
        float2 *b32 = nullptr, *x32 = nullptr;
        STEP(dev_alloc_n(ctx, &r64, (size_t)n));
        STEP(dev_alloc_n(ctx, &b32, (size_t)n));
        STEP(dev_alloc_n(ctx, &x32, (size_t)n));
        for (outer = 1; outer <= 30; ++outer) {
            if (outer > 1) {
                STEP(su_lrho(ctx, Ap->m, x, 0, w_used, r0, d, tidx_d, y, scr, trace_d, &lr, nullptr));
                if (lr <= opt.tol) { status = SS_OK; break; }
            }
            if (total >= opt.maxiter) break;
            double rn = 0.0;
            STEP(su_refine_residual(ctx, Ap->m, b, x, y, r64, b32, x32, scr, &rn));
            if (rn == 0.0) { status = SS_OK; lr = 0.0; break; }
            // a stalled FP32 inner solve returns after a bounded number of iterations
            const int cap = std::min(opt.maxiter - total, std::max(50, opt.maxiter / 5));
            STEP(bicgstab_dev32(ctx, Ap->m, Ap->val32, M, kw, b32, x32, opt.inner_rtol > 0 ? opt.inner_rtol : 1e-5,
                                cap, &res));
            total += res.iters;
            STEP(su_refine_update(ctx, n, x, scr, x32));
            if (res.status == SS_BREAKDOWN && res.iters == 0) { status = SS_BREAKDOWN; break; }
            // an FP32 inner solve that cannot reach its tolerance within its cap
            // has met the limit of FP32 for this system: the remaining
            // iterations run in FP64 from the refined x
            if (res.status == SS_NOT_CONVERGED && total < opt.maxiter) {
                fp64_fallback = true;
                break;
            }
        }
        if (outer > 30) outer = 30;
        dev_free(ctx, r64);
        dev_free(ctx, b32);
        dev_free(ctx, x32);
        if (fp64_fallback) {
            STEP(su_lrho(ctx, Ap->m, x, 0, w_used, r0, d, tidx_d, y, scr, trace_d, &lr, nullptr));
            if (lr <= opt.tol) status = SS_OK;
            else STEP(fp64_passes());
        }
    } else if (!power) {
        STEP(su_zero(ctx, n, b));
        double2 wb = make_double2(w_used, 0.0);
        SS_CUDA(ctx, cudaMemcpyAsync(b + r0, &wb, sizeof(double2), cudaMemcpyHostToDevice, ctx->stream));
        STEP(initial(x));
        outer = 1;
        STEP(fp64_passes());
    } else {
        // x_0 random (SplitMix64 counters), ||x_0|| = 1; b holds x_k, x holds v
        if (opt.warm_start) STEP(initial(b));
        else STEP(su_start_vector(ctx, n, opt.seed, perm_d, b));
        STEP(su_normalise(ctx, n, b, scr));
        double2* oc_y = nullptr;
        double* oc_scr = nullptr;
        STEP(dev_alloc_n(ctx, &oc_y, (size_t)n));
        STEP(dev_alloc_n(ctx, &oc_scr, (size_t)su_scratch_doubles()));
        OuterCheck oc;
        oc.A = &Ap->m;
        oc.sigma = opt.sigma;
        oc.d = d;
        oc.tidx = tidx_d;
        oc.y = oc_y;
        oc.scratch = oc_scr;
        oc.trace = trace_d;
        oc.tol = 0.1 * opt.tol;
        for (outer = 1; outer <= 100; ++outer) {
            if (outer > 1) std::swap(b, x);        // b <- the latest normalised iterate
            STEP(su_zero(ctx, n, x));
            if (krylov == SS_KRYLOV_GMRES)
                STEP(gmres_dev(ctx, Ap->m, M, kw, b, x, 0.1 * opt.tol, opt.maxiter, opt.restart, &res, &oc, kaug));
            else
                STEP(bicgstab_dev(ctx, Ap->m, M, kw, b, x, 0.1 * opt.tol, opt.maxiter, &res, &oc));
            total += res.iters;
            STEP(su_normalise(ctx, n, x, scr));
            STEP(su_lrho(ctx, Ap->m, x, 1, opt.sigma, r0, d, tidx_d, y, scr, trace_d, &lr, nullptr));
            if (lr <= opt.tol) { status = SS_OK; break; }
        }
        if (outer > 100) outer = 100;
        dev_free(ctx, oc_y);
        dev_free(ctx, oc_scr);
    }
    // rho = unpermute(x) / tr(x)
    STEP(su_trace(ctx, d, tidx_d, x, trace_d));
    STEP(su_finalise(ctx, n, perm_d, x, trace_d, rho));
    SS_CUDA(ctx, cudaMemcpyAsync(rho_out, rho, sizeof(double2) * n,
                                 rho_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, ctx->stream));
    SS_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    const double t2 = now_ms();
    inf.status = status;
    inf.iters = total;
    inf.outer_iters = outer;
    inf.fp64_fallback = fp64_fallback ? 1 : 0;
    inf.resid_Lrho = lr;
    inf.ms_setup = t1 - t0;
    inf.ms_solve = t2 - t1;
    if (info) *info = inf;
    cleanup();
#undef STEP
    if (status != SS_OK)
        ctx->last_error = status == SS_BREAKDOWN ? "BiCGSTAB breakdown" : "not converged within maxiter";
    return (ss_status)status;
}
