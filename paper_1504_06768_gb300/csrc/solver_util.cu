// Small vector kernels of the steady-state driver: right-hand side, start
// vector, trace, the FP64 acceptance residual ||L rho||_2, and the final
// unpermute + trace normalisation (column-major rho, Eq. eigval).
#include "common.cuh"
#include "solver_util.cuh"
#include "spmv.cuh"

namespace {

inline unsigned grid_for(int64_t n, int b) { return (unsigned)((n + b - 1) / b); }

__global__ void fill_zero(int64_t n, double2* __restrict__ v) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        v[i] = make_double2(0.0, 0.0);
}

__global__ void fill_ones(int64_t n, double2* __restrict__ v) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        v[i] = make_double2(1.0, 0.0);
}

// SplitMix64 (Steele, Lea and Flood, OOPSLA 2014) at counter c + 1.
__device__ __forceinline__ unsigned long long splitmix64_at(unsigned long long seed, unsigned long long c) {
    unsigned long long z = seed + (c + 1ull) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// Element k of the natural-order start vector goes to permuted position iperm[k].
__global__ void start_vec(int64_t n, unsigned long long seed, const int32_t* __restrict__ perm,
                          double2* __restrict__ x) {
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x) {
        unsigned long long k = (unsigned long long)perm[r];
        double re = 2.0 * ((double)(splitmix64_at(seed, 2 * k) >> 11) * 0x1.0p-53) - 1.0;
        double im = 2.0 * ((double)(splitmix64_at(seed, 2 * k + 1) >> 11) * 0x1.0p-53) - 1.0;
        x[r] = make_double2(re, im);
    }
}

__global__ void norm2_partial(int64_t n, const double2* __restrict__ x, double* __restrict__ part) {
    __shared__ double sh[256];
    double s = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        s += cabs2(x[i]);
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
}

// part[b] = sum |y_r + corr_r|^2 with corr = sigma x_r (shift) or -w tr(x) at r0 (trace row)
__global__ void lrho_partial(int64_t n, const double2* __restrict__ y, const double2* __restrict__ x, int mode,
                             double w_or_sigma, int64_t r0, const double2* __restrict__ trace,
                             double* __restrict__ part) {
    __shared__ double sh[256];
    double s = 0.0;
    const double2 tr = *trace;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        double2 v = y[i];
        if (mode == 1) {
            v.x += w_or_sigma * x[i].x;
            v.y += w_or_sigma * x[i].y;
        } else if (i == r0) {
            v.x -= w_or_sigma * tr.x;
            v.y -= w_or_sigma * tr.y;
        }
        s += cabs2(v);
    }
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
}

__global__ void sum_part(const double* __restrict__ part, int np, double* __restrict__ out) {
    __shared__ double sh[256];
    double s = 0.0;
    for (int t = threadIdx.x; t < np; t += blockDim.x) s += part[t];
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = sh[0];
}

// tr(x) = sum_i x[tidx[i]] (one block, fixed order)
__global__ void trace_kernel(int64_t d, const int32_t* __restrict__ tidx, const double2* __restrict__ x,
                             double2* __restrict__ out) {
    __shared__ double2 sh[256];
    double2 s = make_double2(0.0, 0.0);
    for (int64_t i = threadIdx.x; i < d; i += blockDim.x) s = cadd(s, x[tidx[i]]);
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) sh[threadIdx.x] = cadd(sh[threadIdx.x], sh[threadIdx.x + o]);
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = sh[0];
}

__global__ void scale_by(int64_t n, double2* __restrict__ x, const double* __restrict__ nrm2) {
    const double inv = 1.0 / sqrt(*nrm2);
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        x[i] = cscale(x[i], inv);
}

// rho[perm[r]] = x[r] / tr   (natural column-major order)
__global__ void unpermute_normalise(int64_t n, const int32_t* __restrict__ perm, const double2* __restrict__ x,
                                    const double2* __restrict__ trace, double2* __restrict__ rho) {
    const double2 tr = *trace;
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x)
        rho[perm[r]] = cdiv(x[r], tr);
}

// tr(rho) of a natural-order column-major rho (one block, fixed order)
__global__ void natural_trace(int64_t d, const double2* __restrict__ rho, double2* __restrict__ out) {
    __shared__ double2 sh[256];
    double2 s = make_double2(0.0, 0.0);
    for (int64_t i = threadIdx.x; i < d; i += blockDim.x) s = cadd(s, rho[i * (d + 1)]);
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) sh[threadIdx.x] = cadd(sh[threadIdx.x], sh[threadIdx.x + o]);
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = sh[0];
}

// x[r] = rho[perm[r]] / tr (the warm start), or 0 when tr = 0
__global__ void permute_scaled(int64_t n, const int32_t* __restrict__ perm, const double2* __restrict__ rho,
                               const double2* __restrict__ trace, double2* __restrict__ x) {
    const double2 tr = *trace;
    const bool use = tr.x != 0.0 || tr.y != 0.0;
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x)
        x[r] = use ? cdiv(rho[perm[r]], tr) : make_double2(0.0, 0.0);
}

__global__ void max_abs_partial(int64_t n, const double2* __restrict__ x, double* __restrict__ part) {
    __shared__ double sh[256];
    double s = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        s = fmax(s, hypot(x[i].x, x[i].y));
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) sh[threadIdx.x] = fmax(sh[threadIdx.x], sh[threadIdx.x + o]);
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
}

__global__ void max_part(const double* __restrict__ part, int np, double* __restrict__ out) {
    double s = 0.0;
    for (int t = 0; t < np; ++t) s = fmax(s, part[t]);
    *out = s;
}

constexpr int NB = 256;

// r = b - y and partial ||r||^2 per block
__global__ void resid_partial(int64_t n, const double2* __restrict__ b, const double2* __restrict__ y,
                              double2* __restrict__ r, double* __restrict__ part) {
    __shared__ double sh[256];
    double s = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        double2 v = csub(b[i], y[i]);
        r[i] = v;
        s += cabs2(v);
    }
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
}

// b32 = r / ||r|| (FP32), x32 = 0
__global__ void scale_to32(int64_t n, const double2* __restrict__ r, const double* __restrict__ nrm2,
                           float2* __restrict__ b32, float2* __restrict__ x32) {
    const double inv = 1.0 / sqrt(*nrm2);
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        b32[i] = make_float2((float)(r[i].x * inv), (float)(r[i].y * inv));
        x32[i] = make_float2(0.f, 0.f);
    }
}

// x += ||r|| c (c in FP32)
__global__ void axpy_from32(int64_t n, double2* __restrict__ x, const double* __restrict__ nrm2,
                            const float2* __restrict__ c) {
    const double a = sqrt(*nrm2);
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        x[i].x += a * (double)c[i].x;
        x[i].y += a * (double)c[i].y;
    }
}

}  // namespace

// r = b - A x (FP64), b32 = r / ||r||, x32 = 0; ||r|| to the host and kept in scratch[NB]
ss_status su_refine_residual(ss_ctx ctx, const DeviceCSR& A, const double2* b, const double2* x, double2* y,
                             double2* r, float2* b32, float2* x32, double* scratch, double* rnorm) {
    { ProfScope ps_(ctx, PROF_SPMV); spmv_launch(A, x, y, nullptr, ctx->stream); }
    resid_partial<<<(ss_count_launch(), NB), 256, 0, ctx->stream>>>(A.n_rows, b, y, r, scratch);
    sum_part<<<(ss_count_launch(), 1), 256, 0, ctx->stream>>>(scratch, NB, scratch + NB);
    double h = 0.0;
    SS_CUDA(ctx, cudaMemcpyAsync(&h, scratch + NB, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    SS_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    *rnorm = sqrt(h);
    if (h > 0.0) scale_to32<<<(ss_count_launch(), 1024), 256, 0, ctx->stream>>>(A.n_rows, r, scratch + NB, b32, x32);
    SS_CUDA(ctx, cudaGetLastError());
    return SS_OK;
}

ss_status su_refine_update(ss_ctx ctx, int64_t n, double2* x, const double* scratch, const float2* c) {
    axpy_from32<<<(ss_count_launch(), 1024), 256, 0, ctx->stream>>>(n, x, scratch + NB, c);
    SS_CUDA(ctx, cudaGetLastError());
    return SS_OK;
}

ss_status su_zero(ss_ctx ctx, int64_t n, double2* v) {
    fill_zero<<<(ss_count_launch(), grid_for(n, 256) > 1024 ? 1024 : grid_for(n, 256)), 256, 0, ctx->stream>>>(n, v);
    SS_CUDA(ctx, cudaGetLastError());
    return SS_OK;
}

ss_status su_start_vector(ss_ctx ctx, int64_t n, uint64_t seed, const int32_t* perm_dev, double2* x) {
    start_vec<<<(ss_count_launch(), 1024), 256, 0, ctx->stream>>>(n, seed, perm_dev, x);
    SS_CUDA(ctx, cudaGetLastError());
    return SS_OK;
}

ss_status su_normalise(ss_ctx ctx, int64_t n, double2* x, double* scratch /* NB + 1 */) {
    norm2_partial<<<(ss_count_launch(), NB), 256, 0, ctx->stream>>>(n, x, scratch);
    sum_part<<<(ss_count_launch(), 1), 256, 0, ctx->stream>>>(scratch, NB, scratch + NB);
    scale_by<<<(ss_count_launch(), 1024), 256, 0, ctx->stream>>>(n, x, scratch + NB);
    SS_CUDA(ctx, cudaGetLastError());
    return SS_OK;
}

ss_status su_trace(ss_ctx ctx, int64_t d, const int32_t* tidx, const double2* x, double2* out) {
    trace_kernel<<<(ss_count_launch(), 1), 256, 0, ctx->stream>>>(d, tidx, x, out);
    SS_CUDA(ctx, cudaGetLastError());
    return SS_OK;
}

// ||L rho||_2 for rho = x / tr(x).  mode 0: A = L + w T (row r0 carries T);
// mode 1: A = L - sigma I.  y is scratch (n).  Result on the host.
ss_status su_lrho(ss_ctx ctx, const DeviceCSR& A, const double2* x, int mode, double w_or_sigma, int64_t r0,
                  int64_t d, const int32_t* tidx, double2* y, double* scratch /* NB + 1 */, double2* trace_dev,
                  double* out, double2* trace_host) {
    { ProfScope ps_(ctx, PROF_SPMV); spmv_launch(A, x, y, nullptr, ctx->stream); }
    trace_kernel<<<(ss_count_launch(), 1), 256, 0, ctx->stream>>>(d, tidx, x, trace_dev);
    lrho_partial<<<(ss_count_launch(), NB), 256, 0, ctx->stream>>>(A.n_rows, y, x, mode, w_or_sigma, r0, trace_dev, scratch);
    sum_part<<<(ss_count_launch(), 1), 256, 0, ctx->stream>>>(scratch, NB, scratch + NB);
    double h = 0.0;
    double2 tr;
    SS_CUDA(ctx, cudaMemcpyAsync(&h, scratch + NB, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    SS_CUDA(ctx, cudaMemcpyAsync(&tr, trace_dev, sizeof(double2), cudaMemcpyDeviceToHost, ctx->stream));
    SS_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    double trm = hypot(tr.x, tr.y);
    *out = trm > 0.0 ? sqrt(h) / trm : INFINITY;
    if (trace_host) *trace_host = tr;
    return SS_OK;
}

ss_status su_warm_start(ss_ctx ctx, int64_t n, int64_t d, const int32_t* perm_dev, const double2* rho_dev,
                        double2* trace_dev, double2* x) {
    natural_trace<<<(ss_count_launch(), 1), 256, 0, ctx->stream>>>(d, rho_dev, trace_dev);
    permute_scaled<<<(ss_count_launch(), 1024), 256, 0, ctx->stream>>>(n, perm_dev, rho_dev, trace_dev, x);
    SS_CUDA(ctx, cudaGetLastError());
    return SS_OK;
}

ss_status su_finalise(ss_ctx ctx, int64_t n, const int32_t* perm_dev, const double2* x, const double2* trace_dev,
                      double2* rho_dev) {
    unpermute_normalise<<<(ss_count_launch(), 1024), 256, 0, ctx->stream>>>(n, perm_dev, x, trace_dev, rho_dev);
    SS_CUDA(ctx, cudaGetLastError());
    return SS_OK;
}

ss_status su_condest(ss_ctx ctx, ss_prec M, int64_t n, double2* ones, double2* z, double* scratch, double* out) {
    fill_ones<<<(ss_count_launch(), 1024), 256, 0, ctx->stream>>>(n, ones);
    SS_TRY(prec_apply_dev(ctx, M, ones, z));
    max_abs_partial<<<(ss_count_launch(), NB), 256, 0, ctx->stream>>>(n, z, scratch);
    max_part<<<(ss_count_launch(), 1), 1, 0, ctx->stream>>>(scratch, NB, scratch + NB);
    SS_CUDA(ctx, cudaMemcpyAsync(out, scratch + NB, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    SS_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    SS_TRY(prec_check_error(ctx, M));
    return SS_OK;
}

int su_scratch_doubles() { return NB + 8; }
