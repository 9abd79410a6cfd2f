// Right-preconditioned Krylov solvers on the device (section "Iterative
// solvers"): BiCGSTAB (van der Vorst 1992) and restarted GMRES(m) (Saad and
// Schultz 1986), solving A M^{-1} u = b, x = M^{-1} u, so that the updated
// residual is the residual of A x = b itself.  GMRES optionally augments each
// cycle with the corrections of the k previous cycles (LGMRES(m, k), Baker,
// Jessup and Manteuffel 2005).
//
// All scalars live in device memory (KrylovState) and every reduction is a
// deterministic two-stage sum: each block writes its partial sums, the last
// block to finish adds the partials in block order and applies the scalar
// update of the algorithm.  A `halt` word lets the host queue several
// iterations ahead; once a solve has converged or broken down, the queued
// kernels return immediately.  Inner products are <a, b> = sum conj(a_i) b_i.
#include <cmath>
#include <vector>

#include "common.cuh"
#include "krylov.cuh"
#include "solver_util.cuh"
#include "spmv.cuh"

namespace {

constexpr int RED_THREADS = 256;

inline unsigned grid_for(int64_t n, int b) { return (unsigned)((n + b - 1) / b); }

__host__ __device__ inline int red_blocks(int64_t n) {
    int64_t b = (n + 2047) / 2048;
    if (b < 1) b = 1;
    if (b > 512) b = 512;
    return (int)b;
}

__device__ __forceinline__ double2 d2(double a, double b) { return make_double2(a, b); }

// Block-wide sum of NV complex values in fixed order; result in thread 0.
template <int NV>
__device__ void block_sum(double2 (&v)[NV], double2* sh /* [NV][32] */) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < NV; ++k) {
        for (int o = 16; o > 0; o >>= 1) {
            v[k].x += __shfl_down_sync(0xffffffffu, v[k].x, o);
            v[k].y += __shfl_down_sync(0xffffffffu, v[k].y, o);
        }
        if (lane == 0) sh[k * 32 + wid] = v[k];
    }
    __syncthreads();
    if (wid == 0) {
        const int nw = blockDim.x >> 5;
#pragma unroll
        for (int k = 0; k < NV; ++k) {
            double2 t = lane < nw ? sh[k * 32 + lane] : d2(0, 0);
            for (int o = 16; o > 0; o >>= 1) {
                t.x += __shfl_down_sync(0xffffffffu, t.x, o);
                t.y += __shfl_down_sync(0xffffffffu, t.y, o);
            }
            v[k] = t;
        }
    }
    __syncthreads();
}

// Writes this block's partials; returns true in thread 0 of the last block,
// with the totals in v.
template <int NV>
__device__ bool reduce_last_block(double2 (&v)[NV], double2* partials, unsigned* counter) {
    __shared__ double2 sh[NV * 32];
    __shared__ bool last;
    block_sum<NV>(v, sh);
    if (threadIdx.x == 0) {
#pragma unroll
        for (int k = 0; k < NV; ++k) partials[blockIdx.x * NV + k] = v[k];
        __threadfence();
        unsigned t = atomicAdd(counter, 1u);
        last = (t == gridDim.x - 1);
    }
    __syncthreads();
    if (!last) return false;
    __threadfence();
    double2 acc[NV];
#pragma unroll
    for (int k = 0; k < NV; ++k) acc[k] = d2(0, 0);
    for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x)
#pragma unroll
        for (int k = 0; k < NV; ++k) {
            double2 p = __ldcg(&partials[b * NV + k]);
            acc[k].x += p.x;
            acc[k].y += p.y;
        }
    block_sum<NV>(acc, sh);
    if (threadIdx.x == 0) {
#pragma unroll
        for (int k = 0; k < NV; ++k) v[k] = acc[k];
        *counter = 0u;
        return true;
    }
    return false;
}

__device__ __forceinline__ bool negligible(double2 a, double nu, double nv) {
    double m = hypot(a.x, a.y);
    return m == 0.0 || m < 1e-15 * nu * nv;
}

// ----------------------------------------------------------- BiCGSTAB
// Vector type T is double2 (FP64) or float2 (the inner solve of the mixed
// path); updates run in T's precision, inner products accumulate in FP64.

__device__ __forceinline__ double2 dd(double2 a) { return a; }
__device__ __forceinline__ double2 dd(float2 a) { return make_double2(a.x, a.y); }
template <class T> __device__ __forceinline__ T tt(double2 a);
template <> __device__ __forceinline__ double2 tt<double2>(double2 a) { return a; }
template <> __device__ __forceinline__ float2 tt<float2>(double2 a) { return make_float2((float)a.x, (float)a.y); }
__device__ __forceinline__ double2 tmul(double2 a, double2 b) { return cmul(a, b); }
__device__ __forceinline__ float2 tmul(float2 a, float2 b) { return fcmul(a, b); }
__device__ __forceinline__ double2 tadd(double2 a, double2 b) { return cadd(a, b); }
__device__ __forceinline__ float2 tadd(float2 a, float2 b) { return fcadd(a, b); }
__device__ __forceinline__ double2 tsub(double2 a, double2 b) { return csub(a, b); }
__device__ __forceinline__ float2 tsub(float2 a, float2 b) { return fcsub(a, b); }

// r = b - y (y = A x), rhat = r, rho = <r, r>
template <class T>
__global__ void bicg_init(int64_t n, const T* __restrict__ b, const T* __restrict__ y,
                          T* __restrict__ r, T* __restrict__ rhat, KrylovState* st) {
    double2 v[1] = {d2(0, 0)};
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        T ri = tsub(b[i], y[i]);
        r[i] = ri;
        rhat[i] = ri;
        v[0].x += cabs2(dd(ri));
    }
    if (reduce_last_block<1>(v, st->partials, &st->counter)) {
        double rn = sqrt(v[0].x);
        st->rnorm = rn;
        st->rhat_norm = rn;
        st->rho = d2(v[0].x, 0.0);
        st->iters = 0;
        st->sconv = 0;
        if (rn <= st->tol) { st->status = SS_OK; st->done = 1; st->halt = 1; }
        else if (st->maxiter <= 0) { st->status = SS_NOT_CONVERGED; st->done = 1; st->halt = 1; }
        else { st->status = SS_NOT_CONVERGED; st->done = 0; st->halt = 0; }
    }
}

// p = r (first iteration) or p = r + beta (p - omega v)
template <class T>
__global__ void bicg_p(int64_t n, const T* __restrict__ r, const T* __restrict__ v, T* __restrict__ p,
                       const KrylovState* st) {
    if (st->halt) return;
    const bool first = st->iters == 0;
    const T beta = tt<T>(st->beta), omega = tt<T>(st->omega);
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        if (first) p[i] = r[i];
        else p[i] = tadd(r[i], tmul(beta, tsub(p[i], tmul(omega, v[i]))));
    }
}

// alpha = rho / <rhat, v>
template <class T>
__global__ void bicg_rv(int64_t n, const T* __restrict__ rhat, const T* __restrict__ v, KrylovState* st) {
    if (st->halt) return;
    double2 acc[2] = {d2(0, 0), d2(0, 0)};
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double2 h = dd(rhat[i]), vi = dd(v[i]);
        double2 a = cmulc(h, vi);
        acc[0].x += a.x;
        acc[0].y += a.y;
        acc[1].x += cabs2(vi);
    }
    if (reduce_last_block<2>(acc, st->partials, &st->counter)) {
        if (negligible(acc[0], st->rhat_norm, sqrt(acc[1].x))) {
            st->status = SS_BREAKDOWN; st->done = 1; st->halt = 1;
        } else {
            st->alpha = cdiv(st->rho, acc[0]);
        }
    }
}

// s = r - alpha v; stop early when ||s|| <= tol
template <class T>
__global__ void bicg_s(int64_t n, const T* __restrict__ r, const T* __restrict__ v, T* __restrict__ s,
                       KrylovState* st) {
    if (st->halt) return;
    const T alpha = tt<T>(st->alpha);
    double2 acc[1] = {d2(0, 0)};
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        T si = tsub(r[i], tmul(alpha, v[i]));
        s[i] = si;
        acc[0].x += cabs2(dd(si));
    }
    if (reduce_last_block<1>(acc, st->partials, &st->counter)) {
        double sn = sqrt(acc[0].x);
        st->snorm = sn;
        if (sn <= st->tol) { st->sconv = 1; st->halt = 1; }
    }
}

// omega = <t, s> / <t, t>
template <class T>
__global__ void bicg_ts(int64_t n, const T* __restrict__ t, const T* __restrict__ s, KrylovState* st) {
    if (st->halt) return;
    double2 acc[2] = {d2(0, 0), d2(0, 0)};
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double2 ti = dd(t[i]);
        double2 a = cmulc(ti, dd(s[i]));
        acc[0].x += a.x;
        acc[0].y += a.y;
        acc[1].x += cabs2(ti);
    }
    if (reduce_last_block<2>(acc, st->partials, &st->counter)) {
        if (acc[1].x == 0.0) {
            st->iters += 1;
            st->status = SS_BREAKDOWN; st->done = 1; st->halt = 1;
        } else {
            st->omega = cscale(acc[0], 1.0 / acc[1].x);
        }
    }
}

// x += alpha phat + omega shat; r = s - omega t; rho_new = <rhat, r>
template <class T>
__global__ void bicg_xr(int64_t n, T* __restrict__ x, const T* __restrict__ phat,
                        const T* __restrict__ shat, const T* __restrict__ s, const T* __restrict__ t,
                        T* __restrict__ r, const T* __restrict__ rhat, KrylovState* st) {
    if (st->done) return;
    const double2 alpha = st->alpha, omega = st->omega;
    const T al = tt<T>(alpha), om = tt<T>(omega);
    const bool sconv = st->sconv;
    double2 acc[2] = {d2(0, 0), d2(0, 0)};
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        if (sconv) {
            x[i] = tadd(x[i], tmul(al, phat[i]));
            r[i] = s[i];
        } else {
            x[i] = tadd(x[i], tadd(tmul(al, phat[i]), tmul(om, shat[i])));
            T ri = tsub(s[i], tmul(om, t[i]));
            r[i] = ri;
            const double2 rd = dd(ri);
            double2 a = cmulc(dd(rhat[i]), rd);
            acc[0].x += a.x;
            acc[0].y += a.y;
            acc[1].x += cabs2(rd);
        }
    }
    if (reduce_last_block<2>(acc, st->partials, &st->counter)) {
        st->iters += 1;
        if (sconv) {
            st->rnorm = st->snorm;
            st->status = SS_OK; st->done = 1; st->halt = 1;
            return;
        }
        double rn = sqrt(acc[1].x);
        st->rnorm = rn;
        if (rn <= st->tol) { st->status = SS_OK; st->done = 1; st->halt = 1; return; }
        if (omega.x == 0.0 && omega.y == 0.0) { st->status = SS_BREAKDOWN; st->done = 1; st->halt = 1; return; }
        if (st->iters >= st->maxiter) { st->status = SS_NOT_CONVERGED; st->done = 1; st->halt = 1; return; }
        if (negligible(acc[0], st->rhat_norm, rn)) { st->status = SS_BREAKDOWN; st->done = 1; st->halt = 1; return; }
        st->beta = cmul(cdiv(acc[0], st->rho), cdiv(alpha, omega));
        st->rho = acc[0];
    }
}

// --------------------------------------------------------------- GMRES

// r = b - y; beta = ||r||; v0 = r / beta (second pass); g = beta e1
__global__ void gm_restart(int64_t n, const double2* __restrict__ b, const double2* __restrict__ y,
                           double2* __restrict__ r, KrylovState* st) {
    if (st->done) return;
    double2 acc[1] = {d2(0, 0)};
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        double2 ri = csub(b[i], y[i]);
        r[i] = ri;
        acc[0].x += cabs2(ri);
    }
    if (reduce_last_block<1>(acc, st->partials, &st->counter)) {
        double beta = sqrt(acc[0].x);
        st->rnorm = beta;
        st->k = 0;
        if (beta <= st->tol) { st->status = SS_OK; st->done = 1; st->halt = 1; return; }
        if (st->iters >= st->maxiter) { st->status = SS_NOT_CONVERGED; st->done = 1; st->halt = 1; return; }
        st->halt = 0;
        for (int j = 0; j <= st->m; ++j) st->g[j] = d2(0, 0);
        st->g[0] = d2(beta, 0.0);
        st->hnorm = beta;    // scale for v0
    }
}

// v = r / hnorm
__global__ void gm_scale(int64_t n, const double2* __restrict__ r, double2* __restrict__ v, const KrylovState* st) {
    if (st->halt) return;
    const double inv = 1.0 / st->hnorm;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        v[i] = cscale(r[i], inv);
}

// h_i = <V_i, w> for i <= j (NV at a time); pass 0 writes H[:, j], pass 1 adds
template <int NV>
__global__ void gm_dots(int64_t n, const double2* __restrict__ V, int64_t ldv, int j, int base,
                        const double2* __restrict__ w, KrylovState* st, int pass) {
    if (st->halt) return;
    double2 acc[NV];
#pragma unroll
    for (int k = 0; k < NV; ++k) acc[k] = d2(0, 0);
    const int cnt = min(NV, j + 1 - base);
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double2 wi = w[i];
#pragma unroll
        for (int k = 0; k < NV; ++k)
            if (k < cnt) {
                double2 a = cmulc(V[(int64_t)(base + k) * ldv + i], wi);
                acc[k].x += a.x;
                acc[k].y += a.y;
            }
    }
    if (reduce_last_block<NV>(acc, st->partials, &st->counter)) {
        for (int k = 0; k < cnt; ++k) {
            double2* h = &st->H[(base + k) * KRYLOV_MAX_M + j];
            if (pass == 0) *h = acc[k];
            else *h = cadd(*h, acc[k]);
            st->hwork[base + k] = acc[k];
        }
    }
}

// w -= sum_{i<=j} hwork_i V_i
__global__ void gm_orth_update(int64_t n, const double2* __restrict__ V, int64_t ldv, int j, double2* __restrict__ w,
                               const KrylovState* st) {
    if (st->halt) return;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        double2 wi = w[i];
        for (int k = 0; k <= j; ++k) wi = csub(wi, cmul(st->hwork[k], V[(int64_t)k * ldv + i]));
        w[i] = wi;
    }
}

// H[j+1, j] = ||w||; Givens rotations; residual estimate; end of cycle -> y.
// mt = the cycle's dimension (restart length + augmentation vectors in use).
__global__ void gm_norm(int64_t n, const double2* __restrict__ w, int j, int mt, KrylovState* st) {
    if (st->halt) return;
    double2 acc[1] = {d2(0, 0)};
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        acc[0].x += cabs2(w[i]);
    if (!reduce_last_block<1>(acc, st->partials, &st->counter)) return;
    const int M = KRYLOV_MAX_M;
    double hn = sqrt(acc[0].x);
    st->hnorm = hn;
    double2* H = st->H;
    H[(j + 1) * M + j] = d2(hn, 0.0);
    for (int i = 0; i < j; ++i) {            // previous rotations
        double2 a = H[i * M + j], b = H[(i + 1) * M + j];
        double c = st->cs[i];
        double2 s = st->sn[i];
        H[i * M + j] = cadd(cscale(a, c), cmul(s, b));
        H[(i + 1) * M + j] = csub(cscale(b, c), cmul(cconj(s), a));
    }
    double2 a = H[j * M + j], b = H[(j + 1) * M + j];
    double c;
    double2 s, rr;
    if (b.x == 0.0 && b.y == 0.0) { c = 1.0; s = d2(0, 0); rr = a; }
    else if (a.x == 0.0 && a.y == 0.0) { c = 0.0; s = d2(1, 0); rr = b; }
    else {
        double am = hypot(a.x, a.y), t = hypot(am, hypot(b.x, b.y));
        c = am / t;
        double2 ph = cscale(a, 1.0 / am);
        s = cscale(cmul(ph, cconj(b)), 1.0 / t);
        rr = cscale(ph, t);
    }
    st->cs[j] = c;
    st->sn[j] = s;
    H[j * M + j] = rr;
    H[(j + 1) * M + j] = d2(0, 0);
    double2 gj = st->g[j];
    st->g[j + 1] = cmul(d2(-s.x, s.y), gj);     // -conj(s) g_j
    st->g[j] = cscale(gj, c);
    st->k = j + 1;
    st->iters += 1;
    double res = hypot(st->g[j + 1].x, st->g[j + 1].y);
    st->rnorm = res;
    bool end = res <= st->tol || st->iters >= st->maxiter || j + 1 >= mt || (rr.x == 0.0 && rr.y == 0.0) || hn == 0.0;
    if (end) {
        const int k = j + 1;
        for (int i = k - 1; i >= 0; --i) {   // back substitution H y = g
            double2 acc2 = st->g[i];
            for (int l = i + 1; l < k; ++l) acc2 = csub(acc2, cmul(H[i * M + l], st->y[l]));
            st->y[i] = cdiv(acc2, H[i * M + i]);
        }
        st->halt = 1;
    }
}

// x += sum_{i<k} y_i Z_i
__global__ void gm_update_x(int64_t n, const double2* __restrict__ Z, int64_t ldz, double2* __restrict__ x,
                            const KrylovState* st) {
    if (st->done) return;
    const int k = st->k;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        double2 xi = x[i];
        for (int l = 0; l < k; ++l) xi = cadd(xi, cmul(st->y[l], Z[(int64_t)l * ldz + i]));
        x[i] = xi;
    }
}

// LGMRES end of cycle: dx = sum_{i<k} y_i Z_i, x += dx, dnorm = ||dx||
__global__ void lg_update_x(int64_t n, const double2* __restrict__ Z, int64_t ldz, double2* __restrict__ x,
                            double2* __restrict__ dx, KrylovState* st) {
    if (st->done) return;
    const int k = st->k;
    double2 acc[1] = {d2(0, 0)};
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        double2 di = d2(0, 0);
        for (int l = 0; l < k; ++l) di = cadd(di, cmul(st->y[l], Z[(int64_t)l * ldz + i]));
        dx[i] = di;
        x[i] = cadd(x[i], di);
        acc[0].x += cabs2(di);
    }
    if (reduce_last_block<1>(acc, st->partials, &st->counter)) st->dnorm = sqrt(acc[0].x);
}

// LGMRES: the normalised correction replaces the oldest stored one (slot)
__global__ void lg_store(int64_t n, const double2* __restrict__ dx, double2* __restrict__ slot, const KrylovState* st) {
    if (st->done || !(st->dnorm > 0.0)) return;
    const double inv = 1.0 / st->dnorm;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        slot[i] = cscale(dx[i], inv);
}


}  // namespace

// ------------------------------------------------------------------ host

ss_status krylov_workspace(ss_ctx ctx, KrylovWork& w, int64_t n, int method, int m, int kaug) {
    if (method == SS_KRYLOV_GMRES && (m < 1 || kaug < 0 || m + kaug > KRYLOV_MAX_M))
        return set_error(ctx, SS_ERR_INVALID, "GMRES needs restart >= 1, augmentation >= 0, restart + augmentation <= 64");
    w.n = n;
    w.method = method;
    w.m = m;
    w.kaug = method == SS_KRYLOV_GMRES ? kaug : 0;
    const int nb = red_blocks(n);
    SS_TRY(dev_alloc_n(ctx, &w.st, 1));
    SS_TRY(dev_alloc_n(ctx, &w.partials, (size_t)nb * 32));
    SS_CUDA(ctx, cudaMemsetAsync(w.st, 0, sizeof(KrylovState), ctx->stream));
    size_t nvec = method == SS_KRYLOV_GMRES ? (size_t)(2 * (m + kaug) + 1 + (kaug > 0 ? 1 : 0)) : 8;
    SS_TRY(dev_alloc_n(ctx, &w.vecs, nvec * (size_t)n));
    w.nvec = nvec;
    ss_count_alloc();
    SS_CUDA(ctx, cudaHostAlloc(reinterpret_cast<void**>(&w.host_st), sizeof(KrylovState), cudaHostAllocDefault));
    return SS_OK;
}

void krylov_workspace_free(ss_ctx ctx, KrylovWork& w) {
    dev_free(ctx, w.st);
    dev_free(ctx, w.partials);
    dev_free(ctx, w.vecs);
    if (w.host_st) cudaFreeHost(w.host_st);
    w = KrylovWork();
}

static ss_status read_state(ss_ctx ctx, KrylovWork& w) {
    SS_CUDA(ctx, cudaMemcpyAsync(w.host_st, w.st, sizeof(KrylovState), cudaMemcpyDeviceToHost, ctx->stream));
    SS_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    return SS_OK;
}

static ss_status set_params(ss_ctx ctx, KrylovWork& w, double tol, int maxiter, int m) {
    KrylovState h{};
    h.tol = tol;
    h.maxiter = maxiter;
    h.m = m;
    h.partials = w.partials;
    // only the parameter fields are written; the rest is zeroed
    SS_CUDA(ctx, cudaMemcpyAsync(w.st, &h, sizeof(KrylovState), cudaMemcpyHostToDevice, ctx->stream));
    return SS_OK;
}

static ss_status outer_met(ss_ctx ctx, const OuterCheck* oc, const double2* x, bool* met) {
    *met = false;
    if (!oc) return SS_OK;
    double lr = 0.0;
    SS_TRY(su_lrho(ctx, *oc->A, x, 1, oc->sigma, 0, oc->d, oc->tidx, oc->y, oc->scratch, oc->trace, &lr, nullptr));
    *met = lr <= oc->tol;
    return SS_OK;
}

template <class T>
static void spmv_any(ss_ctx ctx, const DeviceCSR& A, const float2* val32, const T* x, T* y, const int* halt);
template <>
void spmv_any<double2>(ss_ctx ctx, const DeviceCSR& A, const float2*, const double2* x, double2* y, const int* halt) {
    ProfScope ps_(ctx, PROF_SPMV);
    spmv_launch(A, x, y, halt, ctx->stream);
}
template <>
void spmv_any<float2>(ss_ctx ctx, const DeviceCSR& A, const float2* val32, const float2* x, float2* y, const int* halt) {
    ProfScope ps_(ctx, PROF_SPMV);
    spmv_launch32(A, val32, x, y, halt, ctx->stream);
}
static ss_status prec_any(ss_ctx ctx, ss_prec M, const double2* r, double2* z, const int* halt) {
    return prec_apply_dev(ctx, M, r, z, halt);
}
static ss_status prec_any(ss_ctx ctx, ss_prec M, const float2* r, float2* z, const int* halt) {
    return prec_apply_dev32(ctx, M, r, z, halt);
}

template <class T>
static ss_status bicgstab_any(ss_ctx ctx, const DeviceCSR& A, const float2* val32, ss_prec M, KrylovWork& w,
                              const T* b, T* x, double tol, int maxiter, KrylovResultHost* out,
                              const OuterCheck* oc) {
    const int64_t n = A.n_rows;
    T* r = reinterpret_cast<T*>(w.vecs);
    T* rhat = r + n;
    T* p = rhat + n;
    T* v = p + n;
    T* s = v + n;
    T* t = s + n;
    T* phat = t + n;
    T* shat = phat + n;
    const int nb = red_blocks(n);
    const unsigned eg = (unsigned)std::min<int64_t>(grid_for(n, RED_THREADS), 4 * std::max(ctx->num_sms, 1));
    int* halt = &w.st->halt;
    SS_TRY(set_params(ctx, w, tol, maxiter, 0));
    spmv_any<T>(ctx, A, val32, x, v, nullptr);
    bicg_init<T><<<(ss_count_launch(), nb), RED_THREADS, 0, ctx->stream>>>(n, b, v, r, rhat, w.st);
    SS_CUDA(ctx, cudaGetLastError());
    int queued = 0, chunk = 2;
    while (true) {
        for (int c = 0; c < chunk; ++c) {
            bicg_p<T><<<(ss_count_launch(), eg), RED_THREADS, 0, ctx->stream>>>(n, r, v, p, w.st);
            SS_TRY(prec_any(ctx, M, p, phat, halt));
            spmv_any<T>(ctx, A, val32, phat, v, halt);
            bicg_rv<T><<<(ss_count_launch(), nb), RED_THREADS, 0, ctx->stream>>>(n, rhat, v, w.st);
            bicg_s<T><<<(ss_count_launch(), nb), RED_THREADS, 0, ctx->stream>>>(n, r, v, s, w.st);
            SS_TRY(prec_any(ctx, M, s, shat, halt));
            spmv_any<T>(ctx, A, val32, shat, t, halt);
            bicg_ts<T><<<(ss_count_launch(), nb), RED_THREADS, 0, ctx->stream>>>(n, t, s, w.st);
            bicg_xr<T><<<(ss_count_launch(), nb), RED_THREADS, 0, ctx->stream>>>(n, x, phat, shat, s, t, r, rhat, w.st);
        }
        SS_CUDA(ctx, cudaGetLastError());
        queued += chunk;
        SS_TRY(read_state(ctx, w));
        if (w.host_st->done) break;
        bool met = false;
        if (oc) SS_TRY(outer_met(ctx, oc, reinterpret_cast<const double2*>(x), &met));
        if (met) { w.host_st->status = SS_OK; break; }
        if (queued > maxiter + 8) break;   // cannot happen: the state sets done at maxiter
        chunk = std::min(chunk * 2, 32);
    }
    SS_TRY(prec_check_error(ctx, M));
    out->status = w.host_st->status;
    out->iters = w.host_st->iters;
    out->resid = w.host_st->rnorm;
    return SS_OK;
}

ss_status bicgstab_dev(ss_ctx ctx, const DeviceCSR& A, ss_prec M, KrylovWork& w, const double2* b, double2* x,
                       double tol, int maxiter, KrylovResultHost* out, const OuterCheck* oc) {
    return bicgstab_any<double2>(ctx, A, nullptr, M, w, b, x, tol, maxiter, out, oc);
}

ss_status bicgstab_dev32(ss_ctx ctx, const DeviceCSR& A, const float2* val32, ss_prec M, KrylovWork& w,
                         const float2* b, float2* x, double tol, int maxiter, KrylovResultHost* out) {
    return bicgstab_any<float2>(ctx, A, val32, M, w, b, x, tol, maxiter, out, nullptr);
}

ss_status gmres_dev(ss_ctx ctx, const DeviceCSR& A, ss_prec M, KrylovWork& w, const double2* b, double2* x, double tol,
                    int maxiter, int m, KrylovResultHost* out, const OuterCheck* oc, int kaug) {
    const int64_t n = A.n_rows;
    if (m < 1 || kaug < 0 || m + kaug > KRYLOV_MAX_M)
        return set_error(ctx, SS_ERR_INVALID, "GMRES needs restart >= 1, augmentation >= 0, restart + augmentation <= 64");
    if (w.method != SS_KRYLOV_GMRES || w.m != m || w.kaug != kaug || w.n != n)
        return set_error(ctx, SS_ERR_INVALID, "GMRES workspace made for another restart length or augmentation");
    const int mx = m + kaug;
    double2* V = w.vecs;                        // mx + 1 basis vectors
    double2* Z = V + (size_t)(mx + 1) * n;      // mx search directions: m preconditioned, then the stored corrections
    double2* D = Z + (size_t)mx * n;            // this cycle's correction (kaug > 0)
    double2* rv = V + (size_t)m * n;            // v_m doubles as the restart residual buffer
    const int nb = red_blocks(n);
    const unsigned eg = (unsigned)std::min<int64_t>(grid_for(n, RED_THREADS), 4 * std::max(ctx->num_sms, 1));
    int* halt = &w.st->halt;
    int stored = 0, oldest = 0;                 // corrections held in Z[m .. m + stored)
    SS_TRY(set_params(ctx, w, tol, maxiter, mx));
    while (true) {
        // restart: y = A x into V_1 as scratch, r into V_m, v_0 = r / beta
        { ProfScope ps_(ctx, PROF_SPMV); spmv_launch(A, x, V + n, nullptr, ctx->stream); }
        gm_restart<<<(ss_count_launch(), nb), RED_THREADS, 0, ctx->stream>>>(n, b, V + n, rv, w.st);
        gm_scale<<<(ss_count_launch(), eg), RED_THREADS, 0, ctx->stream>>>(n, rv, V, w.st);
        const int mt = m + stored;
        for (int j = 0; j < mt; ++j) {
            double2* vj = V + (size_t)j * n;
            double2* zj = Z + (size_t)j * n;
            double2* wv = V + (size_t)(j + 1) * n;
            if (j < m) SS_TRY(prec_apply_dev(ctx, M, vj, zj, halt));     // else zj is a stored correction
            { ProfScope ps_(ctx, PROF_SPMV); spmv_launch(A, zj, wv, halt, ctx->stream); }
            for (int pass = 0; pass < 2; ++pass) {      // classical Gram-Schmidt, twice
                for (int base = 0; base <= j; base += 8)
                    gm_dots<8><<<(ss_count_launch(), nb), RED_THREADS, 0, ctx->stream>>>(n, V, n, j, base, wv, w.st, pass);
                gm_orth_update<<<(ss_count_launch(), eg), RED_THREADS, 0, ctx->stream>>>(n, V, n, j, wv, w.st);
            }
            gm_norm<<<(ss_count_launch(), nb), RED_THREADS, 0, ctx->stream>>>(n, wv, j, mt, w.st);
            gm_scale<<<(ss_count_launch(), eg), RED_THREADS, 0, ctx->stream>>>(n, wv, wv, w.st);
        }
        int slot = -1;
        if (kaug > 0) {
            slot = m + (stored < kaug ? stored : oldest);
            lg_update_x<<<(ss_count_launch(), nb), RED_THREADS, 0, ctx->stream>>>(n, Z, n, x, D, w.st);
            lg_store<<<(ss_count_launch(), eg), RED_THREADS, 0, ctx->stream>>>(n, D, Z + (size_t)slot * n, w.st);
        } else {
            gm_update_x<<<(ss_count_launch(), eg), RED_THREADS, 0, ctx->stream>>>(n, Z, n, x, w.st);
        }
        SS_CUDA(ctx, cudaGetLastError());
        SS_TRY(read_state(ctx, w));
        if (w.host_st->done) break;
        if (slot >= 0 && w.host_st->dnorm > 0.0) {
            if (stored < kaug) ++stored;
            else oldest = (oldest + 1) % kaug;
        }
        bool met = false;
        SS_TRY(outer_met(ctx, oc, x, &met));
        if (met) { w.host_st->status = SS_OK; break; }
        // a cycle that ended on the iteration cap: the next restart pass sets the status
    }
    SS_TRY(prec_check_error(ctx, M));
    out->status = w.host_st->status;
    out->iters = w.host_st->iters;
    out->resid = w.host_st->rnorm;
    return SS_OK;
}
