// Per-system persistent solver for many small Liouvillians (one CTA per
// system at a time).  Everything one Krylov iteration needs runs inside the
// CTA: the SpMV, the two triangular solves of M^{-1} (section "Iterative
// solvers"), the inner products and the vector updates.
//
// Triangular solves work in place on one shared-memory vector: rows are
// grouped into level-aligned units of 32/G rows (G lanes per row); warp w takes
// units w, w + W, w + 2W, ... in order and each row waits on the shared-memory
// completion flags of the rows it depends on.  A row only depends on rows of
// earlier levels, i.e. on earlier units, which their warps process in order,
// so the earliest unfinished unit can always proceed.  Every wait is bounded.
//
// FP64 mode: BiCGSTAB in complex FP64 with the acceptance loop of the
// single-system driver.  Mixed mode: FP32 matrix, factors and Krylov vectors
// for an inner BiCGSTAB on r / ||r||, refined in FP64 (x += ||r|| c) until the
// FP64 residual ||L rho||_2 <= tol.  Reductions accumulate in FP64 in a fixed
// order.
#include <algorithm>

#include "batched.cuh"

namespace {

constexpr int BT = BATCH_THREADS;
constexpr int NW = BT / 32;
constexpr unsigned FULLM = 0xffffffffu;
constexpr long long SPIN_LIMIT = 1ll << 22;   // with back-off: a wait gives up after ~0.3 s

// ------------------------------------------------------------ arithmetic
__device__ __forceinline__ double2 D(double2 a) { return a; }
__device__ __forceinline__ double2 D(float2 a) { return make_double2(a.x, a.y); }
template <class T> __device__ __forceinline__ T cvt(double2 a);
template <> __device__ __forceinline__ double2 cvt<double2>(double2 a) { return a; }
template <> __device__ __forceinline__ float2 cvt<float2>(double2 a) { return make_float2((float)a.x, (float)a.y); }

__device__ __forceinline__ double2 fmac(double2 a, double2 b, double2 c) {
    return make_double2(c.x + a.x * b.x - a.y * b.y, c.y + a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ float2 fmac(float2 a, float2 b, float2 c) {
    return make_float2(c.x + a.x * b.x - a.y * b.y, c.y + a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 mulc(double2 a, double2 b) { return cmul(a, b); }
__device__ __forceinline__ float2 mulc(float2 a, float2 b) { return fcmul(a, b); }
__device__ __forceinline__ double2 subc(double2 a, double2 b) { return csub(a, b); }
__device__ __forceinline__ float2 subc(float2 a, float2 b) { return fcsub(a, b); }
__device__ __forceinline__ double2 addc(double2 a, double2 b) { return cadd(a, b); }
__device__ __forceinline__ float2 addc(float2 a, float2 b) { return fcadd(a, b); }
__device__ __forceinline__ double2 shd(double2 v, int o) {
    return make_double2(__shfl_down_sync(FULLM, v.x, o), __shfl_down_sync(FULLM, v.y, o));
}
__device__ __forceinline__ float2 shd(float2 v, int o) {
    return make_float2(__shfl_down_sync(FULLM, v.x, o), __shfl_down_sync(FULLM, v.y, o));
}
template <class T> __device__ __forceinline__ T zero();
template <> __device__ __forceinline__ double2 zero<double2>() { return make_double2(0.0, 0.0); }
template <> __device__ __forceinline__ float2 zero<float2>() { return make_float2(0.f, 0.f); }

// Block-wide sums of NV doubles, broadcast to every thread (fixed order).
template <int NV>
__device__ void cta_sum(double (&v)[NV], double* red) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < NV; ++k)
        for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_down_sync(FULLM, v[k], o);
    if (lane == 0)
#pragma unroll
        for (int k = 0; k < NV; ++k) red[w * NV + k] = v[k];
    __syncthreads();
#pragma unroll
    for (int k = 0; k < NV; ++k) {
        double s = 0.0;
        for (int q = 0; q < NW; ++q) s += red[q * NV + k];
        v[k] = s;
    }
    __syncthreads();
}

__device__ __forceinline__ bool negligible(double2 a, double nu, double nv) {
    double m = hypot(a.x, a.y);
    return m == 0.0 || m < 1e-15 * nu * nv;
}

// ------------------------------------------------------ triangular solves
// Waits (bounded) until fl[j] == epoch.  Idle warps sleep between polls so
// that the warps doing the work keep the issue slots and the shared-memory
// pipe.
__device__ __forceinline__ bool wait_flag(volatile uint32_t* fl, int32_t j, uint32_t epoch) {
    if (fl[j] == epoch) return true;
    long long spins = 0;
    unsigned ns = 8;
    while (fl[j] != epoch) {
        __nanosleep(ns);
        if (ns < 64) ns <<= 1;
        if (++spins > SPIN_LIMIT) return false;
    }
    return true;
}

template <bool LOWER, int G, class T>
__device__ void cta_trsv_g(const int32_t* __restrict__ rp, const int32_t* __restrict__ col, const T* __restrict__ val,
                           const int32_t* __restrict__ dpos, const T* __restrict__ inv,
                           const int32_t* __restrict__ units, int32_t nunits, T* buf, volatile uint32_t* fl,
                           uint32_t epoch, int* err) {
    constexpr int R = 32 / G;
    constexpr int MAXE = 4;            // entries per lane held in registers before waiting
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, grp = lane / G, sub = lane % G;
    for (int32_t u = warp; u < nunits; u += NW) {
        const int32_t i = units[u * R + grp];
        int32_t s = 0, e = 0;
        if (i >= 0) {
            if (LOWER) { s = rp[i]; e = dpos[i]; }
            else { s = dpos[i] + 1; e = rp[i + 1]; }
        }
        int32_t jj[MAXE];
        T vv[MAXE];
#pragma unroll
        for (int q = 0; q < MAXE; ++q) {
            const int32_t k = s + sub + q * G;
            const bool ok = k < e;
            jj[q] = ok ? col[k] : -1;
            vv[q] = ok ? val[k] : zero<T>();
        }
        bool bad = false;
#pragma unroll
        for (int q = 0; q < MAXE; ++q)
            if (jj[q] >= 0 && !wait_flag(fl, jj[q], epoch)) bad = true;
        __threadfence_block();
        T acc = zero<T>();
#pragma unroll
        for (int q = 0; q < MAXE; ++q)
            if (jj[q] >= 0) acc = fmac(vv[q], buf[jj[q]], acc);
        for (int32_t k = s + sub + MAXE * G; k < e; k += G) {      // long rows
            const int32_t j = col[k];
            if (!wait_flag(fl, j, epoch)) bad = true;
            __threadfence_block();
            acc = fmac(val[k], buf[j], acc);
        }
#pragma unroll
        for (int o = G / 2; o > 0; o >>= 1) {
            T other = shd(acc, o);
            acc.x += other.x;
            acc.y += other.y;
        }
        if (bad) atomicExch(err, 1);
        if (i >= 0 && sub == 0) {
            T xi = subc(buf[i], acc);
            if (!LOWER) xi = mulc(xi, inv[i]);
            buf[i] = xi;
            __threadfence_block();
            fl[i] = epoch;
        }
    }
    __syncthreads();
}

template <bool LOWER, class T>
__device__ void cta_trsv(int g, const int32_t* rp, const int32_t* col, const T* val, const int32_t* dpos,
                         const T* inv, const int32_t* units, int32_t nunits, T* buf, volatile uint32_t* fl,
                         uint32_t epoch, int* err) {
    switch (g) {
        case 1: cta_trsv_g<LOWER, 1, T>(rp, col, val, dpos, inv, units, nunits, buf, fl, epoch, err); break;
        case 2: cta_trsv_g<LOWER, 2, T>(rp, col, val, dpos, inv, units, nunits, buf, fl, epoch, err); break;
        case 4: cta_trsv_g<LOWER, 4, T>(rp, col, val, dpos, inv, units, nunits, buf, fl, epoch, err); break;
        case 8: cta_trsv_g<LOWER, 8, T>(rp, col, val, dpos, inv, units, nunits, buf, fl, epoch, err); break;
        case 16: cta_trsv_g<LOWER, 16, T>(rp, col, val, dpos, inv, units, nunits, buf, fl, epoch, err); break;
        default: cta_trsv_g<LOWER, 32, T>(rp, col, val, dpos, inv, units, nunits, buf, fl, epoch, err); break;
    }
}

// ------------------------------------------------------------------ SpMV
// y = A x with x in shared memory; accumulates <rhat, y> (dots 0, 1) and
// |y|^2 (dot 2) when rhat is given.
template <int G, class T>
__device__ void cta_spmv_g(const int32_t* __restrict__ rp, const int32_t* __restrict__ col, const T* __restrict__ val,
                           int32_t n, const T* xs, T* __restrict__ y, const T* __restrict__ rhat, double (&dots)[3]) {
    const int lane = threadIdx.x & 31, sub = lane % G;
    const int32_t rows_per_pass = BT / G;
    for (int32_t base = 0; base < n; base += rows_per_pass) {
        const int32_t r = base + threadIdx.x / G;
        T acc = zero<T>();
        if (r < n)
            for (int32_t k = rp[r] + sub; k < rp[r + 1]; k += G) acc = fmac(val[k], xs[col[k]], acc);
#pragma unroll
        for (int o = G / 2; o > 0; o >>= 1) {
            T other = shd(acc, o);
            acc.x += other.x;
            acc.y += other.y;
        }
        if (r < n && sub == 0) {
            y[r] = acc;
            if (rhat) {
                double2 a = D(acc), h = D(rhat[r]);
                dots[0] += h.x * a.x + h.y * a.y;
                dots[1] += h.x * a.y - h.y * a.x;
                dots[2] += a.x * a.x + a.y * a.y;
            }
        }
    }
}

template <class T>
__device__ void cta_spmv(int g, const int32_t* rp, const int32_t* col, const T* val, int32_t n, const T* xs, T* y,
                         const T* rhat, double (&dots)[3]) {
    switch (g) {
        case 1: cta_spmv_g<1, T>(rp, col, val, n, xs, y, rhat, dots); break;
        case 2: cta_spmv_g<2, T>(rp, col, val, n, xs, y, rhat, dots); break;
        case 4: cta_spmv_g<4, T>(rp, col, val, n, xs, y, rhat, dots); break;
        case 8: cta_spmv_g<8, T>(rp, col, val, n, xs, y, rhat, dots); break;
        case 16: cta_spmv_g<16, T>(rp, col, val, n, xs, y, rhat, dots); break;
        default: cta_spmv_g<32, T>(rp, col, val, n, xs, y, rhat, dots); break;
    }
}

// -------------------------------------------------------------- context
template <class T>
struct Ctx {
    const BatchSys* S;
    int32_t n;
    const T* aval;
    const T* fval;
    const T* finv;
    T* buf;                     // shared: n
    volatile uint32_t* fl;      // shared: n
    double* red;                // shared reduction scratch
    uint32_t epoch;
    int* err;
};

// out = M^{-1} in; the result also stays in the shared buffer
template <class T>
__device__ void cta_prec(Ctx<T>& c, const T* in, T* out) {
    const BatchSys& S = *c.S;
    for (int32_t i = threadIdx.x; i < c.n; i += BT) c.buf[i] = in[i];
    __syncthreads();
    cta_trsv<true, T>(S.lo_g, S.f_rp, S.f_col, c.fval, S.f_dpos, c.finv, S.lo_units, S.lo_nunits, c.buf, c.fl,
                      c.epoch, c.err);
    cta_trsv<false, T>(S.up_g, S.f_rp, S.f_col, c.fval, S.f_dpos, c.finv, S.up_units, S.up_nunits, c.buf, c.fl,
                       c.epoch + 1, c.err);
    c.epoch += 2;
    for (int32_t i = threadIdx.x; i < c.n; i += BT) out[i] = c.buf[i];
    // no barrier needed: the shared buffer is only read afterwards
}

struct KResult {
    int status, iters;
    double resid;
};

// Right-preconditioned BiCGSTAB on A x = b (x holds the initial guess),
// stopping at ||b - A x||_2 <= tol.  Same steps and stop/breakdown rules as
// the multi-kernel solver.
template <class T>
__device__ KResult cta_bicgstab(Ctx<T>& c, T* x, const T* b, T* wk, double tol, int maxiter) {
    const BatchSys& S = *c.S;
    const int32_t n = c.n;
    T* r = wk;
    T* rhat = r + n;
    T* p = rhat + n;
    T* v = p + n;
    T* s = v + n;
    T* t = s + n;
    T* phat = t + n;
    T* shat = phat + n;
    KResult res{SS_NOT_CONVERGED, 0, 0.0};
    // r = b - A x
    for (int32_t i = threadIdx.x; i < n; i += BT) c.buf[i] = x[i];
    __syncthreads();
    double dz[3] = {0, 0, 0};
    cta_spmv<T>(S.a_g, S.a_rp, S.a_col, c.aval, n, c.buf, v, nullptr, dz);
    __syncthreads();
    double nr[1] = {0.0};
    for (int32_t i = threadIdx.x; i < n; i += BT) {
        T ri = subc(b[i], v[i]);
        r[i] = ri;
        rhat[i] = ri;
        double2 q = D(ri);
        nr[0] += q.x * q.x + q.y * q.y;
    }
    cta_sum<1>(nr, c.red);
    double rn = sqrt(nr[0]);
    res.resid = rn;
    if (rn <= tol) { res.status = SS_OK; return res; }
    const double rhat_norm = rn;
    double2 rho = make_double2(nr[0], 0.0), alpha = make_double2(1, 0), omega = make_double2(1, 0),
            beta = make_double2(0, 0);
    for (int it = 1; it <= maxiter; ++it) {
        {   // p = r + beta (p - omega v)
            const T bt = cvt<T>(beta), om = cvt<T>(omega);
            for (int32_t i = threadIdx.x; i < n; i += BT)
                p[i] = (it == 1) ? r[i] : addc(r[i], mulc(bt, subc(p[i], mulc(om, v[i]))));
        }
        __syncthreads();
        cta_prec<T>(c, p, phat);
        double dv[3] = {0, 0, 0};
        cta_spmv<T>(S.a_g, S.a_rp, S.a_col, c.aval, n, c.buf, v, rhat, dv);
        cta_sum<3>(dv, c.red);
        const double2 rv = make_double2(dv[0], dv[1]);
        if (negligible(rv, rhat_norm, sqrt(dv[2]))) { res.status = SS_BREAKDOWN; res.iters = it - 1; return res; }
        alpha = cdiv(rho, rv);
        double ns[1] = {0.0};
        {
            const T al = cvt<T>(alpha);
            for (int32_t i = threadIdx.x; i < n; i += BT) {
                T si = subc(r[i], mulc(al, v[i]));
                s[i] = si;
                double2 q = D(si);
                ns[0] += q.x * q.x + q.y * q.y;
            }
        }
        cta_sum<1>(ns, c.red);
        const double sn = sqrt(ns[0]);
        if (sn <= tol) {
            const T al = cvt<T>(alpha);
            for (int32_t i = threadIdx.x; i < n; i += BT) x[i] = addc(x[i], mulc(al, phat[i]));
            __syncthreads();
            res.status = SS_OK;
            res.iters = it;
            res.resid = sn;
            return res;
        }
        cta_prec<T>(c, s, shat);
        double dt[3] = {0, 0, 0};
        cta_spmv<T>(S.a_g, S.a_rp, S.a_col, c.aval, n, c.buf, t, nullptr, dt);
        __syncthreads();
        double tsd[3] = {0, 0, 0};
        for (int32_t i = threadIdx.x; i < n; i += BT) {
            double2 a = D(t[i]), q = D(s[i]);
            tsd[0] += a.x * q.x + a.y * q.y;
            tsd[1] += a.x * q.y - a.y * q.x;
            tsd[2] += a.x * a.x + a.y * a.y;
        }
        cta_sum<3>(tsd, c.red);
        if (tsd[2] == 0.0) { res.status = SS_BREAKDOWN; res.iters = it; return res; }
        omega = make_double2(tsd[0] / tsd[2], tsd[1] / tsd[2]);
        double nr2[3] = {0, 0, 0};
        {
            const T al = cvt<T>(alpha), om = cvt<T>(omega);
            for (int32_t i = threadIdx.x; i < n; i += BT) {
                x[i] = addc(x[i], addc(mulc(al, phat[i]), mulc(om, shat[i])));
                T ri = subc(s[i], mulc(om, t[i]));
                r[i] = ri;
                double2 a = D(rhat[i]), q = D(ri);
                nr2[0] += a.x * q.x + a.y * q.y;
                nr2[1] += a.x * q.y - a.y * q.x;
                nr2[2] += q.x * q.x + q.y * q.y;
            }
        }
        cta_sum<3>(nr2, c.red);
        rn = sqrt(nr2[2]);
        res.iters = it;
        res.resid = rn;
        if (rn <= tol) { res.status = SS_OK; return res; }
        if (omega.x == 0.0 && omega.y == 0.0) { res.status = SS_BREAKDOWN; return res; }
        if (it >= maxiter) { res.status = SS_NOT_CONVERGED; return res; }
        const double2 rho_new = make_double2(nr2[0], nr2[1]);
        if (negligible(rho_new, rhat_norm, rn)) { res.status = SS_BREAKDOWN; return res; }
        beta = cmul(cdiv(rho_new, rho), cdiv(alpha, omega));
        rho = rho_new;
    }
    return res;
}

// FP64 ||L rho||_2 for rho = x / tr(x), x in global memory; also returns tr(x).
__device__ double cta_lrho(const BatchSys& S, const double2* x, double* red, double2* tr_out) {
    double tr[2] = {0, 0};
    for (int32_t i = threadIdx.x; i < S.d; i += BT) {
        double2 v = x[S.tidx[i]];
        tr[0] += v.x;
        tr[1] += v.y;
    }
    cta_sum<2>(tr, red);
    const double2 trc = make_double2(tr[0], tr[1]);
    double acc[1] = {0.0};
    for (int32_t r = threadIdx.x; r < S.n; r += BT) {
        double2 y = make_double2(0.0, 0.0);
        for (int32_t k = S.a_rp[r]; k < S.a_rp[r + 1]; ++k) y = fmac(S.a_val[k], x[S.a_col[k]], y);
        if (S.w != 0.0 && r == S.r0) { y.x -= S.w * trc.x; y.y -= S.w * trc.y; }
        if (S.w == 0.0) { y.x += S.sigma * x[r].x; y.y += S.sigma * x[r].y; }
        acc[0] += y.x * y.x + y.y * y.y;
    }
    cta_sum<1>(acc, red);
    *tr_out = trc;
    const double m = hypot(trc.x, trc.y);
    return m > 0.0 ? sqrt(acc[0]) / m : INFINITY;
}

// ----------------------------------------------------------- iLU(0)
__device__ __forceinline__ int32_t find_col_b(const int32_t* __restrict__ col, int32_t lo, int32_t hi, int32_t c) {
    hi -= 1;
    while (lo <= hi) {
        int32_t mid = (lo + hi) >> 1;
        int32_t v = col[mid];
        if (v == c) return mid;
        if (v < c) lo = mid + 1; else hi = mid - 1;
    }
    return -1;
}

__device__ bool cta_ilu0(const BatchSys& S, bool mixed) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int32_t nnz = S.f_rp[S.n];
    double2* val = S.f_val;
    for (int32_t k = threadIdx.x; k < nnz; k += BT) val[k] = S.a_val[k];
    __syncthreads();
    for (int32_t l = 0; l < S.n_levels; ++l) {
        for (int32_t q = S.lvl_ptr[l] + warp; q < S.lvl_ptr[l + 1]; q += NW) {
            const int32_t i = S.lvl_rows[q];
            const int32_t re = S.f_rp[i + 1], di = S.f_dpos[i];
            for (int32_t t = S.f_rp[i]; t < di; ++t) {
                const int32_t k = S.f_col[t];
                double2 f = make_double2(0.0, 0.0);
                if (lane == 0) {
                    f = cdiv(val[t], val[S.f_dpos[k]]);
                    val[t] = f;
                }
                f.x = __shfl_sync(FULLM, f.x, 0);
                f.y = __shfl_sync(FULLM, f.y, 0);
                for (int32_t u = S.f_dpos[k] + 1 + lane; u < S.f_rp[k + 1]; u += 32) {
                    const int32_t pos = find_col_b(S.f_col, t + 1, re, S.f_col[u]);
                    if (pos >= 0) val[pos] = csub(val[pos], cmul(f, val[u]));
                }
                __syncwarp();
            }
        }
        __syncthreads();
    }
    __shared__ int zero_pivot;
    if (threadIdx.x == 0) zero_pivot = 0;
    __syncthreads();
    for (int32_t i = threadIdx.x; i < S.n; i += BT) {
        double2 dg = val[S.f_dpos[i]];
        if (dg.x == 0.0 && dg.y == 0.0) zero_pivot = 1;
        double2 r = cdiv(make_double2(1.0, 0.0), dg);
        S.f_inv[i] = r;
        if (mixed) S.f_inv32[i] = make_float2((float)r.x, (float)r.y);
    }
    if (mixed) {
        for (int32_t k = threadIdx.x; k < nnz; k += BT) {
            S.f_val32[k] = make_float2((float)val[k].x, (float)val[k].y);
            S.a_val32[k] = make_float2((float)S.a_val[k].x, (float)S.a_val[k].y);
        }
    }
    __syncthreads();
    return zero_pivot == 0;
}

// ------------------------------------------------------------- drivers
__device__ void solve_fp64(BatchSys& S, const BatchParams& P, unsigned char* smem, double* red, int* err) {
    const int32_t n = S.n;
    Ctx<double2> c;
    c.S = &S;
    c.n = n;
    c.aval = S.a_val;
    c.fval = S.f_val;
    c.finv = S.f_inv;
    c.buf = reinterpret_cast<double2*>(smem);
    c.fl = reinterpret_cast<volatile uint32_t*>(smem + sizeof(double2) * n);
    c.red = red;
    c.epoch = 1;
    c.err = err;
    for (int32_t i = threadIdx.x; i < n; i += BT) c.fl[i] = 0u;
    double2* wk = reinterpret_cast<double2*>(S.work);
    double2* b = wk + 8 * (size_t)n;
    double2* x = S.x64;
    for (int32_t i = threadIdx.x; i < n; i += BT) {
        b[i] = make_double2(i == S.r0 ? S.w : 0.0, 0.0);
        x[i] = make_double2(0.0, 0.0);
    }
    __syncthreads();
    double inner = 0.5 * P.tol, lr = INFINITY;
    int total = 0, status = SS_NOT_CONVERGED;
    for (int pass = 0; pass < 8; ++pass) {
        KResult kr = cta_bicgstab<double2>(c, x, b, wk, inner, P.maxiter - total);
        total += kr.iters;
        double2 tr;
        lr = cta_lrho(S, x, red, &tr);
        if (lr <= P.tol) { status = SS_OK; break; }
        if (total >= P.maxiter || kr.status == SS_NOT_CONVERGED || (kr.status == SS_BREAKDOWN && kr.iters == 0)) {
            status = kr.status == SS_OK ? SS_NOT_CONVERGED : kr.status;
            break;
        }
        if (kr.status == SS_OK) inner *= 0.1;
    }
    S.iters = total;
    S.outer = 1;
    S.resid = lr;
    S.status = status;
}

__device__ void solve_mixed(BatchSys& S, const BatchParams& P, unsigned char* smem, double* red, int* err) {
    const int32_t n = S.n;
    Ctx<float2> c;
    c.S = &S;
    c.n = n;
    c.aval = S.a_val32;
    c.fval = S.f_val32;
    c.finv = S.f_inv32;
    c.buf = reinterpret_cast<float2*>(smem);
    c.fl = reinterpret_cast<volatile uint32_t*>(smem + sizeof(float2) * n);
    c.red = red;
    c.epoch = 1;
    c.err = err;
    for (int32_t i = threadIdx.x; i < n; i += BT) c.fl[i] = 0u;
    float2* wk = reinterpret_cast<float2*>(S.work);
    float2* b32 = wk + 8 * (size_t)n;
    float2* x32 = b32 + n;
    double2* x = S.x64;
    double2* r = S.r64;
    for (int32_t i = threadIdx.x; i < n; i += BT) x[i] = make_double2(0.0, 0.0);
    __syncthreads();
    int total = 0, status = SS_NOT_CONVERGED, outer = 0;
    double lr = INFINITY;
    for (outer = 1; outer <= 30; ++outer) {
        // FP64 residual r = b - A x and the acceptance test on x
        double2 tr;
        lr = (outer == 1) ? INFINITY : cta_lrho(S, x, red, &tr);
        if (lr <= P.tol) { status = SS_OK; break; }
        double nrm[1] = {0.0};
        for (int32_t i = threadIdx.x; i < n; i += BT) {
            double2 y = make_double2(i == S.r0 ? S.w : 0.0, 0.0);
            for (int32_t k = S.a_rp[i]; k < S.a_rp[i + 1]; ++k) {
                const double2 a = S.a_val[k], xv = x[S.a_col[k]];
                y.x -= a.x * xv.x - a.y * xv.y;
                y.y -= a.x * xv.y + a.y * xv.x;
            }
            r[i] = y;
            nrm[0] += y.x * y.x + y.y * y.y;
        }
        cta_sum<1>(nrm, red);
        const double rn = sqrt(nrm[0]);
        if (rn == 0.0) { status = SS_OK; lr = 0.0; break; }
        if (total >= P.maxiter) break;
        const double inv = 1.0 / rn;
        for (int32_t i = threadIdx.x; i < n; i += BT) {
            b32[i] = make_float2((float)(r[i].x * inv), (float)(r[i].y * inv));
            x32[i] = make_float2(0.f, 0.f);
        }
        __syncthreads();
        // an FP32 inner solve that stalls above its tolerance returns after a bounded
        // number of iterations so that the FP64 refinement can continue
        const int cap = min(P.maxiter - total, max(50, P.maxiter / 5));
        KResult kr = cta_bicgstab<float2>(c, x32, b32, wk, P.inner_rtol, cap);
        total += kr.iters;
        for (int32_t i = threadIdx.x; i < n; i += BT) {
            x[i].x += rn * (double)x32[i].x;
            x[i].y += rn * (double)x32[i].y;
        }
        __syncthreads();
        if (kr.status == SS_BREAKDOWN && kr.iters == 0) { status = SS_BREAKDOWN; break; }
    }
    if (outer > 30) outer = 30;
    S.iters = total;
    S.outer = outer;
    S.resid = lr;
    S.status = status;
}

__device__ void finalise(const BatchSys& S, double* red) {
    double tr[2] = {0, 0};
    for (int32_t i = threadIdx.x; i < S.d; i += BT) {
        double2 v = S.x64[S.tidx[i]];
        tr[0] += v.x;
        tr[1] += v.y;
    }
    cta_sum<2>(tr, red);
    const double2 t = make_double2(tr[0], tr[1]);
    for (int32_t r = threadIdx.x; r < S.n; r += BT) S.rho_out[S.perm[r]] = cdiv(S.x64[r], t);
    __syncthreads();
}

__global__ void __launch_bounds__(BT, 1) batched_solver(BatchSys* sys, int nsys, BatchParams P, int* queue,
                                                         int* err) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ double red[NW * 3];
    __shared__ int s_idx;
    while (true) {
        if (threadIdx.x == 0) s_idx = atomicAdd(queue, 1);
        __syncthreads();
        const int k = s_idx;
        __syncthreads();
        if (k >= nsys) break;
        BatchSys& S = sys[k];
        bool ok = true;
        if (S.factor_on_device) ok = cta_ilu0(S, P.mixed != 0);
        if (!ok) {
            if (threadIdx.x == 0) { S.status = SS_ZERO_PIVOT; S.iters = 0; S.outer = 0; S.resid = INFINITY; }
            __syncthreads();
            continue;
        }
        if (P.mixed) solve_mixed(S, P, smem, red, err);
        else solve_fp64(S, P, smem, red, err);
        finalise(S, red);
    }
}

}  // namespace

size_t batch_smem_bytes(int n, bool mixed) {
    return (size_t)n * ((mixed ? sizeof(float2) : sizeof(double2)) + sizeof(uint32_t));
}

int batch_max_n(bool mixed) {
    const size_t cap = 227 * 1024 - 2048;
    return (int)(cap / ((mixed ? sizeof(float2) : sizeof(double2)) + sizeof(uint32_t)));
}

ss_status batch_launch(ss_ctx ctx, BatchSys* dsys, int nsys, const BatchParams& p, int max_n, int* queue, int* err) {
    const size_t smem = batch_smem_bytes(max_n, p.mixed != 0);
    SS_CUDA(ctx, cudaFuncSetAttribute(batched_solver, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    const int grid = std::max(1, std::min(nsys, ctx->num_sms > 0 ? ctx->num_sms : 1));
    {
        ProfScope ps(ctx, PROF_BATCHED);
        batched_solver<<<(ss_count_launch(), grid), BT, smem, ctx->stream>>>(dsys, nsys, p, queue, err);
    }
    SS_CUDA(ctx, cudaGetLastError());
    return SS_OK;
}
