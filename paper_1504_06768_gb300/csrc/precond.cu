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
    __device__ static double2 shfl(double2 v, int l) {
        return make_double2(__shfl_sync(FULL, v.x, l), __shfl_sync(FULL, v.y, l));
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
    __device__ static float2 shfl(float2 v, int l) {
        return make_float2(__shfl_sync(FULL, v.x, l), __shfl_sync(FULL, v.y, l));
    }
    __device__ static float2 ldcg(const float2* p) { return __ldcg(p); }
};

__device__ __forceinline__ unsigned long long globaltimer_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
    return t;
}

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

// Sync-free triangular solve.  Each triangle is stored on its own in level
// order, cut into level-aligned units of R = 32 / G rows (G lanes per row); a
// unit's entries are contiguous, so a warp reads them as one coalesced run.
// Blocks take consecutive runs of units in level order through a ticket
// counter (one atomic per block), so a row only ever waits for rows held by
// earlier blocks, which are resident or finished: the solve always
// progresses, whatever else runs on the device (no co-residency is needed).
// The output vector starts filled with the PENDING mark; a row waits
// (bounded) until the values it depends on are no longer PENDING -- the value
// itself is the completion signal, so no flag or fence is needed.  A lane
// issues the loads of its first K entries (columns, values, then the x they
// need) together, so a row costs three dependent round trips (row record,
// entries, x) once its inputs are ready.  The entries of a row beyond its
// first K G (only rows far longer than the triangle's mean, such as the
// trace row) are taken by the whole warp, K per lane at a time.
//   LOWER: x_i = b_i - sum_{j<i} l_ij x_j (unit diagonal); also re-marks
//          `other[i]` (the upper solve's output) PENDING.
//   UPPER: x_i = (b_i - sum_{j>i} u_ij x_j) / u_ii; afterwards re-marks b_i
//          (the lower solve's output) PENDING for the next application.
constexpr int TRSV_THREADS = 256;
constexpr int TRSV_K = 4;      // entries per lane whose loads are issued together
// Systems whose solution vector fits in a block's shared memory (at most this
// many bytes) are solved by one block (sptrsv_block).
constexpr size_t TRSV_BLOCK_MAX_BYTES = 200 * 1024;

template <class T>
struct TrsvArgs {
    const int32_t* urow;
    const int32_t* uptr;
    const int32_t* col;
    const T* val;
    const T* dinv;             // upper: 1 / u_ii per slot
    int64_t n_units;
    const T* b;
    T* x;
    T* other;                  // lower: the upper solve's output (re-marked); upper: the lower's (b)
    int* err;
    unsigned long long* ticket;   // block tickets of this triangle (never reset)
    const int* halt;
    unsigned long long wait_ns;
};

template <int G, int K, class T>
struct UnitPf {                // one lane's share of a unit, prefetched
    int32_t i, s, e;           // row (-1: padding), entry range
    int32_t c[K];
    T v[K];
    T bv, dv;                  // b_i and 1 / u_ii (lane sub == 0)
};

// Slot of this lane's row in unit u (G lanes per row), its row id (-1:
// padding or past the end) and entry range.
template <int G, class T>
__device__ __forceinline__ void unit_rows(const TrsvArgs<T>& a, int64_t u, int grp, int64_t& slot, int32_t& i,
                                          int32_t& s, int32_t& e) {
    i = -1;
    s = e = 0;
    slot = 0;
    if (u < a.n_units) {
        slot = u * (32 / G) + grp;
        i = __ldg(&a.urow[slot]);
        s = __ldg(&a.uptr[slot]);
        e = __ldg(&a.uptr[slot + 1]);
    }
}

template <bool LOWER, int G, int K, class T>
__device__ __forceinline__ void unit_entries(const TrsvArgs<T>& a, int64_t slot, int sub, UnitPf<G, K, T>& p) {
    using C = Cplx<T>;
#pragma unroll
    for (int q = 0; q < K; ++q) {
        const int32_t k = p.s + sub + q * G;
        p.c[q] = k < p.e ? __ldcs(&a.col[k]) : -1;
        p.v[q] = k < p.e ? __ldcs(&a.val[k]) : C::zero();
    }
    p.bv = C::zero();
    p.dv = C::zero();
    if (p.i >= 0 && sub == 0) {
        p.bv = __ldcg(&a.b[p.i]);
        if (!LOWER) p.dv = __ldg(&a.dinv[slot]);
    }
}

// x[c], waiting (bounded) while it is PENDING; 0 after a timeout.
template <class T>
__device__ __forceinline__ T wait_ready(const TrsvArgs<T>& a, int32_t c, T v, bool& timed_out) {
    if (ready(v)) return v;
    const T* xp = &a.x[c];
    const unsigned long long t0 = globaltimer_ns();
    int spins = 0;
    // no back-off between reads: a value is read again as soon as the last
    // read returns (backing off 32, then 256 ns measured 669-671 us in FP32
    // and 1,304-1,309 us in FP64 per M^-1 r of the chain, against 598-599
    // and 1,237-1,241 us)
    while (true) {
        ++spins;
        v = __ldcv(xp);
        if (ready(v)) return v;
        if ((spins & 15) == 0 && (*(volatile int*)a.err != 0 || globaltimer_ns() - t0 > a.wait_ns)) {
            // raised at once, so that every other wait of the launch gives up at its next check
            if (*(volatile int*)a.err == 0) atomicExch(a.err, 1);
            timed_out = true;
            return Cplx<T>::zero();
        }
    }
}

template <bool LOWER, int G, int K, class T>
__global__ void __launch_bounds__(TRSV_THREADS) sptrsv_syncfree(TrsvArgs<T> a) {
    using C = Cplx<T>;
    if (a.halt && *a.halt) return;      // uniform over the launch: no ticket is taken
    __shared__ unsigned long long s_ticket;
    if (threadIdx.x == 0) s_ticket = atomicAdd(a.ticket, 1ull);
    __syncthreads();
    // the k-th block to start takes the k-th run of units (tickets keep
    // counting across launches, each launch takes gridDim.x of them)
    const int64_t u = (int64_t)(s_ticket % (unsigned long long)gridDim.x) * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (u >= a.n_units) return;
    const int lane = threadIdx.x & 31;
    const int grp = lane / G, sub = lane % G;
    bool timed_out = false;
    UnitPf<G, K, T> cur;
    int64_t slot;
    unit_rows<G, T>(a, u, grp, slot, cur.i, cur.s, cur.e);
    unit_entries<LOWER, G, K, T>(a, slot, sub, cur);
    T xj[K];
#pragma unroll
    for (int q = 0; q < K; ++q) xj[q] = cur.c[q] >= 0 ? __ldcv(&a.x[cur.c[q]]) : C::zero();
    T acc = C::zero();
#pragma unroll
    for (int q = 0; q < K; ++q)
        if (cur.c[q] >= 0) acc = C::fma_(cur.v[q], wait_ready(a, cur.c[q], xj[q], timed_out), acc);
    // entries beyond the first K G of a row: the whole warp takes them, one
    // such row after another, K per lane per batch of loads
    unsigned tails = __ballot_sync(FULL, sub == 0 && cur.e - cur.s > K * G);
    while (tails) {
        const int src = __ffs(tails) - 1;
        tails &= tails - 1;
        const int32_t ts = __shfl_sync(FULL, cur.s, src) + K * G, te = __shfl_sync(FULL, cur.e, src);
        T part = C::zero();
        for (int32_t base = ts + lane; base < te; base += 32 * K) {
            int32_t c[K];
            T v[K], xv[K];
#pragma unroll
            for (int q = 0; q < K; ++q) {
                const int32_t k = base + q * 32;
                c[q] = k < te ? __ldcs(&a.col[k]) : -1;
                v[q] = k < te ? __ldcs(&a.val[k]) : C::zero();
            }
#pragma unroll
            for (int q = 0; q < K; ++q) xv[q] = c[q] >= 0 ? __ldcv(&a.x[c[q]]) : C::zero();
#pragma unroll
            for (int q = 0; q < K; ++q)
                if (c[q] >= 0) part = C::fma_(v[q], wait_ready(a, c[q], xv[q], timed_out), part);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const T ov = C::shfl_down(part, o);
            part.x += ov.x;
            part.y += ov.y;
        }
        part = C::shfl(part, 0);
        if (lane == src) {
            acc.x += part.x;
            acc.y += part.y;
        }
    }
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) {
        T ov = C::shfl_down(acc, o);
        acc.x += ov.x;
        acc.y += ov.y;
    }
    if (cur.i >= 0 && sub == 0) {
        T xi = C::sub(cur.bv, acc);
        if (!LOWER) xi = C::mul(xi, cur.dv);
        __stcg(&a.x[cur.i], xi);
        if (a.other) __stcg(&a.other[cur.i], pending<T>());
    }
    if (__any_sync(FULL, timed_out) && lane == 0) atomicExch(a.err, 1);
}

// The same solve by one block for a system whose solution vector fits in
// shared memory: x lives there, pre-marked PENDING, so a dependency is a
// shared-memory store and load (tens of cycles) instead of a round trip
// through L2 -- what counts for factors with many levels (ILUT's upper
// triangle of the Jaynes-Cummings system: 5,703 levels for 6,400 rows).
// Units are dealt to the block's warps round-robin (unit u to warp u mod W,
// each warp in increasing u); every dependency lies in a smaller unit of a
// warp of this block, so the solve progresses, and no barrier separates the
// levels.  Each warp loads its next unit while it solves the current one.
constexpr int TRSV_BLOCK_THREADS = 1024;

template <class T>
__device__ __forceinline__ T smem_ready_value(const TrsvArgs<T>& a, volatile T* xs, int32_t c, bool& timed_out) {
    T v;
    v.x = xs[c].x;
    v.y = xs[c].y;
    if (ready(v) || timed_out) return v;
    const unsigned long long t0 = globaltimer_ns();
    int spins = 0;
    while (true) {
        v.x = xs[c].x;
        v.y = xs[c].y;
        if (ready(v)) return v;
        if ((++spins & 255) == 0 && (*(volatile int*)a.err != 0 || globaltimer_ns() - t0 > a.wait_ns)) {
            if (*(volatile int*)a.err == 0) atomicExch(a.err, 1);
            timed_out = true;
            return Cplx<T>::zero();
        }
    }
}

template <bool LOWER, int G, int K, class T>
__global__ void __launch_bounds__(TRSV_BLOCK_THREADS) sptrsv_block(TrsvArgs<T> a, int64_t n) {
    using C = Cplx<T>;
    if (a.halt && *a.halt) return;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    volatile T* xs = reinterpret_cast<volatile T*>(smem_raw);
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
        const T p = pending<T>();
        xs[i].x = p.x;
        xs[i].y = p.y;
    }
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int grp = lane / G, sub = lane % G;
    const int64_t W = blockDim.x >> 5;
    bool timed_out = false;
    UnitPf<G, K, T> cur, nxt;
    int64_t u = threadIdx.x >> 5, slot;
    unit_rows<G, T>(a, u, grp, slot, cur.i, cur.s, cur.e);
    unit_entries<LOWER, G, K, T>(a, slot, sub, cur);
    for (; u < a.n_units; u += W) {
        unit_rows<G, T>(a, u + W, grp, slot, nxt.i, nxt.s, nxt.e);
        unit_entries<LOWER, G, K, T>(a, slot, sub, nxt);
        T acc = C::zero();
#pragma unroll
        for (int q = 0; q < K; ++q)
            if (cur.c[q] >= 0) acc = C::fma_(cur.v[q], smem_ready_value(a, xs, cur.c[q], timed_out), acc);
        for (int32_t base = cur.s + sub + K * G; base < cur.e; base += K * G) {
#pragma unroll
            for (int q = 0; q < K; ++q) {
                const int32_t k = base + q * G;
                if (k < cur.e) acc = C::fma_(a.val[k], smem_ready_value(a, xs, a.col[k], timed_out), acc);
            }
        }
#pragma unroll
        for (int o = G / 2; o > 0; o >>= 1) {
            T ov = C::shfl_down(acc, o);
            acc.x += ov.x;
            acc.y += ov.y;
        }
        if (cur.i >= 0 && sub == 0) {
            T xi = C::sub(cur.bv, acc);
            if (!LOWER) xi = C::mul(xi, cur.dv);
            xs[cur.i].x = xi.x;
            xs[cur.i].y = xi.y;
        }
        cur = nxt;
    }
    if (__any_sync(FULL, timed_out) && lane == 0) atomicExch(a.err, 1);
    __syncthreads();
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
        T v;
        v.x = xs[i].x;
        v.y = xs[i].y;
        a.x[i] = v;
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

// Lanes per row of a triangle: enough that K entries per lane cover a row of
// twice the triangle's mean length in one batch of loads, at least 2 (G
// divides 32).
int trsv_lanes(double avg_row) {
    int g = 2;
    while (g < 32 && g * TRSV_K < 2.0 * avg_row) g <<= 1;
    return g;
}

// One strict triangle (lower: columns < i, upper: columns > i) of the
// combined factors in unit order: level-aligned units of R rows, each unit's
// entries contiguous.  Only the pattern is needed here; values are gathered
// after the numeric factorisation (pack_triangle).
ss_status build_triangle(ss_ctx ctx, const std::vector<int32_t>& order, const std::vector<int32_t>& lptr,
                         int32_t nlev, bool lower, const std::vector<int32_t>& hrp, const std::vector<int32_t>& hcol,
                         TriLevels& T) {
    const int64_t n = (int64_t)hrp.size() - 1;
    T.n_levels = nlev;
    int64_t nnz_t = 0;
    for (int64_t i = 0; i < n; ++i)
        for (int32_t t = hrp[i]; t < hrp[i + 1]; ++t) nnz_t += lower ? hcol[t] < i : hcol[t] > i;
    T.g = trsv_lanes(n ? (double)nnz_t / n : 1.0);
    const int R = 32 / T.g;
    std::vector<int32_t> urow;
    level_units_host(order, lptr, R, urow);
    T.n_units = (int64_t)urow.size() / R;
    T.nnz = nnz_t;
    std::vector<int32_t> uptr(urow.size() + 1), tcol((size_t)nnz_t), tsrc((size_t)nnz_t);
    int64_t k = 0;
    for (size_t sl = 0; sl < urow.size(); ++sl) {
        uptr[sl] = (int32_t)k;
        const int32_t i = urow[sl];
        if (i < 0) continue;
        for (int32_t t = hrp[i]; t < hrp[i + 1]; ++t)
            if (lower ? hcol[t] < i : hcol[t] > i) {
                tcol[k] = hcol[t];
                tsrc[k] = t;
                ++k;
            }
    }
    uptr[urow.size()] = (int32_t)k;
    SS_TRY(dev_alloc_n(ctx, &T.order, order.size()));
    SS_TRY(dev_alloc_n(ctx, &T.urow, urow.size()));
    SS_TRY(dev_alloc_n(ctx, &T.uptr, uptr.size()));
    SS_TRY(dev_alloc_n(ctx, &T.col, tcol.size()));
    SS_TRY(dev_alloc_n(ctx, &T.src, tsrc.size()));
    SS_CUDA(ctx, cudaMemcpyAsync(T.order, order.data(), sizeof(int32_t) * order.size(), cudaMemcpyHostToDevice,
                                 ctx->stream));
    SS_CUDA(ctx, cudaMemcpyAsync(T.urow, urow.data(), sizeof(int32_t) * urow.size(), cudaMemcpyHostToDevice,
                                 ctx->stream));
    SS_CUDA(ctx, cudaMemcpyAsync(T.uptr, uptr.data(), sizeof(int32_t) * uptr.size(), cudaMemcpyHostToDevice,
                                 ctx->stream));
    if (nnz_t) {
        SS_CUDA(ctx, cudaMemcpyAsync(T.col, tcol.data(), sizeof(int32_t) * tcol.size(), cudaMemcpyHostToDevice,
                                     ctx->stream));
        SS_CUDA(ctx, cudaMemcpyAsync(T.src, tsrc.data(), sizeof(int32_t) * tsrc.size(), cudaMemcpyHostToDevice,
                                     ctx->stream));
    }
    SS_CUDA(ctx, cudaStreamSynchronize(ctx->stream));     // the host vectors go out of scope
    return SS_OK;
}

__global__ void gather_values(const double2* __restrict__ f, const int32_t* __restrict__ src, int64_t nnz,
                              double2* __restrict__ v, float2* __restrict__ v32) {
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < nnz; k += (int64_t)gridDim.x * blockDim.x) {
        const double2 a = f[src[k]];
        v[k] = a;
        if (v32) v32[k] = make_float2((float)a.x, (float)a.y);
    }
}

__global__ void gather_dinv(const double2* __restrict__ inv, const int32_t* __restrict__ urow, int64_t slots,
                            double2* __restrict__ d, float2* __restrict__ d32) {
    for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < slots; s += (int64_t)gridDim.x * blockDim.x) {
        const int32_t i = urow[s];
        const double2 a = i >= 0 ? inv[i] : make_double2(0.0, 0.0);
        d[s] = a;
        if (d32) d32[s] = make_float2((float)a.x, (float)a.y);
    }
}

// Values of one triangle in unit order (FP64, and FP32 when asked), and for
// the upper triangle 1 / u_ii per slot, from the combined factors.
ss_status pack_triangle(ss_ctx ctx, ss_prec M, TriLevels& T, bool upper, bool fp32) {
    const int64_t slots = T.n_units * (32 / T.g);
    if (!T.val) SS_TRY(dev_alloc_n(ctx, &T.val, (size_t)T.nnz));
    if (fp32 && !T.val32) SS_TRY(dev_alloc_n(ctx, &T.val32, (size_t)T.nnz));
    if (T.nnz)
        gather_values<<<(ss_count_launch(), std::min<unsigned>(grid_for(T.nnz, 256), 4096)), 256, 0, ctx->stream>>>(
            M->f.val, T.src, T.nnz, T.val, fp32 ? T.val32 : nullptr);
    if (upper) {
        if (!T.dinv) SS_TRY(dev_alloc_n(ctx, &T.dinv, (size_t)slots));
        if (fp32 && !T.dinv32) SS_TRY(dev_alloc_n(ctx, &T.dinv32, (size_t)slots));
        if (slots)
            gather_dinv<<<(ss_count_launch(), std::min<unsigned>(grid_for(slots, 256), 4096)), 256, 0, ctx->stream>>>(
                M->inv_diag, T.urow, slots, T.dinv, fp32 ? T.dinv32 : nullptr);
    }
    SS_CUDA(ctx, cudaGetLastError());
    return SS_OK;
}

void free_triangle(ss_ctx ctx, TriLevels& T) {
    dev_free(ctx, T.order);
    dev_free(ctx, T.urow);
    dev_free(ctx, T.uptr);
    dev_free(ctx, T.col);
    dev_free(ctx, T.src);
    dev_free(ctx, T.val);
    dev_free(ctx, T.val32);
    dev_free(ctx, T.dinv);
    dev_free(ctx, T.dinv32);
    T = TriLevels();
}

}  // namespace

// Host level analysis of the factor pattern, device buffers of the solves.
static ss_status analyse(ss_ctx ctx, ss_prec M, const std::vector<int32_t>& hrp, const std::vector<int32_t>& hcol,
                         std::vector<int32_t>& lower_order, std::vector<int32_t>& lower_ptr) {
    const int64_t n = M->f.n_rows;
    std::vector<int32_t> upper_order, upper_ptr;
    int32_t nl = level_sets_host(n, hrp.data(), hcol.data(), true, lower_order, lower_ptr);
    int32_t nu = level_sets_host(n, hrp.data(), hcol.data(), false, upper_order, upper_ptr);
    SS_TRY(build_triangle(ctx, lower_order, lower_ptr, nl, true, hrp, hcol, M->lower));
    SS_TRY(build_triangle(ctx, upper_order, upper_ptr, nu, false, hrp, hcol, M->upper));
    SS_TRY(dev_alloc_n(ctx, &M->err, 1));
    SS_TRY(dev_alloc_n(ctx, &M->tickets, 2));
    SS_TRY(dev_alloc_n(ctx, &M->tmp, (size_t)n));
    fill_pending<double2><<<(ss_count_launch(), 256), 256, 0, ctx->stream>>>(n, M->tmp);
    SS_CUDA(ctx, cudaMemsetAsync(M->err, 0, sizeof(int), ctx->stream));
    SS_CUDA(ctx, cudaMemsetAsync(M->tickets, 0, 2 * sizeof(unsigned long long), ctx->stream));
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
        SS_TRY(dev_alloc_n(ctx, &M->tmp32, (size_t)n));
        fill_pending<float2><<<(ss_count_launch(), 256), 256, 0, ctx->stream>>>(n, M->tmp32);
    }
    make_inv_diag<<<(ss_count_launch(), grid_for(n, 256)), 256, 0, ctx->stream>>>(M->f.val, M->diag_pos, n,
                                                                                    M->inv_diag, nullptr, M->err);
    M->fp32 = want_fp32;
    SS_TRY(pack_triangle(ctx, M, M->lower, false, want_fp32));
    SS_TRY(pack_triangle(ctx, M, M->upper, true, want_fp32));
    SS_CUDA(ctx, cudaGetLastError());
    int herr = 0;
    SS_CUDA(ctx, cudaMemcpyAsync(&herr, M->err, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
    SS_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    if (herr == 2) return set_error(ctx, SS_ZERO_PIVOT, "incomplete LU met a zero pivot");
    if (herr) return set_error(ctx, SS_ERR_TIMEOUT, "device wait timed out");
    return SS_OK;
}

template <bool LOWER, int G, class T>
static ss_status launch_trsv_g(ss_ctx ctx, const TriLevels& L, TrsvArgs<T> a, int64_t n) {
    if ((size_t)n * sizeof(T) <= TRSV_BLOCK_MAX_BYTES) {
        // FP64: one entry per lane per step (a padding lane still holds the FP64
        // pipe for a whole warp instruction, and this path is a latency chain)
        auto kern = sptrsv_block<LOWER, G, sizeof(T) == 16 ? 1 : TRSV_K, T>;
        const size_t bytes = std::max<size_t>((size_t)n * sizeof(T), 16);
        SS_CUDA(ctx, cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
        kern<<<(ss_count_launch(), 1), TRSV_BLOCK_THREADS, bytes, ctx->stream>>>(a, n);
        return SS_OK;
    }
    constexpr int wpb = TRSV_THREADS / 32;
    const int64_t blocks = (L.n_units + wpb - 1) / wpb;
    sptrsv_syncfree<LOWER, G, TRSV_K, T><<<(ss_count_launch(), (unsigned)std::max<int64_t>(1, blocks)), TRSV_THREADS, 0,
                                          ctx->stream>>>(a);
    return SS_OK;
}

template <bool LOWER, class T>
static ss_status launch_trsv(ss_ctx ctx, ss_prec M, TriLevels& L, const T* vals, const T* dinv, const T* b, T* x,
                             T* other, const int* halt) {
    TrsvArgs<T> a;
    a.urow = L.urow;
    a.uptr = L.uptr;
    a.col = L.col;
    a.val = vals;
    a.dinv = dinv;
    a.n_units = L.n_units;
    a.b = b;
    a.x = x;
    a.other = other;
    a.err = M->err;
    a.ticket = M->tickets + (LOWER ? 0 : 1);
    a.halt = halt;
    a.wait_ns = ctx->wait_ns;
    switch (L.g) {
        case 2: return launch_trsv_g<LOWER, 2, T>(ctx, L, a, M->f.n_rows);
        case 4: return launch_trsv_g<LOWER, 4, T>(ctx, L, a, M->f.n_rows);
        case 8: return launch_trsv_g<LOWER, 8, T>(ctx, L, a, M->f.n_rows);
        case 16: return launch_trsv_g<LOWER, 16, T>(ctx, L, a, M->f.n_rows);
        default: return launch_trsv_g<LOWER, 32, T>(ctx, L, a, M->f.n_rows);
    }
}

// z = U^{-1} L^{-1} r.  tmp (the lower solve's output) is all PENDING between
// applications; the lower solve marks z PENDING and the upper solve restores
// tmp.  r and z must not alias.
template <class T>
static ss_status apply_impl(ss_ctx ctx, ss_prec M, const T* lv, const T* uv, const T* ud, T* tmp, const T* r, T* z,
                            const int* halt) {
    const int64_t n = M->f.n_rows;
    if (n == 0) return SS_OK;
    {
        ProfScope ps(ctx, PROF_TRSV_LOWER);
        SS_TRY((launch_trsv<true, T>(ctx, M, M->lower, lv, nullptr, r, tmp, z, halt)));
    }
    {
        ProfScope ps(ctx, PROF_TRSV_UPPER);
        SS_TRY((launch_trsv<false, T>(ctx, M, M->upper, uv, ud, tmp, z, tmp, halt)));
    }
    SS_CUDA(ctx, cudaGetLastError());
    return SS_OK;
}

ss_status prec_apply_dev(ss_ctx ctx, ss_prec M, const double2* r, double2* z, const int* halt) {
    return apply_impl<double2>(ctx, M, M->lower.val, M->upper.val, M->upper.dinv, M->tmp, r, z, halt);
}

ss_status prec_apply_dev32(ss_ctx ctx, ss_prec M, const float2* r, float2* z, const int* halt) {
    if (!M->fp32) return set_error(ctx, SS_ERR_INVALID, "preconditioner has no FP32 factors");
    return apply_impl<float2>(ctx, M, M->lower.val32, M->upper.val32, M->upper.dinv32, M->tmp32, r, z, halt);
}

// After a wait gave up, the intermediate vectors no longer hold the PENDING
// mark everywhere: they are re-marked (and the error word cleared) so that
// the next application starts from the invariant again.
ss_status prec_check_error(ss_ctx ctx, ss_prec M) {
    int herr = 0;
    SS_CUDA(ctx, cudaMemcpyAsync(&herr, M->err, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
    SS_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    if (herr == 1) {
        const int64_t n = M->f.n_rows;
        fill_pending<double2><<<(ss_count_launch(), 256), 256, 0, ctx->stream>>>(n, M->tmp);
        if (M->tmp32) fill_pending<float2><<<(ss_count_launch(), 256), 256, 0, ctx->stream>>>(n, M->tmp32);
        SS_CUDA(ctx, cudaMemsetAsync(M->err, 0, sizeof(int), ctx->stream));
        SS_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
        return set_error(ctx, SS_ERR_TIMEOUT, "triangular solve wait timed out");
    }
    return SS_OK;
}

void prec_destroy(ss_ctx ctx, ss_prec M) {
    free_csr(ctx, M->f);
    dev_free(ctx, M->diag_pos);
    dev_free(ctx, M->inv_diag);
    free_triangle(ctx, M->lower);
    free_triangle(ctx, M->upper);
    dev_free(ctx, M->err);
    dev_free(ctx, M->tickets);
    dev_free(ctx, M->tmp);
    dev_free(ctx, M->tmp32);
}

// ------------------------------------------------------------ diagnostics

ss_status prec_skip_row(ss_ctx ctx, ss_prec M, int64_t row, int restore) {
    TriLevels& T = M->lower;
    const int64_t slots = T.n_units * (32 / T.g);
    if (restore) {
        if (M->skipped_slot < 0) return SS_OK;
        SS_CUDA(ctx, cudaMemcpyAsync(T.urow + M->skipped_slot, &M->skipped_row, sizeof(int32_t),
                                     cudaMemcpyHostToDevice, ctx->stream));
        SS_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
        M->skipped_slot = -1;
        return SS_OK;
    }
    if (M->skipped_slot >= 0) return set_error(ctx, SS_ERR_INVALID, "a row is already skipped");
    std::vector<int32_t> urow((size_t)slots);
    SS_CUDA(ctx, cudaMemcpyAsync(urow.data(), T.urow, sizeof(int32_t) * slots, cudaMemcpyDeviceToHost, ctx->stream));
    SS_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    for (int64_t sl = 0; sl < slots; ++sl)
        if (urow[sl] == row) {
            const int32_t none = -1;
            SS_CUDA(ctx, cudaMemcpyAsync(T.urow + sl, &none, sizeof(int32_t), cudaMemcpyHostToDevice, ctx->stream));
            SS_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
            M->skipped_slot = sl;
            M->skipped_row = (int32_t)row;
            return SS_OK;
        }
    return set_error(ctx, SS_ERR_INVALID, "row out of range");
}
