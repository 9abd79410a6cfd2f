// Per-system persistent solver for many small Liouvillians (one CTA per
// system at a time).  Everything one Krylov iteration needs runs inside the
// CTA: the SpMV, the two triangular solves of M^{-1} (section "Iterative
// solvers"), the inner products and the vector updates.
//
// Triangular solves work in place on one shared-memory vector, one level at a
// time with a barrier between levels: rows are grouped into level-aligned
// units of 32/G rows (G lanes per row) stored in a packed lane-major layout
// (one coalesced load per unit and entry slot), and each warp loads its unit
// of the next level before the barrier.  Nothing in the kernel waits on a
// flag.
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

// Block-wide sums of NV values (A = float or double), returned in double to
// every thread.  Warp sums by shuffles, then warp 0 adds the NW warp sums in a
// fixed order and broadcasts them through shared memory (the FP64 pipe is
// scarce on GB300: the final sum is done once, not by every thread).
template <int NV, class A>
__device__ void cta_sum(A (&v)[NV], double (&out)[NV], double* red) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < NV; ++k)
        for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_down_sync(FULLM, v[k], o);
    if (lane == 0)
#pragma unroll
        for (int k = 0; k < NV; ++k) red[w * NV + k] = (double)v[k];
    __syncthreads();
    if (w == 0) {
#pragma unroll
        for (int k = 0; k < NV; ++k) {
            double t = lane < NW ? red[lane * NV + k] : 0.0;
            for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(FULLM, t, o);
            if (lane == 0) red[NW * NV + k] = t;
        }
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < NV; ++k) out[k] = red[NW * NV + k];
    __syncthreads();
}

template <int NV>
__device__ void cta_sum(double (&v)[NV], double* red) {
    double out[NV];
    cta_sum<NV, double>(v, out, red);
#pragma unroll
    for (int k = 0; k < NV; ++k) v[k] = out[k];
}

// Accumulator type of the inner products: the vector type's real type (the
// FP32 inner solve accumulates each thread's share in FP32).
template <class T> struct Acc;
template <> struct Acc<double2> { using type = double; };
template <> struct Acc<float2> { using type = float; };

__device__ __forceinline__ bool negligible(double2 a, double nu, double nv) {
    double m = hypot(a.x, a.y);
    return m == 0.0 || m < 1e-15 * nu * nv;
}

// ------------------------------------------------------ triangular solves
constexpr int MAXE = BATCH_MAXE;    // packed entries per lane and unit
constexpr int RING_MAX = BATCH_RING_MAX;    // shared-memory slots of the level ring, at most

// One unit of a packed operand held in registers (a lane's slots, the row
// and its CSR tail).
template <class T>
struct UnitRegs {
    int32_t jj[MAXE];
    T vv[MAXE];
    int32_t i, ob, oe;
    T dv;                           // upper triangle: 1 / u_ii of the lane's row (packed, prefetched with the unit)
};

template <class T>
__host__ __device__ __forceinline__ int dinv_stride(int R);

// with_dinv: also fetch the row's 1 / u_ii from the packed upper operand, so
// that no global load stays on the critical path of an upper level.
template <int G, class T>
__device__ __forceinline__ void load_unit(const PackedOp& P, int32_t u, int lane, UnitRegs<T>& r,
                                          bool with_dinv = false) {
    constexpr int R = 32 / G;
    const T* __restrict__ pv = reinterpret_cast<const T*>(P.val);
    const int E = P.E;
    const int grp = lane / G;
    r.i = -1;
    r.ob = r.oe = 0;
    r.dv = zero<T>();
#pragma unroll
    for (int q = 0; q < MAXE; ++q) {
        r.jj[q] = -1;
        r.vv[q] = zero<T>();
    }
    if (u >= P.nunits) return;
    const int4 m = P.meta[u * R + grp];
    r.i = m.x;
    r.ob = m.y;
    r.oe = m.z;
#pragma unroll
    for (int q = 0; q < MAXE; ++q)
        if (q < E) {
            const int64_t slot = ((int64_t)u * E + q) * 32 + lane;
            r.jj[q] = P.col[slot];
            r.vv[q] = pv[slot];
        }
    if (with_dinv && (lane % G) == 0) {
        const int ds = dinv_stride<T>(R) / (int)sizeof(T);
        r.dv = reinterpret_cast<const T*>(P.dinv)[(int64_t)u * ds + grp];
    }
}

// Row update of a triangular solve on the shared vector buf: LOWER:
// x_i = b_i - sum_{j<i} l_ij x_j; UPPER: x_i = (b_i - sum_{j>i} u_ij x_j) / u_ii
// (dinv = 1 / u_ii).  The G lanes of a row split its entries and combine
// them by shuffles; ocol/oval hold the CSR entries of long rows that are not
// packed.
template <bool LOWER, int G, class T>
__device__ __forceinline__ void solve_row(const UnitRegs<T>& cu, T dinv, const int32_t* __restrict__ ocol,
                                          const T* __restrict__ oval, T* buf, int sub) {
    T acc = zero<T>();
#pragma unroll
    for (int q = 0; q < MAXE; ++q)
        if (cu.jj[q] >= 0) acc = fmac(cu.vv[q], buf[cu.jj[q]], acc);
    for (int32_t k = cu.ob + sub; k < cu.oe; k += G) acc = fmac(oval[k], buf[ocol[k]], acc);
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) {
        T other = shd(acc, o);
        acc.x += other.x;
        acc.y += other.y;
    }
    if (cu.i >= 0 && sub == 0) {
        T xi = subc(buf[cu.i], acc);
        if (!LOWER) xi = mulc(xi, dinv);
        buf[cu.i] = xi;
    }
}

// Shared-memory ring that stages the packed units of the next levels of a
// triangular solve with bulk asynchronous copies (TMA), so that the data of a
// level was requested nslots - 1 levels earlier and the critical path of a
// level is shared-memory latency, the arithmetic and one barrier.  One thread
// issues a level's copies (values, columns, row records, inverse diagonal)
// into a slot and arms the slot's mbarrier with their byte count; every
// thread waits on the mbarrier's phase before reading the slot.  Levels are
// numbered across calls (seq), slot = seq mod nslots, phase parity =
// (seq / nslots) mod 2.
struct Ring {
    unsigned char* base;
    uint64_t* bars;                 // nslots "full" mbarriers: the slot's copies have landed (shared)
    uint64_t* empty;                // nslots "empty" mbarriers: the slot's level has been solved (shared)
    int* abort;                     // shared flag: a wait ran out of time
    uint32_t* issued;               // shared: staging sequence numbers issued so far (copies requested)
    int* err;                       // global error word
    int32_t slot_bytes;
    int32_t umax;                   // units per staged level (0: no ring)
    int32_t nslots;                 // slots (2 .. RING_MAX)
    uint32_t seq;                   // levels staged so far by this block
    uint64_t wait_ns;               // limit of every wait on the ring's barriers
    int64_t stall_seq;              // failure-detection aid: the staging of this sequence number arms its
                                    // barrier without issuing the copies (-1: never)
};

struct SlotLayout {
    int32_t col, meta, dinv;        // byte offsets inside a slot (values at 0)
};

// Bytes of one unit's inverse diagonal (R values, padded to 16 bytes).
template <class T>
__host__ __device__ __forceinline__ int dinv_stride(int R) {
    return (R * (int)sizeof(T) + 15) & ~15;
}

template <class T>
__host__ __device__ __forceinline__ SlotLayout slot_layout(int E, int R, int umax) {
    SlotLayout L;
    L.col = umax * E * 32 * (int)sizeof(T);
    L.meta = L.col + umax * E * 32 * 4;
    L.dinv = L.meta + umax * R * 16;
    return L;
}

__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ void named_barrier(int id, int threads) {
    asm volatile("bar.sync %0, %1;\n" ::"r"(id), "r"(threads) : "memory");
}
__device__ __forceinline__ void mbar_arrive_tx(uint64_t* bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, unsigned bytes, uint64_t* bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}
__device__ __forceinline__ uint64_t globaltimer_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Wait for a phase of one of the ring's mbarriers; after rg.wait_ns (2 s by
// default: far beyond any copy; only a fault or a missing copy ends there) the
// block gives up, raises the error word and the abort flag, and later waits
// return at once.
__device__ __forceinline__ void ring_wait_on(const Ring& rg, uint64_t* bar, unsigned parity) {
    if (mbar_try_wait(bar, parity)) return;
    const uint64_t t0 = globaltimer_ns();
    while (!mbar_try_wait(bar, parity)) {
        if (*(volatile int*)rg.abort) return;
        if (globaltimer_ns() - t0 > rg.wait_ns) {
            *(volatile int*)rg.abort = 1;
            atomicExch(rg.err, 1);
            return;
        }
    }
}

__device__ __forceinline__ void ring_wait(const Ring& rg, int slot, unsigned parity) {
    ring_wait_on(rg, rg.bars + slot, parity);
}

// One thread: copies of the first min(units, umax) units of level L into slot.
template <bool LOWER, int G, class T>
__device__ __forceinline__ void stage_level(const PackedOp& P, const int32_t* lvl, int32_t L, const Ring& rg,
                                            int slot, const SlotLayout& sl, uint32_t seq) {
    constexpr int R = 32 / G;
    unsigned char* dst = rg.base + (size_t)slot * rg.slot_bytes;
    uint64_t* bar = rg.bars + slot;
    const int32_t beg = lvl[L];
    const int32_t cnt = min(lvl[L + 1] - beg, rg.umax);
    const int E = P.E;
    const unsigned bv = (unsigned)(cnt * E * 32 * (int)sizeof(T));
    const unsigned bc = (unsigned)(cnt * E * 32 * 4);
    const unsigned bm = (unsigned)(cnt * R * 16);
    const unsigned bd = LOWER ? 0u : (unsigned)(cnt * dinv_stride<T>(R));
    mbar_arrive_tx(bar, bv + bc + bm + bd);
    if (cnt > 0 && (int64_t)seq != rg.stall_seq) {
        bulk_g2s(dst, reinterpret_cast<const char*>(P.val) + (size_t)beg * E * 32 * sizeof(T), bv, bar);
        bulk_g2s(dst + sl.col, P.col + (size_t)beg * E * 32, bc, bar);
        bulk_g2s(dst + sl.meta, P.meta + (size_t)beg * R, bm, bar);
        if (!LOWER)
            bulk_g2s(dst + sl.dinv, reinterpret_cast<const char*>(P.dinv) + (size_t)beg * dinv_stride<T>(R), bd, bar);
    }
}

// In-place level-scheduled triangular solve on the shared vector buf: the
// units of a level are spread over the warps and a barrier separates levels,
// so every dependency of a row is complete when its level starts and nothing
// waits on a flag.  lvl: first unit of each level (nlev + 1 entries).
// Warp specialisation: the last warp only stages levels into the ring (it
// runs ahead until every slot is full, refilling a slot once its level has
// been solved); the other NW - 1 warps solve, separated per level by a named
// barrier that the staging warp does not join.
constexpr int CONSUMERS = (NW - 1) * 32;

template <bool LOWER, int G, class T>
__device__ void cta_trsv_ring(const PackedOp& P, const int32_t* lvl, const int32_t* __restrict__ ocol,
                              const T* __restrict__ oval, const T* __restrict__ inv, T* buf, Ring& rg) {
    constexpr int R = 32 / G;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, sub = lane % G, grp = lane / G;
    const int E = P.E, umax = rg.umax;
    const int32_t nlev = P.nlev;
    const SlotLayout sl = slot_layout<T>(E, R, umax);
    const uint32_t s0 = rg.seq;
    const int ns = rg.nslots;
    const int dstride = dinv_stride<T>(R) / (int)sizeof(T);
    if (warp == NW - 1) {
        if (lane == 0)
            for (int32_t L = 0; L < nlev; ++L) {
                const uint32_t q = s0 + L;
                // before its next use, the slot's previous level must be solved
                if (q >= (uint32_t)ns) ring_wait_on(rg, rg.empty + q % ns, ((q / ns) + 1u) & 1u);
                // after an abandoned wait nothing more is staged: a slot whose copies never
                // came keeps its barrier phase open, and it is not armed a second time
                if (*(volatile int*)rg.abort) break;
                stage_level<LOWER, G, T>(P, lvl, L, rg, q % ns, sl, q);
                *(volatile uint32_t*)rg.issued = q + 1;
            }
        __syncwarp();
    } else {
        const T* sv0 = reinterpret_cast<const T*>(rg.base);
        int32_t beg = lvl[0];
        for (int32_t l = 0; l < nlev; ++l) {
            const uint32_t q = s0 + l;
            const int slot = q % ns;
            const int32_t end = lvl[l + 1], cnt = end - beg;
            // warps without a unit do not read the slot; after an abandoned wait
            // (the block is aborting) the slot's contents are not valid and are not read
            if (warp < cnt && (ring_wait(rg, slot, (q / ns) & 1u), *(volatile int*)rg.abort == 0)) {
                const unsigned char* sb = reinterpret_cast<const unsigned char*>(sv0) + (size_t)slot * rg.slot_bytes;
                const T* sv = reinterpret_cast<const T*>(sb) + lane;
                const int32_t* sc = reinterpret_cast<const int32_t*>(sb + sl.col) + lane;
                const int4* sm4 = reinterpret_cast<const int4*>(sb + sl.meta) + grp;
                const T* sd = reinterpret_cast<const T*>(sb + sl.dinv) + grp;
                for (int32_t u = warp; u < cnt; u += NW - 1) {
                    UnitRegs<T> cu;
                    T dinv = zero<T>();
                    if (u < umax) {
                        const int4 m = sm4[u * R];
#pragma unroll
                        for (int q2 = 0; q2 < MAXE; ++q2) {
                            cu.jj[q2] = q2 < E ? sc[(u * E + q2) * 32] : -1;
                            cu.vv[q2] = q2 < E ? sv[(u * E + q2) * 32] : zero<T>();
                        }
                        cu.i = m.x;
                        cu.ob = m.y;
                        cu.oe = m.z;
                        if (!LOWER) dinv = sd[u * dstride];
                    } else {
                        load_unit<G, T>(P, beg + u, lane, cu);
                        if (!LOWER && cu.i >= 0) dinv = inv[cu.i];
                    }
                    solve_row<LOWER, G, T>(cu, dinv, ocol, oval, buf, sub);
                }
            }
            beg = end;
            named_barrier(1, CONSUMERS);
            if (threadIdx.x == 0) mbar_arrive(rg.empty + slot);      // the slot may be refilled
        }
    }
    __syncthreads();
    rg.seq = s0 + (uint32_t)nlev;
}

// Before a block leaves the kernel after an abandoned wait: wait (bounded)
// for the copies still in flight into the ring.
__device__ void ring_drain(const Ring& rg) {
    if (threadIdx.x != 0 || rg.umax == 0 || !*(volatile int*)rg.abort) return;
    // the last nslots stagings the producer issued (earlier ones were waited for
    // before their slots were reused)
    const uint32_t issued = *(volatile uint32_t*)rg.issued;
    for (int k = 1; k <= rg.nslots; ++k) {
        if (issued < (uint32_t)k) break;
        const uint32_t q = issued - k;
        const uint64_t t0 = globaltimer_ns();
        while (!mbar_try_wait(rg.bars + q % rg.nslots, (q / rg.nslots) & 1u))
            if (globaltimer_ns() - t0 > rg.wait_ns) break;
    }
}

// Without a ring: each warp loads its unit of the next level into registers
// before the barrier of the current one.
template <bool LOWER, int G, class T>
__device__ void cta_trsv_pk(const PackedOp& P, const int32_t* lvl, const int32_t* __restrict__ ocol,
                            const T* __restrict__ oval, const T* __restrict__ inv, T* buf) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, sub = lane % G;
    const bool dv = !LOWER && P.dinv != nullptr;   // packed 1 / u_ii, else from inv[] (global, on the level's path)
    UnitRegs<T> ua, ub;
    int32_t beg = lvl[0], end = lvl[1];
    load_unit<G, T>(P, beg + warp < end ? beg + warp : P.nunits, lane, ua, dv);
    for (int32_t l = 0; l < P.nlev; ++l) {
        const int32_t nb = end, ne = (l + 1 < P.nlev) ? lvl[l + 2] : end;
        load_unit<G, T>(P, nb + warp < ne ? nb + warp : P.nunits, lane, ub, dv);
        solve_row<LOWER, G, T>(ua, LOWER || ua.i < 0 ? zero<T>() : (dv ? ua.dv : inv[ua.i]), ocol, oval, buf, sub);
        for (int32_t u = beg + warp + NW; u < end; u += NW) {      // wide levels: more units per warp
            UnitRegs<T> uc;
            load_unit<G, T>(P, u, lane, uc, dv);
            solve_row<LOWER, G, T>(uc, LOWER || uc.i < 0 ? zero<T>() : (dv ? uc.dv : inv[uc.i]), ocol, oval, buf,
                                   sub);
        }
        __syncthreads();
        ua = ub;
        beg = nb;
        end = ne;
    }
}

template <bool LOWER, int G, class T>
__device__ __forceinline__ void cta_trsv_g(const PackedOp& P, const int32_t* lvl, const int32_t* ocol, const T* oval,
                                           const T* inv, T* buf, Ring& rg) {
    if (rg.umax > 0) cta_trsv_ring<LOWER, G, T>(P, lvl, ocol, oval, inv, buf, rg);
    else cta_trsv_pk<LOWER, G, T>(P, lvl, ocol, oval, inv, buf);
}

template <bool LOWER, class T>
__device__ void cta_trsv(const PackedOp& P, const int32_t* lvl, const int32_t* ocol, const T* oval, const T* inv,
                         T* buf, Ring& rg) {
    switch (P.G) {
        case 1: cta_trsv_g<LOWER, 1, T>(P, lvl, ocol, oval, inv, buf, rg); break;
        case 2: cta_trsv_g<LOWER, 2, T>(P, lvl, ocol, oval, inv, buf, rg); break;
        case 4: cta_trsv_g<LOWER, 4, T>(P, lvl, ocol, oval, inv, buf, rg); break;
        case 8: cta_trsv_g<LOWER, 8, T>(P, lvl, ocol, oval, inv, buf, rg); break;
        case 16: cta_trsv_g<LOWER, 16, T>(P, lvl, ocol, oval, inv, buf, rg); break;
        default: cta_trsv_g<LOWER, 32, T>(P, lvl, ocol, oval, inv, buf, rg); break;
    }
}

// ------------------------------- sync-free triangular solves in one block
// Mixed precision, without a barrier per level.  The output vector is first
// filled with SF_PENDING, a NaN payload that no FP32 arithmetic yields (the
// GPU's arithmetic returns its canonical NaN), and a row reads every value it
// depends on until neither part holds that pattern: a value is its own
// completion flag.  Unit u goes to warp u mod NW and each warp walks its
// units in increasing order.  The units are level ordered, so every
// dependency lies in an earlier unit and no row depends on a row of its own
// unit: the earliest unfinished unit always has its inputs, and the block
// cannot stall.  Waits are bounded all the same (the ring's limit; then the
// abort flag and the error word are raised and the row goes on with zeros).
constexpr uint32_t SF_PENDING = 0xFFBADBADu;

__device__ __forceinline__ float2 sf_pending_value() {
    return make_float2(__uint_as_float(SF_PENDING), __uint_as_float(SF_PENDING));
}
__device__ __forceinline__ float2 sf_load(const float2* p) {
    float2 v;
    asm volatile("ld.volatile.shared.v2.f32 {%0, %1}, [%2];\n" : "=f"(v.x), "=f"(v.y) : "r"(smem_u32(p)));
    return v;
}
__device__ __forceinline__ void sf_store(float2* p, float2 v) {
    asm volatile("st.volatile.shared.v2.f32 [%0], {%1, %2};\n" ::"r"(smem_u32(p)), "f"(v.x), "f"(v.y) : "memory");
}
__device__ __forceinline__ bool sf_pending(float2 v) {
    return __float_as_uint(v.x) == SF_PENDING || __float_as_uint(v.y) == SF_PENDING;
}
// The value at p once it is written, waiting at most rg.wait_ns.
__device__ __forceinline__ float2 sf_wait(const float2* p, const Ring& rg) {
    const uint64_t t0 = globaltimer_ns();
    for (uint32_t spin = 0;; ++spin) {
        const float2 v = sf_load(p);
        if (!sf_pending(v)) return v;
        if ((spin & 63) == 63) {
            if (*(volatile int*)rg.abort) break;
            if (globaltimer_ns() - t0 > rg.wait_ns) {
                *(volatile int*)rg.abort = 1;
                atomicExch(rg.err, 1);
                break;
            }
        }
    }
    return make_float2(0.f, 0.f);
}
__device__ __forceinline__ float2 sf_ready(const float2* p, const Ring& rg) {
    const float2 v = sf_load(p);
    return sf_pending(v) ? sf_wait(p, rg) : v;
}

// One unit's row update: x_i = rhs - sum_j t_ij x_j (times 1 / u_ii for the
// upper triangle), all the row's x_j loads issued before any is tested.
template <bool LOWER, int G>
__device__ __forceinline__ void sf_row(const UnitRegs<float2>& cu, float2 rhs, const int32_t* __restrict__ ocol,
                                       const float2* __restrict__ oval, float2* x, int sub, const Ring& rg) {
    float2 xv[MAXE];
#pragma unroll
    for (int q = 0; q < MAXE; ++q) xv[q] = cu.jj[q] >= 0 ? sf_load(x + cu.jj[q]) : make_float2(0.f, 0.f);
    float2 acc = make_float2(0.f, 0.f);
#pragma unroll
    for (int q = 0; q < MAXE; ++q)
        if (cu.jj[q] >= 0) {
            if (sf_pending(xv[q])) xv[q] = sf_wait(x + cu.jj[q], rg);
            acc = fmac(cu.vv[q], xv[q], acc);
        }
    for (int32_t k = cu.ob + sub; k < cu.oe; k += G) acc = fmac(oval[k], sf_ready(x + ocol[k], rg), acc);
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) {
        const float2 other = shd(acc, o);
        acc.x += other.x;
        acc.y += other.y;
    }
    if (cu.i >= 0 && sub == 0) {
        float2 xi = subc(rhs, acc);
        if (!LOWER) xi = mulc(xi, cu.dv);
        sf_store(x + cu.i, xi);
    }
}

// T x = rhs into x (filled with SF_PENDING and synchronised by the caller);
// rhs is in shared memory.  Lower: rhs is complete when the solve starts.
// Upper: rhs is the lower solve's output, waited on like a dependency.  Each
// warp loads its next unit while it solves the current one; nothing on the
// path of a unit waits for a global load.  (Three units in registers, each
// requested two unit solves ahead, put them in local memory: 1,514-1,525
// against 1,964-1,967 solves/s on 608 JC40 systems; bulk L2 prefetches of
// the units three turns ahead, 2,100-2,114 against 2,159-2,175.)
template <bool LOWER, int G>
__device__ void cta_trsv_sfv(const PackedOp& P, const int32_t* __restrict__ ocol, const float2* __restrict__ oval,
                             const float2* __restrict__ inv, const float2* rhs, float2* x, const Ring& rg) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, sub = lane % G;
    const bool dv = !LOWER && P.dinv != nullptr;   // packed 1 / u_ii, else from inv[]
    UnitRegs<float2> ua, ub;
    load_unit<G, float2>(P, warp, lane, ua, dv);
    for (int32_t u = warp; u < P.nunits; u += NW) {
        load_unit<G, float2>(P, u + NW, lane, ub, dv);
        float2 b = make_float2(0.f, 0.f);
        if (ua.i >= 0 && sub == 0) {
            b = LOWER ? sf_load(rhs + ua.i) : sf_ready(rhs + ua.i, rg);
            if (!LOWER && !dv) ua.dv = inv[ua.i];
        }
        sf_row<LOWER, G>(ua, b, ocol, oval, x, sub, rg);
        ua = ub;
    }
}

template <bool LOWER>
__device__ void cta_trsv_sf(const PackedOp& P, const int32_t* ocol, const float2* oval, const float2* inv,
                            const float2* rhs, float2* x, const Ring& rg) {
    switch (P.G) {
        case 1: cta_trsv_sfv<LOWER, 1>(P, ocol, oval, inv, rhs, x, rg); break;
        case 2: cta_trsv_sfv<LOWER, 2>(P, ocol, oval, inv, rhs, x, rg); break;
        case 4: cta_trsv_sfv<LOWER, 4>(P, ocol, oval, inv, rhs, x, rg); break;
        case 8: cta_trsv_sfv<LOWER, 8>(P, ocol, oval, inv, rhs, x, rg); break;
        case 16: cta_trsv_sfv<LOWER, 16>(P, ocol, oval, inv, rhs, x, rg); break;
        default: cta_trsv_sfv<LOWER, 32>(P, ocol, oval, inv, rhs, x, rg); break;
    }
}

// ------------------------------------------------------------------ SpMV
// y = A x with x in shared memory, from the packed operand (consecutive
// units); accumulates <rhat, y> (dots 0, 1) and |y|^2 (dot 2) when rhat is
// given.
constexpr int SPMV_UNROLL = 4;   // units a warp loads before it consumes any
constexpr int VU = 2;            // vector elements a thread loads before it computes
constexpr int MU = 2;            // the same for the FP32 passes that read two or three vectors
constexpr int MU2 = 1;           // and for the FP32 pass that reads six

template <int G, class T, class A>
__device__ void cta_spmv_pk(const PackedOp& P, const int32_t* __restrict__ ocol, const T* __restrict__ oval,
                            const T* xs, T* __restrict__ y, const T* __restrict__ rhat, A (&dots)[3]) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, sub = lane % G;
    for (int32_t base = warp; base < P.nunits; base += NW * SPMV_UNROLL) {
        UnitRegs<T> ur[SPMV_UNROLL];
        T hr[SPMV_UNROLL];
        // every unit's loads first, then the r^ values their row records
        // point to: one round trip for the units instead of one per unit
#pragma unroll
        for (int k = 0; k < SPMV_UNROLL; ++k) load_unit<G, T>(P, base + k * NW, lane, ur[k]);
#pragma unroll
        for (int k = 0; k < SPMV_UNROLL; ++k)
            hr[k] = (rhat && ur[k].i >= 0 && sub == 0) ? rhat[ur[k].i] : zero<T>();
#pragma unroll
        for (int k = 0; k < SPMV_UNROLL; ++k) {
            T acc = zero<T>();
#pragma unroll
            for (int q = 0; q < MAXE; ++q)
                if (ur[k].jj[q] >= 0) acc = fmac(ur[k].vv[q], xs[ur[k].jj[q]], acc);
            for (int32_t kk = ur[k].ob + sub; kk < ur[k].oe; kk += G) acc = fmac(oval[kk], xs[ocol[kk]], acc);
#pragma unroll
            for (int o = G / 2; o > 0; o >>= 1) {
                T other = shd(acc, o);
                acc.x += other.x;
                acc.y += other.y;
            }
            const int32_t r = ur[k].i;
            if (r >= 0 && sub == 0) {
                y[r] = acc;
                if (rhat) {
                    dots[0] += (A)hr[k].x * (A)acc.x + (A)hr[k].y * (A)acc.y;
                    dots[1] += (A)hr[k].x * (A)acc.y - (A)hr[k].y * (A)acc.x;
                    dots[2] += (A)acc.x * (A)acc.x + (A)acc.y * (A)acc.y;
                }
            }
        }
    }
}

template <class T, class A>
__device__ void cta_spmv(const PackedOp& P, const int32_t* ocol, const T* oval, const T* xs, T* y, const T* rhat,
                         A (&dots)[3]) {
    switch (P.G) {
        case 1: cta_spmv_pk<1, T, A>(P, ocol, oval, xs, y, rhat, dots); break;
        case 2: cta_spmv_pk<2, T, A>(P, ocol, oval, xs, y, rhat, dots); break;
        case 4: cta_spmv_pk<4, T, A>(P, ocol, oval, xs, y, rhat, dots); break;
        case 8: cta_spmv_pk<8, T, A>(P, ocol, oval, xs, y, rhat, dots); break;
        case 16: cta_spmv_pk<16, T, A>(P, ocol, oval, xs, y, rhat, dots); break;
        default: cta_spmv_pk<32, T, A>(P, ocol, oval, xs, y, rhat, dots); break;
    }
}

// Packed values of one operand from the CSR values (gathered once per system).
template <class T, class V>
__device__ void cta_pack_values(const PackedOp& P, const V* __restrict__ csr) {
    T* __restrict__ pv = reinterpret_cast<T*>(P.val);
    const int64_t total = (int64_t)P.nunits * P.E * 32;
    for (int64_t s = threadIdx.x; s < total; s += BT) {
        const int32_t k = P.src[s];
        pv[s] = k >= 0 ? cvt<T>(D(csr[k])) : zero<T>();
    }
}

// Inverse diagonal of the upper factor in the packed row order of P (one
// value per unit row; 0 for padding rows).
template <class T>
__device__ void cta_pack_dinv(const PackedOp& P, const T* __restrict__ inv) {
    T* __restrict__ pd = reinterpret_cast<T*>(P.dinv);
    const int R = 32 / P.G, ds = dinv_stride<T>(R) / (int)sizeof(T);
    const int64_t total = (int64_t)P.nunits * R;
    for (int64_t s = threadIdx.x; s < total; s += BT) {
        const int32_t r = P.meta[s].x;
        pd[(s / R) * ds + s % R] = r >= 0 ? inv[r] : zero<T>();
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
    T* buf2;                    // shared: n, the lower solve's output of the sync-free solves (null: level barriers)
    T* buf3;                    // shared: n, the lower solve's right-hand side of the sync-free solves
    double* red;                // shared reduction scratch
    const int32_t* lvl_lo;      // level boundaries of the two triangles (shared, or global)
    const int32_t* lvl_up;
    Ring* ring;
};

// Dynamic shared memory of one system: the solve vector, the level
// boundaries of both triangles (when they fit) and the level ring.
struct SmemPlan {
    unsigned char* buf;
    unsigned char* pbuf;        // mixed precision: p^ (null: kept in global memory)
    unsigned char* buf2;        // mixed precision, sync-free solves: the lower solve's output (else null)
    unsigned char* buf3;        // and its right-hand side
    const int32_t* lvl_lo;
    const int32_t* lvl_up;
    Ring ring;
};

// out = M^{-1} in; the result also stays in the shared buffer
template <class T>
__device__ void cta_prec(Ctx<T>& c, const T* in, T* out) {
    const BatchSys& S = *c.S;
    for (int32_t i = threadIdx.x; i < c.n; i += BT) c.buf[i] = in[i];
    __syncthreads();
    cta_trsv<true, T>(S.lo, c.lvl_lo, S.f_col, c.fval, c.finv, c.buf, *c.ring);
    cta_trsv<false, T>(S.up, c.lvl_up, S.f_col, c.fval, c.finv, c.buf, *c.ring);
    for (int32_t i = threadIdx.x; i < c.n; i += BT) out[i] = c.buf[i];
    // no barrier needed: the shared buffer is only read afterwards
}

// M^{-1} applied in place to the shared buffer, which the caller has filled
// (and synchronised); the result stays there and is also copied to out when
// out is not null (out may be shared or global memory).
template <class T>
__device__ void cta_prec_staged(Ctx<T>& c, T* out) {
    const BatchSys& S = *c.S;
    cta_trsv<true, T>(S.lo, c.lvl_lo, S.f_col, c.fval, c.finv, c.buf, *c.ring);
    cta_trsv<false, T>(S.up, c.lvl_up, S.f_col, c.fval, c.finv, c.buf, *c.ring);
    if (out)
        for (int32_t i = threadIdx.x; i < c.n; i += BT) out[i] = c.buf[i];
}

// Mixed precision, sync-free: L y = b into buf2 (b in buf3), then U z = y
// into buf, each without level barriers; z stays in buf and is also copied to
// out when out is not null.  The caller's pass has written b to buf3, filled
// buf and buf2 with SF_PENDING and synchronised.
__device__ void cta_prec_sf(Ctx<float2>& c, float2* out) {
    const BatchSys& S = *c.S;
    cta_trsv_sf<true>(S.lo, S.f_col, c.fval, c.finv, c.buf3, c.buf2, *c.ring);
    cta_trsv_sf<false>(S.up, S.f_col, c.fval, c.finv, c.buf2, c.buf, *c.ring);
    __syncthreads();
    if (out)
        for (int32_t i = threadIdx.x; i < c.n; i += BT) out[i] = c.buf[i];
}

struct KResult {
    int status, iters;
    double resid;
};

// Right-preconditioned BiCGSTAB on A x = b (x holds the initial guess),
// stopping at ||b - A x||_2 <= tol.  Same steps and stop/breakdown rules as
// the multi-kernel solver.
// re(conj(a) b), im(conj(a) b) and |b|^2 in the accumulator type
template <class T, class A>
__device__ __forceinline__ void acc_dot(const T& a, const T& b, A& re, A& im) {
    re += (A)a.x * (A)b.x + (A)a.y * (A)b.y;
    im += (A)a.x * (A)b.y - (A)a.y * (A)b.x;
}
template <class T, class A>
__device__ __forceinline__ A norm2(const T& a) {
    return (A)a.x * (A)a.x + (A)a.y * (A)a.y;
}

// Right-preconditioned BiCGSTAB on A x = b (x holds the initial guess),
// stopping at ||b - A x||_2 <= tol.  Same steps and stop/breakdown rules as
// the multi-kernel solver.  Each thread accumulates its share of an inner
// product in the vector's precision; the block sums and the scalars are FP64.
template <class T>
__device__ KResult cta_bicgstab(Ctx<T>& c, T* x, const T* b, T* wk, double tol, int maxiter) {
    using A = typename Acc<T>::type;
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
    A dz[3] = {0, 0, 0};
    cta_spmv<T>(S.pa, S.a_col, c.aval, c.buf, v, nullptr, dz);
    __syncthreads();
    A nr[1] = {0};
    for (int32_t i = threadIdx.x; i < n; i += BT) {
        T ri = subc(b[i], v[i]);
        r[i] = ri;
        rhat[i] = ri;
        nr[0] += norm2<T, A>(ri);
    }
    double nrs[1];
    cta_sum<1, A>(nr, nrs, c.red);
    double rn = sqrt(nrs[0]);
    res.resid = rn;
    if (rn <= tol) { res.status = SS_OK; return res; }
    const double rhat_norm = rn;
    double2 rho = make_double2(nrs[0], 0.0), alpha = make_double2(1, 0), omega = make_double2(1, 0),
            beta = make_double2(0, 0);
    for (int it = 1; it <= maxiter; ++it) {
        {   // p = r + beta (p - omega v)
            const T bt = cvt<T>(beta), om = cvt<T>(omega);
            for (int32_t i0 = threadIdx.x; i0 < n; i0 += VU * BT) {
                T ra[VU], pa[VU], va[VU];
#pragma unroll
                for (int k = 0; k < VU; ++k) {
                    const int32_t i = i0 + k * BT;
                    if (i < n) { ra[k] = r[i]; pa[k] = p[i]; va[k] = v[i]; }
                }
#pragma unroll
                for (int k = 0; k < VU; ++k) {
                    const int32_t i = i0 + k * BT;
                    if (i < n) p[i] = (it == 1) ? ra[k] : addc(ra[k], mulc(bt, subc(pa[k], mulc(om, va[k]))));
                }
            }
        }
        __syncthreads();
        cta_prec<T>(c, p, phat);
        if (c.ring->umax > 0 && *(volatile int*)c.ring->abort) { res.status = SS_ERR_TIMEOUT; res.iters = it; return res; }
        A dv[3] = {0, 0, 0};
        cta_spmv<T>(S.pa, S.a_col, c.aval, c.buf, v, rhat, dv);
        double dvs[3];
        cta_sum<3, A>(dv, dvs, c.red);
        const double2 rv = make_double2(dvs[0], dvs[1]);
        if (negligible(rv, rhat_norm, sqrt(dvs[2]))) { res.status = SS_BREAKDOWN; res.iters = it - 1; return res; }
        alpha = cdiv(rho, rv);
        A ns[1] = {0};
        {
            const T al = cvt<T>(alpha);
            for (int32_t i0 = threadIdx.x; i0 < n; i0 += VU * BT) {
                T ra[VU], va[VU];
#pragma unroll
                for (int k = 0; k < VU; ++k) {
                    const int32_t i = i0 + k * BT;
                    if (i < n) { ra[k] = r[i]; va[k] = v[i]; }
                }
#pragma unroll
                for (int k = 0; k < VU; ++k) {
                    const int32_t i = i0 + k * BT;
                    if (i < n) {
                        T si = subc(ra[k], mulc(al, va[k]));
                        s[i] = si;
                        ns[0] += norm2<T, A>(si);
                    }
                }
            }
        }
        double nss[1];
        cta_sum<1, A>(ns, nss, c.red);
        const double sn = sqrt(nss[0]);
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
        A dt[3] = {0, 0, 0};
        cta_spmv<T>(S.pa, S.a_col, c.aval, c.buf, t, nullptr, dt);
        __syncthreads();
        A tsd[3] = {0, 0, 0};
        for (int32_t i0 = threadIdx.x; i0 < n; i0 += VU * BT) {
            T ta[VU], sa[VU];
#pragma unroll
            for (int k = 0; k < VU; ++k) {
                const int32_t i = i0 + k * BT;
                if (i < n) { ta[k] = t[i]; sa[k] = s[i]; }
            }
#pragma unroll
            for (int k = 0; k < VU; ++k)
                if (i0 + k * BT < n) {
                    acc_dot<T, A>(ta[k], sa[k], tsd[0], tsd[1]);
                    tsd[2] += norm2<T, A>(ta[k]);
                }
        }
        double tss[3];
        cta_sum<3, A>(tsd, tss, c.red);
        if (tss[2] == 0.0) { res.status = SS_BREAKDOWN; res.iters = it; return res; }
        omega = make_double2(tss[0] / tss[2], tss[1] / tss[2]);
        A nr2[3] = {0, 0, 0};
        {
            const T al = cvt<T>(alpha), om = cvt<T>(omega);
            for (int32_t i0 = threadIdx.x; i0 < n; i0 += VU * BT) {
                T xa[VU], pa[VU], sa[VU], sha[VU], ta[VU], ha[VU];
#pragma unroll
                for (int k = 0; k < VU; ++k) {
                    const int32_t i = i0 + k * BT;
                    if (i < n) { xa[k] = x[i]; pa[k] = phat[i]; sha[k] = shat[i]; sa[k] = s[i]; ta[k] = t[i]; ha[k] = rhat[i]; }
                }
#pragma unroll
                for (int k = 0; k < VU; ++k) {
                    const int32_t i = i0 + k * BT;
                    if (i < n) {
                        x[i] = addc(xa[k], addc(mulc(al, pa[k]), mulc(om, sha[k])));
                        T ri = subc(sa[k], mulc(om, ta[k]));
                        r[i] = ri;
                        acc_dot<T, A>(ha[k], ri, nr2[0], nr2[1]);
                        nr2[2] += norm2<T, A>(ri);
                    }
                }
            }
        }
        double nrs2[3];
        cta_sum<3, A>(nr2, nrs2, c.red);
        rn = sqrt(nrs2[2]);
        res.iters = it;
        res.resid = rn;
        if (rn <= tol) { res.status = SS_OK; return res; }
        if (omega.x == 0.0 && omega.y == 0.0) { res.status = SS_BREAKDOWN; return res; }
        if (it >= maxiter) { res.status = SS_NOT_CONVERGED; return res; }
        const double2 rho_new = make_double2(nrs2[0], nrs2[1]);
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

// IKJ elimination restricted to the pattern, level by level, from the
// elimination schedule (no column search): a row's pivots in ascending
// order, l_ik = a_ik / u_kk (as a_ik times the stored 1 / u_kk), then
// a_ij -= l_ik u_kj for the entries the schedule lists.  Rows of a level go
// to groups of ILU_GS lanes (32 / ILU_GS rows per warp at a time); a group stages
// its row, the 1 / u_kk of its pivots and the u_kj its updates read in its
// share of the shared memory (free until the solve starts), so the pivot
// chain runs on shared memory; a row too long for the share is eliminated
// in global memory in the same order.  When a row is done its 1 / u_ii is
// stored for the rows of later levels.  Four lanes per row (JC40, 608
// systems: 2,853-2,879 solves/s; 16 lanes 2,738-2,762, 8 lanes 2,818, 2
// lanes 2,829-2,848, one lane 2,765-2,782).
constexpr int ILU_GS = 4;
constexpr int ILU_GROUPS = BT / ILU_GS;

// stage: the shared memory may be used (not while bulk copies of an abandoned
// ring might still land in it).
__device__ bool cta_ilu0(const BatchSys& S, bool mixed, unsigned char* smem, int smem_bytes, bool stage) {
    const int sub = threadIdx.x % ILU_GS, grp = threadIdx.x / ILU_GS;
    const unsigned gmask = ILU_GS == 32 ? FULLM : (((1u << ILU_GS) - 1u) << ((threadIdx.x & 31) & ~(ILU_GS - 1)));
    const int32_t nnz = S.f_rp[S.n];
    double2* val = S.f_val;
    for (int32_t k = threadIdx.x; k < nnz; k += BT) val[k] = S.a_val[k];
    __syncthreads();
    // this group's share: row values, 1 / u_kk per pivot, pivot ranges of the
    // schedule (rebased to the row), and per update its target and u_kj
    const int region = (smem_bytes / ILU_GROUPS) & ~15;
    unsigned char* base = smem + (size_t)grp * region;
    for (int32_t l = 0; l < S.n_levels; ++l) {
        const int32_t lb = S.lvl_ptr[l], le = S.lvl_ptr[l + 1];
        // every group of a warp runs the same number of rounds (the warp's
        // groups meet at __syncwarp), idle groups with no row
        const int32_t rounds = (le - lb + ILU_GROUPS - 1) / ILU_GROUPS;
        for (int32_t rd = 0; rd < rounds; ++rd) {
            const int32_t q = lb + rd * ILU_GROUPS + grp;
            const bool have = q < le;
            int32_t i = 0, rb = 0, re = 0, di = 0, ub = 0, ue = 0;
            if (have) {
                i = S.lvl_rows[q];
                rb = S.f_rp[i];
                re = S.f_rp[i + 1];
                di = S.f_dpos[i];
                ub = S.ilu_ptr[rb];
                ue = S.ilu_ptr[di];
            }
            const int32_t len = re - rb, npiv = di - rb, np = ue - ub;
            const size_t need = (size_t)len * 32 + (size_t)(npiv + 1) * 4 + (size_t)np * 20 + 64;
            const bool staged = stage && have && need <= (size_t)region;
            double2* rv = reinterpret_cast<double2*>(base);                 // len
            double2* pinv = rv + len;                                        // npiv
            double2* uval = pinv + npiv;                                     // np
            int32_t* tptr = reinterpret_cast<int32_t*>(uval + np);           // npiv + 1
            int32_t* utgt = tptr + npiv + 1;                                 // np
            if (staged) {
                for (int32_t e = sub; e < len; e += ILU_GS) {
                    rv[e] = val[rb + e];
                    if (e < npiv) pinv[e] = S.f_inv[S.f_col[rb + e]];
                }
                for (int32_t e = sub; e <= npiv; e += ILU_GS) tptr[e] = S.ilu_ptr[rb + e] - ub;
                for (int32_t p = sub; p < np; p += ILU_GS) {
                    utgt[p] = S.ilu_tgt[ub + p];
                    uval[p] = val[S.ilu_src[ub + p]];
                }
            }
            __syncwarp();
            const int32_t pmax = __reduce_max_sync(FULLM, have ? npiv : 0);
            for (int32_t t = 0; t < pmax; ++t) {
                // every lane of the group reads a_it; l_it replaces it after the
                // warp has met (the updates only touch entries after t)
                double2 f = make_double2(0.0, 0.0);
                if (t < npiv) {
                    if (staged) {
                        f = cmul(rv[t], pinv[t]);
                        for (int32_t p = tptr[t] + sub; p < tptr[t + 1]; p += ILU_GS) {
                            const int32_t tg = utgt[p];
                            if (tg < len) rv[tg] = csub(rv[tg], cmul(f, uval[p]));
                        }
                    } else {
                        f = cmul(val[rb + t], S.f_inv[S.f_col[rb + t]]);
                        for (int32_t p = S.ilu_ptr[rb + t] + sub; p < S.ilu_ptr[rb + t + 1]; p += ILU_GS) {
                            const int32_t tg = rb + S.ilu_tgt[p];
                            val[tg] = csub(val[tg], cmul(f, val[S.ilu_src[p]]));
                        }
                    }
                }
                __syncwarp();
                if (t < npiv && sub == 0) {
                    if (staged) rv[t] = f;
                    else val[rb + t] = f;
                }
            }
            __syncwarp();
            if (staged)
                for (int32_t e = sub; e < len; e += ILU_GS) val[rb + e] = rv[e];
            __syncwarp(gmask);
            if (have && sub == 0) {
                const double2 dg = staged ? rv[npiv] : val[di];
                S.f_inv[i] = (dg.x == 0.0 && dg.y == 0.0) ? make_double2(0.0, 0.0) : cdiv(make_double2(1.0, 0.0), dg);
            }
            __syncwarp();
        }
        __syncthreads();
    }
    __shared__ int zero_pivot;
    if (threadIdx.x == 0) zero_pivot = 0;
    __syncthreads();
    for (int32_t i = threadIdx.x; i < S.n; i += BT) {
        const double2 dg = val[S.f_dpos[i]];
        if (dg.x == 0.0 && dg.y == 0.0) zero_pivot = 1;
        if (mixed) {
            const double2 r = S.f_inv[i];
            S.f_inv32[i] = make_float2((float)r.x, (float)r.y);
        }
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
// Initial iterate x (FP64, permuted order): zero, or with a warm start the
// caller's rho (natural column-major order, in rho_out) scaled to unit trace,
// the normalisation the solution of Eq. (linear) has.  A guess of zero trace
// gives the zero start.
__device__ void cta_initial_guess(const BatchSys& S, bool warm, double2* x, double* red) {
    double tr[2] = {0.0, 0.0};
    if (warm) {
        for (int32_t i = threadIdx.x; i < S.d; i += BT) {
            const double2 v = S.rho_out[(int64_t)i * (S.d + 1)];
            tr[0] += v.x;
            tr[1] += v.y;
        }
        cta_sum<2>(tr, red);
    }
    const bool use = warm && (tr[0] != 0.0 || tr[1] != 0.0);
    const double2 t = make_double2(tr[0], tr[1]);
    for (int32_t r = threadIdx.x; r < S.n; r += BT)
        x[r] = use ? cdiv(S.rho_out[S.perm[r]], t) : make_double2(0.0, 0.0);
    __syncthreads();
}

__device__ void solve_fp64(BatchSys& S, const BatchParams& P, SmemPlan& sm, double* red) {
    const int32_t n = S.n;
    Ctx<double2> c;
    c.S = &S;
    c.n = n;
    c.aval = S.a_val;
    c.fval = S.f_val;
    c.finv = S.f_inv;
    c.buf = reinterpret_cast<double2*>(sm.buf);
    c.buf2 = nullptr;
    c.buf3 = nullptr;
    c.red = red;
    c.lvl_lo = sm.lvl_lo;
    c.lvl_up = sm.lvl_up;
    c.ring = &sm.ring;
    double2* wk = reinterpret_cast<double2*>(S.work);
    double2* b = wk + 8 * (size_t)n;
    double2* x = S.x64;
    for (int32_t i = threadIdx.x; i < n; i += BT) b[i] = make_double2(i == S.r0 ? S.w : 0.0, 0.0);
    cta_initial_guess(S, S.warm != 0, x, red);
    double inner = 0.5 * P.tol, lr = INFINITY;
    int total = 0, status = SS_NOT_CONVERGED;
    for (int pass = 0; pass < 8; ++pass) {
        KResult kr = cta_bicgstab<double2>(c, x, b, wk, inner, P.maxiter - total);
        total += kr.iters;
        double2 tr;
        lr = cta_lrho(S, x, red, &tr);
        if (lr <= P.tol) { status = SS_OK; break; }
        if (total >= P.maxiter || kr.status == SS_NOT_CONVERGED || kr.status == SS_ERR_TIMEOUT ||
            (kr.status == SS_BREAKDOWN && kr.iters == 0)) {
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

// r64 = b - A x64 over the packed A (G lanes per row): the slots' columns
// and CSR positions, then the FP64 values (gathered from the CSR) and the x
// they select, TRU units per warp with their loads in flight together; the
// entries of long rows beyond their slots come from the CSR.  Adds |r_i|^2
// of this thread's rows to nrm.
constexpr int TRU = 2;

template <int G>
__device__ void cta_residual_pk(const BatchSys& S, const double2* __restrict__ x64, double2* __restrict__ r64,
                                float2* __restrict__ r32, double& nrm) {
    const PackedOp& P = S.pa;
    constexpr int R = 32 / G;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, grp = lane / G, sub = lane % G;
    const int E = P.E;
    const double2* __restrict__ av = S.a_val;
    const int32_t* __restrict__ ac = S.a_col;
    for (int32_t base = warp; base < P.nunits; base += NW * TRU) {
        int4 m[TRU];
        int32_t jj[TRU][MAXE], kk[TRU][MAXE];
#pragma unroll
        for (int t = 0; t < TRU; ++t) {
            const int32_t u = base + t * NW;
            m[t] = make_int4(-1, 0, 0, 0);
#pragma unroll
            for (int q = 0; q < MAXE; ++q) jj[t][q] = kk[t][q] = -1;
            if (u < P.nunits) {
                m[t] = P.meta[u * R + grp];
#pragma unroll
                for (int q = 0; q < MAXE; ++q)
                    if (q < E) {
                        const int64_t slot = ((int64_t)u * E + q) * 32 + lane;
                        jj[t][q] = P.col[slot];
                        kk[t][q] = P.src[slot];
                    }
            }
        }
        double2 a[TRU][MAXE], xv[TRU][MAXE];
#pragma unroll
        for (int t = 0; t < TRU; ++t)
#pragma unroll
            for (int q = 0; q < MAXE; ++q) {
                a[t][q] = kk[t][q] >= 0 ? av[kk[t][q]] : zero<double2>();
                xv[t][q] = jj[t][q] >= 0 ? x64[jj[t][q]] : zero<double2>();
            }
#pragma unroll
        for (int t = 0; t < TRU; ++t) {
            double2 acc = zero<double2>();
#pragma unroll
            for (int q = 0; q < MAXE; ++q)
                if (jj[t][q] >= 0) acc = fmac(a[t][q], xv[t][q], acc);
#pragma unroll 4
            for (int32_t k = m[t].y + sub; k < m[t].z; k += G) acc = fmac(av[k], x64[ac[k]], acc);
#pragma unroll
            for (int o = G / 2; o > 0; o >>= 1) {
                const double2 other = shd(acc, o);
                acc.x += other.x;
                acc.y += other.y;
            }
            const int32_t i = m[t].x;
            if (i >= 0 && sub == 0) {
                const double2 y = make_double2((i == S.r0 ? S.w : 0.0) - acc.x, -acc.y);
                r64[i] = y;
                r32[i] = make_float2((float)y.x, (float)y.y);
                nrm += y.x * y.x + y.y * y.y;
            }
        }
    }
}

// True residual in FP64: r64 = b - A x64 (b = w e_r0), r32 = r64 rounded to
// FP32; returns ||r64||_2 and, in *lr, ||L rho||_2 for rho = x64 / tr(x64)
// (L x = b - r64 - w tr(x) e_r0, so no second product is needed).
__device__ double true_residual(const BatchSys& S, const double2* __restrict__ x64, double2* __restrict__ r64,
                                float2* __restrict__ r32, double* red, double* lr) {
    double acc[3] = {0.0, 0.0, 0.0};
    switch (S.pa.G) {
        case 1: cta_residual_pk<1>(S, x64, r64, r32, acc[0]); break;
        case 2: cta_residual_pk<2>(S, x64, r64, r32, acc[0]); break;
        case 4: cta_residual_pk<4>(S, x64, r64, r32, acc[0]); break;
        case 8: cta_residual_pk<8>(S, x64, r64, r32, acc[0]); break;
        case 16: cta_residual_pk<16>(S, x64, r64, r32, acc[0]); break;
        default: cta_residual_pk<32>(S, x64, r64, r32, acc[0]); break;
    }
    for (int32_t i = threadIdx.x; i < S.d; i += BT) {
        const double2 v = x64[S.tidx[i]];
        acc[1] += v.x;
        acc[2] += v.y;
    }
    cta_sum<3>(acc, red);
    const double2 tr = make_double2(acc[1], acc[2]);
    const double2 y0 = r64[S.r0];
    const double2 c0 = make_double2(-y0.x + S.w * (1.0 - tr.x), -y0.y - S.w * tr.y);
    const double l2 = acc[0] - (y0.x * y0.x + y0.y * y0.y) + (c0.x * c0.x + c0.y * c0.y);
    const double m = hypot(tr.x, tr.y);
    *lr = m > 0.0 ? sqrt(fmax(l2, 0.0)) / m : INFINITY;
    return sqrt(acc[0]);
}

// Mixed precision: one BiCGSTAB whose vectors, matrix, factors and inner
// products run in FP32 while the iterate x accumulates in FP64.  Whenever the
// FP32 recursive residual has dropped by DELTA since the last replacement (or
// every REFRESH iterations), it is replaced by the true FP64 residual
// b - A x (reliable updating); the solve stops when the FP64 ||L rho||_2 <= tol.
// A breakdown restarts the recurrence from the current x.  DELTA = 0.2 (JC40,
// 608 systems: 116.8 iterations, 2,144-2,151 solves/s; 0.1: 121.3 and
// 2,127; 0.05: 124.9 and 2,094-2,104; 0.3 and 0.5: 115.6 and 113.7
// iterations, no faster).
constexpr double DELTA = 0.2;
constexpr int REFRESH = 50;

__device__ void solve_mixed(BatchSys& S, const BatchParams& P, SmemPlan& sm, double* red) {
    using T = float2;
    using A = float;
    const int32_t n = S.n;
    Ctx<float2> c;
    c.S = &S;
    c.n = n;
    c.aval = S.a_val32;
    c.fval = S.f_val32;
    c.finv = S.f_inv32;
    c.buf = reinterpret_cast<float2*>(sm.buf);
    c.buf2 = reinterpret_cast<float2*>(sm.buf2);
    c.buf3 = reinterpret_cast<float2*>(sm.buf3);
    const bool sf = c.buf2 != nullptr;
    const float2 pend = sf_pending_value();
    c.red = red;
    c.lvl_lo = sm.lvl_lo;
    c.lvl_up = sm.lvl_up;
    c.ring = &sm.ring;
    T* r = reinterpret_cast<float2*>(S.work);
    T* rhat = r + n;
    T* p = rhat + n;
    T* v = p + n;
    T* s = v + n;
    T* t = s + n;
    T* phat = t + n;
    T* shat = phat + n;
    T* xd = shat + n;            // FP32 increment of x since the last replacement
    T* ph = sm.pbuf ? reinterpret_cast<T*>(sm.pbuf) : phat;     // p^: shared memory when it fits
    double2* x = S.x64;
    double2* r64 = S.r64;
    for (int32_t i = threadIdx.x; i < n; i += BT) xd[i] = make_float2(0.f, 0.f);
    cta_initial_guess(S, S.warm != 0, x, red);
    // x += xd in FP64, xd = 0
    auto fold = [&]() {
        for (int32_t i = threadIdx.x; i < n; i += BT) {
            const T d = xd[i];
            x[i].x += (double)d.x;
            x[i].y += (double)d.y;
            xd[i] = make_float2(0.f, 0.f);
        }
        __syncthreads();
    };
    int it = 0, status = SS_NOT_CONVERGED, restarts = 0, replacements = 0;
    double lr = INFINITY;
    while (it < P.maxiter) {
        // (re)start: true residual, shadow residual r^ = r
        fold();
        double rn = true_residual(S, x, r64, r, red, &lr);
        ++replacements;
        if (lr <= P.tol) { status = SS_OK; break; }
        for (int32_t i = threadIdx.x; i < n; i += BT) rhat[i] = r[i];
        __syncthreads();
        double rhat_norm = rn, rn_ref = rn;
        double2 rho = make_double2(rn * rn, 0.0), alpha = make_double2(1, 0), omega = make_double2(1, 0),
                beta = make_double2(0, 0);
        bool restart = false;
        for (int k = 1; it < P.maxiter; ++k) {
            ++it;
            {   // p = r + beta (p - omega v), written to p and to the solve buffer
                const T bt = cvt<T>(beta), om = cvt<T>(omega);
                for (int32_t i0 = threadIdx.x; i0 < n; i0 += MU * BT) {
                    T ra[MU], pa[MU], va[MU];
#pragma unroll
                    for (int u = 0; u < MU; ++u) {
                        const int32_t i = i0 + u * BT;
                        if (i < n) {
                            ra[u] = r[i];
                            if (k > 1) { pa[u] = p[i]; va[u] = v[i]; }
                        }
                    }
#pragma unroll
                    for (int u = 0; u < MU; ++u) {
                        const int32_t i = i0 + u * BT;
                        if (i < n) {
                            const T pi = (k == 1) ? ra[u] : addc(ra[u], mulc(bt, subc(pa[u], mulc(om, va[u]))));
                            p[i] = pi;
                            if (sf) {
                                c.buf[i] = pend;
                                c.buf2[i] = pend;
                                c.buf3[i] = pi;
                            } else {
                                c.buf[i] = pi;
                            }
                        }
                    }
                }
            }
            __syncthreads();
            if (sf) cta_prec_sf(c, ph);         // p^ = M^{-1} p, kept in ph
            else cta_prec_staged<T>(c, ph);
            if ((sf || c.ring->umax > 0) && *(volatile int*)c.ring->abort) { status = SS_ERR_TIMEOUT; break; }
            A dv[3] = {0, 0, 0};
            cta_spmv<T>(S.pa, S.a_col, c.aval, c.buf, v, rhat, dv);
            double dvs[3];
            cta_sum<3, A>(dv, dvs, c.red);
            const double2 rv = make_double2(dvs[0], dvs[1]);
            if (negligible(rv, rhat_norm, sqrt(dvs[2]))) { restart = true; break; }
            alpha = cdiv(rho, rv);
            {   // s = r - alpha v, written to s and to the solve buffer
                const T al = cvt<T>(alpha);
                for (int32_t i0 = threadIdx.x; i0 < n; i0 += MU * BT) {
                    T ra[MU], va[MU];
#pragma unroll
                    for (int u = 0; u < MU; ++u) {
                        const int32_t i = i0 + u * BT;
                        if (i < n) { ra[u] = r[i]; va[u] = v[i]; }
                    }
#pragma unroll
                    for (int u = 0; u < MU; ++u) {
                        const int32_t i = i0 + u * BT;
                        if (i < n) {
                            const T si = subc(ra[u], mulc(al, va[u]));
                            s[i] = si;
                            if (sf) {
                                c.buf[i] = pend;
                                c.buf2[i] = pend;
                                c.buf3[i] = si;
                            } else {
                                c.buf[i] = si;
                            }
                        }
                    }
                }
            }
            __syncthreads();
            if (sf) cta_prec_sf(c, nullptr);    // s^ = M^{-1} s stays in the solve buffer
            else cta_prec_staged<T>(c, nullptr);
            A dz[3] = {0, 0, 0};
            cta_spmv<T>(S.pa, S.a_col, c.aval, c.buf, t, nullptr, dz);     // t = A s^
            __syncthreads();
            A tsd[3] = {0, 0, 0};
            for (int32_t i0 = threadIdx.x; i0 < n; i0 += MU * BT) {
                T ta[MU], sa[MU];
#pragma unroll
                for (int u = 0; u < MU; ++u) {
                    const int32_t i = i0 + u * BT;
                    if (i < n) { ta[u] = t[i]; sa[u] = s[i]; }
                }
#pragma unroll
                for (int u = 0; u < MU; ++u)
                    if (i0 + u * BT < n) {
                        acc_dot<T, A>(ta[u], sa[u], tsd[0], tsd[1]);
                        tsd[2] += norm2<T, A>(ta[u]);
                    }
            }
            double tss[3];
            cta_sum<3, A>(tsd, tss, c.red);
            omega = tss[2] > 0.0 ? make_double2(tss[0] / tss[2], tss[1] / tss[2]) : make_double2(0.0, 0.0);
            A nr2[3] = {0, 0, 0};
            {   // xd += alpha p^ + omega s^, r = s - omega t, with (r^, r) and |r|^2
                const T al = cvt<T>(alpha), om = cvt<T>(omega);
                for (int32_t i0 = threadIdx.x; i0 < n; i0 += MU2 * BT) {
                    T xa[MU2], pa[MU2], sha[MU2], sa[MU2], ta[MU2], ha[MU2];
#pragma unroll
                    for (int u = 0; u < MU2; ++u) {
                        const int32_t i = i0 + u * BT;
                        if (i < n) {
                            xa[u] = xd[i];
                            pa[u] = ph[i];
                            sha[u] = c.buf[i];
                            sa[u] = s[i];
                            ta[u] = t[i];
                            ha[u] = rhat[i];
                        }
                    }
#pragma unroll
                    for (int u = 0; u < MU2; ++u) {
                        const int32_t i = i0 + u * BT;
                        if (i < n) {
                            xd[i] = addc(xa[u], addc(mulc(al, pa[u]), mulc(om, sha[u])));
                            const T ri = subc(sa[u], mulc(om, ta[u]));
                            r[i] = ri;
                            acc_dot<T, A>(ha[u], ri, nr2[0], nr2[1]);
                            nr2[2] += norm2<T, A>(ri);
                        }
                    }
                }
            }
            double nrs2[3];
            cta_sum<3, A>(nr2, nrs2, c.red);
            double rn32 = sqrt(nrs2[2]);
            double2 rho_new = make_double2(nrs2[0], nrs2[1]);
            if (rn32 <= DELTA * rn_ref || k % REFRESH == 0 || tss[2] == 0.0) {
                fold();
                rn = true_residual(S, x, r64, r, red, &lr);   // reliable update of r
                ++replacements;
                rn_ref = rn;
                if (lr <= P.tol) { status = SS_OK; break; }
                A nr3[2] = {0, 0};
                for (int32_t i = threadIdx.x; i < n; i += BT) acc_dot<T, A>(rhat[i], r[i], nr3[0], nr3[1]);
                double nrs3[2];
                cta_sum<2, A>(nr3, nrs3, c.red);
                rho_new = make_double2(nrs3[0], nrs3[1]);
                rn32 = rn;
            }
            if (tss[2] == 0.0 || (omega.x == 0.0 && omega.y == 0.0) || negligible(rho_new, rhat_norm, rn32)) {
                restart = true;
                break;
            }
            beta = cmul(cdiv(rho_new, rho), cdiv(alpha, omega));
            rho = rho_new;
        }
        if (status == SS_OK || status == SS_ERR_TIMEOUT) break;
        if (restart) {
            fold();
            if (++restarts > 8) { status = SS_BREAKDOWN; break; }
            continue;
        }
    }
    if (status != SS_OK && status != SS_ERR_TIMEOUT) {       // final acceptance test on the last iterate
        fold();
        true_residual(S, x, r64, r, red, &lr);
        if (lr <= P.tol) status = SS_OK;
    }
    S.iters = it;
    S.outer = replacements;
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

template <bool MIXED>
__global__ void __launch_bounds__(BT, BATCH_BLOCKS_PER_SM) batched_solver(BatchSys* sys, int nsys, BatchParams P, int* queue,
                                                         int* err) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ double red[NW * 3 + 3];
    __shared__ int s_idx;
    // The system's descriptor is copied to shared memory: kept in global
    // memory, its pointer fields would be re-read from L2 after every store.
    __shared__ __align__(16) BatchSys S;
    __shared__ __align__(8) uint64_t ring_bars[RING_MAX];
    __shared__ __align__(8) uint64_t ring_empty[RING_MAX];
    __shared__ int ring_abort;
    __shared__ uint32_t ring_issued;
    if (threadIdx.x == 0) {
        for (int r = 0; r < RING_MAX; ++r) {
            mbar_init(ring_bars + r, 1);
            mbar_init(ring_empty + r, 1);
        }
        ring_abort = 0;
        ring_issued = 0;
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    __syncthreads();
    uint32_t ring_seq = 0;          // levels staged by this block (identical in every thread)
    Ring last{};
    while (true) {
        if (threadIdx.x == 0) {
            const int t = atomicAdd(queue, 1);
            s_idx = (t < nsys && P.order) ? P.order[t] : t;
        }
        __syncthreads();
        const int k = s_idx;
        __syncthreads();
        if (k >= nsys) break;
        {
            const int* src = reinterpret_cast<const int*>(&sys[k]);
            int* dst = reinterpret_cast<int*>(&S);
            for (int w = threadIdx.x; w < (int)(sizeof(BatchSys) / sizeof(int)); w += BT) dst[w] = src[w];
        }
        __syncthreads();
        bool ok = true;
        if (S.factor_on_device) ok = cta_ilu0(S, MIXED, smem, P.smem_bytes, *(volatile int*)&ring_abort == 0);
        if (!ok) {
            if (threadIdx.x == 0) {
                sys[k].status = SS_ZERO_PIVOT;
                sys[k].iters = 0;
                sys[k].outer = 0;
                sys[k].resid = INFINITY;
            }
            __syncthreads();
            continue;
        }
        if (MIXED) {
            cta_pack_values<float2>(S.lo, S.f_val32);
            cta_pack_values<float2>(S.up, S.f_val32);
            cta_pack_values<float2>(S.pa, S.a_val32);
            cta_pack_dinv<float2>(S.up, S.f_inv32);
        } else {
            cta_pack_values<double2>(S.lo, S.f_val);
            cta_pack_values<double2>(S.up, S.f_val);
            cta_pack_values<double2>(S.pa, S.a_val);
            cta_pack_dinv<double2>(S.up, S.f_inv);
        }
        // the packed operands are read by bulk copies (the async proxy) from here on
        asm volatile("fence.proxy.async.global;\n" ::: "memory");
        // shared memory of this system: vector, level boundaries, ring
        SmemPlan sm;
        {
            const size_t vb = ((size_t)S.n * (MIXED ? sizeof(float2) : sizeof(double2)) + 15) & ~size_t(15);
            sm.buf = smem;
            size_t off = vb;
            sm.pbuf = nullptr;
            if (MIXED && P.pbuf_smem) {
                sm.pbuf = smem + off;
                off += vb;
            }
            sm.buf2 = sm.buf3 = nullptr;
            if (MIXED && P.sf) {
                sm.buf2 = smem + off;
                sm.buf3 = smem + off + vb;
                off += 2 * vb;
            }
            int32_t* lv = reinterpret_cast<int32_t*>(smem + off);
            if (P.lvl_smem) {
                const int nlo = S.lo.nlev + 1, nup = S.up.nlev + 1;
                for (int t = threadIdx.x; t < nlo; t += BT) lv[t] = S.lo.lvl[t];
                for (int t = threadIdx.x; t < nup; t += BT) lv[nlo + t] = S.up.lvl[t];
                sm.lvl_lo = lv;
                sm.lvl_up = lv + nlo;
                off += ((size_t)(nlo + nup) * 4 + 15) & ~size_t(15);
            } else {
                sm.lvl_lo = S.lo.lvl;
                sm.lvl_up = S.up.lvl;
            }
            sm.ring.base = smem + off;
            sm.ring.bars = ring_bars;
            sm.ring.empty = ring_empty;
            sm.ring.abort = &ring_abort;
            sm.ring.issued = &ring_issued;
            sm.ring.err = err;
            sm.ring.slot_bytes = P.ring_slot_bytes;
            sm.ring.umax = P.ring_umax;
            sm.ring.nslots = P.ring_slots;
            sm.ring.seq = ring_seq;
            sm.ring.wait_ns = P.wait_ns;
            sm.ring.stall_seq = P.diag_stall_seq;
        }
        __syncthreads();
        if (MIXED) solve_mixed(S, P, sm, red);
        else solve_fp64(S, P, sm, red);
        ring_seq = sm.ring.seq;
        last = sm.ring;
        finalise(S, red);
        if (threadIdx.x == 0) {
            sys[k].status = S.status;
            sys[k].iters = S.iters;
            sys[k].outer = S.outer;
            sys[k].resid = S.resid;
        }
        __syncthreads();
    }
    ring_drain(last);
}

}  // namespace

int batch_max_n(bool mixed) {
    const size_t cap = 227 * 1024 - 2048;
    return (int)(cap / ((mixed ? sizeof(float2) : sizeof(double2)) + sizeof(uint32_t)));
}

namespace {

template <class T>
size_t slot_bytes_of(int E, int R, int umax) {
    const SlotLayout L = slot_layout<T>(E, R, umax);
    return (size_t)L.dinv + (size_t)umax * dinv_stride<T>(R);
}

// Dynamic shared memory of a launch for a given plan: the solve vector, p^
// (pbuf), the level boundaries (lvl_smem) and nslots ring slots of umax units.
template <class T>
size_t plan_bytes(const std::vector<BatchShape>& shapes, int pbuf, int lvl_smem, int umax, int nslots,
                  size_t* slot_out, int sf = 0) {
    size_t base = 0, slot = 0;
    for (const BatchShape& b : shapes) {
        const size_t vb = ((size_t)b.n * sizeof(T) + 15) & ~size_t(15);
        size_t v = vb * (1 + (pbuf ? 1 : 0) + (sf ? 2 : 0));
        if (lvl_smem) v += ((size_t)(b.nlev_lo + b.nlev_up + 2) * 4 + 15) & ~size_t(15);
        base = std::max(base, v);
        if (umax > 0)
            slot = std::max(slot, std::max(slot_bytes_of<T>(b.E_lo, b.R_lo, umax), slot_bytes_of<T>(b.E_up, b.R_up, umax)));
    }
    *slot_out = slot;
    return base + (size_t)nslots * slot;
}

// Units per staged level: the widest level of any system (at most one per warp).
int widest_level(const std::vector<BatchShape>& shapes) {
    int u = 1;
    for (const BatchShape& b : shapes) u = std::max(u, b.umax);
    return std::min(u, NW);
}

// Mixed precision (FP32 operands): the sync-free solves (three more shared
// vectors, and p^ in shared memory when it fits; JC40, 608 systems: 313-317
// against 338-344 ms per step with level barriers), else level barriers with
// each warp loading its unit of the next level into registers before the
// current level's barrier, which is faster than the ring for these operands
// (347.5 against 360.1 ms); p^ and the level boundaries go to shared memory.
// FP64: a deep ring (every level's data is requested nslots - 1 levels
// ahead, which has to cover the memory latency; 449.9 against 632.1 ms
// without it), level boundaries in shared memory first.
template <class T>
size_t choose_plan(const std::vector<BatchShape>& shapes, size_t cap, BatchParams& p) {
    const bool ring_first = p.mixed ? p.stage_flip != 0 : p.stage_flip == 0;
    p.sf = 0;
    if (p.mixed && !ring_first)
        for (int pbuf = 1; pbuf >= 0; --pbuf) {
            size_t slot = 0;
            const size_t b = plan_bytes<T>(shapes, pbuf, 0, 0, 0, &slot, 1);
            if (b <= cap) {
                p.sf = 1;
                p.lvl_smem = 0;
                p.pbuf_smem = pbuf;
                p.ring_umax = 0;
                p.ring_slots = 0;
                p.ring_slot_bytes = 0;
                return b;
            }
        }
    if (!ring_first)
        for (int pbuf = 1; pbuf >= 0; --pbuf)
            for (int lvl_smem = 1; lvl_smem >= 0; --lvl_smem) {
                size_t slot = 0;
                const size_t b = plan_bytes<T>(shapes, pbuf, lvl_smem, 0, 0, &slot);
                if (b <= cap) {
                    p.lvl_smem = lvl_smem;
                    p.pbuf_smem = pbuf;
                    p.ring_umax = 0;
                    p.ring_slots = 0;
                    p.ring_slot_bytes = 0;
                    return b;
                }
            }
    struct Try { int pbuf, min_slots; };
    const Try tries[] = {{0, 12}, {0, 4}, {0, 2}};
    for (int lvl_smem = 1; lvl_smem >= 0; --lvl_smem)
        for (int umax = p.ring_allowed ? widest_level(shapes) : 0; umax >= 1; umax = umax > 4 ? umax / 2 : umax - 1)
            for (const Try& t : tries)
                for (int ns = RING_MAX; ns >= t.min_slots; --ns) {
                    size_t slot = 0;
                    const size_t b = plan_bytes<T>(shapes, t.pbuf, lvl_smem, umax, ns, &slot);
                    if (b <= cap) {
                        p.lvl_smem = lvl_smem;
                        p.pbuf_smem = t.pbuf;
                        p.ring_umax = umax;
                        p.ring_slots = ns;
                        p.ring_slot_bytes = (int)slot;
                        return b;
                    }
                }
    size_t slot = 0;
    p.lvl_smem = 0;
    p.pbuf_smem = 0;
    p.ring_umax = 0;
    p.ring_slots = 0;
    p.ring_slot_bytes = 0;
    return plan_bytes<T>(shapes, 0, 0, 0, 0, &slot);
}

}  // namespace

ss_status batch_launch(ss_ctx ctx, BatchSys* dsys, int nsys, BatchParams p, const std::vector<BatchShape>& shapes,
                       int* queue, int* err) {
    int optin = 0, per_sm = 0;
    SS_CUDA(ctx, cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, ctx->device));
    SS_CUDA(ctx, cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, ctx->device));
    // every resident block needs its share of the SM (and 1 KiB the system reserves per block)
    optin = std::min(optin, per_sm / BATCH_BLOCKS_PER_SM - 1024);
    cudaFuncAttributes fa;
    if (p.mixed) SS_CUDA(ctx, cudaFuncGetAttributes(&fa, batched_solver<true>));
    else SS_CUDA(ctx, cudaFuncGetAttributes(&fa, batched_solver<false>));
    const size_t cap = (size_t)optin > fa.sharedSizeBytes + 256 ? (size_t)optin - fa.sharedSizeBytes - 256 : 0;
    const size_t smem = p.mixed ? choose_plan<float2>(shapes, cap, p) : choose_plan<double2>(shapes, cap, p);
    if (smem > cap) return set_error(ctx, SS_ERR_UNSUPPORTED, "system too large for the per-system solver's shared memory");
    p.smem_bytes = (int)smem;
    const int grid = std::max(1, std::min(nsys, BATCH_BLOCKS_PER_SM * (ctx->num_sms > 0 ? ctx->num_sms : 1)));
    if (p.mixed) {
        SS_CUDA(ctx, cudaFuncSetAttribute(batched_solver<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        ProfScope ps(ctx, PROF_BATCHED);
        batched_solver<true><<<(ss_count_launch(), grid), BT, smem, ctx->stream>>>(dsys, nsys, p, queue, err);
    } else {
        SS_CUDA(ctx, cudaFuncSetAttribute(batched_solver<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        ProfScope ps(ctx, PROF_BATCHED);
        batched_solver<false><<<(ss_count_launch(), grid), BT, smem, ctx->stream>>>(dsys, nsys, p, queue, err);
    }
    SS_CUDA(ctx, cudaGetLastError());
    return SS_OK;
}
