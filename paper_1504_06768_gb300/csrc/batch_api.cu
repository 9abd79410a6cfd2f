// steady_state_batched: many independent systems solved by one persistent
// launch of the per-system CTA solver, organised as a wave (batch_wave.cuh).
// Systems that share a sparsity pattern (parameter sweeps) share the RCM
// ordering, the level schedule and the triangular-solve units, computed once
// per pattern on the host (and, in the serving loop, once per pattern across
// waves through the PatternCache).
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <map>
#include <memory>
#include <new>
#include <string>
#include <thread>
#include <tuple>
#include <vector>

#include "batch_wave.cuh"

namespace {

double now_ms() {
    using namespace std::chrono;
    return duration<double, std::milli>(steady_clock::now().time_since_epoch()).count();
}

// Lanes per row of a packed operand: the fewest whose BATCH_MAXE packed slots
// hold 99 % of the rows (fewer lanes: less padding and fewer shuffle rounds;
// the longer rows finish from the CSR).
int lanes_for_triangle(std::vector<int32_t> lens) {
    if (lens.empty()) return 1;
    std::sort(lens.begin(), lens.end());
    const int32_t p99 = lens[(size_t)(0.99 * (double)(lens.size() - 1))];
    int g = 1;
    while (g < 32 && g * BATCH_MAXE < p99) g <<= 1;
    return g;
}

// Lane-major packing of one CSR operand (see PackedOp): unit_rows holds R = 32/G
// row ids per unit; range(i) gives the CSR range [s, e) of row i's entries.
// First unit of each level when each level's rows are cut into units of R.
std::vector<int32_t> unit_levels(const std::vector<int32_t>& lptr, int R) {
    std::vector<int32_t> lvl(1, 0);
    for (size_t l = 0; l + 1 < lptr.size(); ++l) lvl.push_back(lvl.back() + (lptr[l + 1] - lptr[l] + R - 1) / R);
    return lvl;
}

template <class F>
void pack_host(const std::vector<int32_t>& unit_rows, int G, const std::vector<int32_t>& pcol, F range,
               PackedHost& P) {
    const int R = 32 / G;
    P.G = G;
    P.nunits = (int32_t)(unit_rows.size() / R);
    std::vector<int32_t> lens;
    for (int32_t i : unit_rows)
        if (i >= 0) {
            auto se = range(i);
            lens.push_back(se.second - se.first);
        }
    std::sort(lens.begin(), lens.end());
    const int32_t p99 = lens.empty() ? 1 : lens[(size_t)(0.99 * (double)(lens.size() - 1))];
    P.E = std::max(1, std::min(BATCH_MAXE, (p99 + G - 1) / G));
    P.rows = unit_rows;
    const size_t slots = (size_t)P.nunits * P.E * 32;
    P.col.assign(slots, -1);
    P.src.assign(slots, -1);
    P.ovb.assign(unit_rows.size(), 0);
    P.ove.assign(unit_rows.size(), 0);
    for (int32_t u = 0; u < P.nunits; ++u)
        for (int g = 0; g < R; ++g) {
            const int32_t i = unit_rows[(size_t)u * R + g];
            if (i < 0) continue;
            auto se = range(i);
            const int32_t s = se.first, e = se.second;
            for (int sub = 0; sub < G; ++sub)
                for (int q = 0; q < P.E; ++q) {
                    const int32_t k = s + sub + q * G;
                    if (k >= e) continue;
                    const size_t slot = ((size_t)u * P.E + q) * 32 + (size_t)g * G + sub;
                    P.col[slot] = pcol[k];
                    P.src[slot] = k;
                }
            const int32_t pe = s + P.E * G;
            P.ovb[(size_t)u * R + g] = std::min(pe, e);
            P.ove[(size_t)u * R + g] = e;
        }
}

template <class T>
ss_status upload_vec(ss_ctx ctx, const std::vector<T>& h, T** d) {
    SS_TRY(dev_alloc_n(ctx, d, h.size()));
    if (!h.empty())
        SS_CUDA(ctx, cudaMemcpyAsync(*d, h.data(), sizeof(T) * h.size(), cudaMemcpyHostToDevice, ctx->stream));
    return SS_OK;
}

// Host analysis of one pattern: RCM ordering (section "Direct
// factorization"), the permuted pattern with the gather map of its values,
// the level sets of the two triangles and the packed operands.  Runs on any
// host thread; touches nothing on the device.
// Lanes per row scaled by 2^shift (the autotuner's choice), within 1..32.
int shifted_lanes(int g, int shift) {
    while (shift > 0 && g < 32) { g <<= 1; --shift; }
    while (shift < 0 && g > 1) { g >>= 1; ++shift; }
    return g;
}

void build_pattern_host(Pattern& P, int use_rcm, const TuneChoice& tune) {
    const int64_t n = (int64_t)P.rp.size() - 1, d = P.d;
    P.perm.resize(n);
    if (use_rcm) rcm_host(n, P.rp.data(), P.col.data(), P.perm.data());
    else for (int64_t i = 0; i < n; ++i) P.perm[i] = (int32_t)i;
    P.iperm.resize(n);
    for (int64_t r = 0; r < n; ++r) P.iperm[P.perm[r]] = (int32_t)r;
    P.tidx.resize(d);
    for (int64_t i = 0; i < d; ++i) P.tidx[i] = P.iperm[i * (d + 1)];
    P.r0 = P.iperm[0];
    // permuted pattern (rows gathered, columns relabelled and sorted) and the
    // natural-order position each permuted entry comes from
    std::vector<int32_t>& prp = P.prp;
    std::vector<int32_t>& pcol = P.pcol;
    prp.assign(n + 1, 0);
    pcol.resize(P.col.size());
    P.map.resize(P.col.size());
    for (int64_t r = 0; r < n; ++r) prp[r + 1] = prp[r] + (P.rp[P.perm[r] + 1] - P.rp[P.perm[r]]);
    P.dpos.assign(n, -1);
    std::vector<std::pair<int32_t, int32_t>> row;
    for (int64_t r = 0; r < n; ++r) {
        const int32_t i = P.perm[r];
        row.clear();
        for (int32_t t = P.rp[i]; t < P.rp[i + 1]; ++t) row.emplace_back(P.iperm[P.col[t]], t);
        std::sort(row.begin(), row.end());
        int32_t o = prp[r];
        for (const auto& e : row) {
            if (e.first == r) P.dpos[r] = o;
            pcol[o] = e.first;
            P.map[o] = e.second;
            ++o;
        }
    }
    int64_t lo = 0, up = 0;
    for (int64_t r = 0; r < n; ++r) {
        if (P.dpos[r] < 0) {
            P.status = SS_ZERO_PIVOT;
            P.error = "iLU(0): missing diagonal entry in row " + std::to_string(r);
            return;
        }
        lo += P.dpos[r] - prp[r];
        up += prp[r + 1] - P.dpos[r] - 1;
    }
    // elimination schedule of iLU(0) on the permuted pattern (the updates of
    // the IKJ elimination, in its order; shared by the pattern's systems)
    ilu0_schedule_host(n, prp.data(), pcol.data(), P.dpos.data(), P.ilu_ptr, P.ilu_tgt, P.ilu_src);
    std::vector<int32_t> uorder, uptr;
    P.n_levels = level_sets_host(n, prp.data(), pcol.data(), true, P.lorder, P.lptr);
    P.up_levels = level_sets_host(n, prp.data(), pcol.data(), false, uorder, uptr);
    {
        std::vector<int32_t> llen(n), ulen(n);
        for (int64_t r = 0; r < n; ++r) {
            llen[r] = P.dpos[r] - prp[r];
            ulen[r] = prp[r + 1] - P.dpos[r] - 1;
        }
        P.lo_g = shifted_lanes(lanes_for_triangle(std::move(llen)), tune.lo);
        P.up_g = shifted_lanes(lanes_for_triangle(std::move(ulen)), tune.up);
    }
    {
        std::vector<int32_t> alen(n);
        for (int64_t r = 0; r < n; ++r) alen[r] = prp[r + 1] - prp[r];
        P.a_g = shifted_lanes(lanes_for_triangle(std::move(alen)), tune.a);
    }
    level_units_host(P.lorder, P.lptr, 32 / P.lo_g, P.lunits);
    level_units_host(uorder, uptr, 32 / P.up_g, P.uunits);
    P.lo_nunits = (int32_t)(P.lunits.size() / (32 / P.lo_g));
    P.up_nunits = (int32_t)(P.uunits.size() / (32 / P.up_g));
    // packed operands: the two triangles (level-aligned units) and A (consecutive rows)
    const std::vector<int32_t>& dpos = P.dpos;
    pack_host(P.lunits, P.lo_g, pcol, [&](int32_t i) { return std::make_pair(prp[i], dpos[i]); }, P.hl);
    pack_host(P.uunits, P.up_g, pcol, [&](int32_t i) { return std::make_pair(dpos[i] + 1, prp[i + 1]); }, P.hu);
    P.hl.lvl = unit_levels(P.lptr, 32 / P.lo_g);
    P.hu.lvl = unit_levels(uptr, 32 / P.up_g);
    P.hl.nlev = (int32_t)P.hl.lvl.size() - 1;
    P.hu.nlev = (int32_t)P.hu.lvl.size() - 1;
    {
        const int R = 32 / P.a_g;
        std::vector<int32_t> arows(((n + R - 1) / R) * R, -1);
        for (int64_t i = 0; i < n; ++i) arows[i] = (int32_t)i;
        pack_host(arows, P.a_g, pcol, [&](int32_t i) { return std::make_pair(prp[i], prp[i + 1]); }, P.ha);
    }
}

ss_status upload_pattern(ss_ctx ctx, Pattern& P) {
    auto up_packed = [&](PackedHost& h, PackedDev& dv) -> ss_status {
        dv.nunits = h.nunits;
        dv.G = h.G;
        dv.E = h.E;
        h.meta.resize(h.rows.size());
        for (size_t k = 0; k < h.meta.size(); ++k) h.meta[k] = make_int4(h.rows[k], h.ovb[k], h.ove[k], 0);
        SS_TRY(upload_vec(ctx, h.meta, &dv.meta));
        SS_TRY(upload_vec(ctx, h.col, &dv.col));
        SS_TRY(upload_vec(ctx, h.src, &dv.src));
        dv.nlev = h.nlev;
        if (h.nlev > 0) SS_TRY(upload_vec(ctx, h.lvl, &dv.lvl));
        return SS_OK;
    };
    SS_TRY(up_packed(P.hl, P.lo));
    SS_TRY(up_packed(P.hu, P.up));
    SS_TRY(up_packed(P.ha, P.pa));
    SS_TRY(upload_vec(ctx, P.prp, &P.prp_d));
    SS_TRY(upload_vec(ctx, P.pcol, &P.pcol_d));
    SS_TRY(upload_vec(ctx, P.map, &P.map_d));
    SS_TRY(upload_vec(ctx, P.perm, &P.perm_d));
    SS_TRY(upload_vec(ctx, P.tidx, &P.tidx_d));
    SS_TRY(upload_vec(ctx, P.dpos, &P.dpos_d));
    SS_TRY(upload_vec(ctx, P.lunits, &P.lo_units));
    SS_TRY(upload_vec(ctx, P.uunits, &P.up_units));
    SS_TRY(upload_vec(ctx, P.lptr, &P.lvl_ptr));
    SS_TRY(upload_vec(ctx, P.lorder, &P.lvl_rows));
    SS_TRY(upload_vec(ctx, P.ilu_ptr, &P.ilu_ptr_d));
    SS_TRY(upload_vec(ctx, P.ilu_tgt, &P.ilu_tgt_d));
    SS_TRY(upload_vec(ctx, P.ilu_src, &P.ilu_src_d));
    SS_TRY(upload_vec(ctx, P.rp, &P.rp_d));
    SS_TRY(upload_vec(ctx, P.col, &P.col_d));
    return SS_OK;
}

}  // namespace

Pattern::~Pattern() {
    cudaSetDevice(device);
    void* ptrs[] = {rp_d, col_d, prp_d, pcol_d, map_d, perm_d, tidx_d, dpos_d, lo_units, up_units, lvl_ptr, lvl_rows,
                    ilu_ptr_d, ilu_tgt_d, ilu_src_d,
                    lo.col, lo.src, lo.lvl, lo.meta, up.col, up.src, up.lvl, up.meta, pa.col, pa.src, pa.lvl, pa.meta};
    for (void* q : ptrs)
        if (q) cudaFreeAsync(q, 0);
}

void PatternCache::touch(const PatternKey& k, const std::shared_ptr<Pattern>& p) {
    for (size_t i = 0; i < lru.size(); ++i)
        if (lru[i].second == p) {
            auto e = lru[i];
            lru.erase(lru.begin() + (long)i);
            lru.push_back(e);
            return;
        }
    lru.emplace_back(k, p);
}

void PatternCache::insert(const PatternKey& k, const std::shared_ptr<Pattern>& p) {
    by_key[k].push_back(p);
    touch(k, p);
    while (lru.size() > max_patterns) {          // evict the least recently used (waves keep their own references)
        auto e = lru.front();
        lru.erase(lru.begin());
        auto& v = by_key[e.first];
        v.erase(std::remove(v.begin(), v.end(), e.second), v.end());
        if (v.empty()) by_key.erase(e.first);
    }
}

const SolutionCache::Entry* SolutionCache::nearest(const PatternKey& k, double2 fp) {
    auto it = by_key.find(k);
    if (it == by_key.end()) return nullptr;
    const Entry* best = nullptr;
    double bd = INFINITY;
    for (const Entry& e : it->second) {
        const double dd = std::fabs(e.fp.x - fp.x) / std::max(std::max(e.fp.x, fp.x), 1e-300) +
                          std::fabs(e.fp.y - fp.y) / std::max(std::max(e.fp.y, fp.y), 1e-300);
        if (dd < bd) {
            bd = dd;
            best = &e;
        }
    }
    return best;
}

ss_status SolutionCache::insert(ss_ctx ctx, const PatternKey& k, double2 fp, const double2* rho, int64_t n) {
    std::lock_guard<std::mutex> lock(mu);
    const size_t sz = sizeof(double2) * (size_t)n;
    if (sz > max_bytes) return SS_OK;
    auto evict_oldest = [&](std::vector<Entry>* only) {
        std::vector<Entry>* from = nullptr;
        size_t at = 0;
        uint64_t oldest = UINT64_MAX;
        for (auto& kv : by_key) {
            if (only && &kv.second != only) continue;
            for (size_t i = 0; i < kv.second.size(); ++i)
                if (kv.second[i].stamp < oldest) {
                    oldest = kv.second[i].stamp;
                    from = &kv.second;
                    at = i;
                }
        }
        if (!from) return false;
        dev_free(ctx, (*from)[at].rho);
        bytes -= sizeof(double2) * (size_t)(*from)[at].n;
        from->erase(from->begin() + (ptrdiff_t)at);
        return true;
    };
    std::vector<Entry>& v = by_key[k];
    while (v.size() >= per_key && evict_oldest(&v)) {
    }
    while (bytes + sz > max_bytes && evict_oldest(nullptr)) {
    }
    Entry e;
    e.fp = fp;
    e.n = n;
    e.stamp = ++clock;
    SS_TRY(dev_alloc_n(ctx, &e.rho, (size_t)n));
    SS_CUDA(ctx, cudaMemcpyAsync(e.rho, rho, sz, cudaMemcpyDeviceToDevice, ctx->stream));
    bytes += sz;
    by_key[k].push_back(e);
    return SS_OK;
}

void SolutionCache::clear(ss_ctx ctx) {
    std::lock_guard<std::mutex> lock(mu);
    for (auto& kv : by_key)
        for (Entry& e : kv.second) dev_free(ctx, e.rho);
    by_key.clear();
    bytes = 0;
}

size_t wave_footprint_bytes(int64_t d, int64_t nnz_h, const std::vector<int64_t>& nnz_c,
                            const std::vector<int64_t>& ctc_c, bool mixed) {
    // nnz(L) <= 2 d nnz(H) + sum_k (nnz(C_k)^2 + 2 d nnz(C_k^+ C_k)) + d (trace row), the
    // candidate count of the assembly; ctc_c bounds nnz(C_k^+ C_k)
    double nnz = 2.0 * (double)d * (double)nnz_h + (double)d;
    for (size_t k = 0; k < nnz_c.size(); ++k)
        nnz += (double)nnz_c[k] * (double)nnz_c[k] + 2.0 * (double)d * (double)ctc_c[k];
    const double n = (double)d * (double)d;
    // per stored entry: A and the factors (FP64), their FP32 copies, three
    // packed operands with lane padding, and the assembly's candidates
    // (transient); per row: the Krylov vectors and the per-row arrays
    const double per_nnz = 16.0 + 16.0 + (mixed ? 16.0 : 0.0) + 4.0 * (mixed ? 8.0 : 16.0) + 24.0;
    const double per_row = 10.0 * (mixed ? 8.0 : 16.0) + 5.0 * 16.0;
    return (size_t)(std::min(nnz, n * n) * per_nnz + n * per_row) + (1u << 16);
}

size_t wave_pinned_bytes(const BatchWave& w) {
    size_t b = ((w.H.size() * sizeof(BatchSys) + 255) & ~size_t(255)) + 256;
    if (!w.rho_on_device)
        for (const ss_csr_view* h : w.H) b += (size_t)h->n_rows * h->n_rows * sizeof(double2);
    return b;
}

bool wave_ready(BatchWave& w) {
    if (!w.launched) return true;
    return cudaEventQuery(w.done) != cudaErrorNotReady;
}

void wave_release(BatchWave& w) {
    ss_ctx ctx = w.ctx;
    batch_lt_free(ctx, w.blt);
    for (void* p : w.owned) dev_free(ctx, p);
    w.owned.clear();
    w.pats.clear();
    w.pat_of.clear();
    if (w.done) {
        cudaEventDestroy(w.done);
        w.done = nullptr;
    }
    for (cudaEvent_t* e : {&w.k0, &w.k1})
        if (*e) {
            cudaEventDestroy(*e);
            *e = nullptr;
        }
    w.launched = false;
}

ss_status wave_begin(BatchWave& w) {
    ss_ctx ctx = w.ctx;
    const ss_options& opt = w.opt;
    const bool mixed = opt.precision == SS_PREC_MIXED;
    const size_t ns = w.H.size();
    w.t0 = now_ms();
    w.launched = false;
#define WSTEP(call) do { ss_status _st = (call); if (_st != SS_OK) { wave_release(w); return _st; } } while (0)
    // (1) every system's L~ with a fixed number of launches
    WSTEP(batch_trace_systems(ctx, w.H, w.n_c, w.C, opt.w, w.blt));
    BatchLt& blt = w.blt;
    // (2) distinct patterns: hash, then an exact check on the device, within
    // the wave and against the cache
    w.pat_of.assign(ns, -1);
    std::vector<int> rep_sys;
    std::vector<PatternKey> rep_key;
    {
        std::map<PatternKey, int> first;
        std::vector<std::pair<int, int>> pairs;
        for (size_t q = 0; q < ns; ++q) {
            const PatternKey key = std::make_tuple(blt.d[q], blt.n[q], blt.meta[q].nnz, blt.meta[q].hash);
            auto it = first.find(key);
            if (it == first.end()) {
                first.emplace(key, (int)rep_sys.size());
                w.pat_of[q] = (int)rep_sys.size();
                rep_sys.push_back((int)q);
                rep_key.push_back(key);
            } else {
                w.pat_of[q] = it->second;
                pairs.emplace_back((int)q, rep_sys[it->second]);
            }
        }
        std::vector<int> mismatch;
        WSTEP(batch_verify_patterns(ctx, blt, pairs, mismatch));
        for (size_t k = 0; k < pairs.size(); ++k)
            if (mismatch[k]) {                 // equal hashes, different patterns: a pattern of its own
                w.pat_of[pairs[k].first] = (int)rep_sys.size();
                rep_sys.push_back(pairs[k].first);
                rep_key.push_back(std::make_tuple(blt.d[pairs[k].first], blt.n[pairs[k].first],
                                                  blt.meta[pairs[k].first].nnz, blt.meta[pairs[k].first].hash));
            }
    }
    w.pats.assign(rep_sys.size(), nullptr);
    if (w.cache) {
        std::lock_guard<std::mutex> lock(w.cache->mu);
        for (size_t p = 0; p < rep_sys.size(); ++p) {
            auto it = w.cache->by_key.find(rep_key[p]);
            if (it == w.cache->by_key.end()) continue;
            for (const auto& cand : it->second) {
                int mism = 1;
                WSTEP(batch_verify_against(ctx, blt, rep_sys[p], cand->rp_d, cand->col_d, &mism));
                if (!mism) {
                    w.pats[p] = cand;
                    w.cache->touch(rep_key[p], cand);
                    break;
                }
            }
        }
    }
    std::vector<size_t> fresh;
    for (size_t p = 0; p < rep_sys.size(); ++p)
        if (!w.pats[p]) {
            w.pats[p] = std::make_shared<Pattern>();
            w.pats[p]->d = blt.d[rep_sys[p]];
            w.pats[p]->device = ctx->device;
            WSTEP(batch_download_pattern(ctx, blt, rep_sys[p], w.pats[p]->rp, w.pats[p]->col));
            fresh.push_back(p);
        }
    if (!fresh.empty()) {
        SS_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
        const size_t nth = std::max<size_t>(1, std::min<size_t>(fresh.size(), std::min<unsigned>(16u, std::max(1u, std::thread::hardware_concurrency()))));
        if (nth <= 1) {
            for (size_t p : fresh) build_pattern_host(*w.pats[p], opt.use_rcm, w.tune);
        } else {
            std::vector<std::thread> th;
            for (size_t t = 0; t < nth; ++t)
                th.emplace_back([&, t]() {
                    for (size_t k = t; k < fresh.size(); k += nth) build_pattern_host(*w.pats[fresh[k]], opt.use_rcm, w.tune);
                });
            for (auto& x : th) x.join();
        }
        for (size_t p : fresh) {
            Pattern& P = *w.pats[p];
            if (P.status != SS_OK) { ss_status e = set_error(ctx, P.status, P.error); wave_release(w); return e; }
            WSTEP(upload_pattern(ctx, P));
        }
        if (w.cache) {
            // a cached pattern is used by later waves on other streams: its upload must be complete
            SS_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
            std::lock_guard<std::mutex> lock(w.cache->mu);
            for (size_t p : fresh) w.cache->insert(rep_key[p], w.pats[p]);
        }
    }
    w.key_of.resize(ns);
    for (size_t q = 0; q < ns; ++q) w.key_of[q] = rep_key[w.pat_of[q]];
    // the queue takes the systems by estimated cost, largest first
    std::vector<int32_t> order;
    WSTEP(batch_cost_order(ctx, blt, order, &w.fp));
    int32_t* order_d = nullptr;
    WSTEP(dev_alloc_n(ctx, &order_d, ns));
    w.owned.push_back(order_d);
    SS_CUDA(ctx, cudaMemcpyAsync(order_d, order.data(), sizeof(int32_t) * ns, cudaMemcpyHostToDevice, ctx->stream));
    // (3) per-system buffers (one allocation) and descriptors; describe() lays
    // out system q's buffers from address base and returns the bytes used
    const size_t inner = mixed ? sizeof(float2) : sizeof(double2);
    auto describe = [&](size_t q, uintptr_t base, BatchSys& b, GatherEntry& g) -> size_t {
        const Pattern& P = *w.pats[w.pat_of[q]];
        const int64_t n = blt.n[q], nnz = blt.meta[q].nnz;
        size_t off = 0;
        auto take = [&](size_t sz) { uintptr_t p = base + off; off += (sz + 255) & ~size_t(255); return p; };
        std::memset(&b, 0, sizeof(b));
        double2* aval = reinterpret_cast<double2*>(take(nnz * sizeof(double2)));
        g = GatherEntry{P.map_d, aval, blt.meta[q].nz_off, nnz};
        b.n = (int32_t)n;
        b.d = (int32_t)blt.d[q];
        b.a_rp = P.prp_d;
        b.a_col = P.pcol_d;
        b.a_val = aval;
        b.f_rp = P.prp_d;
        b.f_col = P.pcol_d;
        b.f_dpos = P.dpos_d;
        b.factor_on_device = 1;
        b.f_val = reinterpret_cast<double2*>(take(nnz * sizeof(double2)));
        b.f_inv = reinterpret_cast<double2*>(take(n * sizeof(double2)));
        if (mixed) {
            b.f_val32 = reinterpret_cast<float2*>(take(nnz * sizeof(float2)));
            b.a_val32 = reinterpret_cast<float2*>(take(nnz * sizeof(float2)));
            b.f_inv32 = reinterpret_cast<float2*>(take(n * sizeof(float2)));
        }
        b.work = reinterpret_cast<void*>(take(10 * n * inner));
        b.x64 = reinterpret_cast<double2*>(take(n * sizeof(double2)));
        b.r64 = reinterpret_cast<double2*>(take(n * sizeof(double2)));
        b.rho_out = w.rho_on_device ? reinterpret_cast<double2*>(w.rho_out[q])
                                    : reinterpret_cast<double2*>(take(n * sizeof(double2)));
        auto set_op = [&](PackedOp& o, const PackedDev& dv) {
            o.meta = dv.meta;
            o.col = dv.col;
            o.src = dv.src;
            o.dinv = nullptr;
            o.nunits = dv.nunits;
            o.G = dv.G;
            o.E = dv.E;
            o.lvl = dv.lvl;
            o.nlev = dv.nlev;
            o.val = reinterpret_cast<void*>(take((size_t)dv.nunits * dv.E * 32 * inner));
        };
        set_op(b.lo, P.lo);
        set_op(b.up, P.up);
        set_op(b.pa, P.pa);
        b.up.dinv = reinterpret_cast<void*>(take((size_t)P.up.nunits * (((32 / P.up.G) * inner + 15) & ~size_t(15))));
        b.lvl_ptr = P.lvl_ptr;
        b.lvl_rows = P.lvl_rows;
        b.ilu_ptr = P.ilu_ptr_d;
        b.ilu_tgt = P.ilu_tgt_d;
        b.ilu_src = P.ilu_src_d;
        b.n_levels = P.n_levels;
        b.r0 = P.r0;
        b.w = blt.w[q];
        b.sigma = 0.0;
        b.perm = P.perm_d;
        b.tidx = P.tidx_d;
        return off;
    };
    w.hs.assign(ns, BatchSys{});
    std::vector<GatherEntry> gather(ns);
    std::vector<size_t> boff(ns + 1, 0);
    for (size_t q = 0; q < ns; ++q) boff[q + 1] = boff[q] + describe(q, 0, w.hs[q], gather[q]);
    char* blk_all = nullptr;
    WSTEP(dev_alloc(ctx, reinterpret_cast<void**>(&blk_all), boff[ns]));
    w.owned.push_back(blk_all);
    for (size_t q = 0; q < ns; ++q) describe(q, reinterpret_cast<uintptr_t>(blk_all) + boff[q], w.hs[q], gather[q]);
    WSTEP(batch_gather_values(ctx, blt, gather));
    // warm starts: the caller's guesses (in rho_out), or, in the serving loop,
    // the stored state of the closest earlier request with the same pattern
    bool cache_copies = false;
    for (size_t q = 0; q < ns; ++q) {
        if (opt.warm_start) {
            w.hs[q].warm = 1;
            if (!w.rho_on_device)
                SS_CUDA(ctx, cudaMemcpyAsync(w.hs[q].rho_out, w.rho_out[q], sizeof(double2) * blt.n[q],
                                             cudaMemcpyHostToDevice, ctx->stream));
        } else if (w.sols) {
            std::lock_guard<std::mutex> lock(w.sols->mu);
            const SolutionCache::Entry* e = w.sols->nearest(w.key_of[q], w.fp[q]);
            if (e && e->n == blt.n[q]) {
                SS_CUDA(ctx, cudaMemcpyAsync(w.hs[q].rho_out, e->rho, sizeof(double2) * e->n, cudaMemcpyDeviceToDevice,
                                             ctx->stream));
                w.hs[q].warm = 1;
                cache_copies = true;
            }
        }
    }
    // a stored state may be evicted by a later wave: its copy is complete before this wave goes on
    if (cache_copies) SS_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    WSTEP(dev_alloc_n(ctx, &w.dsys, ns));
    w.owned.push_back(w.dsys);
    WSTEP(dev_alloc_n(ctx, &w.ctl, 4));
    w.owned.push_back(w.ctl);
    SS_CUDA(ctx, cudaMemcpyAsync(w.dsys, w.hs.data(), sizeof(BatchSys) * ns, cudaMemcpyHostToDevice, ctx->stream));
    SS_CUDA(ctx, cudaMemsetAsync(w.ctl, 0, sizeof(int) * 4, ctx->stream));
    w.t1 = now_ms();

    BatchParams bp;
    std::memset(&bp, 0, sizeof(bp));
    bp.order = order_d;
    bp.tol = opt.tol;
    bp.maxiter = opt.maxiter;
    bp.mixed = mixed ? 1 : 0;
    bp.inner_rtol = opt.inner_rtol > 0 ? opt.inner_rtol : 1e-5;
    bp.power = 0;
    bp.seed = opt.seed;
    // bulk copies stage the triangles' packed arrays: all must start on 16 bytes
    bp.ring_allowed = 1;
    auto a16 = [](const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15) == 0; };
    for (const BatchSys& b : w.hs)
        for (const PackedOp* o : {&b.lo, &b.up})
            if (!a16(o->meta) || !a16(o->col) || !a16(o->val) || (o->dinv && !a16(o->dinv))) bp.ring_allowed = 0;
    std::vector<BatchShape> shapes(ns);
    for (size_t q = 0; q < ns; ++q) {
        const Pattern& P = *w.pats[w.pat_of[q]];
        int32_t wide = 1;
        for (const std::vector<int32_t>* lv : {&P.hl.lvl, &P.hu.lvl})
            for (size_t l = 0; l + 1 < lv->size(); ++l) wide = std::max(wide, (*lv)[l + 1] - (*lv)[l]);
        shapes[q] = BatchShape{(int32_t)blt.n[q], P.lo.nlev, P.up.nlev, P.lo.E, 32 / P.lo.G, P.up.E, 32 / P.up.G, wide};
    }
    bp.stage_flip = w.tune.stage;
    bp.wait_ns = ctx->wait_ns;
    bp.diag_stall_seq = ctx->diag_stall_seq;
    if (w.time_kernel) {
        if (!w.k0) SS_CUDA(ctx, cudaEventCreate(&w.k0));
        if (!w.k1) SS_CUDA(ctx, cudaEventCreate(&w.k1));
        SS_CUDA(ctx, cudaEventRecord(w.k0, ctx->stream));
    }
    WSTEP(batch_launch(ctx, w.dsys, (int)ns, bp, shapes, w.ctl, w.ctl + 1));
    if (w.time_kernel) SS_CUDA(ctx, cudaEventRecord(w.k1, ctx->stream));
    if (w.stage_pinned) {
        // results to pinned memory, asynchronously: [descriptors][error word][rho ...]
        const size_t hs_bytes = (ns * sizeof(BatchSys) + 255) & ~size_t(255);
        unsigned char* base = reinterpret_cast<unsigned char*>(w.stage);
        SS_CUDA(ctx, cudaMemcpyAsync(base, w.dsys, sizeof(BatchSys) * ns, cudaMemcpyDeviceToHost, ctx->stream));
        SS_CUDA(ctx, cudaMemcpyAsync(base + hs_bytes, w.ctl + 1, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
        w.stage_off.assign(ns, 0);
        size_t off = hs_bytes + 256;
        if (!w.rho_on_device)
            for (size_t q = 0; q < ns; ++q) {
                w.stage_off[q] = off;
                SS_CUDA(ctx, cudaMemcpyAsync(base + off, w.hs[q].rho_out, sizeof(double2) * blt.n[q],
                                             cudaMemcpyDeviceToHost, ctx->stream));
                off += sizeof(double2) * blt.n[q];
            }
    }
    if (!w.done) SS_CUDA(ctx, cudaEventCreateWithFlags(&w.done, cudaEventDisableTiming));
    SS_CUDA(ctx, cudaEventRecord(w.done, ctx->stream));
    w.launched = true;
#undef WSTEP
    return SS_OK;
}

ss_status wave_end(BatchWave& w, ss_info* infos) {
    ss_ctx ctx = w.ctx;
    const size_t ns = w.H.size();
    cudaError_t e = w.launched ? cudaEventSynchronize(w.done) : cudaSuccess;
    int herr = 0;
    if (e == cudaSuccess) {
        if (w.stage_pinned) {
            const unsigned char* base = reinterpret_cast<const unsigned char*>(w.stage);
            const size_t hs_bytes = (ns * sizeof(BatchSys) + 255) & ~size_t(255);
            std::memcpy(w.hs.data(), base, sizeof(BatchSys) * ns);
            std::memcpy(&herr, base + hs_bytes, sizeof(int));
            if (!w.rho_on_device) {
                // large results are copied out by several host threads
                size_t total = 0;
                for (size_t q = 0; q < ns; ++q) total += sizeof(double2) * w.blt.n[q];
                const unsigned hw = std::max(1u, std::thread::hardware_concurrency());
                const size_t nt = std::min<size_t>({ns, (size_t)std::min(8u, hw), total / ((size_t)4 << 20) + 1});
                auto copy = [&](size_t t) {
                    for (size_t q = t; q < ns; q += nt)
                        std::memcpy(w.rho_out[q], base + w.stage_off[q], sizeof(double2) * w.blt.n[q]);
                };
                std::vector<std::thread> th;
                for (size_t t = 1; t < nt; ++t) th.emplace_back(copy, t);
                copy(0);
                for (std::thread& x : th) x.join();
            }
        } else {
            e = cudaMemcpyAsync(w.hs.data(), w.dsys, sizeof(BatchSys) * ns, cudaMemcpyDeviceToHost, ctx->stream);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(&herr, w.ctl + 1, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream);
            if (!w.rho_on_device)
                for (size_t q = 0; q < ns && e == cudaSuccess; ++q)
                    e = cudaMemcpyAsync(w.rho_out[q], w.hs[q].rho_out, sizeof(double2) * w.blt.n[q],
                                        cudaMemcpyDeviceToHost, ctx->stream);
            if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
        }
    }
    if (e != cudaSuccess) {
        wave_release(w);
        return cuda_check(ctx, e, "steady_state_batched");
    }
    w.t2 = now_ms();
    if (w.time_kernel && w.k0 && w.k1) cudaEventElapsedTime(&w.kernel_ms, w.k0, w.k1);
    if (w.sols && !herr) {
        for (size_t q = 0; q < ns; ++q)
            if (w.hs[q].status == SS_OK) {
                ss_status cs = w.sols->insert(ctx, w.key_of[q], w.fp[q], w.hs[q].rho_out, w.blt.n[q]);
                if (cs != SS_OK) break;           // the cache is an aid: a failed copy only ends its filling
            }
        cudaStreamSynchronize(ctx->stream);
    }
    ss_status worst = SS_OK;
    for (size_t q = 0; q < ns; ++q) {
        const Pattern& P = *w.pats[w.pat_of[q]];
        if (herr) w.hs[q].status = SS_ERR_TIMEOUT;
        if (infos) {
            ss_info& inf = infos[q];
            std::memset(&inf, 0, sizeof(inf));
            inf.status = w.hs[q].status;
            inf.method = SS_METHOD_ITER_BICGSTAB;
            inf.iters = w.hs[q].iters;
            inf.outer_iters = w.hs[q].outer;
            inf.resid_Lrho = w.hs[q].resid;
            inf.w_used = w.blt.w[q];
            inf.n = w.hs[q].n;
            inf.nnz = w.blt.meta[q].nnz;
            inf.nnz_factors = w.blt.meta[q].nnz;
            inf.levels_lower = P.n_levels;
            inf.levels_upper = P.up_levels;
            inf.ms_setup = (w.t1 - w.t0) / ns;
            inf.ms_solve = (w.t2 - w.t1) / ns;
            inf.tune_lanes_shift[0] = w.tune.lo;
            inf.tune_lanes_shift[1] = w.tune.up;
            inf.tune_lanes_shift[2] = w.tune.a;
            inf.tune_stage = w.tune.stage;
        }
        if (w.hs[q].status != SS_OK) {
            if (w.hs[q].status != SS_NOT_CONVERGED && w.hs[q].status != SS_BREAKDOWN) worst = (ss_status)w.hs[q].status;
            else if (worst == SS_OK) worst = (ss_status)w.hs[q].status;
        }
    }
    wave_release(w);
    if (worst != SS_OK) ctx->last_error = "at least one system did not converge (see infos)";
    return worst;
}

extern "C" ss_status steady_state(ss_ctx, const ss_csr_view*, int, const ss_csr_view*, const ss_options*, double*, int,
                                  ss_info*);

namespace {

// One probe of the autotuner: the batch's first systems (up to one per SM)
// with a capped iteration count under the candidate choice; the cost is the
// persistent kernel's device time per system-iteration.
struct TuneProbe {
    ss_ctx ctx;
    ss_options opt;
    std::vector<const ss_csr_view*> H, C;
    std::vector<int> n_c;
    std::vector<double*> rho;             // device scratch, one per system
};

double probe_cost(const TuneChoice& c, void* user) {
    TuneProbe& t = *static_cast<TuneProbe*>(user);
    BatchWave w;
    w.ctx = t.ctx;
    w.opt = t.opt;
    w.rho_on_device = 1;
    w.H = t.H;
    w.C = t.C;
    w.n_c = t.n_c;
    w.rho_out = t.rho;
    w.tune = c;
    w.time_kernel = true;
    if (wave_begin(w) != SS_OK) return INFINITY;
    std::vector<ss_info> inf(t.H.size());
    const ss_status st = wave_end(w, inf.data());
    if (st != SS_OK && st != SS_NOT_CONVERGED && st != SS_BREAKDOWN) return INFINITY;
    double iters = 0.0;
    for (const ss_info& i : inf) iters += i.iters;
    return iters > 0.0 ? (double)w.kernel_ms / iters : INFINITY;
}

// Shape of a batch for the tuning table: precision, and per system the
// dimension and the operators' entry counts (FNV-1a).
unsigned long long batch_shape_key(const ss_options& opt, const std::vector<const ss_csr_view*>& H,
                                   const std::vector<int>& n_c, const std::vector<const ss_csr_view*>& C) {
    unsigned long long h = 1469598103934665603ull;
    auto mix = [&](long long v) {
        for (int b = 0; b < 8; ++b) {
            h ^= (unsigned long long)((v >> (8 * b)) & 0xff);
            h *= 1099511628211ull;
        }
    };
    mix(opt.precision);
    for (size_t k = 0; k < H.size(); ++k) {
        mix(H[k]->n_rows);
        mix(H[k]->nnz);
        mix(n_c[k]);
        for (int c = 0; c < n_c[k]; ++c) mix(C[k][c].nnz);
    }
    return h;
}

// The autotuner (ss_options.autotune): coordinate descent from the rules'
// choice over probes of the batch's first systems; the result is kept in the
// context's table for batches of the same shape.
ss_status autotune_batch(ss_ctx ctx, const BatchWave& w, TuneChoice* out) {
    const unsigned long long key = batch_shape_key(w.opt, w.H, w.n_c, w.C);
    auto it = ctx->tune_table.find(key);
    if (it != ctx->tune_table.end()) {
        *out = TuneChoice{it->second[0], it->second[1], it->second[2], it->second[3]};
        return SS_OK;
    }
    TuneProbe t;
    t.ctx = ctx;
    t.opt = w.opt;
    t.opt.maxiter = 8;
    t.opt.warm_start = 0;
    t.opt.autotune = 0;
    const size_t k = std::min<size_t>(w.H.size(), (size_t)std::max(1, ctx->num_sms));
    size_t total = 0;
    for (size_t q = 0; q < k; ++q) total += (size_t)w.H[q]->n_rows * w.H[q]->n_rows;
    double2* scratch = nullptr;
    SS_TRY(dev_alloc_n(ctx, &scratch, total));
    size_t off = 0;
    for (size_t q = 0; q < k; ++q) {
        t.H.push_back(w.H[q]);
        t.C.push_back(w.C[q]);
        t.n_c.push_back(w.n_c[q]);
        t.rho.push_back(reinterpret_cast<double*>(scratch + off));
        off += (size_t)w.H[q]->n_rows * w.H[q]->n_rows;
    }
    TuneChoice best{0, 0, 0, 0};
    tune_search(TuneChoice{0, 0, 0, 0}, probe_cost, &t, 10, &best, nullptr);
    dev_free(ctx, scratch);
    SS_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    ctx->tune_table[key] = {best.lo, best.up, best.a, best.stage};
    *out = best;
    return SS_OK;
}

}  // namespace

extern "C" ss_status steady_state_batched(ss_ctx ctx, int n_sys, const ss_csr_view* H, const int* n_c,
                                          const ss_csr_view* const* c_ops, const ss_options* opt_in,
                                          double* const* rho_out, int rho_on_device, ss_info* infos) {
    if (!ctx) return SS_ERR_INVALID;
    SS_CUDA(ctx, cudaSetDevice(ctx->device));
    if (n_sys < 0 || (n_sys > 0 && (!H || !n_c || !rho_out))) return set_error(ctx, SS_ERR_INVALID, "null argument");
    ss_options opt;
    ss_options_default(&opt);
    if (opt_in) opt = *opt_in;
    const bool mixed = opt.precision == SS_PREC_MIXED;
    const bool fast = opt.method == SS_METHOD_ITER_BICGSTAB && opt.precond == SS_PRECOND_ILU0;
    const int max_n_fast = batch_max_n(mixed);
    std::vector<int> slow;
    std::vector<int> fastidx;
    for (int k = 0; k < n_sys; ++k) {
        const int64_t d = H[k].n_rows;
        if (fast && d > 0 && d * d <= max_n_fast) fastidx.push_back(k);
        else slow.push_back(k);
    }
    // systems outside the persistent kernel's scope: the single-system path
    ss_status worst = SS_OK;
    for (int k : slow) {
        ss_info inf{};
        ss_status st = steady_state(ctx, &H[k], n_c[k], n_c[k] ? c_ops[k] : nullptr, &opt, rho_out[k],
                                    rho_on_device, &inf);
        if (infos) infos[k] = inf;
        if (st != SS_OK && st != SS_NOT_CONVERGED && st != SS_BREAKDOWN) return st;
        if (st != SS_OK) worst = st;
    }
    if (fastidx.empty()) return worst;
    BatchWave w;
    w.ctx = ctx;
    w.opt = opt;
    w.rho_on_device = rho_on_device;
    for (int k : fastidx) {
        w.H.push_back(&H[k]);
        w.n_c.push_back(n_c[k]);
        w.C.push_back(n_c[k] ? c_ops[k] : nullptr);
        w.rho_out.push_back(rho_out[k]);
    }
    if (opt.autotune) SS_TRY(autotune_batch(ctx, w, &w.tune));
    if (!rho_on_device) {
        // host results come back through the context's pinned buffer: one
        // asynchronous copy per system there, then host copies (pageable
        // destinations would make every device copy a staged, blocking one)
        const size_t need = wave_pinned_bytes(w);
        if (ctx->host_stage_bytes < need) {
            if (ctx->host_stage) cudaFreeHost(ctx->host_stage);
            ctx->host_stage = nullptr;
            ctx->host_stage_bytes = 0;
            if (cudaHostAlloc(&ctx->host_stage, need, cudaHostAllocDefault) == cudaSuccess)
                ctx->host_stage_bytes = need;
            else
                cudaGetLastError();          // no pinned memory: pageable copies instead
        }
        if (ctx->host_stage) {
            w.stage_pinned = true;
            w.stage = static_cast<double2*>(ctx->host_stage);
        }
    }
    SS_TRY(wave_begin(w));
    std::vector<ss_info> winf(fastidx.size());
    ss_status st = wave_end(w, winf.data());
    if (infos)
        for (size_t q = 0; q < fastidx.size(); ++q) infos[fastidx[q]] = winf[q];
    if (st != SS_OK && st != SS_NOT_CONVERGED && st != SS_BREAKDOWN) return st;
    if (st != SS_OK && worst == SS_OK) worst = st;
    if (worst != SS_OK) ctx->last_error = "at least one system did not converge (see infos)";
    return worst;
}

extern "C" ss_status assemble_trace_batched(ss_ctx ctx, int n_sys, const ss_csr_view* H, const int* n_c,
                                            const ss_csr_view* const* c_ops, double w, ss_mat* out,
                                            double* w_used) {
    if (!ctx) return SS_ERR_INVALID;
    SS_CUDA(ctx, cudaSetDevice(ctx->device));
    if (n_sys < 0 || (n_sys > 0 && (!H || !n_c || !out))) return set_error(ctx, SS_ERR_INVALID, "null argument");
    for (int k = 0; k < n_sys; ++k) out[k] = nullptr;
    if (n_sys == 0) return SS_OK;
    std::vector<const ss_csr_view*> Hv(n_sys), Cv(n_sys);
    std::vector<int> ncv(n_sys);
    for (int k = 0; k < n_sys; ++k) {
        Hv[k] = &H[k];
        ncv[k] = n_c[k];
        Cv[k] = n_c[k] ? (c_ops ? c_ops[k] : nullptr) : nullptr;
    }
    BatchLt blt;
    SS_TRY(batch_trace_systems(ctx, Hv, ncv, Cv, w, blt));
    ss_status st = SS_OK;
    for (int k = 0; k < n_sys && st == SS_OK; ++k) {
        DeviceCSR m;
        m.n_rows = m.n_cols = blt.n[k];
        m.nnz = blt.meta[k].nnz;
        st = dev_alloc_n(ctx, &m.row_ptr, (size_t)m.n_rows + 1);
        if (st == SS_OK) st = dev_alloc_n(ctx, &m.col, (size_t)m.nnz);
        if (st == SS_OK) st = dev_alloc_n(ctx, &m.val, (size_t)m.nnz);
        cudaError_t e = cudaSuccess;
        if (st == SS_OK)
            e = cudaMemcpyAsync(m.row_ptr, blt.rp + blt.row_off[k] + k, sizeof(int32_t) * (m.n_rows + 1),
                                cudaMemcpyDeviceToDevice, ctx->stream);
        if (st == SS_OK && e == cudaSuccess && m.nnz > 0)
            e = cudaMemcpyAsync(m.col, blt.col + blt.meta[k].nz_off, sizeof(int32_t) * m.nnz, cudaMemcpyDeviceToDevice,
                                ctx->stream);
        if (st == SS_OK && e == cudaSuccess && m.nnz > 0)
            e = cudaMemcpyAsync(m.val, blt.val + blt.meta[k].nz_off, sizeof(double2) * m.nnz,
                                cudaMemcpyDeviceToDevice, ctx->stream);
        if (st == SS_OK && e != cudaSuccess) st = cuda_check(ctx, e, "assemble_trace_batched");
        ss_mat h = nullptr;
        if (st == SS_OK) {
            h = new (std::nothrow) ss_mat_s();
            if (!h) st = set_error(ctx, SS_ERR_OOM, "host allocation failed");
        }
        if (st != SS_OK) {
            free_csr(ctx, m);
            break;
        }
        h->m = m;
        h->d = blt.d[k];
        out[k] = h;
    }
    if (w_used && st == SS_OK)
        for (int k = 0; k < n_sys; ++k) w_used[k] = blt.w[k];
    cudaError_t e = cudaStreamSynchronize(ctx->stream);
    batch_lt_free(ctx, blt);
    if (st == SS_OK && e != cudaSuccess) st = cuda_check(ctx, e, "assemble_trace_batched");
    if (st != SS_OK)
        for (int k = 0; k < n_sys; ++k)
            if (out[k]) {
                ss_mat_free(out[k]);
                out[k] = nullptr;
            }
    return st;
}
