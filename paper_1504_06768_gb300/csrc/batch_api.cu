// steady_state_batched: many independent systems solved by one persistent
// launch of the per-system CTA solver.  Systems that share a sparsity pattern
// (parameter sweeps) share the RCM ordering, the level schedule and the
// triangular-solve units, which are computed once per pattern on the host.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <map>
#include <memory>
#include <thread>
#include <vector>

#include "batched.cuh"
#include "common.cuh"

namespace {

double now_ms() {
    using namespace std::chrono;
    return duration<double, std::milli>(steady_clock::now().time_since_epoch()).count();
}

struct PackedDev {                        // device arrays of one packed operand (per pattern)
    int32_t *rows = nullptr, *col = nullptr, *src = nullptr, *ovb = nullptr, *ove = nullptr, *lvl = nullptr;
    int32_t nunits = 0, G = 1, E = 1, nlev = 0;
};

struct Pattern {                          // per distinct pattern of L~ (before ordering)
    std::vector<int32_t> rp, col;         // natural-order pattern (for exact comparison)
    std::vector<int32_t> perm, iperm, tidx;
    int32_t r0 = 0;
    int64_t bw = 0, profile = 0;
    // device arrays of the permuted structure
    int32_t *perm_d = nullptr, *tidx_d = nullptr, *dpos_d = nullptr;
    int32_t *lo_units = nullptr, *up_units = nullptr, *lvl_ptr = nullptr, *lvl_rows = nullptr;
    int32_t lo_nunits = 0, up_nunits = 0, lo_g = 1, up_g = 1, a_g = 1, n_levels = 0, up_levels = 0;
    PackedDev lo, up, pa;
};

uint64_t fnv1a(const std::vector<int32_t>& a, uint64_t h) {
    for (int32_t v : a) {
        h ^= (uint32_t)v;
        h *= 1099511628211ull;
    }
    return h;
}

int lanes_for(double avg) {
    int g = 1;
    while (g < 32 && 2.0 * g < avg) g <<= 1;
    return g;
}

// Lane-major packing of one CSR operand (see PackedOp): unit_rows holds R = 32/G
// row ids per unit; range(i) gives the CSR range [s, e) of row i's entries.
struct PackedHost {
    std::vector<int32_t> rows, col, src, ovb, ove, lvl;
    int32_t nunits = 0, G = 1, E = 1, nlev = 0;
};

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
    P.E = std::max(1, std::min(4, (p99 + G - 1) / G));
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

ss_status build_pattern(ss_ctx ctx, Pattern& P, const DeviceCSR& A, int64_t d, int use_rcm) {
    const int64_t n = A.n_rows;
    P.perm.resize(n);
    if (use_rcm) rcm_host(n, P.rp.data(), P.col.data(), P.perm.data());
    else for (int64_t i = 0; i < n; ++i) P.perm[i] = (int32_t)i;
    P.iperm.resize(n);
    for (int64_t r = 0; r < n; ++r) P.iperm[P.perm[r]] = (int32_t)r;
    P.tidx.resize(d);
    for (int64_t i = 0; i < d; ++i) P.tidx[i] = P.iperm[i * (d + 1)];
    P.r0 = P.iperm[0];
    // permuted pattern on the host (rows gathered, columns relabelled and sorted)
    std::vector<int32_t> prp(n + 1, 0), pcol(P.col.size());
    for (int64_t r = 0; r < n; ++r) prp[r + 1] = prp[r] + (P.rp[P.perm[r] + 1] - P.rp[P.perm[r]]);
    std::vector<int32_t> dpos(n, -1);
    for (int64_t r = 0; r < n; ++r) {
        int32_t o = prp[r], i = P.perm[r];
        for (int32_t t = P.rp[i]; t < P.rp[i + 1]; ++t) pcol[o++] = P.iperm[P.col[t]];
        std::sort(pcol.begin() + prp[r], pcol.begin() + prp[r + 1]);
        for (int32_t t = prp[r]; t < prp[r + 1]; ++t)
            if (pcol[t] == r) dpos[r] = t;
    }
    int64_t lo = 0, up = 0;
    P.bw = 0;
    for (int64_t r = 0; r < n; ++r) {
        if (dpos[r] < 0) return set_error(ctx, SS_ZERO_PIVOT, "iLU(0): missing diagonal entry in row " + std::to_string(r));
        lo += dpos[r] - prp[r];
        up += prp[r + 1] - dpos[r] - 1;
    }
    std::vector<int32_t> lorder, lptr, uorder, uptr, lunits, uunits;
    P.n_levels = level_sets_host(n, prp.data(), pcol.data(), true, lorder, lptr);
    P.up_levels = level_sets_host(n, prp.data(), pcol.data(), false, uorder, uptr);
    P.lo_g = lanes_for(n ? (double)lo / n : 1.0);
    P.up_g = lanes_for(n ? (double)up / n : 1.0);
    P.a_g = lanes_for(n ? (double)P.col.size() / n : 1.0);
    level_units_host(lorder, lptr, 32 / P.lo_g, lunits);
    level_units_host(uorder, uptr, 32 / P.up_g, uunits);
    P.lo_nunits = (int32_t)(lunits.size() / (32 / P.lo_g));
    P.up_nunits = (int32_t)(uunits.size() / (32 / P.up_g));
    // packed operands: the two triangles (level-aligned units) and A (consecutive rows)
    PackedHost hl, hu, ha;
    pack_host(lunits, P.lo_g, pcol, [&](int32_t i) { return std::make_pair(prp[i], dpos[i]); }, hl);
    pack_host(uunits, P.up_g, pcol, [&](int32_t i) { return std::make_pair(dpos[i] + 1, prp[i + 1]); }, hu);
    hl.lvl = unit_levels(lptr, 32 / P.lo_g);
    hu.lvl = unit_levels(uptr, 32 / P.up_g);
    hl.nlev = (int32_t)hl.lvl.size() - 1;
    hu.nlev = (int32_t)hu.lvl.size() - 1;
    {
        const int R = 32 / P.a_g;
        std::vector<int32_t> arows(((n + R - 1) / R) * R, -1);
        for (int64_t i = 0; i < n; ++i) arows[i] = (int32_t)i;
        pack_host(arows, P.a_g, pcol, [&](int32_t i) { return std::make_pair(prp[i], prp[i + 1]); }, ha);
    }
    auto up_packed = [&](PackedHost& h, PackedDev& dv) -> ss_status {
        dv.nunits = h.nunits;
        dv.G = h.G;
        dv.E = h.E;
        SS_TRY(upload_vec(ctx, h.rows, &dv.rows));
        SS_TRY(upload_vec(ctx, h.col, &dv.col));
        SS_TRY(upload_vec(ctx, h.src, &dv.src));
        SS_TRY(upload_vec(ctx, h.ovb, &dv.ovb));
        SS_TRY(upload_vec(ctx, h.ove, &dv.ove));
        dv.nlev = h.nlev;
        if (h.nlev > 0) SS_TRY(upload_vec(ctx, h.lvl, &dv.lvl));
        return SS_OK;
    };
    SS_TRY(up_packed(hl, P.lo));
    SS_TRY(up_packed(hu, P.up));
    SS_TRY(up_packed(ha, P.pa));
    SS_TRY(upload_vec(ctx, P.perm, &P.perm_d));
    SS_TRY(upload_vec(ctx, P.tidx, &P.tidx_d));
    SS_TRY(upload_vec(ctx, dpos, &P.dpos_d));
    SS_TRY(upload_vec(ctx, lunits, &P.lo_units));
    SS_TRY(upload_vec(ctx, uunits, &P.up_units));
    SS_TRY(upload_vec(ctx, lptr, &P.lvl_ptr));
    SS_TRY(upload_vec(ctx, lorder, &P.lvl_rows));
    return SS_OK;
}

void free_packed(ss_ctx ctx, PackedDev& d) {
    dev_free(ctx, d.rows);
    dev_free(ctx, d.col);
    dev_free(ctx, d.src);
    dev_free(ctx, d.ovb);
    dev_free(ctx, d.ove);
    dev_free(ctx, d.lvl);
}

void free_pattern(ss_ctx ctx, Pattern& P) {
    free_packed(ctx, P.lo);
    free_packed(ctx, P.up);
    free_packed(ctx, P.pa);
    dev_free(ctx, P.perm_d);
    dev_free(ctx, P.tidx_d);
    dev_free(ctx, P.dpos_d);
    dev_free(ctx, P.lo_units);
    dev_free(ctx, P.up_units);
    dev_free(ctx, P.lvl_ptr);
    dev_free(ctx, P.lvl_rows);
}

}  // namespace

extern "C" ss_status steady_state(ss_ctx, const ss_csr_view*, int, const ss_csr_view*, const ss_options*, double*, int,
                                  ss_info*);

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
    const double t0 = now_ms();
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

    // ------------------------------------------------------------ setup
    struct Sys {
        ss_mat L = nullptr, A = nullptr;
        DeviceCSR Ap;
        int pat = -1;
        double w = 0.0;
    };
    std::vector<Sys> sys(fastidx.size());
    std::vector<std::unique_ptr<Pattern>> pats;
    std::map<uint64_t, std::vector<int>> by_hash;
    std::vector<void*> owned;
    auto cleanup = [&]() {
        for (auto& s : sys) {
            if (s.L) ss_mat_free(s.L);
            if (s.A) ss_mat_free(s.A);
            free_csr(ctx, s.Ap);
        }
        for (auto& p : pats) free_pattern(ctx, *p);
        for (void* p : owned) dev_free(ctx, p);
        cudaStreamSynchronize(ctx->stream);
    };
#define BSTEP(call) do { ss_status _st = (call); if (_st != SS_OK) { cleanup(); return _st; } } while (0)
    // Setup runs on worker threads, each with its own stream: (A) assembly,
    // trace row and the pattern of L~; (B, serial) one RCM ordering and level
    // schedule per distinct pattern; (C) the symmetric permutations.
    const size_t ns = fastidx.size();
    const int nthreads = (int)std::max<size_t>(
        1, std::min<size_t>(ns, std::min<unsigned>(16u, std::max(1u, std::thread::hardware_concurrency()))));
    std::vector<ss_ctx_s> wctx(nthreads);
    for (auto& w : wctx) {
        w.device = ctx->device;
        w.num_sms = ctx->num_sms;
        SS_CUDA(ctx, cudaStreamCreateWithFlags(&w.stream, cudaStreamNonBlocking));
    }
    auto drop_streams = [&]() {
        for (auto& w : wctx) {
            cudaStreamSynchronize(w.stream);
            cudaStreamDestroy(w.stream);
        }
    };
    std::vector<std::vector<int32_t>> prps(ns), pcols(ns);
    std::vector<ss_status> wst(ns, SS_OK);
    std::vector<std::string> werr(ns);
    std::vector<int64_t> dims(ns, 0);
    auto run_workers = [&](auto&& body) {
        std::vector<std::thread> th;
        for (int t = 0; t < nthreads; ++t)
            th.emplace_back([&, t]() {
                cudaSetDevice(ctx->device);
                for (size_t q = t; q < ns; q += nthreads) body(&wctx[t], q);
                cudaStreamSynchronize(wctx[t].stream);
            });
        for (auto& x : th) x.join();
        for (size_t q = 0; q < ns; ++q)
            if (wst[q] != SS_OK) return (ss_status)set_error(ctx, wst[q], werr[q]);
        return SS_OK;
    };
    ss_status pst = run_workers([&](ss_ctx wc, size_t q) {
        const int k = fastidx[q];
        ss_status st = assemble_liouvillian(wc, &H[k], n_c[k], n_c[k] ? c_ops[k] : nullptr, &sys[q].L);
        if (st == SS_OK) st = add_trace_row(wc, sys[q].L, opt.w, &sys[q].A, &sys[q].w);
        if (st == SS_OK) {
            const DeviceCSR& A = sys[q].A->m;
            dims[q] = sys[q].L->d;
            prps[q].resize(A.n_rows + 1);
            pcols[q].resize(A.nnz);
            cudaMemcpyAsync(prps[q].data(), A.row_ptr, sizeof(int32_t) * prps[q].size(), cudaMemcpyDeviceToHost,
                            wc->stream);
            cudaMemcpyAsync(pcols[q].data(), A.col, sizeof(int32_t) * pcols[q].size(), cudaMemcpyDeviceToHost,
                            wc->stream);
            cudaError_t e = cudaStreamSynchronize(wc->stream);
            if (e != cudaSuccess) st = cuda_check(wc, e, "pattern download");
        }
        if (sys[q].L) {
            ss_mat_free(sys[q].L);
            sys[q].L = nullptr;
        }
        wst[q] = st;
        if (st != SS_OK) werr[q] = wc->last_error;
    });
    if (pst != SS_OK) { drop_streams(); cleanup(); return pst; }
    int max_n = 0;
    for (size_t q = 0; q < ns; ++q) {
        const uint64_t h = fnv1a(pcols[q], fnv1a(prps[q], 1469598103934665603ull));
        int found = -1;
        for (int pi : by_hash[h])
            if (pats[pi]->rp == prps[q] && pats[pi]->col == pcols[q]) { found = pi; break; }
        if (found < 0) {
            pats.emplace_back(new Pattern());
            Pattern& P = *pats.back();
            P.rp.swap(prps[q]);
            P.col.swap(pcols[q]);
            ss_status st = build_pattern(ctx, P, sys[q].A->m, dims[q], opt.use_rcm);
            if (st != SS_OK) { drop_streams(); cleanup(); return st; }
            found = (int)pats.size() - 1;
            by_hash[h].push_back(found);
        }
        sys[q].pat = found;
        max_n = std::max<int>(max_n, (int)sys[q].A->m.n_rows);
    }
    pst = run_workers([&](ss_ctx wc, size_t q) {
        wst[q] = permute_impl(wc, sys[q].A->m, pats[sys[q].pat]->perm.data(), sys[q].Ap);
        if (wst[q] != SS_OK) werr[q] = wc->last_error;
    });
    drop_streams();
    if (pst != SS_OK) { cleanup(); return pst; }
    // per-system buffers and descriptors
    std::vector<BatchSys> hs(fastidx.size());
    for (size_t q = 0; q < fastidx.size(); ++q) {
        const Pattern& P = *pats[sys[q].pat];
        const DeviceCSR& Ap = sys[q].Ap;
        const int64_t n = Ap.n_rows, nnz = Ap.nnz;
        BatchSys& b = hs[q];
        std::memset(&b, 0, sizeof(b));
        b.n = (int32_t)n;
        b.d = (int32_t)sys[q].A->d;
        b.a_rp = Ap.row_ptr;
        b.a_col = Ap.col;
        b.a_val = Ap.val;
        b.f_rp = Ap.row_ptr;
        b.f_col = Ap.col;
        b.f_dpos = P.dpos_d;
        b.factor_on_device = 1;
        const size_t inner = mixed ? sizeof(float2) : sizeof(double2);
        char* blk = nullptr;
        const size_t pk_slots = ((size_t)P.lo.nunits * P.lo.E + (size_t)P.up.nunits * P.up.E +
                                 (size_t)P.pa.nunits * P.pa.E) * 32;
        const size_t bytes = nnz * sizeof(double2) + n * sizeof(double2) + (mixed ? 2 * nnz * sizeof(float2) + n * sizeof(float2) : 0) +
                             10 * n * inner + 2 * n * sizeof(double2) + (rho_on_device ? 0 : n * sizeof(double2)) +
                             pk_slots * inner + 8 * 256;
        BSTEP(dev_alloc(ctx, reinterpret_cast<void**>(&blk), bytes));
        owned.push_back(blk);
        size_t off = 0;
        auto take = [&](size_t sz) { char* p = blk + off; off += (sz + 15) & ~size_t(15); return p; };
        b.f_val = reinterpret_cast<double2*>(take(nnz * sizeof(double2)));
        b.f_inv = reinterpret_cast<double2*>(take(n * sizeof(double2)));
        if (mixed) {
            b.f_val32 = reinterpret_cast<float2*>(take(nnz * sizeof(float2)));
            b.a_val32 = reinterpret_cast<float2*>(take(nnz * sizeof(float2)));
            b.f_inv32 = reinterpret_cast<float2*>(take(n * sizeof(float2)));
        }
        b.work = take(10 * n * inner);
        b.x64 = reinterpret_cast<double2*>(take(n * sizeof(double2)));
        b.r64 = reinterpret_cast<double2*>(take(n * sizeof(double2)));
        b.rho_out = rho_on_device ? reinterpret_cast<double2*>(rho_out[fastidx[q]])
                                  : reinterpret_cast<double2*>(take(n * sizeof(double2)));
        auto set_op = [&](PackedOp& o, const PackedDev& dv) {
            o.rows = dv.rows;
            o.col = dv.col;
            o.src = dv.src;
            o.ovb = dv.ovb;
            o.ove = dv.ove;
            o.nunits = dv.nunits;
            o.G = dv.G;
            o.E = dv.E;
            o.lvl = dv.lvl;
            o.nlev = dv.nlev;
            o.val = take((size_t)dv.nunits * dv.E * 32 * inner);
        };
        set_op(b.lo, P.lo);
        set_op(b.up, P.up);
        set_op(b.pa, P.pa);
        b.lvl_ptr = P.lvl_ptr;
        b.lvl_rows = P.lvl_rows;
        b.n_levels = P.n_levels;
        b.r0 = P.r0;
        b.w = sys[q].w;
        b.sigma = 0.0;
        b.perm = P.perm_d;
        b.tidx = P.tidx_d;
    }
    BatchSys* dsys = nullptr;
    int* ctl = nullptr;
    BSTEP(dev_alloc_n(ctx, &dsys, hs.size()));
    owned.push_back(dsys);
    BSTEP(dev_alloc_n(ctx, &ctl, 4));
    owned.push_back(ctl);
    SS_CUDA(ctx, cudaMemcpyAsync(dsys, hs.data(), sizeof(BatchSys) * hs.size(), cudaMemcpyHostToDevice, ctx->stream));
    SS_CUDA(ctx, cudaMemsetAsync(ctl, 0, sizeof(int) * 4, ctx->stream));
    const double t1 = now_ms();

    BatchParams bp;
    bp.tol = opt.tol;
    bp.maxiter = opt.maxiter;
    bp.mixed = mixed ? 1 : 0;
    bp.inner_rtol = opt.inner_rtol > 0 ? opt.inner_rtol : 1e-5;
    bp.power = 0;
    bp.seed = opt.seed;
    BSTEP(batch_launch(ctx, dsys, (int)hs.size(), bp, max_n, ctl, ctl + 1));
    SS_CUDA(ctx, cudaMemcpyAsync(hs.data(), dsys, sizeof(BatchSys) * hs.size(), cudaMemcpyDeviceToHost, ctx->stream));
    int herr = 0;
    SS_CUDA(ctx, cudaMemcpyAsync(&herr, ctl + 1, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
    if (!rho_on_device)
        for (size_t q = 0; q < fastidx.size(); ++q)
            SS_CUDA(ctx, cudaMemcpyAsync(rho_out[fastidx[q]], hs[q].rho_out, sizeof(double2) * hs[q].n,
                                         cudaMemcpyDeviceToHost, ctx->stream));
    cudaError_t e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) { cleanup(); return cuda_check(ctx, e, "steady_state_batched"); }
    // (the copies above read hs[q].rho_out, which the kernel does not change)
    const double t2 = now_ms();
    for (size_t q = 0; q < fastidx.size(); ++q) {
        const int k = fastidx[q];
        const Pattern& P = *pats[sys[q].pat];
        if (herr) hs[q].status = SS_ERR_TIMEOUT;
        if (infos) {
            ss_info& inf = infos[k];
            std::memset(&inf, 0, sizeof(inf));
            inf.status = hs[q].status;
            inf.iters = hs[q].iters;
            inf.outer_iters = hs[q].outer;
            inf.resid_Lrho = hs[q].resid;
            inf.w_used = sys[q].w;
            inf.n = hs[q].n;
            inf.nnz = sys[q].Ap.nnz;
            inf.nnz_factors = sys[q].Ap.nnz;
            inf.levels_lower = P.n_levels;
            inf.levels_upper = P.up_levels;
            inf.ms_setup = (t1 - t0) / fastidx.size();
            inf.ms_solve = (t2 - t1) / fastidx.size();
        }
        if (hs[q].status != SS_OK) {
            if (hs[q].status != SS_NOT_CONVERGED && hs[q].status != SS_BREAKDOWN) worst = (ss_status)hs[q].status;
            else if (worst == SS_OK) worst = (ss_status)hs[q].status;
        }
    }
    cleanup();
#undef BSTEP
    if (worst != SS_OK) ctx->last_error = "at least one system did not converge (see infos)";
    return worst;
}
