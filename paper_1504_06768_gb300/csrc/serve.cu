// Serving loop: steady-state requests arrive at any time (ss_submit) and are
// solved while others are on the device.  A worker thread admits queued
// requests in arrival order whenever a wave slot is free and their estimated
// device footprint fits the memory budget, and launches them as one wave of
// the persistent per-system solver on the slot's own stream.  A wave holds one
// SM per system, so several waves run side by side and a new wave fills the
// SMs an earlier one leaves idle (continuous batching at the granularity of
// SMs).  Pattern analyses (RCM ordering, level schedule, packing) stay
// resident across waves for requests with the same structure.  Systems beyond
// the persistent solver's scope, or options it does not run, go to a second
// lane that uses the single-system path.  Results go to the caller's host
// buffer; ss_poll and ss_wait report completion.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <memory>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

#include "batch_wave.cuh"

extern "C" ss_status steady_state(ss_ctx, const ss_csr_view*, int, const ss_csr_view*, const ss_options*, double*, int,
                                  ss_info*);

namespace {

double now_ms() {
    using namespace std::chrono;
    return duration<double, std::milli>(steady_clock::now().time_since_epoch()).count();
}

struct OwnedCsr {                        // a host CSR view and the arrays it points at
    std::vector<int32_t> rp, col;
    std::vector<double> val;
    ss_csr_view view{};
    void copy(const ss_csr_view& v) {
        rp.assign(v.row_ptr, v.row_ptr + v.n_rows + 1);
        col.assign(v.col, v.col + v.nnz);
        val.assign(v.val, v.val + 2 * v.nnz);
        view = v;
        view.row_ptr = rp.data();
        view.col = col.data();
        view.val = val.data();
        view.on_device = 0;
    }
};

struct Request {
    uint64_t id = 0;
    OwnedCsr H;
    std::vector<OwnedCsr> C;
    std::vector<ss_csr_view> cviews;
    double* rho_out = nullptr;
    size_t footprint = 0;
    bool fast = false;
    double t_submit = 0, t_done = 0;
    ss_info info{};
    ss_status status = SS_OK;
    bool done = false;
};

struct Slot {
    std::unique_ptr<ss_ctx_s> ctx;
    BatchWave wave;
    std::vector<std::shared_ptr<Request>> reqs;
    double2* pinned = nullptr;
    size_t pinned_bytes = 0;
    bool busy = false;
};

}  // namespace

struct ss_server_s {
    int device = 0;
    ss_options opt{};
    ss_server_options so{};
    size_t budget = 0, in_use = 0;
    PatternCache cache;
    SolutionCache sols;                  // warm starts (so.warm_start)
    std::vector<Slot> slots;
    std::vector<std::unique_ptr<ss_ctx_s>> large_ctx;   // one context (stream) per single-system worker
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<std::shared_ptr<Request>> q_fast, q_large;
    std::unordered_map<uint64_t, std::shared_ptr<Request>> live;
    uint64_t next_id = 1;
    bool stop = false;
    std::thread worker;
    std::vector<std::thread> large_workers;
    std::string last_error;
    uint64_t waves = 0, completed = 0;
};

namespace {

void finish(ss_server s, const std::shared_ptr<Request>& r, ss_status st, const ss_info* inf) {
    std::lock_guard<std::mutex> lock(s->mu);
    if (inf) r->info = *inf;
    r->status = st;
    r->info.status = st;
    r->t_done = now_ms();
    r->done = true;
    s->in_use -= std::min(s->in_use, r->footprint);
    ++s->completed;
    s->cv_done.notify_all();
    s->cv_work.notify_all();
}

// Retire every slot whose wave has completed.
void retire(ss_server s) {
    for (Slot& sl : s->slots) {
        if (!sl.busy || !wave_ready(sl.wave)) continue;
        std::vector<ss_info> inf(sl.reqs.size());
        const ss_status st = wave_end(sl.wave, inf.data());
        for (size_t q = 0; q < sl.reqs.size(); ++q) {
            ss_status rs = (ss_status)inf[q].status;
            if (st != SS_OK && st != SS_NOT_CONVERGED && st != SS_BREAKDOWN) rs = st;   // the wave itself failed
            finish(s, sl.reqs[q], rs, &inf[q]);
        }
        sl.reqs.clear();
        sl.busy = false;
    }
}

void fast_lane(ss_server s) {
    cudaSetDevice(s->device);
    while (true) {
        retire(s);
        Slot* free_slot = nullptr;
        bool busy = false;
        for (Slot& sl : s->slots) {
            busy = busy || sl.busy;
            if (!sl.busy && !free_slot) free_slot = &sl;
        }
        std::vector<std::shared_ptr<Request>> take;
        {
            std::unique_lock<std::mutex> lock(s->mu);
            if (s->stop && s->q_fast.empty() && !busy) return;
            if (free_slot) {
                // arrival order; the head waits until it fits the budget
                while (!s->q_fast.empty() && (int)take.size() < s->so.max_wave_systems &&
                       s->in_use + s->q_fast.front()->footprint <= s->budget) {
                    s->in_use += s->q_fast.front()->footprint;
                    take.push_back(s->q_fast.front());
                    s->q_fast.pop_front();
                }
            }
            if (take.empty()) {
                if (busy) s->cv_work.wait_for(lock, std::chrono::microseconds(50));
                else
                    s->cv_work.wait(lock, [&] {
                        return s->stop ||
                               (!s->q_fast.empty() && s->in_use + s->q_fast.front()->footprint <= s->budget);
                    });
                continue;
            }
        }
        Slot& sl = *free_slot;
        BatchWave& w = sl.wave;
        w = BatchWave();
        w.ctx = sl.ctx.get();
        w.opt = s->opt;
        w.rho_on_device = 0;
        w.stage_pinned = true;
        w.cache = &s->cache;
        w.sols = s->so.warm_start ? &s->sols : nullptr;
        for (auto& r : take) {
            w.H.push_back(&r->H.view);
            w.n_c.push_back((int)r->cviews.size());
            w.C.push_back(r->cviews.empty() ? nullptr : r->cviews.data());
            w.rho_out.push_back(r->rho_out);
        }
        const size_t need = wave_pinned_bytes(w);
        ss_status st = SS_OK;
        if (need > sl.pinned_bytes) {
            const size_t grow = std::max(need, (size_t)2 * sl.pinned_bytes);
            if (sl.pinned) cudaFreeHost(sl.pinned);
            sl.pinned = nullptr;
            sl.pinned_bytes = 0;
            ss_count_alloc();
            if (cudaMallocHost(reinterpret_cast<void**>(&sl.pinned), grow) != cudaSuccess) {
                cudaGetLastError();
                st = SS_ERR_OOM;
            } else {
                sl.pinned_bytes = grow;
            }
        }
        w.stage = sl.pinned;
        if (st == SS_OK) st = wave_begin(w);
        if (st != SS_OK) {
            {
                std::lock_guard<std::mutex> lock(s->mu);
                s->last_error = sl.ctx->last_error;
            }
            for (auto& r : take) finish(s, r, st, nullptr);
            continue;
        }
        sl.reqs = std::move(take);
        sl.busy = true;
        std::lock_guard<std::mutex> lock(s->mu);
        ++s->waves;
    }
}

// Single-system requests: LARGE_WORKERS threads, each with its own stream, so
// that several large solves (latency-bound chains of small launches) overlap.
constexpr int LARGE_WORKERS = 2;

void large_lane(ss_server s, int wid) {
    cudaSetDevice(s->device);
    while (true) {
        std::shared_ptr<Request> r;
        {
            std::unique_lock<std::mutex> lock(s->mu);
            s->cv_work.wait(lock, [&] {
                return (s->stop && s->q_large.empty()) ||
                       (!s->q_large.empty() && s->in_use + s->q_large.front()->footprint <= s->budget);
            });
            if (s->q_large.empty()) return;
            r = s->q_large.front();
            s->q_large.pop_front();
            s->in_use += r->footprint;
        }
        // FP64 here: the single-system mixed form pays more iterations than it saves on
        // systems this large (optomechanics 10 x 40: 2.6 against 0.96 s per solve)
        ss_info inf{};
        ss_options o = s->opt;
        o.precision = SS_PREC_FP64;
        const ss_status st = steady_state(s->large_ctx[wid].get(), &r->H.view, (int)r->cviews.size(),
                                          r->cviews.empty() ? nullptr : r->cviews.data(), &o, r->rho_out, 0, &inf);
        if (st != SS_OK && st != SS_NOT_CONVERGED && st != SS_BREAKDOWN) {
            std::lock_guard<std::mutex> lock(s->mu);
            s->last_error = s->large_ctx[wid]->last_error;
        }
        finish(s, r, st, &inf);
    }
}

// high: the waves' streams (their blocks are scheduled first when SMs free
// up); otherwise the lowest priority (the single-system lane, whose many small
// launches would otherwise hold SMs a wave's whole-SM blocks are waiting for)
std::unique_ptr<ss_ctx_s> make_ctx(int device, int num_sms, bool high) {
    std::unique_ptr<ss_ctx_s> c(new (std::nothrow) ss_ctx_s());
    if (!c) return nullptr;
    c->device = device;
    c->num_sms = num_sms;
    int least = 0, greatest = 0;
    if (cudaDeviceGetStreamPriorityRange(&least, &greatest) != cudaSuccess) {
        cudaGetLastError();
        least = greatest = 0;
    }
    if (cudaStreamCreateWithPriority(&c->stream, cudaStreamNonBlocking, high ? greatest : least) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    c->pool = device_pool(device);
    return c;
}

}  // namespace

extern "C" void ss_server_options_default(ss_server_options* so) {
    if (!so) return;
    so->hbm_budget_mb = 0.0;
    so->max_waves = 4;
    so->max_wave_systems = 0;
    so->warm_start = 0;
}

extern "C" ss_status ss_server_create(int device, const ss_options* opt, const ss_server_options* so_in,
                                      ss_server* out) {
    if (!out) return SS_ERR_INVALID;
    *out = nullptr;
    int count = 0;
    if (cudaGetDeviceCount(&count) != cudaSuccess || device < 0 || device >= count) {
        cudaGetLastError();
        return SS_ERR_CUDA;
    }
    if (cudaSetDevice(device) != cudaSuccess) return SS_ERR_CUDA;
    std::unique_ptr<ss_server_s> s(new (std::nothrow) ss_server_s());
    if (!s) return SS_ERR_OOM;
    s->device = device;
    ss_options_default(&s->opt);
    if (opt) s->opt = *opt;
    s->opt.warm_start = 0;          // a request's output buffer carries no initial guess
    ss_server_options_default(&s->so);
    if (so_in) s->so = *so_in;
    int sms = 1;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    if (s->so.max_waves < 1) s->so.max_waves = 1;
    if (s->so.max_wave_systems < 1) s->so.max_wave_systems = std::max(1, sms / s->so.max_waves);
    size_t free_b = 0, total_b = 0;
    if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) return SS_ERR_CUDA;
    s->budget = s->so.hbm_budget_mb > 0 ? (size_t)(s->so.hbm_budget_mb * 1048576.0) : (size_t)(0.8 * (double)free_b);
    s->slots.resize(s->so.max_waves);
    for (Slot& sl : s->slots) {
        sl.ctx = make_ctx(device, sms, true);
        if (!sl.ctx) return SS_ERR_CUDA;
    }
    for (int k = 0; k < LARGE_WORKERS; ++k) {
        s->large_ctx.push_back(make_ctx(device, sms, false));
        if (!s->large_ctx.back()) return SS_ERR_CUDA;
    }
    ss_server raw = s.get();
    s->worker = std::thread(fast_lane, raw);
    for (int k = 0; k < LARGE_WORKERS; ++k) s->large_workers.emplace_back(large_lane, raw, k);
    *out = s.release();
    return SS_OK;
}

extern "C" ss_status ss_server_destroy(ss_server s) {
    if (!s) return SS_ERR_INVALID;
    {
        std::lock_guard<std::mutex> lock(s->mu);
        s->stop = true;
    }
    s->cv_work.notify_all();
    if (s->worker.joinable()) s->worker.join();
    for (auto& t : s->large_workers)
        if (t.joinable()) t.join();
    cudaSetDevice(s->device);
    if (!s->slots.empty() && s->slots[0].ctx) {
        s->sols.clear(s->slots[0].ctx.get());       // stream-ordered frees on a slot stream, synchronised below
    }
    for (Slot& sl : s->slots) {
        if (sl.ctx && sl.ctx->stream) {
            cudaStreamSynchronize(sl.ctx->stream);
            cudaStreamDestroy(sl.ctx->stream);
        }
        if (sl.pinned) cudaFreeHost(sl.pinned);
    }
    for (auto& c : s->large_ctx)
        if (c && c->stream) {
            cudaStreamSynchronize(c->stream);
            cudaStreamDestroy(c->stream);
        }
    delete s;
    return SS_OK;
}

extern "C" ss_status ss_submit(ss_server s, const ss_csr_view* H, int n_c, const ss_csr_view* c_ops, double* rho_out,
                               uint64_t* ticket) {
    if (!s || !H || !rho_out || !ticket || n_c < 0 || (n_c > 0 && !c_ops)) return SS_ERR_INVALID;
    *ticket = 0;
    auto fail = [&](ss_status st, const char* msg) {
        std::lock_guard<std::mutex> lock(s->mu);
        s->last_error = msg;
        return st;
    };
    const int64_t d = H->n_rows;
    if (d <= 0 || H->n_cols != d) return fail(SS_ERR_INVALID, "H must be square and non-empty");
    if (H->on_device) return fail(SS_ERR_INVALID, "ss_submit takes host CSR views");
    for (int c = 0; c < n_c; ++c)
        if (c_ops[c].n_rows != d || c_ops[c].n_cols != d || c_ops[c].on_device)
            return fail(SS_ERR_INVALID, "collapse operators must be d x d host CSR views");
    auto r = std::make_shared<Request>();
    r->H.copy(*H);
    r->C.resize(n_c);
    std::vector<int64_t> nnz_c, ctc_c;
    std::vector<int64_t> colcount(d);
    for (int c = 0; c < n_c; ++c) {
        r->C[c].copy(c_ops[c]);
        r->cviews.push_back(r->C[c].view);
        nnz_c.push_back(c_ops[c].nnz);
        // nnz(C^+ C) <= min(d^2, sum over columns of (entries in the column)^2)
        std::fill(colcount.begin(), colcount.end(), 0);
        for (int64_t t = 0; t < c_ops[c].nnz; ++t) {
            const int32_t j = c_ops[c].col[t];
            if (j >= 0 && j < d) ++colcount[j];
        }
        int64_t b = 0;
        for (int64_t k : colcount) b += k * k;
        ctc_c.push_back(std::min(b, d * d));
    }
    r->rho_out = rho_out;
    const bool mixed = s->opt.precision == SS_PREC_MIXED;
    r->fast = s->opt.method == SS_METHOD_ITER_BICGSTAB && s->opt.precond == SS_PRECOND_ILU0 &&
              d * d <= batch_max_n(mixed);
    r->footprint = wave_footprint_bytes(d, H->nnz, nnz_c, ctc_c, mixed);
    r->t_submit = now_ms();
    {
        std::lock_guard<std::mutex> lock(s->mu);
        if (r->footprint > s->budget) {
            s->last_error = "request footprint exceeds the server's device-memory budget";
            return SS_ERR_OOM;
        }
        r->id = s->next_id++;
        s->live[r->id] = r;
        (r->fast ? s->q_fast : s->q_large).push_back(r);
        *ticket = r->id;
    }
    s->cv_work.notify_all();
    return SS_OK;
}

extern "C" ss_status ss_poll(ss_server s, uint64_t ticket, int* done) {
    if (!s || !done) return SS_ERR_INVALID;
    std::lock_guard<std::mutex> lock(s->mu);
    auto it = s->live.find(ticket);
    if (it == s->live.end()) return SS_ERR_INVALID;
    *done = it->second->done ? 1 : 0;
    return SS_OK;
}

extern "C" ss_status ss_wait(ss_server s, uint64_t ticket, int64_t timeout_us, ss_info* info, double* latency_ms) {
    if (!s) return SS_ERR_INVALID;
    std::unique_lock<std::mutex> lock(s->mu);
    auto it = s->live.find(ticket);
    if (it == s->live.end()) return SS_ERR_INVALID;
    std::shared_ptr<Request> r = it->second;
    auto pred = [&] { return r->done; };
    if (timeout_us < 0) s->cv_done.wait(lock, pred);
    else if (!s->cv_done.wait_for(lock, std::chrono::microseconds(timeout_us), pred)) return SS_ERR_TIMEOUT;
    if (info) *info = r->info;
    if (latency_ms) *latency_ms = r->t_done - r->t_submit;
    s->live.erase(ticket);
    return r->status;
}

extern "C" const char* ss_server_last_error(ss_server s) { return s ? s->last_error.c_str() : "null server"; }

extern "C" ss_status ss_server_stats(ss_server s, uint64_t* waves, uint64_t* completed, double* in_use_mb,
                                     double* budget_mb) {
    if (!s) return SS_ERR_INVALID;
    std::lock_guard<std::mutex> lock(s->mu);
    if (waves) *waves = s->waves;
    if (completed) *completed = s->completed;
    if (in_use_mb) *in_use_mb = (double)s->in_use / 1048576.0;
    if (budget_mb) *budget_mb = (double)s->budget / 1048576.0;
    return SS_OK;
}
