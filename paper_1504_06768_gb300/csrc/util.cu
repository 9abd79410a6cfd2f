// Errors, device allocation, scans and small CSR helpers.
#include <atomic>
#include <cstdio>
#include <cstring>

#include <map>
#include <mutex>

#include "common.cuh"

ss_status set_error(ss_ctx ctx, ss_status st, const std::string& msg) {
    if (ctx) ctx->last_error = msg;
    return st;
}

ss_status cuda_check(ss_ctx ctx, cudaError_t e, const char* what) {
    std::string msg = std::string("CUDA error in ") + what + ": " + cudaGetErrorString(e);
    if (e == cudaErrorMemoryAllocation) return set_error(ctx, SS_ERR_OOM, msg);
    return set_error(ctx, SS_ERR_CUDA, msg);
}

// Stream-ordered allocations: freed memory returns to the device pool and is
// reused by later calls on the same stream without a device synchronisation.
ss_status dev_alloc(ss_ctx ctx, void** p, size_t bytes) {
    *p = nullptr;
    ss_count_alloc();
    cudaError_t e = ctx->pool ? cudaMallocFromPoolAsync(p, bytes, ctx->pool, ctx->stream)
                              : cudaMallocAsync(p, bytes, ctx->stream);
    if (e != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return set_error(ctx, SS_ERR_OOM, "device allocation of " + std::to_string(bytes) + " bytes failed");
    }
    return SS_OK;
}

cudaMemPool_t device_pool(int device) {
    static std::mutex mu;
    static std::map<int, cudaMemPool_t> pools;
    std::lock_guard<std::mutex> lock(mu);
    const auto it = pools.find(device);
    if (it != pools.end()) return it->second;
    cudaMemPoolProps props = {};
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = device;
    cudaMemPool_t pool = nullptr;
    if (cudaMemPoolCreate(&pool, &props) == cudaSuccess) {
        // keep every freed block: a batched step allocates and frees the same
        // gigabytes each time
        uint64_t keep = UINT64_MAX;
        if (cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep) != cudaSuccess) cudaGetLastError();
    } else {
        cudaGetLastError();
        pool = nullptr;
    }
    pools[device] = pool;
    return pool;
}

void dev_free(ss_ctx ctx, void* p) {
    if (p) cudaFreeAsync(p, ctx->stream);
}

void dev_free_nostream(void* p) {
    if (p) cudaFreeAsync(p, 0);
}

void free_csr(ss_ctx ctx, DeviceCSR& m) {
    dev_free(ctx, m.row_ptr);
    dev_free(ctx, m.col);
    dev_free(ctx, m.val);
    csr_split_free(ctx, m);
    m = DeviceCSR();
}

// ------------------------------------------------------------------ scan
// Three-phase exclusive scan: per-block sums, one block scans the block sums,
// then every block adds its offset.  int64 accumulation, int32 output.

static constexpr int SCAN_BLOCK = 1024;

__global__ void scan_block_sums(const int32_t* __restrict__ in, int64_t n, long long* __restrict__ sums) {
    __shared__ long long warp_tot[32];
    int64_t i = (int64_t)blockIdx.x * SCAN_BLOCK + threadIdx.x;
    long long v = (i < n) ? (long long)in[i] : 0;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) warp_tot[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x < 32) {
        long long t = warp_tot[threadIdx.x];
        for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
        if (threadIdx.x == 0) sums[blockIdx.x] = t;
    }
}

__global__ void scan_sums_single(long long* __restrict__ sums, int64_t nb, long long* __restrict__ total) {
    // one block of 1024 threads scans nb values in chunks
    __shared__ long long buf[SCAN_BLOCK];
    __shared__ long long carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int64_t base = 0; base < nb; base += SCAN_BLOCK) {
        int64_t i = base + threadIdx.x;
        long long v = (i < nb) ? sums[i] : 0;
        buf[threadIdx.x] = v;
        __syncthreads();
        for (int off = 1; off < SCAN_BLOCK; off <<= 1) {
            long long t = (threadIdx.x >= off) ? buf[threadIdx.x - off] : 0;
            __syncthreads();
            buf[threadIdx.x] += t;
            __syncthreads();
        }
        if (i < nb) sums[i] = carry + buf[threadIdx.x] - v;   // exclusive
        __syncthreads();
        if (threadIdx.x == SCAN_BLOCK - 1) carry += buf[SCAN_BLOCK - 1];
        __syncthreads();
    }
    if (threadIdx.x == 0) *total = carry;
}

__global__ void scan_apply(const int32_t* __restrict__ in, int64_t n, const long long* __restrict__ sums,
                           int32_t* __restrict__ out, const long long* __restrict__ total) {
    __shared__ long long buf[SCAN_BLOCK];
    int64_t i = (int64_t)blockIdx.x * SCAN_BLOCK + threadIdx.x;
    long long v = (i < n) ? (long long)in[i] : 0;
    buf[threadIdx.x] = v;
    __syncthreads();
    for (int off = 1; off < SCAN_BLOCK; off <<= 1) {
        long long t = (threadIdx.x >= off) ? buf[threadIdx.x - off] : 0;
        __syncthreads();
        buf[threadIdx.x] += t;
        __syncthreads();
    }
    if (i < n) out[i] = (int32_t)(sums[blockIdx.x] + buf[threadIdx.x] - v);
    if (i == n - 1 || (n == 0 && i == 0)) out[n] = (int32_t)(*total);
}

ss_status exclusive_scan_i32(ss_ctx ctx, const int32_t* counts, int32_t* out, int64_t n, int64_t* total) {
    int64_t nb = (n + SCAN_BLOCK - 1) / SCAN_BLOCK;
    if (nb == 0) nb = 1;
    long long* sums = nullptr;
    SS_TRY(dev_alloc_n(ctx, &sums, (size_t)nb + 1));
    long long* tot = sums + nb;
    scan_block_sums<<<(ss_count_launch(), (unsigned)nb), SCAN_BLOCK, 0, ctx->stream>>>(counts, n, sums);
    scan_sums_single<<<(ss_count_launch(), 1), SCAN_BLOCK, 0, ctx->stream>>>(sums, nb, tot);
    scan_apply<<<(ss_count_launch(), (unsigned)nb), SCAN_BLOCK, 0, ctx->stream>>>(counts, n, sums, out, tot);
    SS_CUDA(ctx, cudaGetLastError());
    if (!total) {              // the caller knows the total fits: stay asynchronous
        dev_free(ctx, sums);
        return SS_OK;
    }
    long long h = 0;
    SS_CUDA(ctx, cudaMemcpyAsync(&h, tot, sizeof(long long), cudaMemcpyDeviceToHost, ctx->stream));
    SS_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    dev_free(ctx, sums);
    *total = h;
    if (h > INT32_MAX) return set_error(ctx, SS_ERR_UNSUPPORTED, "more than 2^31-1 stored entries");
    return SS_OK;
}

__global__ void find_diag_kernel(const int32_t* __restrict__ rp, const int32_t* __restrict__ col, int64_t n,
                                 int32_t* __restrict__ pos) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int lo = rp[i], hi = rp[i + 1] - 1, found = -1;
    while (lo <= hi) {
        int mid = (lo + hi) >> 1;
        int c = col[mid];
        if (c == i) { found = mid; break; }
        if (c < i) lo = mid + 1; else hi = mid - 1;
    }
    pos[i] = found;
}

ss_status find_diag(ss_ctx ctx, const DeviceCSR& m, int32_t* diag_pos) {
    if (m.n_rows == 0) return SS_OK;
    unsigned g = (unsigned)((m.n_rows + 255) / 256);
    find_diag_kernel<<<(ss_count_launch(), g), 256, 0, ctx->stream>>>(m.row_ptr, m.col, m.n_rows, diag_pos);
    SS_CUDA(ctx, cudaGetLastError());
    return SS_OK;
}

ss_status check_csr_view(ss_ctx ctx, const ss_csr_view* v) {
    if (!v) return set_error(ctx, SS_ERR_INVALID, "null CSR view");
    if (v->n_rows < 0 || v->n_cols < 0 || v->nnz < 0 || v->nnz > INT32_MAX)
        return set_error(ctx, SS_ERR_INVALID, "bad CSR sizes");
    if (!v->row_ptr || (v->nnz > 0 && (!v->col || !v->val)))
        return set_error(ctx, SS_ERR_INVALID, "null CSR array");
    if (!v->on_device) {   // host views can be checked cheaply
        if (v->row_ptr[0] != 0 || v->row_ptr[v->n_rows] != v->nnz)
            return set_error(ctx, SS_ERR_INVALID, "row_ptr does not span nnz");
        for (int64_t i = 0; i < v->n_rows; ++i) {
            int32_t a = v->row_ptr[i], b = v->row_ptr[i + 1];
            if (b < a) return set_error(ctx, SS_ERR_INVALID, "row_ptr not monotone");
            for (int32_t t = a; t < b; ++t) {
                if (v->col[t] < 0 || v->col[t] >= v->n_cols)
                    return set_error(ctx, SS_ERR_INVALID, "column index out of range");
                if (t > a && v->col[t] <= v->col[t - 1])
                    return set_error(ctx, SS_ERR_INVALID, "columns not sorted/unique within a row");
            }
        }
        for (int64_t t = 0; t < 2 * v->nnz; ++t)
            if (!(v->val[t] == v->val[t]) || v->val[t] - v->val[t] != 0.0)
                return set_error(ctx, SS_ERR_INVALID, "non-finite value in CSR view");
    }
    return SS_OK;
}

// Validate and copy a CSR view into library-owned device memory.
ss_status upload_csr(ss_ctx ctx, const ss_csr_view* v, DeviceCSR& out) {
    out = DeviceCSR();
    SS_TRY(check_csr_view(ctx, v));
    cudaMemcpyKind kind = v->on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    out.n_rows = v->n_rows;
    out.n_cols = v->n_cols;
    out.nnz = v->nnz;
    SS_TRY(dev_alloc_n(ctx, &out.row_ptr, (size_t)v->n_rows + 1));
    SS_TRY(dev_alloc_n(ctx, &out.col, (size_t)v->nnz));
    SS_TRY(dev_alloc_n(ctx, &out.val, (size_t)v->nnz));
    SS_CUDA(ctx, cudaMemcpyAsync(out.row_ptr, v->row_ptr, sizeof(int32_t) * (v->n_rows + 1), kind, ctx->stream));
    if (v->nnz > 0) {
        SS_CUDA(ctx, cudaMemcpyAsync(out.col, v->col, sizeof(int32_t) * v->nnz, kind, ctx->stream));
        SS_CUDA(ctx, cudaMemcpyAsync(out.val, v->val, sizeof(double2) * v->nnz, kind, ctx->stream));
    }
    return SS_OK;
}

// ----------------------------------------------------------------- profiler

static cudaEvent_t prof_event(ss_ctx ctx) {
    if (!ctx->prof_pool.empty()) {
        cudaEvent_t e = ctx->prof_pool.back();
        ctx->prof_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return e;
}

ProfScope::ProfScope(ss_ctx ctx, int k) : c(ctx), kind(k) {
    if (c && c->prof) {
        a = prof_event(c);
        if (a) cudaEventRecord(a, c->stream);
    }
}

ProfScope::~ProfScope() {
    if (!a) return;
    cudaEvent_t b = prof_event(c);
    if (!b) return;
    cudaEventRecord(b, c->stream);
    c->prof_recs.push_back(ProfRec{a, b, kind});
}

extern "C" ss_status ss_profile_enable(ss_ctx ctx, int enable) {
    if (!ctx) return SS_ERR_INVALID;
    ctx->prof = enable ? 1 : 0;
    return SS_OK;
}

extern "C" ss_status ss_profile_read(ss_ctx ctx, int kind, int64_t* launches, double* total_ms) {
    if (!ctx || kind < 0 || kind >= PROF_NKINDS) return SS_ERR_INVALID;
    SS_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    int64_t cnt = 0;
    double ms = 0.0;
    std::vector<ProfRec> keep;
    for (const ProfRec& r : ctx->prof_recs) {
        if (r.kind != kind) {
            keep.push_back(r);
            continue;
        }
        float t = 0.f;
        if (cudaEventElapsedTime(&t, r.a, r.b) == cudaSuccess) {
            ms += t;
            ++cnt;
        } else {
            cudaGetLastError();
        }
        ctx->prof_pool.push_back(r.a);
        ctx->prof_pool.push_back(r.b);
    }
    ctx->prof_recs.swap(keep);
    if (launches) *launches = cnt;
    if (total_ms) *total_ms = ms;
    return SS_OK;
}

// ------------------------------------------------------------ launch count

static std::atomic<unsigned long long> g_launches{0};

int ss_count_launch() {
    g_launches.fetch_add(1, std::memory_order_relaxed);
    return 0;
}

extern "C" unsigned long long ss_launch_count(void) { return g_launches.load(std::memory_order_relaxed); }

// ------------------------------------------------------- allocation count

static std::atomic<unsigned long long> g_allocs{0};

void ss_count_alloc() { g_allocs.fetch_add(1, std::memory_order_relaxed); }

extern "C" unsigned long long ss_alloc_count(void) { return g_allocs.load(std::memory_order_relaxed); }
