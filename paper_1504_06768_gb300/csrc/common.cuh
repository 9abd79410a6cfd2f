// Internal declarations shared by the solver's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <array>
#include <map>
#include <string>
#include <vector>

#include "../../include/lindblad_ss.h"

// ------------------------------------------------------------ complex math
// Complex FP64 / FP32 numbers are double2 / float2 (x = re, y = im).

__host__ __device__ __forceinline__ double2 cmake(double re, double im) { return make_double2(re, im); }
__host__ __device__ __forceinline__ double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__host__ __device__ __forceinline__ double2 csub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__host__ __device__ __forceinline__ double2 cmul(double2 a, double2 b) {
    return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// conj(a) * b
__host__ __device__ __forceinline__ double2 cmulc(double2 a, double2 b) {
    return make_double2(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x);
}
__host__ __device__ __forceinline__ double2 cconj(double2 a) { return make_double2(a.x, -a.y); }
__host__ __device__ __forceinline__ double2 cscale(double2 a, double s) { return make_double2(a.x * s, a.y * s); }
__host__ __device__ __forceinline__ double cabs2(double2 a) { return a.x * a.x + a.y * a.y; }

// Smith's algorithm (R. L. Smith, "Algorithm 116: Complex division", CACM 1962).
__host__ __device__ __forceinline__ double2 cdiv(double2 a, double2 b) {
    if (fabs(b.x) >= fabs(b.y)) {
        double r = b.y / b.x, den = b.x + b.y * r;
        return make_double2((a.x + a.y * r) / den, (a.y - a.x * r) / den);
    } else {
        double r = b.x / b.y, den = b.y + b.x * r;
        return make_double2((a.x * r + a.y) / den, (a.y * r - a.x) / den);
    }
}

__host__ __device__ __forceinline__ float2 fcadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__host__ __device__ __forceinline__ float2 fcsub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__host__ __device__ __forceinline__ float2 fcmul(float2 a, float2 b) {
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

// ---------------------------------------------------------------- handles

struct DeviceCSR {          // complex FP64 CSR on the device
    int64_t n_rows = 0, n_cols = 0, nnz = 0;
    int32_t* row_ptr = nullptr;
    int32_t* col = nullptr;
    double2* val = nullptr;
    // Part-split copy for the FP64 SpMV (built on demand by csr_split): each
    // stored entry becomes one real "part" per nonzero component; a row holds
    // its real parts, then (from s_mid[i]) its imaginary parts.  Entries of
    // the Liouvillian are mostly purely real (dissipators) or purely
    // imaginary (the Hamiltonian commutator), so a part costs 12 bytes and
    // 2 FMAs where a complex entry costs 20 bytes and 4 FMAs.
    int32_t* s_row_ptr = nullptr;
    int32_t* s_mid = nullptr;
    uint32_t* s_col = nullptr;
    double* s_val = nullptr;
    int64_t s_nnz = 0;
    int s_state = 0;       // 0: not examined; 1: built; -1: not worth it (too many two-part entries)
};

// Kernel classes timed by the optional per-launch profiler.
enum ProfKind { PROF_SPMV = 0, PROF_TRSV_LOWER = 1, PROF_TRSV_UPPER = 2, PROF_BATCHED = 3, PROF_NKINDS = 4 };

struct ProfRec {
    cudaEvent_t a, b;
    int kind;
};

struct ss_ctx_s {
    int device = 0;
    cudaStream_t stream = nullptr;
    std::string last_error;
    int num_sms = 0;
    int prof = 0;                       // record events around SpMV / triangular-solve launches
    std::vector<ProfRec> prof_recs;
    std::vector<cudaEvent_t> prof_pool;
    // persistent scratch (grown on demand)
    void* scratch = nullptr;
    size_t scratch_bytes = 0;
    double* h_pinned = nullptr;      // small pinned host buffer for scalars
    // limit of every bounded device-side wait (triangular-solve dependencies,
    // staging barriers), after which the kernel reports SS_ERR_TIMEOUT
    unsigned long long wait_ns = 2000000000ull;
    // failure-detection aid (ss_diag_batched_stall): the batched solver's level
    // staging of this sequence number arms its barrier but issues no copies
    long long diag_stall_seq = -1;
    // the batched solver's autotuned choices (lanes-per-row shifts, staging
    // flip) per batch shape, kept for later batches of the same shape
    std::map<unsigned long long, std::array<int, 4>> tune_table;
    // pinned host memory through which steady_state_batched returns host
    // results (grown on demand, kept until the context is destroyed)
    void* host_stage = nullptr;
    size_t host_stage_bytes = 0;
    // device memory pool of the context's device (see device_pool; null: the
    // device's default pool)
    cudaMemPool_t pool = nullptr;
};

struct ss_mat_s {
    DeviceCSR m;
    int32_t* diag_pos = nullptr;      // position of the diagonal entry per row (-1 if absent)
    float2* val32 = nullptr;          // FP32 copy of the values (made on demand)
    int64_t d = 0;                    // Hilbert dimension when the matrix is a Liouvillian (n = d^2)
};

struct TriLevels {                    // one level-scheduled strict triangle of the factors
    int32_t n_levels = 0;
    int32_t* order = nullptr;         // rows sorted by level (device, n)
    int g = 32;                       // lanes per row in the solve (R = 32 / g rows per unit)
    int64_t n_units = 0;              // level-aligned units of R rows
    // The triangle in unit order, stored on its own: slot s = u R + k is the
    // k-th row of unit u (urow[s] = -1 pads a unit at the end of a level);
    // its entries are col/val[uptr[s] .. uptr[s + 1]), so a unit's entries
    // are contiguous.  src maps each entry to its position in the combined
    // factors (values are gathered from there after every factorisation).
    int32_t* urow = nullptr;          // n_units R
    int32_t* uptr = nullptr;          // n_units R + 1
    int32_t* col = nullptr;           // nnz
    int32_t* src = nullptr;           // nnz
    double2* val = nullptr;           // nnz
    float2* val32 = nullptr;          // nnz (mixed precision)
    double2* dinv = nullptr;          // upper triangle: 1 / u_ii per slot (0 for padding)
    float2* dinv32 = nullptr;
    int64_t nnz = 0;
};

struct ss_prec_s {
    DeviceCSR f;                      // combined factors: strict lower = L (unit), rest = U
    int32_t* diag_pos = nullptr;      // device, n
    double2* inv_diag = nullptr;      // 1 / u_ii (device, n)
    bool fp32 = false;                // FP32 copies of the triangles exist
    TriLevels lower, upper;
    int* err = nullptr;               // device error word (bounded waits)
    unsigned long long* tickets = nullptr;  // block tickets of the lower [0] and upper [1] solves
    double2* tmp = nullptr;           // intermediate vector of the two solves (PENDING between uses)
    float2* tmp32 = nullptr;
    int64_t skipped_slot = -1;        // diagnostics: lower-solve slot whose row is not computed (-1: none)
    int32_t skipped_row = -1;
};

// ----------------------------------------------------------------- errors

ss_status set_error(ss_ctx ctx, ss_status st, const std::string& msg);
ss_status cuda_check(ss_ctx ctx, cudaError_t e, const char* what);

#define SS_CUDA(ctx, call)                                              \
    do {                                                                \
        cudaError_t _e = (call);                                        \
        if (_e != cudaSuccess) return cuda_check((ctx), _e, #call);     \
    } while (0)

#define SS_TRY(call)                                                    \
    do {                                                                \
        ss_status _s = (call);                                          \
        if (_s != SS_OK) return _s;                                     \
    } while (0)

// Every kernel launch of the library goes through ss_count_launch() (in the
// grid expression of the launch), so the total is available to callers.
int ss_count_launch();
// Every device or pinned-host allocation the library makes is counted
// (ss_alloc_count), so a caller can check that a call allocated nothing.
void ss_count_alloc();
// Loads the allocation-free entry point's fixed workspace onto the context's
// device and records its address (once per device); called by ss_ctx_create.
ss_status noalloc_prepare(ss_ctx ctx);

// RAII event pair around one launch when the context's profiler is on.
struct ProfScope {
    ss_ctx c;
    int kind;
    cudaEvent_t a = nullptr;
    ProfScope(ss_ctx ctx, int k);
    ~ProfScope();
};

// ------------------------------------------------------------ allocation

ss_status dev_alloc(ss_ctx ctx, void** p, size_t bytes);
// The process-wide memory pool of a device from which the library's
// contexts allocate: freed blocks stay in it for later allocations instead
// of going back to the driver at every synchronisation.  Created on first
// use, never destroyed (memory freed after its context is gone still returns
// to a live pool).  Null when the device cannot make one.
cudaMemPool_t device_pool(int device);
void dev_free(ss_ctx ctx, void* p);
void dev_free_nostream(void* p);
template <class T> ss_status dev_alloc_n(ss_ctx ctx, T** p, size_t n) {
    return dev_alloc(ctx, reinterpret_cast<void**>(p), n * sizeof(T) + (n == 0 ? 16 : 0));
}
void free_csr(ss_ctx ctx, DeviceCSR& m);

// --------------------------------------------------------- device helpers

// Exclusive scan of n int32 counts into n+1 offsets (out[0] = 0, out[n] = total).
// With total != NULL the call waits for the result, returns it in *total and
// fails with SS_ERR_UNSUPPORTED past 2^31-1; with total == NULL it stays
// asynchronous (for sums already known to fit, e.g. a permutation of rows).
ss_status exclusive_scan_i32(ss_ctx ctx, const int32_t* counts, int32_t* out, int64_t n, int64_t* total);
// Position of the diagonal entry in each row (-1 when absent).
ss_status find_diag(ss_ctx ctx, const DeviceCSR& m, int32_t* diag_pos);
// Sizes and pointers of a CSR view; a host view's contents too (row pointers
// spanning nnz, sorted unique in-range columns, finite values).
ss_status check_csr_view(ss_ctx ctx, const ss_csr_view* v);
ss_status upload_csr(ss_ctx ctx, const ss_csr_view* v, DeviceCSR& out);

// ----------------------------------------------------------- kernels API

ss_status assemble_impl(ss_ctx ctx, const DeviceCSR& H, const std::vector<DeviceCSR>& C, DeviceCSR& L);

// Liouvillian rows of a batch of systems whose operators are stacked
// block-diagonally (H and each C_k of all systems, an absent operator being
// an empty block).  System s owns operator rows [doff[s], doff[s+1]) and rows
// [row_off[s], row_off[s+1]) of the concatenated Liouvillians (device arrays
// of nsys + 1 entries, P = row_off[nsys]).  Row p's stored entries are
// key[off[p] .. off[p] + cnt[p]) (key = local column) and val at the same
// positions; each system's row 0 has reserve_row0 ? d : 0 spare slots after
// its candidates.  The arithmetic of every entry is that of assemble_impl.
struct BatchRows {
    int32_t* off = nullptr;               // P + 1 candidate offsets
    int32_t* cnt = nullptr;               // P stored counts
    unsigned long long* key = nullptr;
    double2* val = nullptr;
    int64_t total = 0;                    // candidate slots
};
ss_status batch_lrows(ss_ctx ctx, const DeviceCSR& H, const std::vector<DeviceCSR>& C, const int64_t* row_off_d,
                      const int64_t* doff_d, int64_t nsys, int64_t P, int32_t reserve_row0, BatchRows& out);
void batch_rows_free(ss_ctx ctx, BatchRows& r);
ss_status add_trace_row_impl(ss_ctx ctx, const DeviceCSR& L, int64_t d, double w, DeviceCSR& out);
ss_status mean_abs_diag(ss_ctx ctx, const DeviceCSR& L, double* w);
ss_status add_shift_impl(ss_ctx ctx, const DeviceCSR& L, double sigma, DeviceCSR& out);
ss_status permute_impl(ss_ctx ctx, const DeviceCSR& A, const int32_t* perm_host, DeviceCSR& out);
ss_status bandwidth_profile_impl(ss_ctx ctx, const DeviceCSR& A, int64_t* bw, int64_t* prof);

#include "host_algos.h"

// preconditioner
ss_status ilu0_device(ss_ctx ctx, const DeviceCSR& A, ss_prec M);
ss_status prec_finish(ss_ctx ctx, ss_prec M, bool want_fp32);
ss_status prec_apply_dev(ss_ctx ctx, ss_prec M, const double2* r, double2* z, const int* halt = nullptr);
ss_status prec_apply_dev32(ss_ctx ctx, ss_prec M, const float2* r, float2* z, const int* halt = nullptr);
ss_status prec_from_host(ss_ctx ctx, ss_prec M, int64_t n, const std::vector<int32_t>& rp,
                         const std::vector<int32_t>& col, const std::vector<double>& val);
ss_status prec_check_error(ss_ctx ctx, ss_prec M);
// Test aid: the lower solve stops computing `row` (its output keeps the
// PENDING mark, so the rows depending on it wait until their limit), or with
// restore != 0 computes it again.
ss_status prec_skip_row(ss_ctx ctx, ss_prec M, int64_t row, int restore);
void prec_destroy(ss_ctx ctx, ss_prec M);

// SpMV
ss_status spmv_dev(ss_ctx ctx, const DeviceCSR& A, const double2* x, double2* y);
ss_status spmv_dev32(ss_ctx ctx, const DeviceCSR& A, const float2* val32, const float2* x, float2* y);
// Builds A's part-split copy when it pays (at most 1.6 parts per entry);
// later FP64 SpMVs of A use it.
ss_status csr_split(ss_ctx ctx, DeviceCSR& A);
void csr_split_free(ss_ctx ctx, DeviceCSR& A);
