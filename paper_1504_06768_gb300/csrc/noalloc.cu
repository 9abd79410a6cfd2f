// krylov_solve_noalloc: the preconditioned BiCGSTAB solve of krylov_solve,
// for callers that must not allocate memory during the call -- for example a
// control loop with a fixed memory budget, or a host that hands every device
// allocation to its own pool and forbids cudaMalloc behind its back.
//
// The Krylov workspace (eight vectors of at most SS_NOALLOC_MAX_N complex
// doubles, the device-side solver state and the reduction partials) lives in
// one file-scope __device__ array.  Every GPU that loads the library holds
// that array until the process exits.  With lazy module loading (the CUDA
// default) the array only comes into existence when its module is first
// touched, so ss_ctx_create touches it (noalloc_prepare): the call that
// creates a context loads the array and looks up its device address, and no
// krylov_solve_noalloc call ever allocates.  The array is shared by all calls
// on a device and keeps the last call's contents; the solver initialises
// every word it reads, so nothing from an earlier call leaks into a result.
// Two calls whose work overlaps on the same GPU (different streams or host
// threads) race on the array, and on the per-device host mirror of the
// solver state as well.
#include <mutex>

#include "common.cuh"
#include "krylov.cuh"

namespace {

constexpr int64_t MAX_N = SS_NOALLOC_MAX_N;
constexpr size_t VEC_BYTES = 8ull * MAX_N * sizeof(double2);
constexpr size_t STATE_BYTES = (sizeof(KrylovState) + 255) & ~size_t(255);
constexpr size_t PART_BYTES = 512ull * 32 * sizeof(double2);
constexpr size_t SCRATCH_BYTES = VEC_BYTES + STATE_BYTES + PART_BYTES;

static __device__ __align__(256) unsigned char g_noalloc_scratch[SCRATCH_BYTES];

constexpr int MAX_DEVICES = 64;
std::mutex g_mu;
void* g_ptr[MAX_DEVICES] = {};       // device address of the array, per device
KrylovState g_host_state[MAX_DEVICES];  // host mirror of the solver state (not pinned)

// Device address of the scratch array on ctx's device, looked up once per
// device with that device current.  In host code the array's name is only a
// host-side stand-in, so the address must come from cudaGetSymbolAddress.
ss_status scratch_for(ss_ctx ctx, void** out) {
    if (ctx->device < 0 || ctx->device >= MAX_DEVICES)
        return set_error(ctx, SS_ERR_UNSUPPORTED, "device index beyond the no-allocation table");
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_ptr[ctx->device]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) return cuda_check(ctx, e, "cudaGetSymbolAddress(no-allocation scratch)");
        g_ptr[ctx->device] = p;
    }
    *out = g_ptr[ctx->device];
    return SS_OK;
}

}  // namespace

ss_status noalloc_prepare(ss_ctx ctx) {
    void* p = nullptr;
    return scratch_for(ctx, &p);
}

extern "C" ss_status krylov_solve_noalloc(ss_ctx ctx, ss_mat A, ss_prec M, const double* b, double* x, double tol,
                                          int maxiter, int* iters_out, double* resid_out) {
    if (!ctx) return SS_ERR_INVALID;
    SS_CUDA(ctx, cudaSetDevice(ctx->device));
    if (!A || !M || !b || !x) return set_error(ctx, SS_ERR_INVALID, "null argument");
    const int64_t n = A->m.n_rows;
    if (M->f.n_rows != n) return set_error(ctx, SS_ERR_INVALID, "preconditioner size mismatch");
    if (n > MAX_N)
        return set_error(ctx, SS_ERR_INVALID,
                         "n = " + std::to_string(n) + " exceeds the no-allocation limit of " + std::to_string(MAX_N) +
                             " unknowns; use krylov_solve");
    void* base = nullptr;
    SS_TRY(scratch_for(ctx, &base));
    unsigned char* p = static_cast<unsigned char*>(base);
    KrylovWork w;
    w.n = n;
    w.method = SS_KRYLOV_BICGSTAB;
    w.m = 0;
    w.vecs = reinterpret_cast<double2*>(p);
    w.st = reinterpret_cast<KrylovState*>(p + VEC_BYTES);
    w.partials = reinterpret_cast<double2*>(p + VEC_BYTES + STATE_BYTES);
    w.nvec = 8;
    w.host_st = &g_host_state[ctx->device];
    const int prof = ctx->prof;       // the event profiler would create CUDA events: keep it off here
    ctx->prof = 0;
    KrylovResultHost res;
    ss_status st = bicgstab_dev(ctx, A->m, M, w, reinterpret_cast<const double2*>(b), reinterpret_cast<double2*>(x),
                                tol, maxiter, &res);
    ctx->prof = prof;
    SS_TRY(st);
    if (iters_out) *iters_out = res.iters;
    if (resid_out) *resid_out = res.resid;
    if (res.status != SS_OK) {
        ctx->last_error = res.status == SS_BREAKDOWN ? "BiCGSTAB breakdown" : "iteration cap reached";
        return (ss_status)res.status;
    }
    return SS_OK;
}
