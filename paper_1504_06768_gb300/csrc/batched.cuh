// Per-system persistent solver: one CTA takes one system at a time from a
// work queue and runs the numeric iLU(0), the preconditioned BiCGSTAB (FP64,
// or FP32 inner + FP64 refinement), the acceptance test and the
// finalisation without leaving the kernel.
#pragma once

#include <utility>
#include <vector>

#include "common.cuh"

constexpr int BATCH_THREADS = 512;     // threads of one solver block
constexpr int BATCH_BLOCKS_PER_SM = 1; // solver blocks resident per SM (each solves its own system)
constexpr int BATCH_MAXE = 3;       // packed entry slots per lane and unit (longer rows overflow to the CSR)
constexpr int BATCH_RING_MAX = 16;  // shared-memory slots staging triangular-solve levels, at most

// Lane-major packed layout of one CSR operand (a strict triangle of the
// factors, or A itself).  Rows are grouped into units of R = 32 / G rows
// (level-aligned for the triangles, consecutive for A); slot (u*E + q)*32 +
// lane holds the q-th entry handled by that lane, so a warp reads a whole unit
// with E coalesced loads.  Entries of a long row beyond its first E*G stay in
// the CSR and are visited from ovb to ove.
struct PackedOp {
    const int4* meta;       // nunits * R row records {row (-1 pads a unit), first CSR position
                            // not packed, end of the row's CSR range, 0}
    const int32_t* col;     // nunits * E * 32 column ids (-1: empty slot)
    const int32_t* src;     // nunits * E * 32 CSR positions of the slots (-1: empty)
    void* val;              // per system: nunits * E * 32 values of the inner type
    void* dinv;             // per system, upper triangle: nunits * R values 1 / u_ii (else null)
    int32_t nunits, G, E;
    const int32_t* lvl;     // triangles: first unit of each level (nlev + 1 entries)
    int32_t nlev;
};

struct BatchSys {
    int32_t n, d;
    // system matrix A (RCM-permuted L + wT or L - sigma I)
    const int32_t* a_rp;
    const int32_t* a_col;
    const double2* a_val;
    float2* a_val32;            // written by the kernel (mixed precision)
    // combined incomplete factors (pattern of A for iLU(0)); values written by the kernel
    const int32_t* f_rp;
    const int32_t* f_col;
    const int32_t* f_dpos;
    double2* f_val;
    double2* f_inv;
    float2* f_val32;
    float2* f_inv32;
    int32_t factor_on_device;   // 1: iLU(0) computed in the kernel from a_val; 0: factors given
    int32_t warm;               // 1: rho_out holds the initial guess (natural order, column-major)
    // packed operands of the two triangular solves and of the SpMV
    PackedOp lo, up, pa;
    const int32_t* lvl_ptr;     // lower level boundaries in lvl_rows (factorisation schedule)
    const int32_t* lvl_rows;
    int32_t n_levels;
    // elimination schedule: the pivot at CSR position t updates the entries
    // ilu_tgt[p] (index within its row) with the values at ilu_src[p] (CSR
    // positions in the pivot's row), p in [ilu_ptr[t], ilu_ptr[t + 1])
    const int32_t* ilu_ptr;
    const int32_t* ilu_tgt;
    const int32_t* ilu_src;
    // right-hand side / trace
    int32_t r0;                 // permuted position of row 0
    double w;                   // weight of the trace row (0: shifted system)
    double sigma;
    const int32_t* perm;        // perm[new] = old
    const int32_t* tidx;        // permuted positions of the diagonal elements rho_ii
    // work: 10 vectors of n elements of the inner type + x64, r64 (FP64)
    void* work;
    double2* x64;
    double2* r64;
    double2* rho_out;           // natural column-major order, device
    // results
    int status, iters, outer;
    double resid;
};

struct BatchParams {
    double tol;
    int maxiter;
    int mixed;                  // 0: FP64, 1: FP32 inner + FP64 refinement
    double inner_rtol;          // mixed: inner relative tolerance
    int power;                  // inverse power (FP64 only)
    uint64_t seed;
    int ring_allowed;           // every staged array is 16-byte aligned (bulk copies may be used)
    const int32_t* order;       // device: the k-th system taken is order[k] (null: submission order)
    int stage_flip;             // 1: the level staging the rule would not choose (ring for FP32, none for FP64)
    unsigned long long wait_ns; // limit of the staging barriers' waits
    long long diag_stall_seq;   // failure-detection aid: this staging sequence number gets no copies (-1: none)
    // shared-memory plan of the launch (set by batch_launch)
    int ring_umax;              // units per staged level (0: no ring)
    int ring_slots;             // slots of the ring
    int ring_slot_bytes;
    int lvl_smem;               // level boundaries copied to shared memory
    int pbuf_smem;              // mixed precision: p^ kept in shared memory
    int smem_bytes;             // dynamic shared memory of a block (staging of the factorisation's rows)
    int sf;                     // mixed precision: triangular solves without level barriers (values as flags)
};

struct BatchShape {             // what the shared-memory plan needs of one system
    int32_t n, nlev_lo, nlev_up, E_lo, R_lo, E_up, R_up;
    int32_t umax;               // units in the widest level of either triangle
};

// ------------------------------------------------------- batched setup

struct BatchMeta {                  // per system, from the device
    int64_t nz_off, nnz;            // entries of the system in BatchLt::col / val
    unsigned long long hash;        // hash of the pattern (equal patterns, equal hashes)
};

// Trace-row systems L~ = L + wT (Eq. linear) of a batch, concatenated on the
// device: system s has n[s] = d[s]^2 rows, local row pointers at
// rp[row_off[s] + s ...] (n[s] + 1 entries, starting at 0), local columns and
// values at col / val[meta[s].nz_off ...].
struct BatchLt {
    int64_t ns = 0;
    std::vector<int64_t> d, n, row_off;
    std::vector<BatchMeta> meta;
    std::vector<double> w;
    int32_t* rp = nullptr;
    int32_t* col = nullptr;
    double2* val = nullptr;
    int64_t* row_off_d = nullptr;
    BatchMeta* meta_d = nullptr;
};

struct GatherEntry {                // dst[k] = val[src_off + map[k]], k < nnz
    const int32_t* map;
    double2* dst;
    int64_t src_off, nnz;
};

// Assembly (Eq. lindblad), weight w (w_in > 0: as given, else mean |L_ii|) and
// trace row of every system, with a number of launches that does not grow
// with the number of systems.  Each system's L~ is entry for entry the one
// assemble_liouvillian + add_trace_row give.
ss_status batch_trace_systems(ss_ctx ctx, const std::vector<const ss_csr_view*>& H, const std::vector<int>& n_c,
                              const std::vector<const ss_csr_view*>& C, double w_in, BatchLt& out);
void batch_lt_free(ss_ctx ctx, BatchLt& b);
// mismatch[k] = 1 when the patterns of systems pairs[k] differ (same n, nnz).
ss_status batch_verify_patterns(ss_ctx ctx, const BatchLt& b, const std::vector<std::pair<int, int>>& pairs,
                                std::vector<int>& mismatch);
// Asynchronous copy of system s's pattern to the host (synchronise the stream before use).
ss_status batch_download_pattern(ss_ctx ctx, const BatchLt& b, int s, std::vector<int32_t>& rp,
                                 std::vector<int32_t>& col);
ss_status batch_gather_values(ss_ctx ctx, const BatchLt& b, const std::vector<GatherEntry>& tab);
// *mismatch = 1 unless system s's pattern equals the natural-order pattern
// (rp_d: n + 1 row pointers, col_d: nnz columns) on the device.
ss_status batch_verify_against(ss_ctx ctx, const BatchLt& b, int s, const int32_t* rp_d, const int32_t* col_d,
                               int* mismatch);

// Order in which the persistent solver takes the systems: largest estimated
// cost first (longest-processing-time-first list scheduling, so that no long
// system starts last and holds one SM while the others idle).  The estimate
// is the entry count of L~ times (1 + ||offdiag(L~)||_F / ||diag(L~)||_F):
// iLU(0)-preconditioned Krylov methods need more iterations the weaker the
// diagonal.  Ties keep the submission order.  Results do not depend on it.
// fp (may be null) receives each system's (||diag||_F^2, ||offdiag||_F^2).
ss_status batch_cost_order(ss_ctx ctx, const BatchLt& b, std::vector<int32_t>& order,
                           std::vector<double2>* fp = nullptr);

int batch_max_n(bool mixed);
// Chooses the shared-memory plan (ring size, level boundaries in shared
// memory) for the systems' shapes and launches the persistent solver.
ss_status batch_launch(ss_ctx ctx, BatchSys* dsys, int nsys, BatchParams p, const std::vector<BatchShape>& shapes,
                       int* queue, int* err);
