// A batch of systems for the persistent per-system solver ("wave"), split into
// begin (setup on the device, pattern analysis on the host, launch and the
// asynchronous copies of the results), ready (completion test) and end
// (results and release).  steady_state_batched runs one wave to completion;
// the serving loop keeps several waves in flight on separate streams and
// shares the pattern analyses between them through a PatternCache.
#pragma once

#include <cuda_runtime.h>

#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "batched.cuh"
#include "common.cuh"
#include "host_algos.h"

struct PackedDev {                        // device arrays of one packed operand (per pattern)
    int32_t *col = nullptr, *src = nullptr, *lvl = nullptr;
    int4* meta = nullptr;
    int32_t nunits = 0, G = 1, E = 1, nlev = 0;
};

struct PackedHost {
    std::vector<int32_t> rows, col, src, ovb, ove, lvl;
    std::vector<int4> meta;               // {row, ovb, ove, 0} per unit row, as uploaded
    int32_t nunits = 0, G = 1, E = 1, nlev = 0;
};

// Analysis of one sparsity pattern of L~: RCM ordering, permuted structure,
// level schedule, packed operands.  Owns its device arrays (freed on
// destruction, stream-ordered on the legacy stream, after every wave that
// used it has completed).
struct Pattern {
    std::vector<int32_t> rp, col;         // natural-order pattern
    int64_t d = 0;
    std::vector<int32_t> perm, iperm, tidx;
    int32_t r0 = 0;
    std::vector<int32_t> prp, pcol, map, dpos, lorder, lptr, lunits, uunits;
    std::vector<int32_t> ilu_ptr, ilu_tgt, ilu_src;    // iLU(0) elimination schedule (see BatchSys)
    PackedHost hl, hu, ha;
    ss_status status = SS_OK;
    std::string error;
    int32_t *rp_d = nullptr, *col_d = nullptr;          // natural-order pattern (cache verification)
    int32_t *prp_d = nullptr, *pcol_d = nullptr, *map_d = nullptr;
    int32_t *perm_d = nullptr, *tidx_d = nullptr, *dpos_d = nullptr;
    int32_t *lo_units = nullptr, *up_units = nullptr, *lvl_ptr = nullptr, *lvl_rows = nullptr;
    int32_t *ilu_ptr_d = nullptr, *ilu_tgt_d = nullptr, *ilu_src_d = nullptr;
    int32_t lo_nunits = 0, up_nunits = 0, lo_g = 1, up_g = 1, a_g = 1, n_levels = 0, up_levels = 0;
    PackedDev lo, up, pa;
    int device = 0;
    ~Pattern();
};

using PatternKey = std::tuple<int64_t, int64_t, int64_t, unsigned long long>;   // d, n, nnz, hash

// Pattern analyses shared by the waves of a serving loop, keyed by
// (d, n, nnz, hash) and checked entry for entry on the device before reuse.
struct PatternCache {
    std::mutex mu;
    std::map<PatternKey, std::vector<std::shared_ptr<Pattern>>> by_key;
    std::vector<std::pair<PatternKey, std::shared_ptr<Pattern>>> lru;   // most recent last
    size_t max_patterns = 64;
    void touch(const PatternKey& k, const std::shared_ptr<Pattern>& p);
    void insert(const PatternKey& k, const std::shared_ptr<Pattern>& p);
};

// Steady states of earlier requests kept on the device by the serving loop,
// per sparsity pattern, each with the fingerprint of its L~ (squared
// Frobenius norms of the diagonal and the off-diagonal part): a new request
// of the same pattern starts from the stored state with the closest
// fingerprint (a neighbouring point of a parameter sweep).  Bounded in
// entries per pattern and in bytes; the oldest entry goes first.
struct SolutionCache {
    struct Entry {
        double2 fp;                   // (||diag||^2, ||offdiag||^2) of L~
        double2* rho = nullptr;       // device, natural column-major order, n values
        int64_t n = 0;
        uint64_t stamp = 0;
    };
    std::mutex mu;
    std::map<PatternKey, std::vector<Entry>> by_key;
    size_t bytes = 0, max_bytes = (size_t)256 << 20;
    size_t per_key = 8;
    uint64_t clock = 0;
    // the closest entry of key k to fingerprint fp (null: none)
    const Entry* nearest(const PatternKey& k, double2 fp);
    // stores a copy of rho (device, on ctx's stream), evicting old entries
    ss_status insert(ss_ctx ctx, const PatternKey& k, double2 fp, const double2* rho, int64_t n);
    void clear(ss_ctx ctx);
};

struct BatchWave {
    // inputs (borrowed for the duration of wave_begin; the views' arrays are read there)
    ss_ctx ctx = nullptr;                 // its stream carries the wave
    ss_options opt{};
    std::vector<const ss_csr_view*> H, C;
    std::vector<int> n_c;
    std::vector<double*> rho_out;         // per system: device (rho_on_device) or host memory
    int rho_on_device = 0;
    bool stage_pinned = false;            // host results: copy through pinned memory, asynchronously
    PatternCache* cache = nullptr;
    SolutionCache* sols = nullptr;        // serving: warm starts from earlier requests (null: off)
    TuneChoice tune{0, 0, 0, 0};          // lanes-per-row shifts and staging flip (autotuner; 0: the rules)
    bool time_kernel = false;             // record the persistent kernel's device time (kernel_ms)
    float kernel_ms = 0.f;
    // state
    BatchLt blt;
    std::vector<std::shared_ptr<Pattern>> pats;
    std::vector<int> pat_of;
    std::vector<PatternKey> key_of;       // per system: its pattern's cache key
    std::vector<double2> fp;              // per system: fingerprint of L~ (see SolutionCache)
    std::vector<void*> owned;
    std::vector<BatchSys> hs;
    BatchSys* dsys = nullptr;
    int* ctl = nullptr;
    double2* stage = nullptr;             // caller-owned pinned buffer of wave_pinned_bytes (stage_pinned)
    std::vector<size_t> stage_off;
    cudaEvent_t done = nullptr;
    cudaEvent_t k0 = nullptr, k1 = nullptr;   // around the persistent kernel (time_kernel)
    double t0 = 0, t1 = 0, t2 = 0;
    bool launched = false;
};

// Device bytes a wave holds for a system of Hilbert dimension d whose
// operators have the given nonzero counts (ctc_c: bounds of nnz(C_k^+ C_k));
// an upper bound, for admission.
size_t wave_footprint_bytes(int64_t d, int64_t nnz_h, const std::vector<int64_t>& nnz_c,
                            const std::vector<int64_t>& ctc_c, bool mixed);
// Pinned bytes a wave with stage_pinned needs (descriptors, error word, host results).
size_t wave_pinned_bytes(const BatchWave& w);
// Sets up and launches the wave; on success the solve and the result copies
// are queued on ctx's stream and `done` is recorded after them.
ss_status wave_begin(BatchWave& w);
bool wave_ready(BatchWave& w);
// Waits for the wave, writes rho (host results) and infos (wave order), releases.
ss_status wave_end(BatchWave& w, ss_info* infos);
void wave_release(BatchWave& w);
