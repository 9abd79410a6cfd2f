// Host-side (C++) algorithms of the solver: ordering, level analysis, ILUT.
// Plain C++17, no CUDA types, so these translation units build with g++.
#pragma once

#include <stdint.h>

#include <vector>

// Reverse Cuthill-McKee order of the pattern of A + A^T (A: n x n CSR).
// perm[new] = old.  Start node: highest-index unvisited node of minimum
// degree; neighbours in ascending (degree, index); degree counts the stored
// diagonal.
void rcm_host(int64_t n, const int32_t* row_ptr, const int32_t* col, int32_t* perm);

// Level sets of the strict lower (lower = true) or strict upper triangle of
// a CSR pattern: level(i) = 1 + max level of the rows i depends on.  Fills
// `order` with the rows sorted by (level, row) -- for the upper triangle the
// rows are visited from the last to the first -- and returns the number of
// levels.  level_ptr (size levels + 1) receives the start of each level in
// `order`.
int32_t level_sets_host(int64_t n, const int32_t* row_ptr, const int32_t* col, bool lower,
                        std::vector<int32_t>& order, std::vector<int32_t>& level_ptr);

// Level-aligned units of R rows for the triangular solves: every unit holds
// up to R rows of one level (padded with -1), units follow level order.
void level_units_host(const std::vector<int32_t>& order, const std::vector<int32_t>& level_ptr, int R,
                      std::vector<int32_t>& units);

// Elimination schedule of iLU(0) (IKJ elimination restricted to the pattern
// of an n x n CSR with ascending columns; dpos[i]: position of row i's
// diagonal).  For the pivot at position t of row i (k = col[t] < i): the
// entries j > t of row i whose column row k's upper part (after its
// diagonal) also holds, as tgt = j - row_ptr[i] and src = the position in
// row k, at tgt/src[ptr[t] .. ptr[t + 1]) in ascending order of the row k
// position; ptr has row_ptr[n] + 1 entries (empty ranges for non-pivots).
// The elimination is: for each row, for each pivot t in ascending order,
// l = a[t] / a[dpos[k]], a[t] = l, a[row_ptr[i] + tgt] -= l a[src] for the
// listed pairs.
void ilu0_schedule_host(int64_t n, const int32_t* row_ptr, const int32_t* col, const int32_t* dpos,
                        std::vector<int32_t>& ptr, std::vector<int32_t>& tgt, std::vector<int32_t>& src);

// ILUT(drop_tol, fill_factor) without pivoting on an n x n CSR matrix with
// interleaved complex values.  Output: combined factors (strict lower part =
// L with unit diagonal, diagonal and upper part = U), sorted columns.
// Returns 0, or 1 + the row index of a zero or missing pivot.
int64_t ilut_host(int64_t n, const int32_t* row_ptr, const int32_t* col, const double* val,
                  double drop_tol, double fill_factor, std::vector<int32_t>& f_row_ptr,
                  std::vector<int32_t>& f_col, std::vector<double>& f_val);

// Weighted maximum bipartite matching (section "Direct factorization"):
// match[j] = the row assigned to column j (-1 if none), so that A[match, :]
// has a zero-free diagonal when A is structurally nonsingular.  Columns go in
// descending order of their largest |a_ij|^2 (ties: ascending column); each
// runs a breadth-first augmenting-path search trying rows in descending
// |a_ij|^2 (ties: ascending row).  val: interleaved complex.  Returns the
// number of matched columns (n when the diagonal can be made zero-free).
int64_t mbm_host(int64_t n, const int32_t* row_ptr, const int32_t* col, const double* val, int32_t* match);

// Autotuner search of the batched solver's launch choices.  A choice is four
// small integers: the lanes-per-row shifts of the lower triangle, the upper
// triangle and A (G = rule G * 2^shift, shift in [TUNE_SHIFT_MIN,
// TUNE_SHIFT_MAX]) and the level-staging flag (0: the rule's staging, 1: the
// other one: the shared-memory ring for FP32, register prefetch for FP64).
// Coordinate descent from `start`: each coordinate in turn tries its two
// neighbours (cost evaluated once per choice, memoised) and moves while the
// cost drops by more than 1 %; it stops when a full sweep improves nothing or
// after max_probes evaluations.  Returns the number of evaluations.
constexpr int TUNE_SHIFT_MIN = -1;
constexpr int TUNE_SHIFT_MAX = 2;
struct TuneChoice {
    int lo, up, a, stage;
};
int tune_search(TuneChoice start, double (*cost)(const TuneChoice&, void*), void* user, int max_probes,
                TuneChoice* best, double* best_cost);
