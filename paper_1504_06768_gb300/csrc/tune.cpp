// Autotuner search of the batched solver's launch choices (host, no CUDA):
// coordinate descent over the lanes per row of the three packed operands and
// the level-staging method, each evaluation a measured probe (see
// batch_api.cu) or, in tests, a table.
#include <map>
#include <tuple>

#include "host_algos.h"

namespace {
std::tuple<int, int, int, int> key(const TuneChoice& c) { return std::make_tuple(c.lo, c.up, c.a, c.stage); }
}  // namespace

int tune_search(TuneChoice start, double (*cost)(const TuneChoice&, void*), void* user, int max_probes,
                TuneChoice* best, double* best_cost) {
    std::map<std::tuple<int, int, int, int>, double> seen;
    int probes = 0;
    auto eval = [&](const TuneChoice& c, double* out) {
        auto it = seen.find(key(c));
        if (it != seen.end()) { *out = it->second; return true; }
        if (probes >= max_probes) return false;
        ++probes;
        *out = cost(c, user);
        seen[key(c)] = *out;
        return true;
    };
    TuneChoice cur = start;
    double cur_cost = 0.0;
    if (!eval(cur, &cur_cost)) { *best = cur; if (best_cost) *best_cost = 0.0; return probes; }
    bool improved = true;
    while (improved && probes < max_probes) {
        improved = false;
        for (int dim = 0; dim < 4; ++dim) {
            const int lo = dim < 3 ? TUNE_SHIFT_MIN : 0, hi = dim < 3 ? TUNE_SHIFT_MAX : 1;
            int* field = dim == 0 ? &cur.lo : dim == 1 ? &cur.up : dim == 2 ? &cur.a : &cur.stage;
            bool moved = true;
            while (moved) {
                moved = false;
                for (int step : {-1, 1}) {
                    const int v = *field + step;
                    if (v < lo || v > hi) continue;
                    TuneChoice c = cur;
                    int* cf = dim == 0 ? &c.lo : dim == 1 ? &c.up : dim == 2 ? &c.a : &c.stage;
                    *cf = v;
                    double cc = 0.0;
                    if (!eval(c, &cc)) break;
                    if (cc < 0.99 * cur_cost) {
                        cur = c;
                        cur_cost = cc;
                        moved = improved = true;
                        break;
                    }
                }
            }
        }
    }
    *best = cur;
    if (best_cost) *best_cost = cur_cost;
    return probes;
}
