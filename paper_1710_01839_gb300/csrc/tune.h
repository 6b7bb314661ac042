// Algorithm / block-size selection for MPGEMM_AUTO.
#pragma once

#include <cstdint>

#include "../../include/mpgemm.h"

namespace mpg {

struct Choice {
    int algo;
    int n_min;
    int depth;
};

// Pick (algo, n_min, depth) for a problem: the tuned table if one was loaded
// for this shape, else the cost model if trained, else a fixed heuristic.
// Remembered tuner choice for (kind, bits, m, l, n) on `sms` SMs, else the
// cost model's, else the default block configuration.
int auto_choice(int kind, int prec_bits, int64_t m, int64_t l, int64_t n, int sms, Choice* out);

int default_n_min(int kind);

// Stores a choice for MPGEMM_AUTO (as MPGEMM_TUNE_REMEMBER does).
void remember_choice(int kind, int prec_bits, int64_t m, int64_t l, int64_t n, int sms, Choice ch);

// Persistent tuning cache (tune_cache.cu): lookups fail and appends do
// nothing while no cache file is open.
struct TuneKey {
    int kind, bits;
    int64_t m, l, n;
    int sms;
};
bool tune_cache_lookup_meas(const TuneKey& k, int algo, int n_min, int depth, int64_t rows, int reps, double* ms);
void tune_cache_append_meas(const TuneKey& k, int algo, int n_min, int depth, int64_t rows, int reps, double ms);
bool tune_cache_lookup_choice(const TuneKey& k, mpgemm_tune_report* rep);
void tune_cache_append_choice(const TuneKey& k, const mpgemm_tune_report* rep);

}  // namespace mpg
