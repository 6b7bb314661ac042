// Algorithm / block-size selection for MPGEMM_AUTO.
#pragma once

#include <cstdint>
#include <vector>

#include <cuda_runtime.h>

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

// MPGEMM_AUTO for a call with operands (device pointers in the format of
// `kind`; C may be overwritten): the remembered choice; else the cost
// model's short list of configurations predicted within its own error of
// the best, where a list of more than one is timed once on the operands
// (not while the stream captures a graph, and not in model-only mode) and
// its fastest member remembered; without a model, the default.
int auto_choice_measured(int kind, int prec_bits, int64_t m, int64_t l, int64_t n, const void* A, const void* B,
                         void* C, cudaStream_t s, Choice* out);

// Stores a choice for MPGEMM_AUTO (as MPGEMM_TUNE_REMEMBER does).
void remember_choice(int kind, int prec_bits, int64_t m, int64_t l, int64_t n, int sms, Choice ch);

// Persistent tuning cache (tune_cache.cu): lookups fail and appends do
// nothing while no cache file is open.
struct TuneKey {
    int kind, bits;
    int64_t m, l, n;
    int sms;
};
// Cost model (mlp.cu): the configurations predicted within (1 + margin) of
// the best, fastest first, and the best of each algorithm family predicted
// within (1 + 2 margin) or below cheap_ms, at most kmax; false without a
// model.
bool cost_model_shortlist(int kind, int prec_bits, int64_t m, int64_t l, int64_t n, int sms, double margin,
                          double cheap_ms, int kmax, std::vector<Choice>* out, std::vector<float>* pred_ms);

bool tune_cache_lookup_meas(const TuneKey& k, int algo, int n_min, int depth, int64_t rows, int reps, double* ms);
void tune_cache_append_meas(const TuneKey& k, int algo, int n_min, int depth, int64_t rows, int reps, double ms);
bool tune_cache_lookup_choice(const TuneKey& k, mpgemm_tune_report* rep);
void tune_cache_append_choice(const TuneKey& k, const mpgemm_tune_report* rep);

}  // namespace mpg
