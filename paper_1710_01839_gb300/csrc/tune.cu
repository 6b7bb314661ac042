// The tuning procedure of the paper's Section 3, on the GPU:
//   1. for every candidate block size n_min, time the block algorithm on A's
//      first r rows against the whole of B and predict the full time as
//      T_sample * m / r (Fig. 1; the paper's tables imply r = 2 n_min);
//   2. keep the n_min with the smallest prediction;
//   3. time the simple algorithm, the block algorithm with that n_min and
//      Strassen (depths 1..4, leaves at that n_min) and pick the fastest.
// GPU adaptation of step 1: a reduced-row launch must still fill the machine,
// so r is at least the rows that give one full wave of CTAs (same per-CTA
// work as the full run), rounded up to the CTA tile; and the scale factor
// m / r becomes the ratio of per-SM rounds of CTAs (full run / sample), which
// equals m / r when both are whole rounds and also covers the partly filled
// last round.
//
// Choices can be remembered per problem shape; MPGEMM_AUTO then uses them,
// else the cost model if one is installed, else a fixed default.
#include <algorithm>
#include <cstring>
#include <chrono>
#include <cmath>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "common.cuh"
#include "kernels.h"
#include "strassen.h"
#include "tune.h"

namespace mpg {

// (kind, bits, m, l, n, SMs): choices are remembered per SM count, so a run
// on an SM partition (partition.cu) keeps its own.
using Key = std::tuple<int, int, int64_t, int64_t, int64_t, int>;
static std::mutex g_tmu;
static std::map<Key, Choice> g_table;

// Installed cost model (mlp.cu); returns false when none is installed.
bool cost_model_choice(int kind, int prec_bits, int64_t m, int64_t l, int64_t n, int sms, Choice* out,
                       float* pred_ms = nullptr);

void remember_choice(int kind, int prec_bits, int64_t m, int64_t l, int64_t n, int sms, Choice ch) {
    std::lock_guard<std::mutex> lk(g_tmu);
    g_table[Key(kind, prec_bits, m, l, n, sms)] = ch;
}

// MPGEMM_AUTO's selection mode (mpgemm_auto_mode): 1 = the cost model's
// short list timed on the operands when it holds more than one
// configuration, 0 = the cost model's pick alone (never times).
static int g_auto_mode = 1;
// The short list: configurations predicted within this fraction of the best
// (about twice the model's 90th-percentile error on held-out timings) and
// the best of each algorithm family within twice it or predicted cheap to
// time, at most this many.
constexpr double AUTO_MARGIN = 0.30;
constexpr double AUTO_CHEAP_MS = 2.0;   // a family's best predicted below this is timed anyway
constexpr int AUTO_MAX_TIMED = 6;

// Replacement timer (mpgemm_tune_set_timer): simulated or recorded timings.
static std::mutex g_timer_mu;
static mpgemm_timer_fn g_timer = nullptr;
static void* g_timer_ctx = nullptr;

int auto_choice(int kind, int prec_bits, int64_t m, int64_t l, int64_t n, int sms, Choice* out) {
    {
        std::lock_guard<std::mutex> lk(g_tmu);
        auto it = g_table.find(Key(kind, prec_bits, m, l, n, sms));
        if (it != g_table.end()) {
            *out = it->second;
            return MPGEMM_OK;
        }
    }
    if (cost_model_choice(kind, prec_bits, m, l, n, sms, out)) return MPGEMM_OK;
    out->algo = MPGEMM_BLOCK;
    out->n_min = default_n_min(kind);
    out->depth = 0;
    return MPGEMM_OK;
}

// CTA tile edge used by the block kernel for a given n_min (mirrors the
// launch selection in gemm_ddqd.cu / gemm_mp.cu).
int block_tile(int kind, int n_min) {
    if (kind == MPGEMM_KIND_DD) return n_min <= 16 ? 16 : n_min <= 32 ? 32 : 64;
    if (kind == MPGEMM_KIND_QD) return n_min <= 16 ? 16 : 32;
    return 16;
}

// Resident CTAs per SM assumed for a full wave (measured occupancy of the
// block kernels: 256-thread CTAs; DD 64-tiles use ~180 registers per thread).
static int ctas_per_sm(int kind, int tile) {
    if (kind == MPGEMM_KIND_DD) return tile == 64 ? 1 : tile == 32 ? 3 : 4;
    if (kind == MPGEMM_KIND_QD) return tile == 32 ? 2 : 3;
    return 2;
}

// Per-SM rounds of CTAs for `rows` rows of C: the block kernels are bound
// by one pipe per SM (FP64 for DD/QD, integer for multi-limb), so an SM's
// co-resident CTAs share it and the run time follows the largest number of
// CTAs any SM receives, ceil(CTAs / SMs).
static double rounds(int kind, int64_t rows, int64_t n, int n_min, int sms) {
    int tile = block_tile(kind, n_min);
    int64_t ctas = ((rows + tile - 1) / tile) * ((n + tile - 1) / tile);
    return (double)((ctas + sms - 1) / sms);
}

int64_t sample_rows_rule(int64_t m, int n_min, int64_t wave_rows, int tile) {
    int64_t r = 2 * (int64_t)n_min;
    if (r < wave_rows) r = wave_rows;
    if (tile > 0) r = (r + tile - 1) / tile * tile;
    if (r > m) r = m;
    return r;
}

namespace {

struct Problem {
    int kind, prec_bits;
    int64_t m, l, n;
    const void* A;
    const void* B;
    void* C;
    cudaStream_t s;
};

int run_once(const Problem& P, int algo, int n_min, int depth, int64_t rows) {
    if (P.kind == MPGEMM_KIND_MP) {
        int w = P.prec_bits / 32;
        const size_t eb = sizeof(uint32_t) * (size_t)(2 + w);
        View<const uint32_t> a = bounded(View<const uint32_t>{(const uint32_t*)P.A, P.l, P.m * P.l, 0}, P.A,
                                         eb * P.m * P.l);
        View<const uint32_t> b = bounded(planes_view((const uint32_t*)P.B, P.l, P.n), P.B, eb * P.l * P.n);
        View<uint32_t> c = bounded(View<uint32_t>{(uint32_t*)P.C, P.n, P.m * P.n, 0}, P.C, eb * P.m * P.n);
        if (algo == MPGEMM_STRASSEN) return strassen_mp(w, P.m, P.l, P.n, a, b, c, n_min, depth, P.s);
        return mp_gemm(w, algo, rows, P.l, P.n, 1, a, b, c, n_min, P.s);
    }
    const size_t eb = sizeof(double) * (P.kind == MPGEMM_KIND_DD ? 2 : 4);
    View<const double> a = bounded(View<const double>{(const double*)P.A, P.l, P.m * P.l, 0}, P.A, eb * P.m * P.l);
    View<const double> b = bounded(planes_view((const double*)P.B, P.l, P.n), P.B, eb * P.l * P.n);
    View<double> c = bounded(View<double>{(double*)P.C, P.n, P.m * P.n, 0}, P.C, eb * P.m * P.n);
    if (algo == MPGEMM_STRASSEN) return strassen_ddqd(P.kind, P.m, P.l, P.n, a, b, c, n_min, depth, P.s);
    return ddqd_gemm(P.kind, algo, rows, P.l, P.n, 1, a, b, c, n_min, P.s);
}

// Time per run, in ms, of `reps` runs issued back to back between two
// events (after one warm-up run): the steady-state cost of a repeated call,
// with the host's launch overhead overlapped by the device's work as it is
// in a loop of calls.
int time_it(const Problem& P, int algo, int n_min, int depth, int64_t rows, int reps, double* ms) {
    cudaEvent_t e0, e1;
    MPG_CUDA(cudaEventCreate(&e0));
    MPG_CUDA(cudaEventCreate(&e1));
    int rc = run_once(P, algo, n_min, depth, rows);
    if (rc == MPGEMM_OK && cudaStreamSynchronize(P.s) != cudaSuccess) rc = MPGEMM_ECUDA;
    float f = 0.f;
    if (rc == MPGEMM_OK) {
        cudaEventRecord(e0, P.s);
        for (int i = 0; i < reps && rc == MPGEMM_OK; i++) rc = run_once(P, algo, n_min, depth, rows);
        cudaEventRecord(e1, P.s);
        if (cudaEventSynchronize(e1) != cudaSuccess) rc = MPGEMM_ECUDA;
        cudaEventElapsedTime(&f, e0, e1);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc) return rc;
    *ms = reps > 0 ? (double)f / reps : 0.0;
    return MPGEMM_OK;
}

// One timing of the procedure: from the open tuning cache when it holds
// this measurement, else from the replacement timer if one is set, else
// timed on the device; new timings are appended to the cache at once.
int measure(const Problem& P, const TuneKey& key, int algo, int n_min, int depth, int64_t rows, int reps, double* ms,
            int* measured) {
    if (tune_cache_lookup_meas(key, algo, n_min, depth, rows, reps, ms)) return MPGEMM_OK;
    mpgemm_timer_fn fn;
    void* ctx;
    {
        std::lock_guard<std::mutex> lk(g_timer_mu);
        fn = g_timer;
        ctx = g_timer_ctx;
    }
    if (fn) {
        const double t = fn(ctx, P.kind, P.prec_bits, P.m, P.l, P.n, algo, n_min, depth, rows, reps);
        if (!(t >= 0.0)) return MPGEMM_ECUDA;
        *ms = t;
    } else {
        int rc = time_it(P, algo, n_min, depth, rows, reps, ms);
        if (rc) return rc;
    }
    (*measured)++;
    tune_cache_append_meas(key, algo, n_min, depth, rows, reps, *ms);
    return MPGEMM_OK;
}

}  // namespace

int auto_choice_measured(int kind, int prec_bits, int64_t m, int64_t l, int64_t n, const void* A, const void* B,
                         void* C, cudaStream_t s, Choice* out) {
    const int sms = stream_sms(s);
    {
        std::lock_guard<std::mutex> lk(g_tmu);
        auto it = g_table.find(Key(kind, prec_bits, m, l, n, sms));
        if (it != g_table.end()) {
            *out = it->second;
            return MPGEMM_OK;
        }
    }
    std::vector<Choice> list;
    std::vector<float> pred;
    if (!cost_model_shortlist(kind, prec_bits, m, l, n, sms, AUTO_MARGIN, AUTO_CHEAP_MS, AUTO_MAX_TIMED, &list,
                              &pred) ||
        list.empty())
        return auto_choice(kind, prec_bits, m, l, n, sms, out);
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cap) != cudaSuccess) {
        cudaGetLastError();
        cap = cudaStreamCaptureStatusActive;
    }
    int mode;
    {
        std::lock_guard<std::mutex> lk(g_tmu);
        mode = g_auto_mode;
    }
    if (list.size() == 1 || mode == 0 || cap != cudaStreamCaptureStatusNone)
        return auto_choice(kind, prec_bits, m, l, n, sms, out);   // the model's rule, nothing timed
    Problem P{kind, kind == MPGEMM_KIND_MP ? prec_bits : 0, m, l, n, A, B, C, s};
    const TuneKey key{kind, P.prec_bits, m, l, n, sms};
    int measured = 0;
    std::vector<double> t(list.size());
    for (size_t i = 0; i < list.size(); i++) {
        const float p = pred[i];
        const int reps = p < 1.0f ? 10 : p < 20.0f ? 3 : 1;
        int rc = measure(P, key, list[i].algo, list[i].n_min, list[i].depth, m, reps, &t[i], &measured);
        if (rc) return rc;
    }
    // the fastest; among those within 3 % of it (timing noise), the fewest
    // launches (a caller with more launch overhead than this timer pays less)
    const double tmin = *std::min_element(t.begin(), t.end());
    auto launches = [](const Choice& c) { return c.algo == MPGEMM_STRASSEN ? 3 * c.depth + 1 : 1; };
    int best = -1;
    for (size_t i = 0; i < list.size(); i++) {
        if (t[i] > 1.03 * tmin) continue;
        if (best < 0 || launches(list[i]) < launches(list[best]) ||
            (launches(list[i]) == launches(list[best]) && t[i] < t[best]))
            best = (int)i;
    }
    const double best_ms = t[best];
    *out = list[best];
    remember_choice(kind, P.prec_bits, m, l, n, sms, *out);
    mpgemm_tune_report rep;
    memset(&rep, 0, sizeof rep);
    rep.algo = out->algo;
    rep.n_min = out->n_min;
    rep.depth = out->depth;
    rep.best_ms = best_ms;
    rep.simple_ms = rep.block_ms = NAN;
    for (int d = 0; d < 5; d++) rep.strassen_ms[d] = NAN;
    tune_cache_append_choice(key, &rep);
    return MPGEMM_OK;
}

}  // namespace mpg

using namespace mpg;

extern "C" {

double mpgemm_predict_time(double t_sample, int64_t m, int64_t rows) {
    if (rows <= 0) return NAN;
    return t_sample * (double)m / (double)rows;
}

int64_t mpgemm_sample_rows(int kind, int64_t m, int64_t n, int n_min, int num_sms) {
    int tile = block_tile(kind, n_min);
    int64_t tiles_n = (n + tile - 1) / tile;
    int64_t wave_ctas = (int64_t)num_sms * ctas_per_sm(kind, tile);
    int64_t wave_rows = tiles_n > 0 ? (wave_ctas + tiles_n - 1) / tiles_n * tile : tile;
    return sample_rows_rule(m, n_min, wave_rows, tile);
}

int mpgemm_tune(int kind, int prec_bits, int64_t m, int64_t l, int64_t n, const void* A, const void* B, void* C,
                int flags, void* stream, mpgemm_tune_report* rep) {
    if (!rep || m <= 0 || l <= 0 || n <= 0 || !A || !B || !C) return MPGEMM_EINVAL;
    if (kind < MPGEMM_KIND_DD || kind > MPGEMM_KIND_MP) return MPGEMM_EINVAL;
    if (kind == MPGEMM_KIND_MP && (prec_bits <= 0 || prec_bits % 32)) return MPGEMM_EINVAL;
    auto t_start = std::chrono::steady_clock::now();
    Problem P{kind, kind == MPGEMM_KIND_MP ? prec_bits : 0, m, l, n, A, B, C, (cudaStream_t)stream};
    PartitionScope pscope(P.s);
    const int sms = stream_sms(P.s);   // the partition's SMs when the stream has one
    const int reps = (flags & MPGEMM_TUNE_QUICK) ? 1 : 3;
    memset(rep, 0, sizeof *rep);
    const TuneKey key{kind, P.prec_bits, m, l, n, sms};
    auto wall_ms = [&] {
        return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t_start).count();
    };
    if (!(flags & MPGEMM_TUNE_FORCE) && tune_cache_lookup_choice(key, rep)) {
        rep->from_cache = 1;
        rep->measured = 0;
        remember_choice(kind, P.prec_bits, m, l, n, sms, Choice{rep->algo, rep->n_min, rep->depth});
        rep->tuning_ms = wall_ms();
        return MPGEMM_OK;
    }
    int measured = 0;
    static const int cands[] = {16, 32, 64, 128, 256, 512};
    constexpr int NC = (int)(sizeof cands / sizeof cands[0]);
    int best = -1;
    double best_pred = 0;
    for (int c = 0; c < NC; c++) {
        int nm = cands[c];
        int64_t r = mpgemm_sample_rows(kind, m, n, nm, sms);
        double ms = 0;
        int rc = measure(P, key, MPGEMM_BLOCK, nm, 0, r, reps, &ms, &measured);
        if (rc) return rc;
        rep->cand_n_min[c] = nm;
        rep->cand_rows[c] = r;
        rep->cand_sample_ms[c] = ms;
        rep->cand_pred_ms[c] = ms * rounds(kind, m, n, nm, sms) / rounds(kind, r, n, nm, sms);
        rep->cand_full_ms[c] = NAN;
        if (flags & MPGEMM_TUNE_VERIFY) {
            rc = measure(P, key, MPGEMM_BLOCK, nm, 0, m, reps, &rep->cand_full_ms[c], &measured);
            if (rc) return rc;
        }
        if (best < 0 || rep->cand_pred_ms[c] < best_pred) {
            best = c;
            best_pred = rep->cand_pred_ms[c];
        }
    }
    rep->n_cand = NC;
    const int nm = cands[best];
    int rc;
    rep->simple_ms = NAN;
    if (!(flags & MPGEMM_TUNE_SKIP_SIMPLE)) {
        rc = measure(P, key, MPGEMM_SIMPLE, nm, 0, m, reps, &rep->simple_ms, &measured);
        if (rc) return rc;
    }
    rc = measure(P, key, MPGEMM_BLOCK, nm, 0, m, reps, &rep->block_ms, &measured);
    if (rc) return rc;
    Choice ch{MPGEMM_BLOCK, nm, 0};
    double best_ms = rep->block_ms;
    if (!std::isnan(rep->simple_ms) && rep->simple_ms < best_ms) {
        ch = Choice{MPGEMM_SIMPLE, nm, 0};
        best_ms = rep->simple_ms;
    }
    for (int d = 1; d <= 4; d++) {
        rep->strassen_ms[d] = NAN;
        // leaves of the zero-extended problem at least 16 on every side
        if (strassen_extended(m, d) >> d < 16 || strassen_extended(l, d) >> d < 16 ||
            strassen_extended(n, d) >> d < 16)
            continue;
        rc = measure(P, key, MPGEMM_STRASSEN, nm, d, m, reps, &rep->strassen_ms[d], &measured);
        if (rc) return rc;
        if (rep->strassen_ms[d] < best_ms) {
            ch = Choice{MPGEMM_STRASSEN, nm, d};
            best_ms = rep->strassen_ms[d];
        }
    }
    rep->algo = ch.algo;
    rep->n_min = ch.n_min;
    rep->depth = ch.depth;
    rep->best_ms = best_ms;
    rep->measured = measured;
    rep->from_cache = 0;
    if (flags & MPGEMM_TUNE_REMEMBER) remember_choice(kind, P.prec_bits, m, l, n, sms, ch);
    tune_cache_append_choice(key, rep);
    rep->tuning_ms = wall_ms();
    return MPGEMM_OK;
}

int mpgemm_time_config(int kind, int prec_bits, int64_t m, int64_t l, int64_t n, const void* A, const void* B,
                       void* C, int algo, int n_min, int depth, int reps, void* stream, double* ms) {
    if (!ms || m <= 0 || l <= 0 || n <= 0 || !A || !B || !C || reps < 1 || reps > 1000) return MPGEMM_EINVAL;
    if (kind < MPGEMM_KIND_DD || kind > MPGEMM_KIND_MP) return MPGEMM_EINVAL;
    if (kind == MPGEMM_KIND_MP && (prec_bits <= 0 || prec_bits % 32)) return MPGEMM_EINVAL;
    if (algo < MPGEMM_SIMPLE || algo > MPGEMM_STRASSEN || n_min < 1 || depth < 0 || depth > 4) return MPGEMM_EINVAL;
    Problem P{kind, kind == MPGEMM_KIND_MP ? prec_bits : 0, m, l, n, A, B, C, (cudaStream_t)stream};
    PartitionScope pscope(P.s);
    return time_it(P, algo, n_min, algo == MPGEMM_STRASSEN ? depth : 0, m, reps, ms);
}

int mpgemm_auto_mode(int mode) {
    if (mode != 0 && mode != 1) return MPGEMM_EINVAL;
    std::lock_guard<std::mutex> lk(g_tmu);
    g_auto_mode = mode;
    return MPGEMM_OK;
}

int mpgemm_tune_set_timer(mpgemm_timer_fn fn, void* ctx) {
    std::lock_guard<std::mutex> lk(g_timer_mu);
    g_timer = fn;
    g_timer_ctx = fn ? ctx : nullptr;
    return MPGEMM_OK;
}

int mpgemm_tune_forget(void) {
    std::lock_guard<std::mutex> lk(g_tmu);
    g_table.clear();
    return MPGEMM_OK;
}

int mpgemm_auto_choice(int kind, int prec_bits, int64_t m, int64_t l, int64_t n, int* algo, int* n_min, int* depth) {
    Choice c;
    int rc = auto_choice(kind, prec_bits, m, l, n, stream_sms(nullptr), &c);
    if (rc) return rc;
    if (algo) *algo = c.algo;
    if (n_min) *n_min = c.n_min;
    if (depth) *depth = c.depth;
    return MPGEMM_OK;
}

}  // extern "C"
