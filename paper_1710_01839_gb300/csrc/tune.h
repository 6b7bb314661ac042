// Algorithm / block-size selection for MPGEMM_AUTO.
#pragma once

#include <cstdint>

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

}  // namespace mpg
