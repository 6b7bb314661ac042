// FP32 MLP cost model (placeholder until trained models are installed).
#include "common.cuh"
#include "tune.h"

namespace mpg {

bool cost_model_choice(int kind, int prec_bits, int64_t m, int64_t l, int64_t n, Choice* out) {
    (void)kind; (void)prec_bits; (void)m; (void)l; (void)n; (void)out;
    return false;
}

}  // namespace mpg
