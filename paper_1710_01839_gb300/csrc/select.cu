// Precision selection from an accuracy target (the paper's outlook: choose
// the precision, not only the algorithm, for the user).
//
// Every configuration the library offers for a real product C = AB gets an
// a-priori elementwise bound |C - AB| <= beta |A||B|, and the configurations
// with beta <= the target are ranked by predicted time.  Bounds (u_p = 2^-p):
//   DD (simple / block)     4 l 2^-104 (the DD kernels' tested bound);
//   QD (simple / block)     4 l 2^-208;
//   p-bit multi-limb        gamma_l = l u_p / (1 - l u_p) (one rounding per
//                           multiply and per add, Eq 1 order);
//   split precision         with an entry at most `spread` binades below the
//                           largest of its row (A) or column (B), the
//                           truncation of one operand costs at most
//                           t = 2^(spread + 1 - 7S) (int8) or
//                           2^(spread + 2 - 5S) (e4m3) of it, the dropped
//                           triangle s + t > S + 1 at most
//                           (S + 1) c 2^(2 spread + 2 - bS) (c = 1.02 / 1.07
//                           for b = 7 / 5), the final DD rounding 2^-106:
//                           beta = 2t + t^2 + triangle + 2^-106 (DD result;
//                           2^-211 for the QD result of the QD split).
//   DD / QD on the integer pipe  (p-bit limbs, T = 2 / 4 result terms)
//                           gamma_l(p) for the multi-limb GEMM, 2^(1-p) for
//                           rounding both operands to p bits, 2^(-53 T) for
//                           the final greedy expansion (each term takes all
//                           but 2^-53 of the remainder), each to first order
//                           (a 2^-40 relative allowance covers the rest).
// Strassen is left out: its bound (2^-96 l max|A| max|B| for DD) is not
// elementwise.  Predicted times: the installed cost model's best simple /
// block configuration for DD, QD and multi-limb, else the block rates
// measured on GB300; split precision from its tensor work at the measured
// level-kernel rates plus its memory passes.
#include <algorithm>
#include <climits>
#include <cmath>
#include <vector>

#include "common.cuh"

namespace mpg {

double cost_model_block_ms(int kind, int prec_bits, int64_t m, int64_t l, int64_t n, int sms);

namespace {

struct Cand {
    int method, bits, slices;
    double log2_bound, ms;
};

// log2 of a sum of terms given as log2 values
double log2_sum(std::initializer_list<double> xs) {
    double mx = -1e300;
    for (double x : xs) mx = std::max(mx, x);
    double s = 0.0;
    for (double x : xs) s += std::exp2(x - mx);
    return mx + std::log2(s);
}

// final_log2: the rounding of the exact result (DD: 2^-106, QD: 2^-211).
double split_log2_bound(int digit_bits, int S, int spread, double final_log2 = -106.0) {
    const double t = (digit_bits == 7 ? spread + 1.0 : spread + 2.0) - (double)digit_bits * S;
    const double c = digit_bits == 7 ? 1.02 : 1.07;
    const double tri = std::log2((S + 1) * c) + 2.0 * spread + 2.0 - (double)digit_bits * S;
    return log2_sum({1.0 + t, 2.0 * t, tri, final_log2});
}

// Block-algorithm rates measured on GB300 (effective GFLOP/s, 1024-2048).
double static_block_gflops(int method, int bits) {
    if (method == MPGEMM_SEL_DD) return 118.0;
    if (method == MPGEMM_SEL_QD) return 13.7;
    switch (bits) {
        case 128: return 108.0;
        case 256: return 75.0;
        case 512: return 27.0;
        default: return 7.5;   // 1024
    }
}

double mp_gamma_log2(int64_t l, int prec_bits) {
    const double lu = std::log2((double)l) - prec_bits;   // log2(l u)
    return lu >= -1.0 ? INFINITY : lu - std::log2(1.0 - std::exp2(lu));
}

double via_mp_log2_bound(int terms, int prec_bits, int64_t l) {
    const double g = mp_gamma_log2(l, prec_bits);
    if (!std::isfinite(g)) return INFINITY;
    const double slack = std::log2(1.0 + std::exp2(-40.0));
    return log2_sum({g, 1.0 - prec_bits, -53.0 * terms}) + slack;
}

// The two conversion passes of mpgemm_{dd,qd}_via_mp, per element as
// measured on GB300 (DD 128-bit: 10 / 12 ps in / out; QD 256-bit: 35 / 43).
double via_mp_convert_ms(int terms, int64_t m, int64_t l, int64_t n) {
    const double tin = terms == 2 ? 10e-12 : 35e-12, tout = terms == 2 ? 12e-12 : 43e-12;
    return 1e3 * (((double)m * l + (double)l * n) * tin + (double)m * n * tout) + 0.01;
}

double split_ms(int digit_bits, int S, int64_t m, int64_t l, int64_t n, int terms = 2) {
    const double lp = (double)((l + 127) / 128 * 128);
    const double ops = 2.0 * (double)m * (double)n * lp * S * (S + 1) / 2.0;
    const double rate = digit_bits == 5 ? 3.4e15 : 1.5e14;   // k_levels_tc / k_ozaki_levels, measured
    const double bytes = 8.0 * terms * ((double)m * l + (double)l * n) + (double)S * (m + n) * lp +
                         8.0 * S * (double)m * n + 8.0 * terms * (double)m * n;
    return 1e3 * (ops / rate + bytes / 3.0e12) + 0.05;
}

// frexp exponent of a nonzero double from its bits (INT_MIN for +-0).
__device__ __forceinline__ int sel_expo(double x) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    if ((((unsigned)__double2hiint(x) << 1) | (unsigned)__double2loint(x)) == 0u) return INT_MIN;
    const int E = (int)((b >> 52) & 0x7ff);
    if (E == 0) return -1022 - (__clzll(b & ((1ull << 52) - 1)) - 12);
    return E - 1022;
}

// Rows of A's hi plane: spread = largest exponent - smallest nonzero one.
__global__ void k_row_spread(int64_t m, int64_t l, const double* hi, int* out) {
    const int64_t row = (int64_t)blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
    const int lane = threadIdx.x & 31;
    if (row >= m) return;
    int mx = INT_MIN, mn = INT_MAX;
    for (int64_t k = lane; k < l; k += 32) {
        const int e = sel_expo(hi[row * l + k]);
        if (e != INT_MIN) {
            mx = max(mx, e);
            mn = min(mn, e);
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        mn = min(mn, __shfl_xor_sync(0xffffffffu, mn, o));
    }
    if (lane == 0 && mx != INT_MIN) atomicMax(out, mx - mn);
}

// Columns of B's hi plane: per-column extremes over 256-row blocks.
__global__ void k_col_extremes(int64_t l, int64_t n, const double* hi, int* cmax, int* cmin) {
    const int64_t j = (int64_t)blockIdx.x * 32 + threadIdx.x;
    if (j >= n) return;
    const int64_t k0 = (int64_t)blockIdx.y * 256, k1 = k0 + 256 < l ? k0 + 256 : l;
    int mx = INT_MIN, mn = INT_MAX;
    for (int64_t k = k0 + threadIdx.y; k < k1; k += blockDim.y) {
        const int e = sel_expo(hi[k * n + j]);
        if (e != INT_MIN) {
            mx = max(mx, e);
            mn = min(mn, e);
        }
    }
    if (mx != INT_MIN) {
        atomicMax(cmax + j, mx);
        atomicMin(cmin + j, mn);
    }
}

__global__ void k_col_spread(int64_t n, const int* cmax, const int* cmin, int* out) {
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j < n && cmax[j] >= cmin[j]) atomicMax(out, cmax[j] - cmin[j]);
}

}  // namespace

}  // namespace mpg

using namespace mpg;

extern "C" {

double mpgemm_precision_log2_bound(int method, int prec_bits, int num_slices, int64_t l, int spread) {
    if (l <= 0 || spread < 0) return NAN;
    const double ll = std::log2((double)l);
    switch (method) {
        case MPGEMM_SEL_DD: return 2.0 + ll - 104.0;
        case MPGEMM_SEL_QD: return 2.0 + ll - 208.0;
        case MPGEMM_SEL_MP:
            return prec_bits <= 0 ? NAN : mp_gamma_log2(l, prec_bits);
        case MPGEMM_SEL_DD_VIA_MP:
        case MPGEMM_SEL_QD_VIA_MP: {
            const int terms = method == MPGEMM_SEL_DD_VIA_MP ? 2 : 4;
            const int bits = prec_bits > 0 ? prec_bits : (terms == 2 ? 128 : 256);
            if (bits % 32 || bits < 64 || bits > 512) return NAN;
            return via_mp_log2_bound(terms, bits, l);
        }
        case MPGEMM_SEL_OZAKI_INT8:
            return (num_slices >= 1 && num_slices <= 18) ? split_log2_bound(7, num_slices, spread) : NAN;
        case MPGEMM_SEL_OZAKI_E4M3:
            return (num_slices >= 1 && num_slices <= 24) ? split_log2_bound(5, num_slices, spread) : NAN;
        case MPGEMM_SEL_OZAKI_QD:
            return (num_slices >= 1 && num_slices <= 48) ? split_log2_bound(5, num_slices, spread, -211.0) : NAN;
        default: return NAN;
    }
}

int mpgemm_dd_exponent_spread(int64_t m, int64_t l, int64_t n, const double* A, const double* B, int* spread,
                              void* stream) {
    if (m < 0 || l < 0 || n < 0 || !spread || (m > 0 && l > 0 && !A) || (l > 0 && n > 0 && !B)) return MPGEMM_EINVAL;
    if (l > 65535 * 256LL) return MPGEMM_EUNSUPPORTED;   // grid.y of the column pass
    *spread = 0;
    if (m == 0 || l == 0 || n == 0) return MPGEMM_OK;
    cudaStream_t s = (cudaStream_t)stream;
    PartitionScope pscope(s);
    int* buf = nullptr;   // [result | column max (n) | column min (n)]
    cudaError_t e = dev_malloc_async((void**)&buf, sizeof(int) * (size_t)(1 + 2 * n), s);
    if (e != cudaSuccess) {
        set_last_cuda_error(e);
        return MPGEMM_ENOMEM;
    }
    int rc = MPGEMM_OK;
    auto ck = [&](cudaError_t x) {
        if (x != cudaSuccess && rc == MPGEMM_OK) {
            set_last_cuda_error(x);
            rc = MPGEMM_ECUDA;
        }
    };
    ck(cudaMemsetAsync(buf, 0, sizeof(int), s));
    ck(cudaMemsetAsync(buf + 1, 0x80, sizeof(int) * (size_t)n, s));       // below every exponent
    ck(cudaMemsetAsync(buf + 1 + n, 0x7F, sizeof(int) * (size_t)n, s));   // above every exponent
    if (rc == MPGEMM_OK) {
        k_row_spread<<<ceil_div(m, 8), 256, 0, s>>>(m, l, A, buf);
        k_col_extremes<<<dim3(ceil_div(n, 32), ceil_div(l, 256)), dim3(32, 8), 0, s>>>(l, n, B, buf + 1, buf + 1 + n);
        k_col_spread<<<ceil_div(n, 256), 256, 0, s>>>(n, buf + 1, buf + 1 + n, buf);
        ck(cudaGetLastError());
        ck(cudaMemcpyAsync(spread, buf, sizeof(int), cudaMemcpyDeviceToHost, s));
    }
    ck(cudaFreeAsync(buf, s));
    ck(cudaStreamSynchronize(s));
    return rc;
}

int mpgemm_select_precision(double log2_target, int64_t m, int64_t l, int64_t n, int spread,
                            mpgemm_precision_choice* out, int max_out) {
    if (m <= 0 || l <= 0 || n <= 0 || spread < 0 || max_out < 0 || (max_out > 0 && !out) || std::isnan(log2_target))
        return MPGEMM_EINVAL;
    const int sms = stream_sms(nullptr);
    std::vector<Cand> cs;
    auto timed = [&](int method, int bits) {
        const int kind = method == MPGEMM_SEL_DD ? MPGEMM_KIND_DD : method == MPGEMM_SEL_QD ? MPGEMM_KIND_QD
                                                                                              : MPGEMM_KIND_MP;
        double ms = cost_model_block_ms(kind, bits, m, l, n, sms);
        if (ms < 0) ms = 2.0 * (double)m * l * n / (static_block_gflops(method, bits) * 1e9) * 1e3;
        return ms;
    };
    // split precision: the fewest slices that meet the target
    for (int db : {5, 7}) {
        const int method = db == 5 ? MPGEMM_SEL_OZAKI_E4M3 : MPGEMM_SEL_OZAKI_INT8;
        const int smax = db == 5 ? 24 : 18;
        if (db == 5 && l > 65536) continue;                                  // exact f32 chunks need 256 l <= 2^24
        if (db == 7 && (double)smax * 16129.0 * (double)l >= 2147483648.0) continue;   // int32 level sums
        for (int S = 1; S <= smax; S++) {
            const double b = mpgemm_precision_log2_bound(method, 0, S, l, spread);
            if (b <= log2_target) {
                cs.push_back({method, 0, S, b, split_ms(db, S, m, l, n)});
                break;
            }
        }
    }
    // QD split (QD operands and result): only for targets the DD splits cannot reach
    bool dd_split = false;
    for (const Cand& c : cs) dd_split |= c.method == MPGEMM_SEL_OZAKI_E4M3 || c.method == MPGEMM_SEL_OZAKI_INT8;
    if (!dd_split && l <= 65536 && 48.0 * 256.0 * (double)l < 2147483648.0) {
        for (int S = 1; S <= 48; S++) {
            const double b = mpgemm_precision_log2_bound(MPGEMM_SEL_OZAKI_QD, 0, S, l, spread);
            if (b <= log2_target) {
                cs.push_back({MPGEMM_SEL_OZAKI_QD, 0, S, b, split_ms(5, S, m, l, n, 4)});
                break;
            }
        }
    }
    for (int method : {MPGEMM_SEL_DD, MPGEMM_SEL_QD}) {
        const double b = mpgemm_precision_log2_bound(method, 0, 0, l, 0);
        if (b <= log2_target) cs.push_back({method, 0, 0, b, timed(method, 0)});
    }
    // DD / QD on the integer pipe (DD / QD operands and result)
    for (int terms : {2, 4}) {
        const int method = terms == 2 ? MPGEMM_SEL_DD_VIA_MP : MPGEMM_SEL_QD_VIA_MP;
        const int bits = terms == 2 ? 128 : 256;
        const double b = via_mp_log2_bound(terms, bits, l);
        if (b <= log2_target)
            cs.push_back({method, bits, 0, b, timed(MPGEMM_SEL_MP, bits) + via_mp_convert_ms(terms, m, l, n)});
    }
    for (int bits : {128, 256, 512, 1024}) {   // the smallest multi-limb precision that meets the target
        const double b = mpgemm_precision_log2_bound(MPGEMM_SEL_MP, bits, 0, l, 0);
        if (b <= log2_target) {
            cs.push_back({MPGEMM_SEL_MP, bits, 0, b, timed(MPGEMM_SEL_MP, bits)});
            break;
        }
    }
    std::stable_sort(cs.begin(), cs.end(), [](const Cand& a, const Cand& b) { return a.ms < b.ms; });
    const int k = std::min<int>(max_out, (int)cs.size());
    for (int i = 0; i < k; i++)
        out[i] = mpgemm_precision_choice{cs[i].method, cs[i].bits, cs[i].slices, cs[i].log2_bound, cs[i].ms};
    return (int)cs.size();
}

}  // extern "C"
