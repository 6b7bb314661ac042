// FP32 MLP cost model: log(time) of a GEMM configuration from its features,
// 2 hidden layers of 64 ReLU units, trained with Adam on timings the library
// measures itself.  It stands in for the paper's time prediction (Section 3)
// when picking algorithm, tile and Strassen depth (MPGEMM_AUTO, batched
// tiles); exhaustive measured tuning stays the fallback and the yardstick of its regret.
//
// Kernels: k_mlp_train runs the whole training in one CTA (1024 threads,
// activations and weights in shared memory, one minibatch of 128 per step:
// forward, backward, Adam); k_mlp_predict evaluates a batch of feature
// vectors, one thread per vector.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <random>
#include <vector>

#include "common.cuh"
#include "kernels.h"
#include "strassen.h"
#include "tune.h"

namespace mpg {

constexpr int NF = 16;     // features
constexpr int NH = 64;     // hidden units per layer
constexpr int MB = 128;    // minibatch
constexpr int NT = 1024;   // training threads
// parameter block layout (floats): W1[NF][NH] b1[NH] W2[NH][NH] b2[NH] W3[NH] b3[1]
constexpr int OFF_W1 = 0, OFF_B1 = OFF_W1 + NF * NH, OFF_W2 = OFF_B1 + NH, OFF_B2 = OFF_W2 + NH * NH,
              OFF_W3 = OFF_B2 + NH, OFF_B3 = OFF_W3 + NH, NPARAM = OFF_B3 + 1;

// Features of one configuration (all inputs of the model, before
// normalisation): log2 m, l, n and mnl; format one-hot; log2 significand
// bits; log2 tile; algorithm one-hot; Strassen depth; log2 CTAs; log2 rounds
// of CTAs over the SMs; log2 kernel launches.  The GPU-specific ones let the
// model see wave quantisation and per-launch overhead directly.
void encode_features(int kind, int prec_bits, int64_t m, int64_t l, int64_t n, int algo, int tile, int depth,
                     int sms, float* f) {
    const double lm = std::log2((double)std::max<int64_t>(m, 1)), ll = std::log2((double)std::max<int64_t>(l, 1)),
                 ln = std::log2((double)std::max<int64_t>(n, 1));
    const int bits = kind == MPGEMM_KIND_DD ? 106 : kind == MPGEMM_KIND_QD ? 212 : prec_bits;
    int64_t mm = (m + ((int64_t)1 << depth) - 1) >> depth, nn = (n + ((int64_t)1 << depth) - 1) >> depth;
    int64_t ctas = ((mm + tile - 1) / tile) * ((nn + tile - 1) / tile);
    if (algo == MPGEMM_STRASSEN) ctas *= (int64_t)std::pow(7.0, depth);
    if (algo == MPGEMM_SIMPLE) ctas = ((m + 7) / 8) * ((n + 31) / 32);
    const double rounds = std::ceil((double)ctas / std::max(sms, 1));
    float v[NF] = {(float)lm, (float)ll, (float)ln, (float)(lm + ll + ln),
                   kind == MPGEMM_KIND_DD ? 1.f : 0.f, kind == MPGEMM_KIND_QD ? 1.f : 0.f,
                   kind == MPGEMM_KIND_MP ? 1.f : 0.f, (float)std::log2((double)bits),
                   (float)std::log2((double)std::max(tile, 1)), algo == MPGEMM_SIMPLE ? 1.f : 0.f,
                   algo == MPGEMM_BLOCK ? 1.f : 0.f, algo == MPGEMM_STRASSEN ? 1.f : 0.f, (float)depth,
                   (float)std::log2((double)std::max<int64_t>(ctas, 1)), (float)std::log2(std::max(rounds, 1.0)),
                   (float)std::log2(algo == MPGEMM_STRASSEN ? 3.0 * depth + 1.0 : 1.0)};   // kernel launches
    std::memcpy(f, v, sizeof v);
}

// ---------------------------------------------------------------- kernels

__device__ __forceinline__ float relu(float x) { return x > 0.f ? x : 0.f; }

struct TrainArgs {
    const float* X;      // [N][NF] normalised features
    const float* Y;      // [N] targets (normalised log time)
    const int* perm;     // [epochs][N] sample order
    int N, epochs;
    float lr, beta1, beta2, eps;
    float* params;       // [NPARAM] in/out
    float* loss_out;     // [epochs] mean loss per epoch
};

__global__ void __launch_bounds__(NT) k_mlp_train(TrainArgs a) {
    extern __shared__ float s[];
    float* P = s;                          // parameters
    float* G = P + NPARAM;                 // gradients
    float* M1 = G + NPARAM;                // Adam first moment
    float* M2 = M1 + NPARAM;               // Adam second moment
    float* X = M2 + NPARAM;                // [MB][NF]
    float* H1 = X + MB * NF;               // [MB][NH]
    float* H2 = H1 + MB * NH;              // [MB][NH]
    float* D2 = H2 + MB * NH;              // [MB][NH] dL/d(pre-activation 2)
    float* Yp = D2 + MB * NH;              // [MB] prediction error
    __shared__ float s_loss;
    const int t = threadIdx.x;
    for (int i = t; i < NPARAM; i += NT) {
        P[i] = a.params[i];
        M1[i] = 0.f;
        M2[i] = 0.f;
    }
    __syncthreads();
    int step = 0;
    const int nb = a.N / MB;
    for (int ep = 0; ep < a.epochs; ep++) {
        if (t == 0) s_loss = 0.f;
        for (int b = 0; b < nb; b++) {
            const int* idx = a.perm + (size_t)ep * a.N + b * MB;
            for (int i = t; i < MB * NF; i += NT) X[i] = a.X[(size_t)idx[i / NF] * NF + i % NF];
            for (int i = t; i < NPARAM; i += NT) G[i] = 0.f;
            __syncthreads();
            // forward 1: H1 = relu(X W1 + b1)
            for (int i = t; i < MB * NH; i += NT) {
                int r = i / NH, h = i % NH;
                float acc = P[OFF_B1 + h];
                for (int f = 0; f < NF; f++) acc = __fmaf_rn(X[r * NF + f], P[OFF_W1 + f * NH + h], acc);
                H1[i] = relu(acc);
            }
            __syncthreads();
            // forward 2: H2 = relu(H1 W2 + b2)
            for (int i = t; i < MB * NH; i += NT) {
                int r = i / NH, h = i % NH;
                float acc = P[OFF_B2 + h];
                for (int k = 0; k < NH; k++) acc = __fmaf_rn(H1[r * NH + k], P[OFF_W2 + k * NH + h], acc);
                H2[i] = relu(acc);
            }
            __syncthreads();
            // output and its error: Yp = (H2 W3 + b3 - y) * 2 / MB
            for (int r = t; r < MB; r += NT) {
                float acc = P[OFF_B3];
                for (int k = 0; k < NH; k++) acc = __fmaf_rn(H2[r * NH + k], P[OFF_W3 + k], acc);
                float e = acc - a.Y[idx[r]];
                Yp[r] = 2.f * e / MB;
                atomicAdd(&s_loss, e * e / (MB * nb));
            }
            __syncthreads();
            // D2 = Yp W3^T (.) [H2 > 0]
            for (int i = t; i < MB * NH; i += NT) {
                int r = i / NH, h = i % NH;
                D2[i] = H2[i] > 0.f ? Yp[r] * P[OFF_W3 + h] : 0.f;
            }
            // gW3 = H2^T Yp, gb3 = sum Yp
            for (int h = t; h < NH; h += NT) {
                float acc = 0.f;
                for (int r = 0; r < MB; r++) acc = __fmaf_rn(H2[r * NH + h], Yp[r], acc);
                G[OFF_W3 + h] = acc;
            }
            if (t == 0) {
                float acc = 0.f;
                for (int r = 0; r < MB; r++) acc += Yp[r];
                G[OFF_B3] = acc;
            }
            __syncthreads();
            // gW2 = H1^T D2, gb2 = sum D2
            for (int i = t; i < NH * NH; i += NT) {
                int k = i / NH, h = i % NH;
                float acc = 0.f;
                for (int r = 0; r < MB; r++) acc = __fmaf_rn(H1[r * NH + k], D2[r * NH + h], acc);
                G[OFF_W2 + i] = acc;
            }
            for (int h = t; h < NH; h += NT) {
                float acc = 0.f;
                for (int r = 0; r < MB; r++) acc += D2[r * NH + h];
                G[OFF_B2 + h] = acc;
            }
            __syncthreads();
            // D1 = D2 W2^T (.) [H1 > 0], stored over H2 (no longer needed)
            float* D1 = H2;
            for (int i = t; i < MB * NH; i += NT) {
                int r = i / NH, k = i % NH;
                float acc = 0.f;
                for (int h = 0; h < NH; h++) acc = __fmaf_rn(D2[r * NH + h], P[OFF_W2 + k * NH + h], acc);
                D1[i] = H1[i] > 0.f ? acc : 0.f;
            }
            __syncthreads();
            // gW1 = X^T D1, gb1 = sum D1
            for (int i = t; i < NF * NH; i += NT) {
                int f = i / NH, h = i % NH;
                float acc = 0.f;
                for (int r = 0; r < MB; r++) acc = __fmaf_rn(X[r * NF + f], D1[r * NH + h], acc);
                G[OFF_W1 + i] = acc;
            }
            for (int h = t; h < NH; h += NT) {
                float acc = 0.f;
                for (int r = 0; r < MB; r++) acc += D1[r * NH + h];
                G[OFF_B1 + h] = acc;
            }
            __syncthreads();
            // Adam
            step++;
            const float c1 = 1.f - powf(a.beta1, (float)step), c2 = 1.f - powf(a.beta2, (float)step);
            for (int i = t; i < NPARAM; i += NT) {
                float g = G[i];
                M1[i] = a.beta1 * M1[i] + (1.f - a.beta1) * g;
                M2[i] = a.beta2 * M2[i] + (1.f - a.beta2) * g * g;
                float mh = M1[i] / c1, vh = M2[i] / c2;
                P[i] -= a.lr * mh / (sqrtf(vh) + a.eps);
            }
            __syncthreads();
        }
        if (t == 0) a.loss_out[ep] = s_loss;
        __syncthreads();
    }
    for (int i = t; i < NPARAM; i += NT) a.params[i] = P[i];
}

__global__ void k_mlp_predict(const float* __restrict__ X, int N, const float* __restrict__ params,
                              const float* __restrict__ norm, float* __restrict__ out) {
    __shared__ float P[NPARAM];
    for (int i = threadIdx.x; i < NPARAM; i += blockDim.x) P[i] = params[i];
    __syncthreads();
    int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= N) return;
    float x[NF];
#pragma unroll
    for (int f = 0; f < NF; f++) x[f] = (X[(size_t)r * NF + f] - norm[f]) / norm[NF + f];
    float h1[NH];
#pragma unroll 4
    for (int h = 0; h < NH; h++) {
        float acc = P[OFF_B1 + h];
#pragma unroll
        for (int f = 0; f < NF; f++) acc = __fmaf_rn(x[f], P[OFF_W1 + f * NH + h], acc);
        h1[h] = relu(acc);
    }
    float y = P[OFF_B3];
    for (int h = 0; h < NH; h++) {
        float acc = P[OFF_B2 + h];
#pragma unroll 8
        for (int k = 0; k < NH; k++) acc = __fmaf_rn(h1[k], P[OFF_W2 + k * NH + h], acc);
        y = __fmaf_rn(relu(acc), P[OFF_W3 + h], y);
    }
    // de-normalise the target: log(ms) = y * sd + mean
    out[r] = expf(y * norm[2 * NF + 1] + norm[2 * NF]);
}

// ---------------------------------------------------------------- model state

struct Model {
    bool ready = false;
    float* d_params = nullptr;   // device
    float* d_norm = nullptr;     // device: mean[NF], sd[NF], y_mean, y_sd
    std::vector<float> params, norm;
    int sms = 152;
};
static std::mutex g_mmu;
static Model g_model;

static int upload_model(Model& M) {
    if (!M.d_params) MPG_CUDA(dev_malloc((void**)&M.d_params, sizeof(float) * NPARAM));
    if (!M.d_norm) MPG_CUDA(dev_malloc((void**)&M.d_norm, sizeof(float) * (2 * NF + 2)));
    MPG_CUDA(cudaMemcpy(M.d_params, M.params.data(), sizeof(float) * NPARAM, cudaMemcpyHostToDevice));
    MPG_CUDA(cudaMemcpy(M.d_norm, M.norm.data(), sizeof(float) * (2 * NF + 2), cudaMemcpyHostToDevice));
    M.ready = true;
    return MPGEMM_OK;
}

// Predicted milliseconds for `count` raw feature vectors (synchronous).
static int predict(const float* feats, int count, float* out) {
    std::lock_guard<std::mutex> lk(g_mmu);
    if (!g_model.ready) return MPGEMM_EUNSUPPORTED;
    float *dX = nullptr, *dO = nullptr;
    MPG_CUDA(dev_malloc((void**)&dX, sizeof(float) * NF * (size_t)count));
    cudaError_t e = dev_malloc((void**)&dO, sizeof(float) * (size_t)count);
    if (e == cudaSuccess) e = cudaMemcpy(dX, feats, sizeof(float) * NF * (size_t)count, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
        k_mlp_predict<<<ceil_div(count, 128), 128>>>(dX, count, g_model.d_params, g_model.d_norm, dO);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpy(out, dO, sizeof(float) * (size_t)count, cudaMemcpyDeviceToHost);
    cudaFree(dX);
    cudaFree(dO);
    if (e != cudaSuccess) {
        set_last_cuda_error(e);
        return MPGEMM_ECUDA;
    }
    return MPGEMM_OK;
}

// Candidate configurations the model chooses among for one GEMM.
struct Cand {
    int algo, tile, depth;
};
static std::vector<Cand> candidates(int kind, int64_t m, int64_t l, int64_t n) {
    std::vector<Cand> c;
    c.push_back({MPGEMM_SIMPLE, 16, 0});
    const int tmax = kind == MPGEMM_KIND_DD ? 64 : kind == MPGEMM_KIND_QD ? 32 : 16;
    for (int t = 16; t <= tmax; t *= 2) c.push_back({MPGEMM_BLOCK, t, 0});
    for (int d = 1; d <= 4; d++) {
        if (strassen_extended(m, d) >> d < 16 || strassen_extended(l, d) >> d < 16 ||
            strassen_extended(n, d) >> d < 16)
            continue;
        for (int t = 16; t <= tmax; t *= 2) c.push_back({MPGEMM_STRASSEN, t, d});
    }
    return c;
}

bool cost_model_choice(int kind, int prec_bits, int64_t m, int64_t l, int64_t n, int sms, Choice* out,
                       float* pred_ms = nullptr) {
    {
        std::lock_guard<std::mutex> lk(g_mmu);
        if (!g_model.ready) return false;
    }
    std::vector<Cand> cs = candidates(kind, m, l, n);
    std::vector<float> F(cs.size() * NF), T(cs.size());
    for (size_t i = 0; i < cs.size(); i++)
        encode_features(kind, prec_bits, m, l, n, cs[i].algo, cs[i].tile, cs[i].depth, sms, &F[i * NF]);
    if (predict(F.data(), (int)cs.size(), T.data()) != MPGEMM_OK) return false;
    const size_t best = (size_t)(std::min_element(T.begin(), T.end()) - T.begin());
    // Among configurations predicted within 10 % of the best, the one with
    // the fewest launches: the model's relative error is largest on small,
    // launch-bound products, where Strassen's 3d + 1 launches decide.
    auto launches = [](const Cand& c) { return c.algo == MPGEMM_STRASSEN ? 3 * c.depth + 1 : 1; };
    size_t pick = best;
    for (size_t i = 0; i < cs.size(); i++) {
        if (T[i] > 1.10f * T[best]) continue;
        const int li = launches(cs[i]), lp = launches(cs[pick]);
        if (li < lp || (li == lp && T[i] < T[pick])) pick = i;
    }
    out->algo = cs[pick].algo;
    out->n_min = cs[pick].tile;
    out->depth = cs[pick].depth;
    if (pred_ms) *pred_ms = T[pick];
    return true;
}

// The configurations predicted within (1 + margin) of the best, fastest
// first, and the fastest of each algorithm family (simple, block, Strassen)
// predicted within (1 + 2 margin) or below cheap_ms (cheap to time), at most
// kmax; false without a model.
bool cost_model_shortlist(int kind, int prec_bits, int64_t m, int64_t l, int64_t n, int sms, double margin,
                          double cheap_ms, int kmax, std::vector<Choice>* out, std::vector<float>* pred_ms) {
    {
        std::lock_guard<std::mutex> lk(g_mmu);
        if (!g_model.ready) return false;
    }
    std::vector<Cand> cs = candidates(kind, m, l, n);
    std::vector<float> F(cs.size() * NF), T(cs.size());
    for (size_t i = 0; i < cs.size(); i++)
        encode_features(kind, prec_bits, m, l, n, cs[i].algo, cs[i].tile, cs[i].depth, sms, &F[i * NF]);
    if (predict(F.data(), (int)cs.size(), T.data()) != MPGEMM_OK) return false;
    std::vector<size_t> order(cs.size());
    for (size_t i = 0; i < cs.size(); i++) order[i] = i;
    std::sort(order.begin(), order.end(), [&](size_t a, size_t b) { return T[a] < T[b]; });
    out->clear();
    if (pred_ms) pred_ms->clear();
    bool family[3] = {false, false, false};
    for (size_t k = 0; k < order.size() && (int)out->size() < kmax; k++) {
        const size_t i = order[k];
        const bool near = k == 0 || T[i] <= (1.0 + margin) * T[order[0]];
        const bool family_best =
            !family[cs[i].algo] && (T[i] <= (1.0 + 2.0 * margin) * T[order[0]] || T[i] <= cheap_ms);
        if (!near && !family_best) continue;
        family[cs[i].algo] = true;
        out->push_back(Choice{cs[i].algo, cs[i].tile, cs[i].depth});
        if (pred_ms) pred_ms->push_back(T[i]);
    }
    return true;
}

// Predicted time (ms) of the model's best simple / block configuration
// (Strassen excluded: its bound is normwise); negative without a model.
double cost_model_block_ms(int kind, int prec_bits, int64_t m, int64_t l, int64_t n, int sms) {
    {
        std::lock_guard<std::mutex> lk(g_mmu);
        if (!g_model.ready) return -1.0;
    }
    std::vector<Cand> cs;
    for (const Cand& c : candidates(kind, m, l, n))
        if (c.algo != MPGEMM_STRASSEN) cs.push_back(c);
    std::vector<float> F(cs.size() * NF), T(cs.size());
    for (size_t i = 0; i < cs.size(); i++)
        encode_features(kind, prec_bits, m, l, n, cs[i].algo, cs[i].tile, cs[i].depth, sms, &F[i * NF]);
    if (predict(F.data(), (int)cs.size(), T.data()) != MPGEMM_OK) return -1.0;
    return (double)*std::min_element(T.begin(), T.end());
}

// Tile (16 or 32) the model prefers for a DD / QD block GEMM; 0 without a model.
int cost_model_tile(int kind, int prec_bits, int64_t m, int64_t l, int64_t n) {
    {
        std::lock_guard<std::mutex> lk(g_mmu);
        if (!g_model.ready) return 0;
    }
    float F[2 * NF], T[2];
    encode_features(kind, prec_bits, m, l, n, MPGEMM_BLOCK, 16, 0, g_model.sms, F);
    encode_features(kind, prec_bits, m, l, n, MPGEMM_BLOCK, 32, 0, g_model.sms, F + NF);
    if (predict(F, 2, T) != MPGEMM_OK) return 0;
    return T[0] < T[1] ? 16 : 32;
}

// ---------------------------------------------------------------- data collection

__global__ void k_fill_random(double* p, size_t count, unsigned long long seed, int mode, int planes) {
    size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    unsigned long long z = seed + i * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    if (mode == 0) {   // DD / QD planes: leading plane U[-1,1), lower planes tiny
        size_t per = count / planes;
        int q = (int)(i / per);
        double u = (double)(z >> 11) * (1.0 / 9007199254740992.0) * 2.0 - 1.0;
        p[i] = q == 0 ? u : ldexp(u, -54 * q);
    } else {           // multi-limb words (as raw bits): exponent 0, flags 0, limbs random, top limb normalised
        reinterpret_cast<unsigned long long*>(p)[i] = z;
    }
}

}  // namespace mpg

using namespace mpg;

extern "C" {

int mpgemm_cost_features(int kind, int prec_bits, int64_t m, int64_t l, int64_t n, int algo, int tile, int depth,
                         float* out) {
    if (!out) return MPGEMM_EINVAL;
    int sms = 152;
    {
        std::lock_guard<std::mutex> lk(g_mmu);
        sms = g_model.sms;
    }
    encode_features(kind, prec_bits, m, l, n, algo, tile, depth, sms, out);
    return MPGEMM_OK;
}

int mpgemm_cost_num_features(void) { return NF; }

int mpgemm_cost_choice(int kind, int prec_bits, int64_t m, int64_t l, int64_t n, void* stream, int* algo, int* n_min,
                       int* depth, float* pred_ms) {
    if (m <= 0 || l <= 0 || n <= 0 || !algo || !n_min || !depth) return MPGEMM_EINVAL;
    if (kind < MPGEMM_KIND_DD || kind > MPGEMM_KIND_MP) return MPGEMM_EINVAL;
    Choice c;
    float ms = 0.f;
    if (!cost_model_choice(kind, prec_bits, m, l, n, stream_sms((cudaStream_t)stream), &c, &ms))
        return MPGEMM_EUNSUPPORTED;   // no model installed
    *algo = c.algo;
    *n_min = c.n_min;
    *depth = c.depth;
    if (pred_ms) *pred_ms = ms;
    return MPGEMM_OK;
}

// Time `count` random configurations: shapes log-uniform in [16, max_dim],
// format uniform over {DD, QD, 256-bit multi-limb}, algorithm / tile /
// Strassen depth uniform over the valid candidates.  Features and median
// times (ms, 2 timed runs after a warm-up) go to host arrays.
int mpgemm_cost_collect(int count, unsigned long long seed, int max_dim, float* features, float* times_ms,
                        void* stream) {
    if (count <= 0 || max_dim < 16 || !features || !times_ms) return MPGEMM_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    int dev = 0, sms = 0;
    MPG_CUDA(cudaGetDevice(&dev));
    MPG_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    {
        std::lock_guard<std::mutex> lk(g_mmu);
        g_model.sms = sms;
    }
    const size_t maxe = (size_t)max_dim * max_dim;
    const size_t bytes = maxe * 4 * 34;   // largest element: 1024-bit multi-limb, 34 words
    void *A = nullptr, *B = nullptr, *C = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int rc = MPGEMM_OK;
    auto ck = [&](cudaError_t e) {   // first failure wins; everything is released below
        if (e != cudaSuccess && rc == MPGEMM_OK) {
            set_last_cuda_error(e);
            rc = MPGEMM_ECUDA;
        }
    };
    ck(dev_malloc((void**)&A, bytes));
    ck(dev_malloc((void**)&B, bytes));
    ck(dev_malloc((void**)&C, bytes));
    ck(cudaEventCreate(&e0));
    ck(cudaEventCreate(&e1));
    std::mt19937_64 rng(seed);
    std::uniform_real_distribution<double> U(std::log(16.0), std::log((double)max_dim));
    for (int i = 0; i < count && rc == MPGEMM_OK; i++) {
        int64_t m = (int64_t)std::lround(std::exp(U(rng))), l = (int64_t)std::lround(std::exp(U(rng))),
                n = (int64_t)std::lround(std::exp(U(rng)));
        int kind = (int)(rng() % 3);
        // multi-limb: 256 bits (the batched workload's width), 128 bits (the
        // width of the integer-pipe DD GEMM), 512 and 1024 bits
        static const int precs[10] = {128, 128, 128, 256, 256, 256, 256, 512, 512, 1024};
        int prec = kind == MPGEMM_KIND_MP ? precs[rng() % 10] : 0;
        if (rng() % 3 == 0) {   // a third of the shapes even enough for Strassen
            m &= ~7LL;
            l &= ~7LL;
            n &= ~7LL;
            m = std::max<int64_t>(m, 16);
            l = std::max<int64_t>(l, 16);
            n = std::max<int64_t>(n, 16);
        }
        std::vector<Cand> cs = candidates(kind, m, l, n);
        Cand c = cs[rng() % cs.size()];
        // operands
        int planes = kind == MPGEMM_KIND_DD ? 2 : kind == MPGEMM_KIND_QD ? 4 : 2 + prec / 32;
        size_t ea = (size_t)(m * l) * planes, eb = (size_t)(l * n) * planes;
        if (kind != MPGEMM_KIND_MP) {
            k_fill_random<<<ceil_div((int64_t)ea, 256), 256, 0, s>>>((double*)A, ea, seed + 2 * i, 0, planes);
            k_fill_random<<<ceil_div((int64_t)eb, 256), 256, 0, s>>>((double*)B, eb, seed + 2 * i + 1, 0, planes);
        } else {
            k_fill_random<<<ceil_div((int64_t)(ea / 2), 256), 256, 0, s>>>((double*)A, ea / 2, seed + 2 * i, 1, 1);
            k_fill_random<<<ceil_div((int64_t)(eb / 2), 256), 256, 0, s>>>((double*)B, eb / 2, seed + 2 * i + 1, 1, 1);
            // exponent plane 0, flags plane 0, top limb with its high bit set
            ck(cudaMemsetAsync(A, 0, sizeof(uint32_t) * 2 * (size_t)(m * l), s));
            ck(cudaMemsetAsync(B, 0, sizeof(uint32_t) * 2 * (size_t)(l * n), s));
            const size_t top = (size_t)(1 + prec / 32);   // plane of the top limb
            if (rc == MPGEMM_OK) rc = fill_u32((uint32_t*)A + top * (size_t)(m * l), (size_t)(m * l), 0x80000001u, s);
            if (rc == MPGEMM_OK) rc = fill_u32((uint32_t*)B + top * (size_t)(l * n), (size_t)(l * n), 0x80000001u, s);
        }
        ck(cudaGetLastError());
        if (rc != MPGEMM_OK) break;
        auto run = [&]() -> int {
            if (kind == MPGEMM_KIND_DD)
                return mpgemm_dd(m, l, n, (const double*)A, (const double*)B, (double*)C, c.algo, c.tile, c.depth, s);
            if (kind == MPGEMM_KIND_QD)
                return mpgemm_qd(m, l, n, (const double*)A, (const double*)B, (double*)C, c.algo, c.tile, c.depth, s);
            return mpgemm_mp(m, l, n, prec, (const uint32_t*)A, (const uint32_t*)B, (uint32_t*)C, c.algo, c.tile,
                             c.depth, s);
        };
        rc = run();
        float t[2] = {0.f, 0.f};
        for (int r = 0; r < 2 && rc == MPGEMM_OK; r++) {
            ck(cudaEventRecord(e0, s));
            if (rc == MPGEMM_OK) rc = run();
            ck(cudaEventRecord(e1, s));
            ck(cudaEventSynchronize(e1));
            ck(cudaEventElapsedTime(&t[r], e0, e1));
        }
        encode_features(kind, prec, m, l, n, c.algo, c.tile, c.depth, sms, features + (size_t)i * NF);
        times_ms[i] = std::min(t[0], t[1]);
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(A);
    cudaFree(B);
    cudaFree(C);
    if (rc == MPGEMM_OK) rc = mpgemm_stream_status(stream);   // a device-side failure of the timed GEMMs
    return rc;
}

// Train a fresh model on (features, times) and install it as the cost model.
int mpgemm_cost_train(const float* features, const float* times_ms, int count, int epochs, unsigned long long seed,
                      float* loss_per_epoch) {
    if (!features || !times_ms || count < MB || epochs <= 0) return MPGEMM_EINVAL;
    const int N = count / MB * MB;
    std::vector<float> mean(NF, 0.f), sd(NF, 0.f), X((size_t)N * NF), Y(N);
    double ym = 0, ys = 0;
    for (int i = 0; i < N; i++) {
        for (int f = 0; f < NF; f++) mean[f] += features[(size_t)i * NF + f] / N;
        double y = std::log(std::max(times_ms[i], 1e-4f));
        ym += y / N;
    }
    for (int i = 0; i < N; i++) {
        for (int f = 0; f < NF; f++) {
            float d = features[(size_t)i * NF + f] - mean[f];
            sd[f] += d * d / N;
        }
        double y = std::log(std::max(times_ms[i], 1e-4f)) - ym;
        ys += y * y / N;
    }
    for (int f = 0; f < NF; f++) sd[f] = sd[f] > 1e-12f ? std::sqrt(sd[f]) : 1.f;
    ys = ys > 1e-12 ? std::sqrt(ys) : 1.0;
    for (int i = 0; i < N; i++) {
        for (int f = 0; f < NF; f++) X[(size_t)i * NF + f] = (features[(size_t)i * NF + f] - mean[f]) / sd[f];
        Y[i] = (float)((std::log(std::max(times_ms[i], 1e-4f)) - ym) / ys);
    }
    std::mt19937_64 rng(seed);
    std::vector<float> params(NPARAM, 0.f);
    auto init = [&](int off, int fan_in, int cnt) {
        std::normal_distribution<float> G(0.f, std::sqrt(2.f / fan_in));
        for (int i = 0; i < cnt; i++) params[off + i] = G(rng);
    };
    init(OFF_W1, NF, NF * NH);
    init(OFF_W2, NH, NH * NH);
    init(OFF_W3, NH, NH);
    std::vector<int> perm((size_t)epochs * N);
    std::vector<int> base(N);
    for (int i = 0; i < N; i++) base[i] = i;
    for (int e = 0; e < epochs; e++) {
        std::shuffle(base.begin(), base.end(), rng);
        std::copy(base.begin(), base.end(), perm.begin() + (size_t)e * N);
    }
    float *dX = nullptr, *dY = nullptr, *dP = nullptr, *dL = nullptr;
    int* dPerm = nullptr;
    int rc = MPGEMM_OK;
    auto ck = [&](cudaError_t e) {
        if (e != cudaSuccess && rc == MPGEMM_OK) {
            set_last_cuda_error(e);
            rc = MPGEMM_ECUDA;
        }
    };
    ck(dev_malloc((void**)&dX, sizeof(float) * X.size()));
    ck(dev_malloc((void**)&dY, sizeof(float) * Y.size()));
    ck(dev_malloc((void**)&dP, sizeof(float) * NPARAM));
    ck(dev_malloc((void**)&dL, sizeof(float) * epochs));
    ck(dev_malloc((void**)&dPerm, sizeof(int) * perm.size()));
    if (rc == MPGEMM_OK) {
        ck(cudaMemcpy(dX, X.data(), sizeof(float) * X.size(), cudaMemcpyHostToDevice));
        ck(cudaMemcpy(dY, Y.data(), sizeof(float) * Y.size(), cudaMemcpyHostToDevice));
        ck(cudaMemcpy(dP, params.data(), sizeof(float) * NPARAM, cudaMemcpyHostToDevice));
        ck(cudaMemcpy(dPerm, perm.data(), sizeof(int) * perm.size(), cudaMemcpyHostToDevice));
    }
    const size_t smem = sizeof(float) * (4 * NPARAM + MB * NF + 3 * MB * NH + MB);
    if (rc == MPGEMM_OK) ck(cudaFuncSetAttribute(k_mlp_train, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    if (rc == MPGEMM_OK) {
        TrainArgs a{dX, dY, dPerm, N, epochs, 2e-3f, 0.9f, 0.999f, 1e-7f, dP, dL};
        k_mlp_train<<<1, NT, smem>>>(a);
        ck(cudaGetLastError());
        ck(cudaDeviceSynchronize());
    }
    if (rc == MPGEMM_OK) {
        ck(cudaMemcpy(params.data(), dP, sizeof(float) * NPARAM, cudaMemcpyDeviceToHost));
        if (loss_per_epoch) ck(cudaMemcpy(loss_per_epoch, dL, sizeof(float) * epochs, cudaMemcpyDeviceToHost));
    }
    cudaFree(dX);
    cudaFree(dY);
    cudaFree(dP);
    cudaFree(dL);
    cudaFree(dPerm);
    if (rc) return rc;
    std::lock_guard<std::mutex> lk(g_mmu);
    g_model.params = params;
    g_model.norm.assign(2 * NF + 2, 0.f);
    for (int f = 0; f < NF; f++) {
        g_model.norm[f] = mean[f];
        g_model.norm[NF + f] = sd[f];
    }
    g_model.norm[2 * NF] = (float)ym;
    g_model.norm[2 * NF + 1] = (float)ys;
    return upload_model(g_model);
}

int mpgemm_cost_predict(const float* features, int count, float* out_ms) {
    if (!features || !out_ms || count <= 0) return MPGEMM_EINVAL;
    return predict(features, count, out_ms);
}

int mpgemm_cost_clear(void) {
    std::lock_guard<std::mutex> lk(g_mmu);
    g_model.ready = false;
    return MPGEMM_OK;
}

// Binary model file: "MPGCOST1", NF, NH, norm[2 NF + 2], params[NPARAM].
int mpgemm_cost_save(const char* path) {
    std::lock_guard<std::mutex> lk(g_mmu);
    if (!g_model.ready || !path) return MPGEMM_EINVAL;
    FILE* f = std::fopen(path, "wb");
    if (!f) return MPGEMM_EINVAL;
    int hdr[2] = {NF, NH};
    bool ok = std::fwrite("MPGCOST1", 1, 8, f) == 8 && std::fwrite(hdr, sizeof hdr, 1, f) == 1 &&
              std::fwrite(g_model.norm.data(), sizeof(float), g_model.norm.size(), f) == g_model.norm.size() &&
              std::fwrite(g_model.params.data(), sizeof(float), NPARAM, f) == (size_t)NPARAM;
    std::fclose(f);
    return ok ? MPGEMM_OK : MPGEMM_EINVAL;
}

int mpgemm_cost_load(const char* path) {
    if (!path) return MPGEMM_EINVAL;
    FILE* f = std::fopen(path, "rb");
    if (!f) return MPGEMM_EINVAL;
    char magic[8];
    int hdr[2];
    std::vector<float> norm(2 * NF + 2), params(NPARAM);
    bool ok = std::fread(magic, 1, 8, f) == 8 && std::memcmp(magic, "MPGCOST1", 8) == 0 &&
              std::fread(hdr, sizeof hdr, 1, f) == 1 && hdr[0] == NF && hdr[1] == NH &&
              std::fread(norm.data(), sizeof(float), norm.size(), f) == norm.size() &&
              std::fread(params.data(), sizeof(float), NPARAM, f) == (size_t)NPARAM;
    std::fclose(f);
    if (!ok) return MPGEMM_EINVAL;
    std::lock_guard<std::mutex> lk(g_mmu);
    g_model.norm = norm;
    g_model.params = params;
    return upload_model(g_model);
}

}  // extern "C"
