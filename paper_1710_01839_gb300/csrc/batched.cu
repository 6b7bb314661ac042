// Batched GEMMs of uneven sizes and mixed precisions in ONE persistent launch.
//
// A plan turns the descriptors into a device table of work items (one per
// CTA tile of C of one GEMM), sorted by estimated cost, heaviest first
// (longest-processing-time order).  The persistent kernel runs one CTA per
// resident slot; each CTA takes the next item from a global atomic counter
// and computes that tile with the same block-tile code as the single-GEMM
// kernels (DD / QD tiles of 16 or 32, 256-bit multi-limb tiles of 16).  No
// CTA ever waits for another: the only shared state is the counter.  The
// launch (counter reset + kernel) can be captured once into a CUDA graph and
// replayed.
//
// A DD or QD descriptor with engine = 1 runs on the integer pipe: the plan
// owns 128-bit (DD) or 256-bit (QD) multi-limb copies of its A, B and C;
// before the persistent launch one conversion pass per format rounds every
// such A and B into them, the persistent kernel computes the multi-limb
// tiles, and one pass per format rounds C back to doubles (the definitions
// of mpgemm_dd_via_mp / mpgemm_qd_via_mp).
#include <algorithm>
#include <cmath>
#include <new>
#include <vector>

#include "common.cuh"
#include "kernels.h"
#include "mp_convert.cuh"
#include "profile.h"
#include "tiles.cuh"

namespace mpg {

// T_MP128 and T_MP256C: the integer pipe's images of DD / QD operands (similar magnitudes:
// the add's alignment shortcut); T_MP256: the caller's 256-bit operands.
enum TileKind : int { T_DD16 = 0, T_DD32 = 1, T_QD16 = 2, T_QD32 = 3, T_MP256 = 4, T_MP128 = 5, T_MP256C = 6 };

struct DevDesc {
    int tk;
    int tile;
    int64_t m, l, n;
    const void* A;
    const void* B;
    void* C;
};

struct Work {
    int desc, tm, tn, pad;
};

// MP_ONLY: the instantiation for plans whose tiles are all multi-limb (its
// registers and shared memory are those of the multi-limb tiles alone, so
// more CTAs fit per SM); a DD / QD tile reaching it is flagged and skipped.
template <bool MP_ONLY>
__global__ void __launch_bounds__(256) k_batched(const DevDesc* __restrict__ descs, const Work* __restrict__ work,
                                                 int nwork, unsigned* counter, unsigned* status) {
    constexpr int SMD_DDQD = ddqd_tile_doubles<DDFmt, 32, 16>() > ddqd_tile_doubles<QDFmt, 32, 8>()
                                 ? ddqd_tile_doubles<DDFmt, 32, 16>()
                                 : ddqd_tile_doubles<QDFmt, 32, 8>();
    constexpr int SMD = MP_ONLY ? (mp_tile_words<8, 8>() + 1) / 2 : SMD_DDQD;
    static_assert(SMD * 8 >= mp_tile_words<8, 8>() * 4, "the 256-bit tile's staging fits too");
    __shared__ __align__(16) double sm[SMD];   // the largest tile's staging
    __shared__ int s_item;
    unsigned st = 0u;
    for (;;) {
        if (threadIdx.x == 0) s_item = (int)atomicAdd(counter, 1u);
        __syncthreads();
        const int it = s_item;
        __syncthreads();
        if (it >= nwork) break;
        const Work w = work[it];
        const DevDesc d = descs[w.desc];
        const int64_t i0 = (int64_t)w.tm * d.tile, j0 = (int64_t)w.tn * d.tile;
        if (d.tk == T_MP256 || d.tk == T_MP128 || d.tk == T_MP256C) {
            View<const uint32_t> a = planes_view((const uint32_t*)d.A, d.m, d.l);
            View<const uint32_t> b = planes_view((const uint32_t*)d.B, d.l, d.n);
            View<uint32_t> c = planes_view((uint32_t*)d.C, d.m, d.n);
            if (d.tk == T_MP256)
                mp_block_tile<8, 8>(d.m, d.l, d.n, a, b, c, 0, i0, j0, reinterpret_cast<uint32_t*>(sm), st);
            else if (d.tk == T_MP256C)
                mp_block_tile<8, 8, true>(d.m, d.l, d.n, a, b, c, 0, i0, j0, reinterpret_cast<uint32_t*>(sm), st);
            else
                mp_block_tile<4, 8, true>(d.m, d.l, d.n, a, b, c, 0, i0, j0, reinterpret_cast<uint32_t*>(sm), st);
        } else if constexpr (!MP_ONLY) {
            View<const double> a = planes_view((const double*)d.A, d.m, d.l);
            View<const double> b = planes_view((const double*)d.B, d.l, d.n);
            View<double> c = planes_view((double*)d.C, d.m, d.n);
            switch (d.tk) {
                case T_DD16: ddqd_block_tile<DDFmt, 16, 1, 16>(d.m, d.l, d.n, a, b, c, 0, i0, j0, sm); break;
                case T_DD32: ddqd_block_tile<DDFmt, 32, 2, 16>(d.m, d.l, d.n, a, b, c, 0, i0, j0, sm); break;
                case T_QD16: ddqd_block_tile<QDFmt, 16, 1, 16>(d.m, d.l, d.n, a, b, c, 0, i0, j0, sm); break;
                default: ddqd_block_tile<QDFmt, 32, 2, 8>(d.m, d.l, d.n, a, b, c, 0, i0, j0, sm); break;
            }
        } else {
            st |= DEV_BAD_DESC;
        }
    }
    if (st) atomicOr(status, st);
}

// Relative cost of one multiply-accumulate, for ordering work items only:
// time per MAC of each tile kind on GB300 in units where a 128-bit
// multi-limb MAC is 8.3 (DD 5.1 and QD 51.25 FP64 operations at 81 - 88 % of
// the FP64 pipe; the 128- and 256-bit multi-limb MACs issue 232 and 377
// instructions at about 43 % of the issue rate).
static double mac_cost(int tk) {
    switch (tk) {
        case T_DD16: case T_DD32: return 6.4;
        case T_QD16: case T_QD32: return 63.5;
        case T_MP128: return 8.3;
        default: return 13.5;
    }
}

// One conversion job of the integer-pipe descriptors: `count` elements
// between T-term double planes and (2 + W)-word multi-limb planes.
struct ConvJob {
    const double* x;   // to multi-limb: source; from: unused
    double* xo;        // from multi-limb: destination
    uint32_t* y;       // multi-limb planes
    int64_t count;
    int64_t first;     // prefix sum of the counts before this job
};

// Element i of the concatenated jobs: its job by binary search on `first`.
__device__ __forceinline__ int conv_job_of(const ConvJob* jobs, int njobs, int64_t i) {
    int lo = 0, hi = njobs - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (jobs[mid].first <= i) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

template <int W, int T>
__global__ void k_batched_to_mp(const ConvJob* __restrict__ jobs, int njobs, int64_t total, unsigned* status) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= total) return;
    const ConvJob j = jobs[conv_job_of(jobs, njobs, i)];
    const int64_t e = i - j.first, cnt = j.count;
    unsigned st = 0u;
    MPV<W> c;
    terms_to_mp<W, T>(j.x + e, cnt, c, st);
    j.y[e] = (uint32_t)c.e;
    j.y[cnt + e] = c.f;
#pragma unroll
    for (int q = 0; q < W; q++) j.y[(2 + q) * cnt + e] = c.m[q];
    if (st) atomicOr(status, st);
}

template <int W, int T>
__global__ void k_batched_from_mp(const ConvJob* __restrict__ jobs, int njobs, int64_t total, unsigned* status) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= total) return;
    const ConvJob j = jobs[conv_job_of(jobs, njobs, i)];
    const int64_t e = i - j.first, cnt = j.count;
    unsigned st = 0u;
    MPV<W> r;
    r.e = (int)j.y[e];
    r.f = j.y[cnt + e];
#pragma unroll
    for (int q = 0; q < W; q++) r.m[q] = j.y[(2 + q) * cnt + e];
    mp_to_terms<W, T>(r, j.xo + e, cnt, st);
    if (st) atomicOr(status, st);
}

// A conversion pass: its device job table and total element count.
struct ConvPass {
    ConvJob* d_jobs = nullptr;
    int njobs = 0;
    int64_t total = 0;
};

}  // namespace mpg

struct mpgemm_plan_s {
    int count = 0, nwork = 0, grid = 0, device = 0;
    bool mp_only = false;   // every tile multi-limb: the k_batched<true> instantiation
    // conversion passes of the integer-pipe descriptors: [0] DD in, [1] QD
    // in, [2] DD out, [3] QD out; the multi-limb copies live in d_limbs
    mpg::ConvPass conv[4];
    uint32_t* d_limbs = nullptr;
    mpg::DevDesc* d_descs = nullptr;
    mpg::Work* d_work = nullptr;
    unsigned* d_counter = nullptr;
    cudaStream_t cap = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    std::vector<mpgemm_desc> descs;
    std::vector<int> tiles;
};

namespace mpg {
int cost_model_tile(int kind, int prec_bits, int64_t m, int64_t l, int64_t n);
}

using namespace mpg;

static int desc_tile_kind(const mpgemm_desc& d, int tile, int* tk) {
    if (d.kind == MPGEMM_KIND_DD) *tk = tile == 16 ? T_DD16 : T_DD32;
    else if (d.kind == MPGEMM_KIND_QD) *tk = tile == 16 ? T_QD16 : T_QD32;
    else if (d.kind == MPGEMM_KIND_MP && d.prec_bits == 256) *tk = T_MP256;
    else return MPGEMM_EUNSUPPORTED;
    return MPGEMM_OK;
}

extern "C" {

static void plan_free(mpgemm_plan P) {
    if (P->exec) cudaGraphExecDestroy(P->exec);
    if (P->graph) cudaGraphDestroy(P->graph);
    if (P->cap) cudaStreamDestroy(P->cap);
    cudaFree(P->d_descs);
    cudaFree(P->d_work);
    cudaFree(P->d_counter);
    cudaFree(P->d_limbs);
    for (auto& c : P->conv) cudaFree(c.d_jobs);
    delete P;
}

int mpgemm_batched_plan(const mpgemm_desc* descs, int count, mpgemm_plan* out) {
    if (!out || count < 0 || (count > 0 && !descs)) return MPGEMM_EINVAL;
    *out = nullptr;
    mpgemm_plan P = new (std::nothrow) mpgemm_plan_s;
    if (!P) return MPGEMM_ENOMEM;
    P->count = count;
    P->descs.assign(descs, descs + count);
    std::vector<DevDesc> dd(count);
    struct Item {
        Work w;
        double cost;
    };
    std::vector<Item> items;
    std::vector<int64_t> limb_off(count, -1);   // word offset of an integer-pipe descriptor's copies
    int64_t limb_words = 0;
    for (int i = 0; i < count; i++) {
        const mpgemm_desc& d = descs[i];
        if (d.m < 0 || d.l < 0 || d.n < 0 || d.m > 65535 * 64 || d.n > 65535 * 64 || d.l > (1LL << 31) ||
            d.engine < 0 || d.engine > 1 ||
            (d.engine == 1 && d.kind == MPGEMM_KIND_MP)) {
            delete P;
            return MPGEMM_EINVAL;
        }
        int tile = d.kind == MPGEMM_KIND_MP || d.engine == 1
                       ? 16
                       : (d.tile == 16 || d.tile == 32 ? d.tile : (d.tile == 0 ? 0 : -1));
        if (tile == 0) {   // the cost model's choice when one is installed, else 32
            tile = cost_model_tile(d.kind, d.prec_bits, d.m, d.l, d.n);
            if (tile == 0) tile = 32;
        }
        if (tile < 0) {
            delete P;
            return MPGEMM_EINVAL;
        }
        int tk;
        if (d.engine == 1) {
            tk = d.kind == MPGEMM_KIND_DD ? T_MP128 : T_MP256C;
        } else if (int rc = desc_tile_kind(d, tile, &tk)) {
            delete P;
            return rc;
        }
        if ((d.m > 0 && d.l > 0 && !d.A) || (d.l > 0 && d.n > 0 && !d.B) || (d.m > 0 && d.n > 0 && !d.C)) {
            delete P;
            return MPGEMM_EINVAL;
        }
        if (d.engine == 1) {
            const int64_t words = 2 + (d.kind == MPGEMM_KIND_DD ? 4 : 8);
            limb_off[i] = limb_words;
            limb_words += words * (d.m * d.l + d.l * d.n + d.m * d.n);
        }
        P->tiles.push_back(tile);
        dd[i] = DevDesc{tk, tile, d.m, d.l, d.n, d.A, d.B, d.C};
        int64_t tm = (d.m + tile - 1) / tile, tn = (d.n + tile - 1) / tile;
        double cost = (double)tile * tile * (double)(d.l + 8) * mac_cost(tk);
        for (int64_t a = 0; a < tm; a++)
            for (int64_t b = 0; b < tn; b++) items.push_back(Item{Work{i, (int)a, (int)b, 0}, cost});
    }
    std::stable_sort(items.begin(), items.end(), [](const Item& x, const Item& y) { return x.cost > y.cost; });
    std::vector<Work> work(items.size());
    for (size_t i = 0; i < items.size(); i++) work[i] = items[i].w;
    P->nwork = (int)work.size();
    int rc = MPGEMM_OK;
    auto fail = [&](cudaError_t e) {
        set_last_cuda_error(e);
        rc = e == cudaErrorMemoryAllocation ? MPGEMM_ENOMEM : MPGEMM_ECUDA;
    };
    cudaError_t e;
    if (limb_words && (e = dev_malloc((void**)&P->d_limbs, sizeof(uint32_t) * (size_t)limb_words)) != cudaSuccess) fail(e);
    // point the integer-pipe descriptors at their copies; conversion jobs
    std::vector<ConvJob> jobs[4];
    for (int i = 0; i < count && !rc; i++) {
        if (limb_off[i] < 0) continue;
        const mpgemm_desc& d = descs[i];
        const bool is_dd = d.kind == MPGEMM_KIND_DD;
        const int64_t words = 2 + (is_dd ? 4 : 8);
        uint32_t* Am = P->d_limbs + limb_off[i];
        uint32_t* Bm = Am + words * d.m * d.l;
        uint32_t* Cm = Bm + words * d.l * d.n;
        dd[i].A = Am;
        dd[i].B = Bm;
        dd[i].C = Cm;
        const int in = is_dd ? 0 : 1, outp = is_dd ? 2 : 3;
        if (d.m > 0 && d.l > 0) jobs[in].push_back(ConvJob{(const double*)d.A, nullptr, Am, d.m * d.l, 0});
        if (d.l > 0 && d.n > 0) jobs[in].push_back(ConvJob{(const double*)d.B, nullptr, Bm, d.l * d.n, 0});
        if (d.m > 0 && d.n > 0) jobs[outp].push_back(ConvJob{nullptr, (double*)d.C, Cm, d.m * d.n, 0});
    }
    for (int k = 0; k < 4 && !rc; k++) {
        int64_t first = 0;
        for (auto& j : jobs[k]) {
            j.first = first;
            first += j.count;
        }
        P->conv[k].njobs = (int)jobs[k].size();
        P->conv[k].total = first;
        if (jobs[k].empty()) continue;
        if ((e = dev_malloc((void**)&P->conv[k].d_jobs, sizeof(ConvJob) * jobs[k].size())) != cudaSuccess) fail(e);
        else if ((e = cudaMemcpy(P->conv[k].d_jobs, jobs[k].data(), sizeof(ConvJob) * jobs[k].size(),
                                 cudaMemcpyHostToDevice)) != cudaSuccess)
            fail(e);
    }
    if (!rc && (e = cudaGetDevice(&P->device)) != cudaSuccess) fail(e);
    int sms = 0, occ = 0;
    if (!rc && (e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, P->device)) != cudaSuccess) fail(e);
    P->mp_only = count > 0;
    for (int i = 0; i < count; i++) P->mp_only &= dd[i].tk == T_MP128 || dd[i].tk == T_MP256 || dd[i].tk == T_MP256C;
    if (!rc && (e = P->mp_only ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_batched<true>, 256, 0)
                               : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_batched<false>, 256, 0)) !=
                   cudaSuccess)
        fail(e);
    P->grid = std::max(1, sms * std::max(occ, 1));
    if (!rc && count && (e = dev_malloc((void**)&P->d_descs, sizeof(DevDesc) * count)) != cudaSuccess) fail(e);
    if (!rc && P->nwork && (e = dev_malloc((void**)&P->d_work, sizeof(Work) * P->nwork)) != cudaSuccess) fail(e);
    if (!rc && (e = dev_malloc((void**)&P->d_counter, sizeof(unsigned))) != cudaSuccess) fail(e);
    if (!rc && count && (e = cudaMemcpy(P->d_descs, dd.data(), sizeof(DevDesc) * count, cudaMemcpyHostToDevice)))
        fail(e);
    if (!rc && P->nwork && (e = cudaMemcpy(P->d_work, work.data(), sizeof(Work) * P->nwork, cudaMemcpyHostToDevice)))
        fail(e);
    if (!rc && (e = cudaStreamCreateWithFlags(&P->cap, cudaStreamNonBlocking)) != cudaSuccess) fail(e);
    if (rc) {
        plan_free(P);
        return rc;
    }
    *out = P;
    return MPGEMM_OK;
}

// Conversion pass k of a plan (0 / 1: DD / QD operands in, 2 / 3: DD / QD
// products out).
static int launch_conv(mpgemm_plan P, int k, cudaStream_t s, unsigned* status) {
    const ConvPass& c = P->conv[k];
    if (c.total == 0) return MPGEMM_OK;
    const unsigned grid = ceil_div(c.total, 128);
    switch (k) {
        case 0: k_batched_to_mp<4, 2><<<grid, 128, 0, s>>>(c.d_jobs, c.njobs, c.total, status); break;
        case 1: k_batched_to_mp<8, 4><<<grid, 128, 0, s>>>(c.d_jobs, c.njobs, c.total, status); break;
        case 2: k_batched_from_mp<4, 2><<<grid, 128, 0, s>>>(c.d_jobs, c.njobs, c.total, status); break;
        default: k_batched_from_mp<8, 4><<<grid, 128, 0, s>>>(c.d_jobs, c.njobs, c.total, status); break;
    }
    return check_launch();
}

// The plan's launches on stream s: counter reset, operand conversions, the
// persistent kernel (bracketed for mpgemm_profile when `prof`), product
// conversions.
static int plan_launches(mpgemm_plan P, cudaStream_t s, unsigned* status, bool prof) {
    MPG_CUDA(cudaMemsetAsync(P->d_counter, 0, sizeof(unsigned), s));
    for (int k = 0; k < 2; k++)
        if (int rc = launch_conv(P, k, s, status)) return rc;
    auto launch = [&]() {
        if (P->mp_only) k_batched<true><<<P->grid, 256, 0, s>>>(P->d_descs, P->d_work, P->nwork, P->d_counter, status);
        else k_batched<false><<<P->grid, 256, 0, s>>>(P->d_descs, P->d_work, P->nwork, P->d_counter, status);
    };
    if (prof) {
        ProfScope ps(s);
        launch();
    } else {
        launch();
    }
    if (int rc = check_launch()) return rc;
    for (int k = 2; k < 4; k++)
        if (int rc = launch_conv(P, k, s, status)) return rc;
    return MPGEMM_OK;
}

int mpgemm_batched_run(mpgemm_plan P, void* stream) {
    if (!P) return MPGEMM_EINVAL;
    if (P->nwork == 0) return MPGEMM_OK;
    unsigned* status = device_status_ptr();
    if (!status) return MPGEMM_ECUDA;
    return plan_launches(P, (cudaStream_t)stream, status, true);
}

int mpgemm_batched_run_graph(mpgemm_plan P, void* stream) {
    if (!P) return MPGEMM_EINVAL;
    if (P->nwork == 0) return MPGEMM_OK;
    if (!P->exec) {
        unsigned* status = device_status_ptr();   // resolve before capture
        if (!status) return MPGEMM_ECUDA;
        MPG_CUDA(cudaStreamBeginCapture(P->cap, cudaStreamCaptureModeThreadLocal));
        int rc = plan_launches(P, P->cap, status, false);
        cudaGraph_t g = nullptr;
        cudaError_t e3 = cudaStreamEndCapture(P->cap, &g);
        if (rc || e3) {
            if (g) cudaGraphDestroy(g);
            if (e3) set_last_cuda_error(e3);
            return rc ? rc : MPGEMM_ECUDA;
        }
        cudaError_t e4 = cudaGraphInstantiate(&P->exec, g, 0);
        if (e4) {
            cudaGraphDestroy(g);
            set_last_cuda_error(e4);
            return MPGEMM_ECUDA;
        }
        P->graph = g;
    }
    MPG_CUDA(cudaGraphLaunch(P->exec, (cudaStream_t)stream));
    return MPGEMM_OK;
}

int mpgemm_batched_destroy(mpgemm_plan P) {
    if (!P) return MPGEMM_OK;
    plan_free(P);
    return MPGEMM_OK;
}

int mpgemm_batched_info(mpgemm_plan P, int* work_items, int* grid, int* tiles, int tiles_len) {
    if (!P) return MPGEMM_EINVAL;
    if (work_items) *work_items = P->nwork;
    if (grid) *grid = P->grid;
    if (tiles)
        for (int i = 0; i < tiles_len && i < (int)P->tiles.size(); i++) tiles[i] = P->tiles[i];
    return MPGEMM_OK;
}

// One launch per GEMM (the baseline the persistent launch is compared with).
int mpgemm_batched_sequential(const mpgemm_desc* descs, int count, void* stream) {
    if (count < 0 || (count > 0 && !descs)) return MPGEMM_EINVAL;
    for (int i = 0; i < count; i++) {
        const mpgemm_desc& d = descs[i];
        int tile = d.tile == 16 || d.tile == 32 ? d.tile : 32;
        int rc;
        if (d.engine == 1 && d.kind == MPGEMM_KIND_DD)
            rc = mpgemm_dd_via_mp(d.m, d.l, d.n, (const double*)d.A, (const double*)d.B, (double*)d.C, 128,
                                  MPGEMM_BLOCK, 16, 0, stream);
        else if (d.engine == 1 && d.kind == MPGEMM_KIND_QD)
            rc = mpgemm_qd_via_mp(d.m, d.l, d.n, (const double*)d.A, (const double*)d.B, (double*)d.C, 256,
                                  MPGEMM_BLOCK, 16, 0, stream);
        else if (d.kind == MPGEMM_KIND_DD)
            rc = mpgemm_dd(d.m, d.l, d.n, (const double*)d.A, (const double*)d.B, (double*)d.C, MPGEMM_BLOCK, tile, 0,
                           stream);
        else if (d.kind == MPGEMM_KIND_QD)
            rc = mpgemm_qd(d.m, d.l, d.n, (const double*)d.A, (const double*)d.B, (double*)d.C, MPGEMM_BLOCK, tile, 0,
                           stream);
        else
            rc = mpgemm_mp(d.m, d.l, d.n, d.prec_bits, (const uint32_t*)d.A, (const uint32_t*)d.B, (uint32_t*)d.C,
                           MPGEMM_BLOCK, 16, 0, stream);
        if (rc) return rc;
    }
    return MPGEMM_OK;
}

}  // extern "C"
