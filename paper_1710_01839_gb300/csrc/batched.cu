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
#include <algorithm>
#include <cmath>
#include <new>
#include <vector>

#include "common.cuh"
#include "kernels.h"
#include "profile.h"
#include "tiles.cuh"

namespace mpg {

enum TileKind : int { T_DD16 = 0, T_DD32 = 1, T_QD16 = 2, T_QD32 = 3, T_MP256 = 4 };

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

__global__ void __launch_bounds__(256) k_batched(const DevDesc* __restrict__ descs, const Work* __restrict__ work,
                                                 int nwork, unsigned* counter, unsigned* status) {
    constexpr int SMD = ddqd_tile_doubles<DDFmt, 32, 16>() > ddqd_tile_doubles<QDFmt, 32, 8>()
                            ? ddqd_tile_doubles<DDFmt, 32, 16>()
                            : ddqd_tile_doubles<QDFmt, 32, 8>();
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
        if (d.tk == T_MP256) {
            View<const uint32_t> a = planes_view((const uint32_t*)d.A, d.m, d.l);
            View<const uint32_t> b = planes_view((const uint32_t*)d.B, d.l, d.n);
            View<uint32_t> c = planes_view((uint32_t*)d.C, d.m, d.n);
            mp_block_tile<8, 8>(d.m, d.l, d.n, a, b, c, 0, i0, j0, reinterpret_cast<uint32_t*>(sm), st);
        } else {
            View<const double> a = planes_view((const double*)d.A, d.m, d.l);
            View<const double> b = planes_view((const double*)d.B, d.l, d.n);
            View<double> c = planes_view((double*)d.C, d.m, d.n);
            switch (d.tk) {
                case T_DD16: ddqd_block_tile<DDFmt, 16, 1, 16>(d.m, d.l, d.n, a, b, c, 0, i0, j0, sm); break;
                case T_DD32: ddqd_block_tile<DDFmt, 32, 2, 16>(d.m, d.l, d.n, a, b, c, 0, i0, j0, sm); break;
                case T_QD16: ddqd_block_tile<QDFmt, 16, 1, 16>(d.m, d.l, d.n, a, b, c, 0, i0, j0, sm); break;
                default: ddqd_block_tile<QDFmt, 32, 2, 8>(d.m, d.l, d.n, a, b, c, 0, i0, j0, sm); break;
            }
        }
    }
    if (st) atomicOr(status, st);
}

// Relative cost of one multiply-accumulate, for ordering work items only
// (FP64 operations per MAC for DD / QD; the 256-bit multi-limb MAC measured
// against DD on this GPU).
static double mac_cost(int tk) {
    switch (tk) {
        case T_DD16: case T_DD32: return 9.4;
        case T_QD16: case T_QD32: return 76.0;
        default: return 40.0;
    }
}

}  // namespace mpg

struct mpgemm_plan_s {
    int count = 0, nwork = 0, grid = 0, device = 0;
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

static size_t desc_elem_bytes(const mpgemm_desc& d) {
    return d.kind == MPGEMM_KIND_DD ? 16 : d.kind == MPGEMM_KIND_QD ? 32 : 4 * (size_t)(2 + d.prec_bits / 32);
}

extern "C" {

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
    for (int i = 0; i < count; i++) {
        const mpgemm_desc& d = descs[i];
        if (d.m < 0 || d.l < 0 || d.n < 0 || d.m > 65535 * 64 || d.n > 65535 * 64) {
            delete P;
            return MPGEMM_EINVAL;
        }
        int tile = d.kind == MPGEMM_KIND_MP ? 16 : (d.tile == 16 || d.tile == 32 ? d.tile : (d.tile == 0 ? 0 : -1));
        if (tile == 0) {   // the cost model's choice when one is installed, else 32
            tile = cost_model_tile(d.kind, d.prec_bits, d.m, d.l, d.n);
            if (tile == 0) tile = 32;
        }
        if (tile < 0) {
            delete P;
            return MPGEMM_EINVAL;
        }
        int tk;
        if (int rc = desc_tile_kind(d, tile, &tk)) {
            delete P;
            return rc;
        }
        size_t eb = desc_elem_bytes(d);
        if ((d.m * d.l && !d.A) || (d.l * d.n && !d.B) || (d.m * d.n && !d.C)) {
            delete P;
            return MPGEMM_EINVAL;
        }
        (void)eb;
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
        rc = MPGEMM_ECUDA;
    };
    cudaError_t e;
    if ((e = cudaGetDevice(&P->device)) != cudaSuccess) fail(e);
    int sms = 0, occ = 0;
    if (!rc && (e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, P->device)) != cudaSuccess) fail(e);
    if (!rc && (e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_batched, 256, 0)) != cudaSuccess) fail(e);
    P->grid = std::max(1, sms * std::max(occ, 1));
    if (!rc && count && (e = cudaMalloc(&P->d_descs, sizeof(DevDesc) * count)) != cudaSuccess) fail(e);
    if (!rc && P->nwork && (e = cudaMalloc(&P->d_work, sizeof(Work) * P->nwork)) != cudaSuccess) fail(e);
    if (!rc && (e = cudaMalloc(&P->d_counter, sizeof(unsigned))) != cudaSuccess) fail(e);
    if (!rc && count && (e = cudaMemcpy(P->d_descs, dd.data(), sizeof(DevDesc) * count, cudaMemcpyHostToDevice)))
        fail(e);
    if (!rc && P->nwork && (e = cudaMemcpy(P->d_work, work.data(), sizeof(Work) * P->nwork, cudaMemcpyHostToDevice)))
        fail(e);
    if (!rc && (e = cudaStreamCreateWithFlags(&P->cap, cudaStreamNonBlocking)) != cudaSuccess) fail(e);
    if (rc) {
        cudaFree(P->d_descs);
        cudaFree(P->d_work);
        cudaFree(P->d_counter);
        if (P->cap) cudaStreamDestroy(P->cap);
        delete P;
        return rc;
    }
    *out = P;
    return MPGEMM_OK;
}

int mpgemm_batched_run(mpgemm_plan P, void* stream) {
    if (!P) return MPGEMM_EINVAL;
    if (P->nwork == 0) return MPGEMM_OK;
    cudaStream_t s = (cudaStream_t)stream;
    unsigned* status = device_status_ptr();
    if (!status) return MPGEMM_ECUDA;
    MPG_CUDA(cudaMemsetAsync(P->d_counter, 0, sizeof(unsigned), s));
    ProfScope ps(s);
    k_batched<<<P->grid, 256, 0, s>>>(P->d_descs, P->d_work, P->nwork, P->d_counter, status);
    return check_launch();
}

int mpgemm_batched_run_graph(mpgemm_plan P, void* stream) {
    if (!P) return MPGEMM_EINVAL;
    if (P->nwork == 0) return MPGEMM_OK;
    if (!P->exec) {
        unsigned* status = device_status_ptr();   // resolve before capture
        if (!status) return MPGEMM_ECUDA;
        MPG_CUDA(cudaStreamBeginCapture(P->cap, cudaStreamCaptureModeThreadLocal));
        cudaError_t e1 = cudaMemsetAsync(P->d_counter, 0, sizeof(unsigned), P->cap);
        k_batched<<<P->grid, 256, 0, P->cap>>>(P->d_descs, P->d_work, P->nwork, P->d_counter, status);
        cudaError_t e2 = cudaGetLastError();
        cudaGraph_t g = nullptr;
        cudaError_t e3 = cudaStreamEndCapture(P->cap, &g);
        if (e1 || e2 || e3) {
            if (g) cudaGraphDestroy(g);
            set_last_cuda_error(e1 ? e1 : e2 ? e2 : e3);
            return MPGEMM_ECUDA;
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
    if (P->exec) cudaGraphExecDestroy(P->exec);
    if (P->graph) cudaGraphDestroy(P->graph);
    if (P->cap) cudaStreamDestroy(P->cap);
    cudaFree(P->d_descs);
    cudaFree(P->d_work);
    cudaFree(P->d_counter);
    delete P;
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
        if (d.kind == MPGEMM_KIND_DD)
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
