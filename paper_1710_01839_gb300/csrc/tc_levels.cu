// Level sums of the FP8-digit split-precision DD GEMM on the 5th-generation
// tensor cores (tcgen05, kind::f8f6f4, e4m3 x e4m3 -> f32 in tensor memory).
//
// One CTA (128 threads) computes one 128 x 256 tile of C for one chunk of
// one level: L_g = sum_{s in chunk} D_s^A (D_{g-s}^B)^T, the K dimension being
// the concatenation of the chunk's slice pairs.  Operands are staged by
// cp.async into shared memory in the K-major, 128-byte-swizzled layout the
// tensor core reads through smem descriptors (4 stages of 128 bytes of K);
// one thread issues the MMAs and tcgen05.commit signals a per-stage mbarrier
// when a stage may be overwritten.  The f32 accumulator lives in tensor
// memory (256 columns); a chunk holds at most Q pairs with Q * 256 * lp <=
// 2^24, so every partial sum is an exact integer.  The epilogue reads the
// accumulator with tcgen05.ld and stores (single-chunk levels) or atomically
// adds (multi-chunk levels, into a zeroed buffer) the int32 level sums.
//
// Every wait is bounded; on a timeout the CTA records DEV_TIMEOUT in the
// status word, skips its epilogue and still frees its tensor memory.
#include <algorithm>
#include <cstdint>
#include <vector>

#include "common.cuh"
#include "profile.h"
#include "tc_levels.h"

namespace mpg {

constexpr int TC_M = 128, TC_N = 256, TC_BK = 128, TC_STAGES = 4, TC_THREADS = 128;
constexpr int TC_STAGE_BYTES = (TC_M + TC_N) * TC_BK;          // 48 KB
constexpr int TC_SMEM = TC_STAGES * TC_STAGE_BYTES + 1024;      // + alignment slack
constexpr uint32_t TC_IDESC = (1u << 4)                         // D: f32
                              | (0u << 7) | (0u << 10)          // A, B: e4m3
                              | ((uint32_t)(TC_N >> 3) << 17)   // N = 256
                              | ((uint32_t)(TC_M >> 4) << 24);  // M = 128
constexpr uint32_t TC_SPIN = 1u << 24;

__device__ __forceinline__ uint32_t su32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row groups
// 1024 bytes apart.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr) {
    return (uint64_t)((addr & 0x3FFFF) >> 4) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) |
           ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}

__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
    for (uint32_t i = 0; i < TC_SPIN; i++) {
        uint32_t done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(bar), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

// byte offset of 16-byte chunk c of row r inside a swizzled operand tile
__device__ __forceinline__ uint32_t sw128(int r, int c) {
    return (uint32_t)((r >> 3) * 1024 + (r & 7) * 128 + ((c ^ (r & 7)) << 4));
}

struct TcItem {
    int tile, g, s0, s1;   // tile index, level, pairs s in [s0, s1)
};

__global__ void __launch_bounds__(TC_THREADS, 1)
    k_levels_tc(int64_t m, int64_t n, int64_t lp, const unsigned char* __restrict__ DA,
                const unsigned char* __restrict__ DB, int* __restrict__ Lv, const TcItem* __restrict__ items,
                const unsigned char* __restrict__ multi, unsigned tiles_n, unsigned* status) {
    extern __shared__ unsigned char dsm[];
    __shared__ __align__(8) uint64_t mbar[TC_STAGES];
    __shared__ uint32_t tmem_base;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    unsigned char* base = (unsigned char*)(((uintptr_t)dsm + 1023) & ~(uintptr_t)1023);
    const TcItem it = items[blockIdx.x];
    const int64_t row0 = (int64_t)(it.tile / tiles_n) * TC_M, col0 = (int64_t)(it.tile % tiles_n) * TC_N;
    const int ksteps = (int)(lp / TC_BK);
    const int total = (it.s1 - it.s0) * ksteps;
    const int64_t planeA = m * lp, planeB = n * lp;

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(&tmem_base)),
                     "r"(TC_N));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        for (int s = 0; s < TC_STAGES; s++) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(su32(&mbar[s])));
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = tmem_base;

    // iteration q: pair s = s0 + q / ksteps, K block kb = (q % ksteps) * 128, into stage q % STAGES
    auto load = [&](int q) {
        const int s = it.s0 + q / ksteps;
        const int64_t kb = (int64_t)(q % ksteps) * TC_BK;
        const unsigned char* Ab = DA + (int64_t)(s - 1) * planeA + kb;
        const unsigned char* Bb = DB + (int64_t)(it.g - s - 1) * planeB + kb;
        unsigned char* sA = base + (q % TC_STAGES) * TC_STAGE_BYTES;
        unsigned char* sB = sA + TC_M * TC_BK;
#pragma unroll
        for (int v = 0; v < (TC_M * 8) / TC_THREADS; v++) {
            int c = tid + v * TC_THREADS, r = c >> 3, ch = c & 7;
            int64_t gr = row0 + r;
            bool ok = gr < m;
            const void* src = ok ? (const void*)(Ab + gr * lp + ch * 16) : (const void*)DA;
            asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(su32(sA + sw128(r, ch))), "l"(src),
                         "r"(ok ? 16 : 0));
        }
#pragma unroll
        for (int v = 0; v < (TC_N * 8) / TC_THREADS; v++) {
            int c = tid + v * TC_THREADS, r = c >> 3, ch = c & 7;
            int64_t gc = col0 + r;
            bool ok = gc < n;
            const void* src = ok ? (const void*)(Bb + gc * lp + ch * 16) : (const void*)DB;
            asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(su32(sB + sw128(r, ch))), "l"(src),
                         "r"(ok ? 16 : 0));
        }
    };

    bool ok = true;
#pragma unroll 1
    for (int q = 0; q < TC_STAGES - 1; q++) {
        if (q < total) load(q);
        asm volatile("cp.async.commit_group;");
    }
#pragma unroll 1
    for (int q = 0; q < total; q++) {
        const int st = q % TC_STAGES;
        asm volatile("cp.async.wait_group %0;" ::"n"(TC_STAGES - 2) : "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        ok = __syncthreads_and(ok);   // also makes a timeout seen by any thread a uniform exit
        if (!ok) break;
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;");
            const uint32_t a0 = su32(base + st * TC_STAGE_BYTES), b0 = a0 + TC_M * TC_BK;
#pragma unroll
            for (int j = 0; j < TC_BK / 32; j++) {
                const uint64_t ad = smem_desc(a0 + 32 * j), bd = smem_desc(b0 + 32 * j);
                const uint32_t acc = (q > 0 || j > 0) ? 1u : 0u;
                asm volatile(
                    "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                    " tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
                    "l"(ad), "l"(bd), "r"(TC_IDESC), "r"(acc));
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                             su32(&mbar[st]))
                         : "memory");
        }
        // refill the stage used by iteration q - 1 once its MMAs have read it
        const int nx = q + TC_STAGES - 1;
        if (nx < total) {
            if (q >= 1) {
                const int pq = q - 1;
                if (!mbar_wait(su32(&mbar[pq % TC_STAGES]), (uint32_t)((pq / TC_STAGES) & 1))) ok = false;
            }
            if (ok) load(nx);
        }
        asm volatile("cp.async.commit_group;");
    }
    asm volatile("cp.async.wait_group 0;" ::: "memory");
    // the last commit covers every MMA issued before it
    if (ok && total > 0) {
        const int lq = total - 1;
        if (!mbar_wait(su32(&mbar[lq % TC_STAGES]), (uint32_t)((lq / TC_STAGES) & 1))) ok = false;
    }
    // a CTA that timed out must not read or free tensor memory another thread's MMAs may still write
    ok = __syncthreads_and(ok);
    asm volatile("tcgen05.fence::after_thread_sync;");
    if (ok && total > 0) {
        int* out = Lv + (int64_t)(it.g - 2) * m * n;
        const bool atomic = multi[it.g] != 0;
        const int64_t r = row0 + warp * 32 + lane;
#pragma unroll 1
        for (int ch = 0; ch < TC_N / 32; ch++) {
            uint32_t v[32];
            const uint32_t ta = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(ch * 32);
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
                "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
                : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
                  "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]),
                  "=r"(v[15]), "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]),
                  "=r"(v[22]), "=r"(v[23]), "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]),
                  "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
                : "r"(ta));
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            if (r < m) {
                const int64_t c0 = col0 + ch * 32;
#pragma unroll
                for (int i = 0; i < 32; i++) {
                    if (c0 + i < n) {
                        const int x = __float2int_rn(__uint_as_float(v[i]));
                        if (atomic) atomicAdd(out + r * n + c0 + i, x);
                        else out[r * n + c0 + i] = x;
                    }
                }
            }
        }
    } else if (!ok && tid == 0) {
        atomicOr(status, DEV_TIMEOUT);
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TC_N));
}

int tc_levels(int64_t m, int64_t n, int64_t lp, int S, const void* DA, const void* DB, int* Lv, cudaStream_t s) {
    if (lp % TC_BK) return MPGEMM_EINVAL;
    unsigned* status = device_status_ptr();
    if (!status) return MPGEMM_ECUDA;
    const int Q = (int)((int64_t)(1 << 24) / (256 * lp));   // pairs per chunk: Q * 256 * lp <= 2^24
    if (Q < 1) return MPGEMM_EUNSUPPORTED;
    const unsigned tm = ceil_div(m, TC_M), tn = ceil_div(n, TC_N);
    std::vector<TcItem> items;
    std::vector<unsigned char> multi(S + 2, 0);
    // heaviest work first: levels with the most pairs (chunks of up to Q pairs)
    for (int g = S + 1; g >= 2; g--) {
        const int pairs = g - 1;
        if (pairs > Q) multi[g] = 1;
        for (int s0 = 1; s0 <= pairs; s0 += Q) {
            const int s1 = s0 + Q <= pairs + 1 ? s0 + Q : pairs + 1;
            for (unsigned t = 0; t < tm * tn; t++) items.push_back(TcItem{(int)t, g, s0, s1});
        }
    }
    // stable heaviest-first order: sort chunks by their pair count
    std::stable_sort(items.begin(), items.end(),
                     [](const TcItem& a, const TcItem& b) { return (a.s1 - a.s0) > (b.s1 - b.s0); });
    bool any_multi = false;
    for (int g = 2; g <= S + 1; g++) any_multi |= multi[g] != 0;
    // the item table and the per-level flags travel in one stream-ordered allocation
    const size_t ib = sizeof(TcItem) * items.size(), mb = multi.size();
    void* dev = nullptr;
    bool owned = false;
    cudaError_t ae = cudaMallocAsync(&dev, ib + mb + 16, s);
    if (ae != cudaSuccess) {
        set_last_cuda_error(ae);
        return MPGEMM_ENOMEM;
    }
    owned = true;
    int rc;
    TcItem* d_items = (TcItem*)dev;
    unsigned char* d_multi = (unsigned char*)dev + ((ib + 15) & ~(size_t)15);
    MPG_CUDA(cudaMemcpyAsync(d_items, items.data(), ib, cudaMemcpyHostToDevice, s));
    MPG_CUDA(cudaMemcpyAsync(d_multi, multi.data(), mb, cudaMemcpyHostToDevice, s));
    if (any_multi) MPG_CUDA(cudaMemsetAsync(Lv, 0, sizeof(int) * (size_t)S * (size_t)(m * n), s));
    static bool attr_set[64];
    int devno = 0;
    MPG_CUDA(cudaGetDevice(&devno));
    if (devno >= 0 && devno < 64 && !attr_set[devno]) {
        MPG_CUDA(cudaFuncSetAttribute(k_levels_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, TC_SMEM));
        attr_set[devno] = true;
    }
    {
        ProfScope ps(s);
        k_levels_tc<<<(unsigned)items.size(), TC_THREADS, TC_SMEM, s>>>(m, n, lp, (const unsigned char*)DA,
                                                                       (const unsigned char*)DB, Lv, d_items, d_multi,
                                                                       tn, status);
    }
    rc = check_launch();
    if (owned) MPG_CUDA(cudaFreeAsync(dev, s));
    return rc;
}

}  // namespace mpg
