// Level sums of the FP8-digit split-precision DD GEMM on the 5th-generation
// tensor cores (tcgen05, kind::f8f6f4, e4m3 x e4m3 -> f32 in tensor memory).
//
// A job is one 128 x 256 tile of one level: L_g = sum_{s=1}^{g-1} D_s^A
// (D_{g-s}^B)^T, the K dimension being the concatenation of the g - 1 slice
// pairs.  The f32 accumulator is exact only while every partial sum stays
// below 2^24, so a job runs as chunks of at most Q pairs (Q * 256 * lp <=
// 2^24); each chunk's sum is converted to int32 and the chunks of a job are
// added in registers-to-memory order by the same epilogue thread.
//
// Persistent, warp-specialised CTA (one per SM, 192 threads):
//   warp 0 (one lane)  TMA producer: 3-D tensor maps over the digit planes
//                      ([S][rows][lp] bytes), 128-byte swizzle, one A box
//                      (128 x 128 B) and one B box (256 x 128 B) per stage,
//                      completion counted on the stage's `full` mbarrier;
//   warp 1 (one lane)  MMA issuer: 4 x tcgen05.mma (K = 32) per stage into
//                      one of two 256-column TMEM accumulators, then
//                      tcgen05.commit to the stage's `empty` mbarrier, and
//                      after a chunk's last stage to the accumulator's
//                      `tmem_full` mbarrier;
//   warps 2-5          epilogue: tcgen05.ld of their 32-lane quarter,
//                      exact f32 -> int32, store (first chunk) or add (later
//                      chunks), then release the accumulator (`tmem_empty`).
// With two accumulators the epilogue of one chunk overlaps the MMAs of the
// next.  Jobs are ordered heaviest level first and dealt to CTAs in snake
// order (round k: CTA c takes job k G + c, or k G + G - 1 - c for odd k), so
// the per-CTA sums of pair counts differ by at most about one job.
//
// Every wait is bounded.  A role that gives up sets a shared abort flag and
// DEV_TIMEOUT in the status word; the other roles leave their loops when
// they see the flag.  Before the CTA exits the producer waits for its last
// TMA copy into each stage and the MMA thread waits for all its MMAs, so no
// asynchronous write is in flight when tensor memory is freed.
#include <cuda.h>

#include <cmath>
#include <cstdint>
#include <mutex>

#include "common.cuh"
#include "profile.h"
#include "tc_levels.h"
#include "tcgen05.cuh"

namespace mpg {

constexpr int TC_M = 128, TC_N = 256, TC_BK = 128, TC_STAGES = 4, TC_THREADS = 192;
constexpr int TC_A_BYTES = TC_M * TC_BK, TC_B_BYTES = TC_N * TC_BK;
constexpr int TC_STAGE_BYTES = TC_A_BYTES + TC_B_BYTES;          // 48 KB
constexpr int TC_SMEM = TC_STAGES * TC_STAGE_BYTES + 1024;      // + 1024-byte alignment slack
constexpr int TC_TMEM_COLS = 2 * TC_N;                          // two accumulators
constexpr uint32_t TC_IDESC = (1u << 4)                         // D: f32
                              | (0u << 7) | (0u << 10)          // A, B: e4m3
                              | ((uint32_t)(TC_N >> 3) << 17)   // N = 256
                              | ((uint32_t)(TC_M >> 4) << 24);  // M = 128
__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap* map, int x, int y, int z, uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
        "[%5];" ::"r"(dst),
        "l"((uint64_t)map), "r"(x), "r"(y), "r"(z), "r"(bar)
        : "memory");
}

__device__ __forceinline__ void tc_fail(volatile int* abort_flag, unsigned* status) {
    *abort_flag = 1;
    atomicOr(status, DEV_TIMEOUT);
}

struct TcJob {
    int g, row0, col0;
};

// Job order: the tiles are grouped into super-tiles of SR x SC tiles (bands
// of SR tile rows, each cut into SC tile columns; the last band and the last
// super-tile of a band may be smaller), super-tiles in row-major order, and
// within a super-tile the levels from g = S + 1 (S pairs) down to g = 2, the
// tiles of a level row-major.  All levels of a super-tile read the same S
// digit planes of its SR row blocks of A and SC column blocks of B, which the
// host sizes to stay in L2 while the super-tile's jobs run.
struct TcOrder {
    int S, tiles_m, tiles_n, SR, SC;
};

__host__ __device__ inline TcJob tc_job(int j, const TcOrder& o) {
    const int band_jobs = o.SR * o.tiles_n * o.S;   // every band but the last is full
    const int b = j / band_jobs;
    const int r = j - b * band_jobs;
    const int h = o.tiles_m - b * o.SR < o.SR ? o.tiles_m - b * o.SR : o.SR;
    const int st_jobs = h * o.SC * o.S;             // every super-tile of a band but the last is full
    const int c = r / st_jobs;
    const int q = r - c * st_jobs;
    const int w = o.tiles_n - c * o.SC < o.SC ? o.tiles_n - c * o.SC : o.SC;
    const int lvl = q / (h * w), t = q - lvl * (h * w);
    return TcJob{o.S + 1 - lvl, (b * o.SR + t / w) * TC_M, (c * o.SC + t % w) * TC_N};
}

// Index of this CTA's job in round k (snake order).
__device__ __forceinline__ int tc_job_index(int k, int G, int c) { return k * G + ((k & 1) ? (G - 1 - c) : c); }

__global__ void __launch_bounds__(TC_THREADS, 1)
    k_levels_tc(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, int m, int n,
                int ksteps, int S, int Q, TcOrder order, int tiles, int vec, int* __restrict__ Lv, unsigned* status) {
    extern __shared__ unsigned char dsm[];
    __shared__ __align__(8) uint64_t full[TC_STAGES], empty[TC_STAGES], tmem_full[2], tmem_empty[2], drain;
    __shared__ uint32_t tmem_base;
    __shared__ volatile int abort_flag;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    unsigned char* base = (unsigned char*)(((uintptr_t)dsm + 1023) & ~(uintptr_t)1023);
    const int J = tiles * S, G = gridDim.x, cta = blockIdx.x;
    const int rounds = (J + G - 1) / G;

    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(&tmem_base)),
                     "r"(TC_TMEM_COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        for (int s = 0; s < TC_STAGES; s++) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(su32(&full[s])));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(su32(&empty[s])));
        }
        for (int a = 0; a < 2; a++) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(su32(&tmem_full[a])));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(&tmem_empty[a])), "r"(128));
        }
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(su32(&drain)));
        abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;");
        asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)&tmA) : "memory");
        asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)&tmB) : "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = tmem_base;

    if (warp == 0) {
        // ------------------------------------------------------------ TMA producer
        if (lane == 0) {
            uint32_t it = 0;
            bool ok = true;
            for (int k = 0; k < rounds && ok; k++) {
                const int j = tc_job_index(k, G, cta);
                if (j >= J) continue;
                const TcJob jb = tc_job(j, order);
                for (int s = 1; s < jb.g && ok; s++) {
                    for (int kb = 0; kb < ksteps; kb++, it++) {
                        const int st = (int)(it % TC_STAGES);
                        if (!mbar_wait(su32(&empty[st]), ((it / TC_STAGES) & 1) ^ 1, &abort_flag)) {
                            ok = false;
                            break;
                        }
                        const uint32_t fb = su32(&full[st]);
                        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(fb),
                                     "r"(TC_STAGE_BYTES)
                                     : "memory");
                        const uint32_t sA = su32(base + st * TC_STAGE_BYTES);
                        tma_load_3d(sA, &tmA, kb * TC_BK, jb.row0, s - 1, fb);
                        tma_load_3d(sA + TC_A_BYTES, &tmB, kb * TC_BK, jb.col0, jb.g - s - 1, fb);
                    }
                }
            }
            if (!ok) tc_fail(&abort_flag, status);
            // the last copy issued into each stage has landed before the CTA may exit
            for (uint32_t i = it > (uint32_t)TC_STAGES ? it - TC_STAGES : 0; i < it; i++)
                if (!mbar_drain(su32(&full[i % TC_STAGES]), (i / TC_STAGES) & 1)) tc_fail(&abort_flag, status);
        }
        __syncwarp();
    } else if (warp == 1) {
        // ------------------------------------------------------------ MMA issuer
        if (lane == 0) {
            uint32_t it = 0, cc = 0;
            bool ok = true, issued = false;
            for (int k = 0; k < rounds && ok; k++) {
                const int j = tc_job_index(k, G, cta);
                if (j >= J) continue;
                const int pairs = tc_job(j, order).g - 1;
                for (int s0 = 1; s0 <= pairs && ok; s0 += Q, cc++) {
                    const int np = (pairs - s0 + 1) < Q ? (pairs - s0 + 1) : Q;
                    const uint32_t acc = cc & 1;
                    if (!mbar_wait(su32(&tmem_empty[acc]), ((cc >> 1) & 1) ^ 1, &abort_flag)) {
                        ok = false;
                        break;
                    }
                    asm volatile("tcgen05.fence::after_thread_sync;");
                    const uint32_t d = tmem + acc * TC_N;
                    const int nst = np * ksteps;
                    for (int q = 0; q < nst; q++, it++) {
                        const int st = (int)(it % TC_STAGES);
                        if (!mbar_wait(su32(&full[st]), (it / TC_STAGES) & 1, &abort_flag)) {
                            ok = false;
                            break;
                        }
                        asm volatile("tcgen05.fence::after_thread_sync;");
                        const uint32_t a0 = su32(base + st * TC_STAGE_BYTES), b0 = a0 + TC_A_BYTES;
#pragma unroll
                        for (int kk = 0; kk < TC_BK / 32; kk++) {
                            const uint64_t ad = smem_desc(a0 + 32 * kk), bd = smem_desc(b0 + 32 * kk);
                            const uint32_t accum = (q > 0 || kk > 0) ? 1u : 0u;
                            asm volatile(
                                "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                                " tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
                                "l"(ad), "l"(bd), "r"(TC_IDESC), "r"(accum));
                        }
                        issued = true;
                        // the stage may be refilled once these MMAs have read it
                        asm volatile(
                            "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                                su32(&empty[st]))
                            : "memory");
                    }
                    if (!ok) break;
                    // the chunk's sum is complete once every MMA issued so far has finished
                    asm volatile(
                        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                            su32(&tmem_full[acc]))
                        : "memory");
                }
            }
            if (!ok) tc_fail(&abort_flag, status);
            if (issued) {
                asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                                 su32(&drain))
                             : "memory");
                if (!mbar_drain(su32(&drain), 0)) tc_fail(&abort_flag, status);
            }
        }
        __syncwarp();
    } else {
        // ------------------------------------------------------------ epilogue
        const int quarter = warp & 3;   // tcgen05.ld reaches TMEM lanes 32 (warp % 4) .. + 31
        uint32_t cc = 0;
        bool ok = true;
        for (int k = 0; k < rounds && ok; k++) {
            const int j = tc_job_index(k, G, cta);
            if (j >= J) continue;
            const TcJob jb = tc_job(j, order);
            const int pairs = jb.g - 1;
            const int64_t r = (int64_t)jb.row0 + quarter * 32 + lane;
            int* out = Lv + (int64_t)(jb.g - 2) * m * n + r * n;
            for (int s0 = 1; s0 <= pairs; s0 += Q, cc++) {
                const uint32_t acc = cc & 1;
                const bool w = mbar_wait(su32(&tmem_full[acc]), (cc >> 1) & 1, &abort_flag);
                if (!__all_sync(0xffffffffu, w)) {
                    ok = false;
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;");
                const bool first = s0 == 1;
#pragma unroll 1
                for (int ch = 0; ch < TC_N / 32; ch++) {
                    uint32_t v[32];
                    const uint32_t ta = tmem + ((uint32_t)(quarter * 32) << 16) + acc * TC_N + (uint32_t)(ch * 32);
                    asm volatile(
                        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,"
                        "%14,%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
                        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
                          "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]),
                          "=r"(v[14]), "=r"(v[15]), "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]),
                          "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]), "=r"(v[24]), "=r"(v[25]),
                          "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
                        : "r"(ta));
                    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                    if (r < m) {
                        const int c0 = jb.col0 + ch * 32;
                        int x[32];
#pragma unroll
                        for (int i = 0; i < 32; i++) x[i] = __float2int_rn(__uint_as_float(v[i]));
                        if (vec && c0 + 32 <= n) {
                            int4* o = (int4*)(out + c0);
#pragma unroll
                            for (int i = 0; i < 8; i++) {
                                int4 t = make_int4(x[4 * i], x[4 * i + 1], x[4 * i + 2], x[4 * i + 3]);
                                if (!first) {
                                    const int4 p = o[i];
                                    t.x += p.x;
                                    t.y += p.y;
                                    t.z += p.z;
                                    t.w += p.w;
                                }
                                o[i] = t;
                            }
                        } else {
#pragma unroll
                            for (int i = 0; i < 32; i++)
                                if (c0 + i < n) out[c0 + i] = first ? x[i] : out[c0 + i] + x[i];
                        }
                    }
                }
                asm volatile("tcgen05.fence::before_thread_sync;");
                asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(su32(&tmem_empty[acc])) : "memory");
            }
        }
        if (!ok && lane == 0) tc_fail(&abort_flag, status);
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    if (warp == 1)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TC_TMEM_COLS));
}

// Self-test of the failure path: one warp waits, with the kernels' bounded
// wait, for an mbarrier phase that nothing completes.  The wait gives up
// after limit_ns, the kernel records DEV_TIMEOUT in the status word and
// returns normally, so the host sees MPGEMM_ETIMEOUT and the context stays
// usable.  Nothing is faulted, trapped or left running.
__global__ void k_wait_selftest(uint64_t limit_ns, unsigned* status) {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(su32(&bar)));
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    __syncwarp();
    const bool ok = mbar_wait(su32(&bar), 0, nullptr, limit_ns);   // no thread ever arrives
    if (!__all_sync(0xffffffffu, ok) && threadIdx.x == 0) atomicOr(status, DEV_TIMEOUT);
}

int wait_selftest(int limit_ms, cudaStream_t s) {
    if (limit_ms < 1 || limit_ms > 2000) return MPGEMM_EINVAL;
    unsigned* status = device_status_ptr();
    if (!status) return MPGEMM_ECUDA;
    k_wait_selftest<<<1, 32, 0, s>>>((uint64_t)limit_ms * 1000000ull, status);
    return check_launch();
}

// ---------------------------------------------------------------- host side

using EncodeTiledFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                   const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

// cuTensorMapEncodeTiled through the runtime's driver entry point (no link
// against the driver library).
static EncodeTiledFn encode_tiled() {
    static EncodeTiledFn fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (EncodeTiledFn)p;
    });
    return fn;
}

// [S][rows][lp] bytes, box = 128 bytes of K x box_rows rows x 1 plane,
// 128-byte swizzle; rows past the end read as zero.
static int digit_map(CUtensorMap* map, const void* D, int64_t rows, int64_t lp, int S, int box_rows) {
    EncodeTiledFn enc = encode_tiled();
    if (!enc) return MPGEMM_ECUDA;
    cuuint64_t dims[3] = {(cuuint64_t)lp, (cuuint64_t)rows, (cuuint64_t)S};
    cuuint64_t strides[2] = {(cuuint64_t)lp, (cuuint64_t)(rows * lp)};
    cuuint32_t box[3] = {(cuuint32_t)TC_BK, (cuuint32_t)box_rows, 1};
    cuuint32_t estr[3] = {1, 1, 1};
    CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_UINT8, 3, const_cast<void*>(D), dims, strides, box, estr,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? MPGEMM_OK : MPGEMM_EINVAL;
}

// Super-tile shape for the job order: SC column blocks (256 x lp x S digit
// bytes each) and SR row blocks (128 x lp x S) whose planes together take at
// most about three quarters of the 129 MB L2.
constexpr double TC_L2_BUDGET = 96.0 * 1024 * 1024;

static TcOrder tc_order(int64_t m, int64_t n, int64_t lp, int S) {
    TcOrder o;
    o.S = S;
    o.tiles_m = (int)ceil_div(m, TC_M);
    o.tiles_n = (int)ceil_div(n, TC_N);
    const double a_blk = (double)TC_M * (double)lp * S, b_blk = (double)TC_N * (double)lp * S;
    double sc = std::floor(TC_L2_BUDGET / 2 / b_blk);
    o.SC = (int)(sc < 1 ? 1 : sc > o.tiles_n ? o.tiles_n : sc);
    double sr = std::floor((TC_L2_BUDGET - o.SC * b_blk) / a_blk);
    o.SR = (int)(sr < 1 ? 1 : sr > o.tiles_m ? o.tiles_m : sr);
    return o;
}

int tc_levels(int64_t m, int64_t n, int64_t lp, int S, const void* DA, const void* DB, int* Lv, cudaStream_t s) {
    if (lp <= 0 || lp % TC_BK || S < 1) return MPGEMM_EINVAL;
    if (((uintptr_t)DA | (uintptr_t)DB) & 15) return MPGEMM_EINVAL;   // tensor-map base alignment
    if (m > 65535 || n > 65535) return MPGEMM_EUNSUPPORTED;   // keeps job counts and offsets in int
    const int Q = (int)((int64_t)(1 << 24) / (256 * lp));   // pairs per chunk: Q * 256 * lp <= 2^24
    if (Q < 1) return MPGEMM_EUNSUPPORTED;
    unsigned* status = device_status_ptr();
    if (!status) return MPGEMM_ECUDA;
    CUtensorMap mA, mB;
    int rc;
    if ((rc = digit_map(&mA, DA, m, lp, S, TC_M))) return rc;
    if ((rc = digit_map(&mB, DB, n, lp, S, TC_N))) return rc;
    // set on every call: the current context may be an SM partition's (partition.cu)
    MPG_CUDA(cudaFuncSetAttribute(k_levels_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, TC_SMEM));
    const int sms = stream_sms(s);   // one persistent CTA per SM of the stream's partition
    const TcOrder order = tc_order(m, n, lp, S);
    const int tiles = order.tiles_m * order.tiles_n;
    const int64_t jobs = (int64_t)tiles * S;
    const int grid = (int)(jobs < sms ? jobs : sms);
    const int vec = ((uintptr_t)Lv % 16 == 0) && (n % 4 == 0);
    {
        ProfScope ps(s);
        k_levels_tc<<<grid, TC_THREADS, TC_SMEM, s>>>(mA, mB, (int)m, (int)n, (int)(lp / TC_BK), S, Q, order,
                                                      tiles, vec, Lv, status);
    }
    return check_launch();
}

}  // namespace mpg

using namespace mpg;

extern "C" int mpgemm_split_job_order(int64_t m, int64_t n, int64_t l, int num_slices, int* jobs, int max_jobs) {
    if (m < 1 || n < 1 || l < 1 || num_slices < 1 || m > 65535 || n > 65535 || max_jobs < 0 || (max_jobs && !jobs))
        return MPGEMM_EINVAL;
    const int64_t lp = (l + TC_BK - 1) / TC_BK * TC_BK;
    const TcOrder o = tc_order(m, n, lp, num_slices);
    const int64_t J = (int64_t)o.tiles_m * o.tiles_n * num_slices;
    if (J > 0x7FFFFFFF) return MPGEMM_EUNSUPPORTED;
    for (int64_t j = 0; j < J && j < max_jobs; j++) {
        const TcJob jb = tc_job((int)j, o);
        jobs[3 * j] = jb.g;
        jobs[3 * j + 1] = jb.row0;
        jobs[3 * j + 2] = jb.col0;
    }
    return (int)J;
}
