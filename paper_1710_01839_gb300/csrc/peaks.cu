// Peak-rate microbenchmarks: the denominators of the library's rooflines,
// measured on the GPU the library runs on instead of taken from data sheets.
//
//   MPGEMM_PEAK_TC_E4M3  tcgen05.mma.cta_group::1.kind::f8f6f4, M 128, N 256,
//                        K 32, e4m3 x e4m3 -> f32 in tensor memory, operands
//                        resident in shared memory (no loads in the loop),
//                        one CTA per SM, one thread issuing back to back;
//                        the split-precision level kernel's instruction;
//   MPGEMM_PEAK_MMA_S8   mma.sync.m16n8k32 s8 x s8 -> s32 on register
//                        operands, 8 independent accumulators per warp (the
//                        int8 split-precision level kernel's instruction);
//   MPGEMM_PEAK_DFMA     FP64 fused multiply-add, 16 independent chains per
//                        thread (the DD / QD kernels' pipe);
//   MPGEMM_PEAK_IMAD     32-bit integer multiply-add (mad.lo.u32), 8
//                        independent chains per thread (the multi-limb
//                        kernels' limb products);
//   MPGEMM_PEAK_DADD / _DMUL  the same with FP64 adds / multiplies: the FP64
//                        pipe's rate is the fastest of the three loops.
//
// Each launch covers every SM of the stream's partition.  The caller times
// it (events on the same stream) and divides the operation count that
// mpgemm_peak_run reports by the time.  The tcgen05 kernel's only wait (for
// its own MMAs to finish before tensor memory is freed) is bounded.
#include <cstdint>

#include "common.cuh"
#include "tcgen05.cuh"

namespace mpg {

constexpr int PK_M = 128, PK_N = 256, PK_KB = 128;                 // K bytes staged (4 MMAs of K = 32)
constexpr int PK_A_BYTES = PK_M * PK_KB, PK_B_BYTES = PK_N * PK_KB;   // 16 KB + 32 KB
constexpr int PK_SMEM = PK_A_BYTES + PK_B_BYTES + 1024 + 100 * 1024;   // + alignment; 149 KB: 1 CTA per SM
constexpr uint32_t PK_IDESC = (1u << 4)                               // D: f32
                              | (0u << 7) | (0u << 10)                // A, B: e4m3
                              | ((uint32_t)(PK_N >> 3) << 17)         // N = 256
                              | ((uint32_t)(PK_M >> 4) << 24);        // M = 128
constexpr int PK_TMEM_COLS = PK_N;

// Written only when a loop's result equals an improbable value: keeps the
// compiler from removing the loops.
static __device__ unsigned long long g_peak_sink[4];

__global__ void __launch_bounds__(128, 1) k_peak_tc_e4m3(int64_t rounds, unsigned* status) {
    extern __shared__ unsigned char dsm[];
    __shared__ __align__(8) uint64_t done;
    __shared__ uint32_t tmem_base;
    unsigned char* base = (unsigned char*)(((uintptr_t)dsm + 1023) & ~(uintptr_t)1023);
    const int tid = threadIdx.x, warp = tid >> 5;
    // e4m3 codes of digits in [-16, 16]: 16, -15, 8, -4, 1, -8, 5, -1
    const unsigned char tab[8] = {0x58, 0xD7, 0x50, 0xC8, 0x38, 0xD0, 0x4A, 0xB8};
    for (int i = tid; i < PK_A_BYTES + PK_B_BYTES; i += blockDim.x)
        base[i] = tab[((uint32_t)i * 2654435761u >> 13) & 7];
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");   // generic-proxy writes -> tensor core reads
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(&tmem_base)),
                     "r"(PK_TMEM_COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(su32(&done)));
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = tmem_base;
    if (tid == 0) {
        const uint32_t a0 = su32(base), b0 = a0 + PK_A_BYTES;
        for (int64_t r = 0; r < rounds; r++) {
#pragma unroll
            for (int kk = 0; kk < PK_KB / 32; kk++) {
                const uint64_t ad = smem_desc(a0 + 32 * kk), bd = smem_desc(b0 + 32 * kk);
                const uint32_t accum = (r > 0 || kk > 0) ? 1u : 0u;
                asm volatile(
                    "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                    " tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
                    "l"(ad), "l"(bd), "r"(PK_IDESC), "r"(accum));
            }
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(su32(&done))
                     : "memory");
        // every MMA has finished before tensor memory is freed; a second
        // bounded wait covers MMAs still running after the first gave up
        if (!mbar_wait(su32(&done), 0, nullptr)) {
            atomicOr(status, DEV_TIMEOUT);
            (void)mbar_wait(su32(&done), 0, nullptr);
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(PK_TMEM_COLS));
}

__global__ void __launch_bounds__(256) k_peak_mma_s8(int64_t iters) {
    unsigned a[4], b[2];
    const unsigned t = threadIdx.x * 0x9E3779B9u + blockIdx.x;
#pragma unroll
    for (int i = 0; i < 4; i++) a[i] = t * (2 * i + 1);
    b[0] = t ^ 0x5A5A5A5Au;
    b[1] = t * 7u;
    int c[8][4] = {};
    for (int64_t it = 0; it < iters; it++) {
#pragma unroll
        for (int j = 0; j < 8; j++)
            asm volatile(
                "mma.sync.aligned.m16n8k32.row.col.s32.s8.s8.s32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
                "{%0,%1,%2,%3};\n"
                : "+r"(c[j][0]), "+r"(c[j][1]), "+r"(c[j][2]), "+r"(c[j][3])
                : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
    }
    int s = 0;
#pragma unroll
    for (int j = 0; j < 8; j++) s += c[j][0] ^ c[j][1] ^ c[j][2] ^ c[j][3];
    if (s == 0x7F3A5C11) g_peak_sink[0] = (unsigned)s;
}

// FP64 loops: 16 independent dependent chains per thread (a chain cannot be
// hoisted out of the loop; 16 of them per thread and every SM full keep the
// pipe fed).  OP 0: DFMA, 1: DADD, 2: DMUL.
template <int OP>
__global__ void __launch_bounds__(256) k_peak_fp64(int64_t iters, double b, double c) {
    double x[16];
#pragma unroll
    for (int j = 0; j < 16; j++) x[j] = 1.0 + 1e-3 * (threadIdx.x + 37 * j);
    for (int64_t it = 0; it < iters; it++) {
#pragma unroll
        for (int j = 0; j < 16; j++) {
            if constexpr (OP == 0) x[j] = fma(x[j], b, c);
            else if constexpr (OP == 1) x[j] = __dadd_rn(x[j], c);
            else x[j] = __dmul_rn(x[j], b);
        }
    }
    double s = 0;
#pragma unroll
    for (int j = 0; j < 16; j++) s += x[j];
    if (s == 1234.5) g_peak_sink[1] = __double_as_longlong(s);
}

__global__ void __launch_bounds__(256) k_peak_imad(int64_t iters, uint32_t b, uint32_t c) {
    uint32_t x[8];
#pragma unroll
    for (int j = 0; j < 8; j++) x[j] = threadIdx.x * 2654435761u + (uint32_t)j;
    for (int64_t it = 0; it < iters; it++) {
#pragma unroll
        for (int j = 0; j < 8; j++) asm volatile("mad.lo.u32 %0, %0, %1, %2;" : "+r"(x[j]) : "r"(b), "r"(c));
    }
    uint32_t s = 0;
#pragma unroll
    for (int j = 0; j < 8; j++) s ^= x[j];
    if (s == 0x2468ACE1u) g_peak_sink[2] = s;
}

}  // namespace mpg

using namespace mpg;

extern "C" int mpgemm_peak_run(int kind, int64_t iters, double* ops, void* stream) {
    if (iters < 1 || iters > (int64_t(1) << 32) || !ops) return MPGEMM_EINVAL;
    if (kind < MPGEMM_PEAK_TC_E4M3 || kind > MPGEMM_PEAK_DMUL) return MPGEMM_EINVAL;
    // keeps one tcgen05 launch well inside its bounded wait
    if (kind == MPGEMM_PEAK_TC_E4M3 && iters > (int64_t(1) << 22)) return MPGEMM_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    PartitionScope pscope(s);
    unsigned* status = device_status_ptr();
    if (!status) return MPGEMM_ECUDA;
    const int sms = stream_sms(s);
    switch (kind) {
        case MPGEMM_PEAK_TC_E4M3: {
            MPG_CUDA(cudaFuncSetAttribute(k_peak_tc_e4m3, cudaFuncAttributeMaxDynamicSharedMemorySize, PK_SMEM));
            k_peak_tc_e4m3<<<sms, 128, PK_SMEM, s>>>(iters, status);
            *ops = 2.0 * PK_M * PK_N * 32 * (PK_KB / 32) * (double)iters * sms;
            break;
        }
        // the others: every SM filled to its resident-CTA limit, so each SM
        // holds the same number of CTAs and none waits for a second wave
        case MPGEMM_PEAK_MMA_S8: {
            int occ = 0;
            MPG_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_peak_mma_s8, 256, 0));
            if (occ < 1) return MPGEMM_ECUDA;
            k_peak_mma_s8<<<occ * sms, 256, 0, s>>>(iters);
            *ops = 2.0 * 16 * 8 * 32 * 8 * (double)iters * ((double)occ * sms * 256 / 32);
            break;
        }
        case MPGEMM_PEAK_DFMA:
        case MPGEMM_PEAK_DADD:
        case MPGEMM_PEAK_DMUL: {
            int occ = 0;
            auto kern = kind == MPGEMM_PEAK_DFMA ? k_peak_fp64<0> : kind == MPGEMM_PEAK_DADD ? k_peak_fp64<1>
                                                                                            : k_peak_fp64<2>;
            MPG_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, 256, 0));
            if (occ < 1) return MPGEMM_ECUDA;
            kern<<<occ * sms, 256, 0, s>>>(iters, 0.999999, 1e-7);
            *ops = 16.0 * (double)iters * (double)occ * sms * 256;
            break;
        }
        case MPGEMM_PEAK_IMAD: {
            int occ = 0;
            MPG_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_peak_imad, 256, 0));
            if (occ < 1) return MPGEMM_ECUDA;
            k_peak_imad<<<occ * sms, 256, 0, s>>>(iters, 2654435761u, 12345u);
            *ops = 8.0 * (double)iters * (double)occ * sms * 256;
            break;
        }
        default: return MPGEMM_EINVAL;
    }
    return check_launch();
}
