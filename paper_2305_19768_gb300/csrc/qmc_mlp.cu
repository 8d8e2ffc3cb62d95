// Tensor-core kernels of the learned lattice-size / amplitude model
// (north-star production form "learned part"): a BF16 GEMM on the 5th-
// generation tensor cores (tcgen05.mma, accumulator in tensor memory, FP32
// accumulation) plus the elementwise kernels of an MLP's forward and
// backward passes and its Adam update.
//
// gemm: C[M][N] (fp32) = A[M][K] . B[N][K]^T with A, B bf16 and K-major
// (row-major [rows][K]). One CTA of 128 threads computes a 128 x N tile
// (N <= 256, multiple of 16; M, K multiples of 128 and 16): K is staged in
// chunks of 64 through shared memory in the canonical no-swizzle K-major
// layout (8 x 16-byte core matrices), one elected thread issues four
// tcgen05.mma (K = 16 each) per chunk, tcgen05.commit signals an mbarrier,
// and the 4 warps read the 128 x N accumulator back with tcgen05.ld.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "qmc_internal.h"

#define QMC_E_INVAL_LOCAL (-1)
#define QMC_E_CUDA_LOCAL (-3)

namespace {

constexpr int kGemmThreads = 128;
constexpr int kChunkK = 64;                       // K elements staged per round
constexpr int kTileM = 128;
constexpr int kMaxN = 256;
constexpr int kAChunkBytes = kTileM * kChunkK * 2;  // 16 KB
constexpr int kBChunkBytes = kMaxN * kChunkK * 2;   // 32 KB
// Dynamic shared memory reserved per CTA: the operand chunks plus headroom, so
// that every address the descriptors can describe stays inside the allocation.
constexpr int kGemmSmem = 200 * 1024;
constexpr unsigned kWaitLimit = 1u << 26;

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

// Shared-memory matrix descriptor (tcgen05): start address, leading byte
// offset (K-direction core-matrix stride), stride byte offset (M/N-direction
// core-matrix stride), version 1, no swizzle.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = 0;
    d |= (uint64_t)((addr & 0x3FFFF) >> 4);
    d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}

// Instruction descriptor, kind::f16: D = F32, A = B = BF16, both K-major.
__host__ __device__ constexpr uint32_t instr_desc_bf16(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t phase) {
    for (unsigned it = 0; it < kWaitLimit; ++it) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}\n"
            : "=r"(done)
            : "r"(mbar), "r"(phase)
            : "memory");
        if (done) return true;
        if (it > 64) __nanosleep(64);
    }
    return false;
}

__global__ void __launch_bounds__(kGemmThreads, 1)
qmc_gemm_bf16_tc(const __nv_bfloat16 *__restrict__ A, const __nv_bfloat16 *__restrict__ B, float *__restrict__ C,
                 int M, int N, int K, int ldc, unsigned *err) {
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ __align__(8) uint64_t mbar;
    __shared__ uint32_t tmem_base;
    unsigned char *sA = smem;
    unsigned char *sB = smem + kAChunkBytes;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int m0 = blockIdx.x * kTileM;

    if (warp == 0) {
        const uint32_t dst = smem_u32(&tmem_base);
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(dst), "r"(kMaxN));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::);
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar)));
        asm volatile("fence.mbarrier_init.release.cluster;" ::);
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::);
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::);
    const uint32_t tmem = tmem_base;
    const uint32_t mb = smem_u32(&mbar);
    const uint32_t idesc = instr_desc_bf16(kTileM, N);
    const int ngroups = N >> 3;
    bool ok = true;
    uint32_t phase = 0;

    for (int k0 = 0; k0 < K; k0 += kChunkK) {
        const int kc = min(kChunkK, K - k0);   // multiple of 16
        const int cgroups = kc >> 3;
        // stage A[m0 .. m0+127][k0 .. k0+kc) : core matrix (g, c) at (c * 16 + g) * 128 bytes
        for (int idx = tid; idx < kTileM * cgroups; idx += kGemmThreads) {
            const int row = idx / cgroups, c = idx % cgroups;
            const uint4 v = *reinterpret_cast<const uint4 *>(A + (size_t)(m0 + row) * K + k0 + c * 8);
            *reinterpret_cast<uint4 *>(sA + ((c * 16 + (row >> 3)) * 128 + (row & 7) * 16)) = v;
        }
        // stage B[0 .. N)[k0 .. k0+kc): core matrix (g, c) at (c * N/8 + g) * 128 bytes
        for (int idx = tid; idx < N * cgroups; idx += kGemmThreads) {
            const int row = idx / cgroups, c = idx % cgroups;
            const uint4 v = *reinterpret_cast<const uint4 *>(B + (size_t)row * K + k0 + c * 8);
            *reinterpret_cast<uint4 *>(sB + ((c * ngroups + (row >> 3)) * 128 + (row & 7) * 16)) = v;
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::);
            for (int ks = 0; ks < kc / 16; ++ks) {
                const uint64_t da = smem_desc(smem_u32(sA) + ks * 2 * 16 * 128, 16 * 128, 128);
                const uint64_t db = smem_desc(smem_u32(sB) + ks * 2 * ngroups * 128, ngroups * 128, 128);
                const uint32_t acc = (k0 > 0 || ks > 0) ? 1u : 0u;
                asm volatile(
                    "{\n\t.reg .pred p;\n\t"
                    "setp.ne.b32 p, %4, 0;\n\t"
                    "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem),
                    "l"(da), "l"(db), "r"(idesc), "r"(acc));
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mb)
                         : "memory");
        }
        // the MMAs must finish reading this chunk before it is overwritten
        if (!mbar_wait(mb, phase)) ok = false;
        phase ^= 1u;
        ok = __syncthreads_and(ok);
        if (!ok) break;
    }
    asm volatile("tcgen05.fence::after_thread_sync;" ::);
    if (ok) {
        // warp w owns TMEM lanes 32w..32w+31 = rows m0 + 32w + lane
        const int row = m0 + warp * 32 + lane;
        for (int c0 = 0; c0 < N; c0 += 16) {
            uint32_t r[16];
            const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0;
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, "
                "%13, %14, %15}, [%16];"
                : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                  "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
                  "=r"(r[15])
                : "r"(taddr));
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            if (row < M) {
                float *dst = C + (size_t)row * ldc + c0;
#pragma unroll
                for (int q = 0; q < 16; ++q) dst[q] = __uint_as_float(r[q]);
            }
        }
    } else if (tid == 0) {
        atomicAdd(err, 1u);
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::);
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kMaxN));
}

}  // namespace

// C[M][N] = A[M][K] B[N][K]^T, device pointers; M % 128 == 0, K % 16 == 0,
// N % 16 == 0 and 16 <= N <= 256; rows/cols contiguous (ldc = N).
extern "C" int qmc_k_gemm_bf16(const void *A, const void *B, float *C, int M, int N, int K, unsigned *err_dev,
                               void *stream) {
    if (M <= 0 || M % 128 || K <= 0 || K % 16 || N < 16 || N > 256 || N % 16) return -2;
    static bool attr_set = false;
    if (!attr_set) {
        if (cudaFuncSetAttribute(qmc_gemm_bf16_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, kGemmSmem) !=
            cudaSuccess)
            return -1;
        attr_set = true;
    }
    qmc_gemm_bf16_tc<<<M / 128, kGemmThreads, kGemmSmem, (cudaStream_t)stream>>>(
        (const __nv_bfloat16 *)A, (const __nv_bfloat16 *)B, C, M, N, K, N, err_dev);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

// Host-buffer wrapper (tests and small callers): copies in, runs, copies out.
extern "C" int qmc_gemm_bf16(const uint16_t *A, const uint16_t *B, float *C, int M, int N, int K) {
    if (!A || !B || !C) return QMC_E_INVAL_LOCAL;
    if (M <= 0 || M % 128 || K <= 0 || K % 16 || N < 16 || N > 256 || N % 16) return QMC_E_INVAL_LOCAL;
    void *dA = nullptr, *dB = nullptr;
    float *dC = nullptr;
    unsigned *derr = nullptr;
    int rc = 0;
    if (cudaMalloc(&dA, (size_t)M * K * 2) || cudaMalloc(&dB, (size_t)N * K * 2) ||
        cudaMalloc(&dC, (size_t)M * N * 4) || cudaMalloc(&derr, 4)) {
        rc = QMC_E_CUDA_LOCAL;
    } else {
        cudaMemcpy(dA, A, (size_t)M * K * 2, cudaMemcpyHostToDevice);
        cudaMemcpy(dB, B, (size_t)N * K * 2, cudaMemcpyHostToDevice);
        cudaMemset(derr, 0, 4);
        if (qmc_k_gemm_bf16(dA, dB, dC, M, N, K, derr, nullptr)) rc = QMC_E_CUDA_LOCAL;
        unsigned herr = 0;
        if (cudaMemcpy(C, dC, (size_t)M * N * 4, cudaMemcpyDeviceToHost) != cudaSuccess) rc = QMC_E_CUDA_LOCAL;
        if (cudaMemcpy(&herr, derr, 4, cudaMemcpyDeviceToHost) != cudaSuccess || herr) rc = QMC_E_CUDA_LOCAL;
    }
    cudaFree(dA);
    cudaFree(dB);
    cudaFree(dC);
    cudaFree(derr);
    return rc;
}
