// Tensor-core kernels of the learned lattice-size / amplitude model of the
// amplitude scan: a BF16 GEMM on the 5th-generation tensor cores and the
// elementwise kernels of an MLP's forward and backward passes and its Adam
// update.
//
// gemm: C[M][N] (fp32) = A[M][K] . B[N][K]^T with A, B bf16 and K-major
// (row-major [rows][K]). One CTA of 128 threads computes a 128 x N tile
// (N <= 256, multiple of 16; M a multiple of 128, K of 16) over a range of
// K (split-K when the M tiles alone cannot fill the GPU):
//  * thread 0 streams 64-wide K chunks of A (128 rows) and B (N rows) into a
//    4-stage shared-memory ring with TMA (cp.async.bulk.tensor, 128-byte
//    swizzle), each stage completing on a transaction-count mbarrier;
//  * thread 32 issues four tcgen05.mma (K = 16 each) per stage into an FP32
//    accumulator in tensor memory and frees the stage with tcgen05.commit;
//  * after the last commit all 4 warps read the accumulator back with
//    tcgen05.ld and store it.
// Split-K partials go to a workspace and a second kernel adds them in split
// order (deterministic). Every mbarrier wait has an iteration limit, after
// which the CTA records an error, waits for its copies in flight, frees its
// tensor memory and exits.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <cmath>
#include <mutex>
#include <vector>

#include "../../include/qmc.h"

#include "qmc_internal.h"

#define QMC_E_INVAL_LOCAL QMC_E_INVAL
#define QMC_E_CUDA_LOCAL QMC_E_CUDA

namespace {

constexpr int kGemmThreads = 128;
constexpr int kStages = 4;
constexpr int kBK = 64;                                  // K elements per stage: one 128-byte swizzle span
constexpr int kTileM = 128;
constexpr int kMaxN = 256;
constexpr int kAStageBytes = kTileM * kBK * 2;           // 16 KB
constexpr int kBStageBytes = kMaxN * kBK * 2;            // 32 KB
constexpr int kStageBytes = kAStageBytes + kBStageBytes;
constexpr int kGemmSmem = kStages * kStageBytes + 1024;  // + slack to align the ring to 1024 B
// Polls of one mbarrier wait before it gives up (with 64 ns sleeps: a few
// seconds). The pipeline's waits take their limit from the launch (this value
// unless a caller asks for fewer); the clean-up after a timeout always waits
// with this one, so that copies and MMAs in flight land before the CTA frees
// its tensor memory and exits.
constexpr unsigned kWaitLimit = 1u << 26;

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

// Shared-memory matrix descriptor (tcgen05) of a K-major operand in the
// 128-byte-swizzled layout that TMA writes: start address, stride between
// 8-row core-matrix groups 1024 B, fixed field 0b001 at bit 46, swizzle mode
// 2 (128 B) at bit 61; the leading-dimension offset is unused for swizzled
// K-major operands (set to 1).
__device__ __forceinline__ uint64_t smem_desc_sw128(uint32_t addr) {
    uint64_t d = 0;
    d |= (uint64_t)((addr & 0x3FFFF) >> 4);
    d |= (uint64_t)1 << 16;
    d |= (uint64_t)(1024 >> 4) << 32;
    d |= (uint64_t)1 << 46;
    d |= (uint64_t)2 << 61;
    return d;
}

// Instruction descriptor, kind::f16: D = F32, A = B = BF16, both K-major.
__host__ __device__ constexpr uint32_t instr_desc_bf16(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t phase, unsigned limit) {
    for (unsigned it = 0; it < limit; ++it) {
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

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap *map, int x, int y, uint32_t mbar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], "
        "[%4];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(mbar)
        : "memory");
}

__global__ void __launch_bounds__(kGemmThreads, 1)
qmc_gemm_bf16_tc(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB, float *C,
                 int N, int K, int chunks_per_split, size_t split_stride, unsigned *err, unsigned wait_limit) {
    extern __shared__ unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t full[kStages], empty[kStages], done;
    __shared__ uint32_t tmem_base;
    __shared__ int issued, consumed;
    unsigned char *ring = reinterpret_cast<unsigned char *>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int m0 = blockIdx.x * kTileM;
    const int nchunks = (K + kBK - 1) / kBK;
    const int c0 = blockIdx.y * chunks_per_split;
    const int nc = min(nchunks, c0 + chunks_per_split) - c0;   // >= 1 by the host's split choice
    float *Cs = C + (size_t)blockIdx.y * split_stride;

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                     "r"(kMaxN));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::);
    }
    if (tid == 0) {
        for (int s = 0; s < kStages; ++s) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&full[s])));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&empty[s])));
        }
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&done)));
        asm volatile("fence.mbarrier_init.release.cluster;" ::);
        issued = 0;
        consumed = 0;
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::);
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::);
    const uint32_t tmem = tmem_base;
    const uint32_t bytes_stage = (uint32_t)((kTileM + N) * kBK * 2);
    bool ok = true;

    if (tid == 0) {
        // producer: TMA into the ring, each stage reused once the MMAs reading it committed
        for (int i = 0; i < nc; ++i) {
            const int s = i % kStages;
            if (i >= kStages && !mbar_wait(smem_u32(&empty[s]), (uint32_t)((i / kStages - 1) & 1), wait_limit)) {
                ok = false;
                break;
            }
            const uint32_t fb = smem_u32(&full[s]);
            asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(fb), "r"(bytes_stage)
                         : "memory");
            const uint32_t sa = smem_u32(ring + s * kStageBytes);
            tma_load_2d(sa, &mapA, (c0 + i) * kBK, m0, fb);
            tma_load_2d(sa + kAStageBytes, &mapB, (c0 + i) * kBK, 0, fb);
            issued = i + 1;
        }
    } else if (tid == 32) {
        // MMA issuer
        const uint32_t idesc = instr_desc_bf16(kTileM, N);
        for (int i = 0; i < nc; ++i) {
            const int s = i % kStages;
            if (!mbar_wait(smem_u32(&full[s]), (uint32_t)((i / kStages) & 1), wait_limit)) {
                ok = false;
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::);
            const uint32_t sa = smem_u32(ring + s * kStageBytes);
#pragma unroll
            for (int ks = 0; ks < kBK / 16; ++ks) {
                const uint64_t da = smem_desc_sw128(sa + ks * 32);
                const uint64_t db = smem_desc_sw128(sa + kAStageBytes + ks * 32);
                const uint32_t acc = (i > 0 || ks > 0) ? 1u : 0u;
                asm volatile(
                    "{\n\t.reg .pred p;\n\t"
                    "setp.ne.b32 p, %4, 0;\n\t"
                    "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem),
                    "l"(da), "l"(db), "r"(idesc), "r"(acc));
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                             smem_u32(&empty[s]))
                         : "memory");
            consumed = i + 1;
        }
        // completion of every MMA issued so far
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                         smem_u32(&done))
                     : "memory");
    }
    if (!mbar_wait(smem_u32(&done), 0, wait_limit)) ok = false;
    ok = __syncthreads_and(ok);
    asm volatile("tcgen05.fence::after_thread_sync;" ::);
    if (ok) {
        // warp w owns TMEM lanes 32w..32w+31 = rows m0 + 32w + lane
        const int row = m0 + warp * 32 + lane;
        for (int c = 0; c < N; c += 16) {
            uint32_t r[16];
            const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c;
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, "
                "%13, %14, %15}, [%16];"
                : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                  "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
                  "=r"(r[15])
                : "r"(taddr));
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            float *dst = Cs + (size_t)row * N + c;
#pragma unroll
            for (int q = 0; q < 16; ++q) dst[q] = __uint_as_float(r[q]);
        }
    } else {
        if (tid == 0) {
            atomicAdd(err, 1u);
            // copies still in flight land before the CTA's shared memory goes
            // away, and the MMAs issued so far finish before the accumulator's
            // tensor memory is freed (the MMA thread always commits `done`)
            for (int i = consumed; i < issued; ++i)
                mbar_wait(smem_u32(&full[i % kStages]), (uint32_t)((i / kStages) & 1), kWaitLimit);
            mbar_wait(smem_u32(&done), 0, kWaitLimit);
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::);
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kMaxN));
}

// C = sum over splits of W[s] (in split order)
__global__ void qmc_gemm_splitk_sum(const float *W, int splits, size_t stride, float *C, size_t n) {
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        float acc = W[i];
        for (int s = 1; s < splits; ++s) acc += W[(size_t)s * stride + i];
        C[i] = acc;
    }
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
    static EncodeTiledFn fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(p);
    });
    return fn;
}

// 2-D bf16 tensor [rows][K] (row stride K), box {64, box_rows}, 128-byte swizzle,
// zero fill beyond K
bool make_map(CUtensorMap *map, const void *ptr, int rows, int K, int box_rows) {
    EncodeTiledFn fn = encode_fn();
    if (!fn) return false;
    const cuuint64_t dims[2] = {(cuuint64_t)K, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)K * 2};
    const cuuint32_t box[2] = {(cuuint32_t)kBK, (cuuint32_t)box_rows};
    const cuuint32_t estr[2] = {1, 1};
    return fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void *>(ptr), dims, strides, box, estr,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// split-K workspace, grown on demand (one per process; calls on one device)
struct SplitWorkspace {
    std::mutex mu;
    float *ptr = nullptr;
    size_t cap = 0;
};
SplitWorkspace &workspace() {
    static SplitWorkspace w;
    return w;
}

}  // namespace

// C[M][N] = A[M][K] B[N][K]^T, device pointers; M % 128 == 0, K % 16 == 0,
// N % 16 == 0 and 16 <= N <= 256; A, B 16-byte aligned; C rows contiguous
// (ldc = N). Split-K when the M tiles leave most SMs idle.
extern "C" int qmc_k_gemm_bf16_limit(const void *A, const void *B, float *C, int M, int N, int K, unsigned *err_dev,
                                     void *stream, unsigned wait_limit) {
    if (M <= 0 || M % 128 || K <= 0 || K % 16 || N < 16 || N > 256 || N % 16) return -2;
    if ((reinterpret_cast<uintptr_t>(A) | reinterpret_cast<uintptr_t>(B)) & 15) return -2;
    static bool attr_set = false;
    if (!attr_set) {
        if (cudaFuncSetAttribute(qmc_gemm_bf16_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, kGemmSmem) !=
            cudaSuccess)
            return -1;
        attr_set = true;
    }
    CUtensorMap mapA, mapB;
    if (!make_map(&mapA, A, M, K, kTileM) || !make_map(&mapB, B, N, K, N)) return -1;
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int mt = M / kTileM, nchunks = (K + kBK - 1) / kBK;
    int splits = std::max(1, std::min(nchunks, sms / mt));
    const int per = (nchunks + splits - 1) / splits;
    splits = (nchunks + per - 1) / per;   // every split has at least one chunk
    const size_t mn = (size_t)M * N;
    float *out = C;
    std::unique_lock<std::mutex> lock(workspace().mu, std::defer_lock);
    if (splits > 1) {
        lock.lock();
        SplitWorkspace &w = workspace();
        if (w.cap < (size_t)splits * mn) {
            cudaStreamSynchronize((cudaStream_t)stream);
            cudaFree(w.ptr);
            w.ptr = nullptr;
            w.cap = 0;
            if (cudaMalloc(&w.ptr, (size_t)splits * mn * sizeof(float)) != cudaSuccess) return -1;
            w.cap = (size_t)splits * mn;
        }
        out = w.ptr;
    }
    qmc_gemm_bf16_tc<<<dim3(mt, splits), kGemmThreads, kGemmSmem, (cudaStream_t)stream>>>(mapA, mapB, out, N, K,
                                                                                           per, mn, err_dev,
                                                                                           wait_limit);
    if (splits > 1) {
        const unsigned blocks = (unsigned)std::min<size_t>((mn + 255) / 256, 4096);
        qmc_gemm_splitk_sum<<<blocks, 256, 0, (cudaStream_t)stream>>>(out, splits, mn, C, mn);
    }
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

extern "C" int qmc_k_gemm_bf16(const void *A, const void *B, float *C, int M, int N, int K, unsigned *err_dev,
                               void *stream) {
    return qmc_k_gemm_bf16_limit(A, B, C, M, N, K, err_dev, stream, kWaitLimit);
}

extern "C" int qmc_gemm_bf16_device(const void *A, const void *B, float *C, int M, int N, int K, unsigned *err_dev,
                                    void *stream) {
    if (!A || !B || !C || !err_dev) return QMC_E_INVAL_LOCAL;
    const int rc = qmc_k_gemm_bf16(A, B, C, M, N, K, err_dev, stream);
    return rc == -2 ? QMC_E_INVAL_LOCAL : (rc ? QMC_E_CUDA_LOCAL : 0);
}

extern "C" int qmc_gemm_bf16_device_limit(const void *A, const void *B, float *C, int M, int N, int K,
                                          unsigned *err_dev, void *stream, unsigned wait_limit) {
    if (!A || !B || !C || !err_dev) return QMC_E_INVAL_LOCAL;
    const int rc = qmc_k_gemm_bf16_limit(A, B, C, M, N, K, err_dev, stream, wait_limit);
    return rc == -2 ? QMC_E_INVAL_LOCAL : (rc ? QMC_E_CUDA_LOCAL : 0);
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

// ============================================================================
// The MLP: x (nin) -> tanh(W0 x + b0) -> [tanh(Wk h + bk)] x (depth-1) -> Wout h + bout
// Layer 0 (K = nin, tiny) runs on the CUDA cores in FP32; every other layer and
// every weight/activation gradient product runs through qmc_gemm_bf16_tc with
// bf16 operands and FP32 accumulation. FP32 master weights, Adam in FP32.
// Batches are padded to a multiple of 128 rows with zero loss weight.
// ============================================================================
namespace {

__device__ __forceinline__ __nv_bfloat16 bf(float x) { return __float2bfloat16_rn(x); }

// h0 = tanh(x W0^T + b0): f32 [Bp][H], bf16 [Bp][H] and [H][Bp]
__global__ void mlp_layer0_fwd(const float *x, const float *W0, const float *b0, int nin, int H, int Bp,
                               float *h, __nv_bfloat16 *hb, __nv_bfloat16 *hbT) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= Bp * H) return;
    const int b = i / H, o = i % H;
    float z = b0[o];
    for (int k = 0; k < nin; ++k) z = fmaf(W0[o * nin + k], x[b * nin + k], z);
    const float a = tanhf(z);
    h[i] = a;
    hb[i] = bf(a);
    hbT[(size_t)o * Bp + b] = bf(a);
}

// a = act(C + bias) for a GEMM output C [Bp][ldc] (columns < N used)
__global__ void mlp_bias_act(const float *C, const float *bias, int N, int ldc, int Bp, int act, float *h,
                             __nv_bfloat16 *hb, __nv_bfloat16 *hbT) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= Bp * N) return;
    const int b = i / N, o = i % N;
    float z = C[(size_t)b * ldc + o] + bias[o];
    if (act) z = tanhf(z);
    h[i] = z;
    if (hb) hb[i] = bf(z);
    if (hbT) hbT[(size_t)o * Bp + b] = bf(z);
}

// weighted squared error: loss += wt_o mask_b (out - y)^2 / B; dout = 2 wt_o mask_b (out - y) / B
__global__ void mlp_loss(const float *out, const float *y, const float *wt, const float *mask, int No, int Nop,
                         int Bp, float invB, __nv_bfloat16 *dob, __nv_bfloat16 *dobT, float *dof, double *loss) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= Bp * Nop) return;
    const int b = i / Nop, o = i % Nop;
    float g = 0.f;
    if (o < No) {
        const float r = out[(size_t)b * No + o] - y[(size_t)b * No + o];
        const float w = wt[o] * mask[b];
        g = 2.f * w * r * invB;
        if (w != 0.f) atomicAdd(loss, (double)(w * r * r * invB));
    }
    dob[i] = bf(g);
    dobT[(size_t)o * Bp + b] = bf(g);
    dof[i] = g;
}

// dz = dh (1 - h^2) for tanh layers: bf16 [Bp][H], bf16 [H][Bp], f32 [Bp][H]
__global__ void mlp_tanh_bwd(const float *dh, const float *h, int H, int Bp, __nv_bfloat16 *dzb,
                             __nv_bfloat16 *dzbT, float *dzf) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= Bp * H) return;
    const int b = i / H, o = i % H;
    const float a = h[i];
    const float g = dh[i] * (1.f - a * a);
    dzb[i] = bf(g);
    dzbT[(size_t)o * Bp + b] = bf(g);
    dzf[i] = g;
}

// column sums: db[o] = sum_b dz[b][o]  (one block per column, fixed order)
__global__ void mlp_colsum(const float *dz, int N, int ld, int Bp, float *db) {
    const int o = blockIdx.x;
    __shared__ float red[256];
    float s = 0.f;
    for (int b = threadIdx.x; b < Bp; b += blockDim.x) s += dz[(size_t)b * ld + o];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) db[o] = red[0];
}

// dW0[o][k] = sum_b dz0[b][o] x[b][k]
__global__ void mlp_layer0_bwd(const float *dz, const float *x, int nin, int H, int Bp, float *dW0) {
    const int o = blockIdx.x, k = blockIdx.y;
    __shared__ float red[256];
    float s = 0.f;
    for (int b = threadIdx.x; b < Bp; b += blockDim.x) s = fmaf(dz[(size_t)b * H + o], x[b * nin + k], s);
    red[threadIdx.x] = s;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) dW0[o * nin + k] = red[0];
}

// copy a [H][Nop] GEMM result (dWout^T) into dWout [No][H]
__global__ void mlp_untranspose(const float *src, int H, int Nop, int No, float *dst) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= No * H) return;
    const int o = i / H, k = i % H;
    dst[i] = src[(size_t)k * Nop + o];
}

// bf16 copies of a weight matrix W [R][C] (rows >= R of the padded copy are 0)
__global__ void mlp_weights_bf16(const float *W, int R, int Rp, int C, __nv_bfloat16 *Wb, __nv_bfloat16 *WbT) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= Rp * C) return;
    const int r = i / C, c = i % C;
    const float v = r < R ? W[(size_t)r * C + c] : 0.f;
    Wb[i] = bf(v);
    WbT[(size_t)c * Rp + r] = bf(v);
}

__global__ void mlp_adam(float *p, const float *g, float *m, float *v, size_t n, float lr, float b1, float b2,
                         float eps, float c1, float c2) {
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

inline unsigned nblk(size_t n, int t = 256) { return (unsigned)((n + t - 1) / t); }

uint64_t mlp_sm64(uint64_t &s) {
    uint64_t z = (s += 0x9E3779B97F4A7C15ULL);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

}  // namespace

struct qmc_mlp {
    int device = 0, nin = 0, H = 0, D = 0, No = 0, Nop = 0;
    cudaStream_t stream = nullptr;
    size_t nparams = 0;
    std::vector<size_t> offW, offb;     // per layer (0..D-1 hidden, D = output)
    float *params = nullptr, *grads = nullptr, *am = nullptr, *av = nullptr;
    std::vector<__nv_bfloat16 *> Wb, WbT;   // layers 1..D (index by layer)
    int Bcap = 0;
    float *x = nullptr, *y = nullptr, *mask = nullptr, *C = nullptr, *tmp = nullptr;
    std::vector<float *> hf;                 // [D] f32 activations
    std::vector<__nv_bfloat16 *> hb, hbT;    // [D]
    float *out = nullptr, *dof = nullptr, *dz = nullptr;
    __nv_bfloat16 *dob = nullptr, *dobT = nullptr, *dzb = nullptr, *dzbT = nullptr;
    float *wt = nullptr;
    double *loss = nullptr;
    unsigned *err = nullptr;
    int t = 0;
};

namespace {

int mlp_free_batch(qmc_mlp *m) {
    cudaFree(m->x);
    cudaFree(m->y);
    cudaFree(m->mask);
    cudaFree(m->C);
    cudaFree(m->tmp);
    cudaFree(m->out);
    cudaFree(m->dof);
    cudaFree(m->dz);
    cudaFree(m->dob);
    cudaFree(m->dobT);
    cudaFree(m->dzb);
    cudaFree(m->dzbT);
    for (float *p : m->hf) cudaFree(p);
    for (auto *p : m->hb) cudaFree(p);
    for (auto *p : m->hbT) cudaFree(p);
    m->hf.assign(m->D, nullptr);
    m->hb.assign(m->D, nullptr);
    m->hbT.assign(m->D, nullptr);
    m->x = m->y = m->mask = m->C = m->tmp = m->out = m->dof = m->dz = nullptr;
    m->dob = m->dobT = m->dzb = m->dzbT = nullptr;
    m->Bcap = 0;
    return 0;
}

int mlp_ensure_batch(qmc_mlp *m, int Bp) {
    if (Bp <= m->Bcap) return 0;
    mlp_free_batch(m);
    const size_t H = m->H, No = m->No, Nop = m->Nop;
    bool bad = false;
    auto A = [&](void **p, size_t bytes) { bad |= cudaMalloc(p, bytes) != cudaSuccess; };
    A((void **)&m->x, (size_t)Bp * m->nin * 4);
    A((void **)&m->y, (size_t)Bp * No * 4);
    A((void **)&m->mask, (size_t)Bp * 4);
    A((void **)&m->C, (size_t)Bp * std::max(H, Nop) * 4);
    A((void **)&m->tmp, (size_t)std::max(H * Nop, (size_t)Bp * H) * 4);
    A((void **)&m->out, (size_t)Bp * No * 4);
    A((void **)&m->dof, (size_t)Bp * Nop * 4);
    A((void **)&m->dz, (size_t)Bp * H * 4);
    A((void **)&m->dob, (size_t)Bp * Nop * 2);
    A((void **)&m->dobT, (size_t)Bp * Nop * 2);
    A((void **)&m->dzb, (size_t)Bp * H * 2);
    A((void **)&m->dzbT, (size_t)Bp * H * 2);
    for (int l = 0; l < m->D; ++l) {
        A((void **)&m->hf[l], (size_t)Bp * H * 4);
        A((void **)&m->hb[l], (size_t)Bp * H * 2);
        A((void **)&m->hbT[l], (size_t)Bp * H * 2);
    }
    if (bad) {
        mlp_free_batch(m);
        return -1;
    }
    m->Bcap = Bp;
    return 0;
}

// refresh the bf16 weight copies of the GEMM layers from the FP32 master weights
int mlp_sync_weights(qmc_mlp *m) {
    for (int l = 1; l <= m->D; ++l) {
        const int R = l == m->D ? m->No : m->H, Rp = l == m->D ? m->Nop : m->H;
        mlp_weights_bf16<<<nblk((size_t)Rp * m->H), 256, 0, m->stream>>>(m->params + m->offW[l], R, Rp, m->H,
                                                                        m->Wb[l], m->WbT[l]);
    }
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

// forward for Bp rows already in m->x; output in m->out [Bp][No]
int mlp_forward_dev(qmc_mlp *m, int Bp) {
    const int H = m->H;
    mlp_layer0_fwd<<<nblk((size_t)Bp * H), 256, 0, m->stream>>>(m->x, m->params + m->offW[0], m->params + m->offb[0],
                                                               m->nin, H, Bp, m->hf[0], m->hb[0], m->hbT[0]);
    for (int l = 1; l < m->D; ++l) {
        if (qmc_k_gemm_bf16(m->hb[l - 1], m->Wb[l], m->C, Bp, H, H, m->err, m->stream)) return -1;
        mlp_bias_act<<<nblk((size_t)Bp * H), 256, 0, m->stream>>>(m->C, m->params + m->offb[l], H, H, Bp, 1,
                                                                 m->hf[l], m->hb[l], m->hbT[l]);
    }
    if (qmc_k_gemm_bf16(m->hb[m->D - 1], m->Wb[m->D], m->C, Bp, m->Nop, H, m->err, m->stream)) return -1;
    mlp_bias_act<<<nblk((size_t)Bp * m->No), 256, 0, m->stream>>>(m->C, m->params + m->offb[m->D], m->No, m->Nop,
                                                                 Bp, 0, m->out, nullptr, nullptr);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

// loss (into *loss_dst) and gradients (into m->grads) for Bp rows with x, y, mask, wt in place
int mlp_backward_dev(qmc_mlp *m, int Bp, int B, double *loss_dst) {
    const int H = m->H, D = m->D, Nop = m->Nop, No = m->No;
    cudaMemsetAsync(loss_dst, 0, sizeof(double), m->stream);
    mlp_loss<<<nblk((size_t)Bp * Nop), 256, 0, m->stream>>>(m->out, m->y, m->wt, m->mask, No, Nop, Bp, 1.f / B,
                                                            m->dob, m->dobT, m->dof, loss_dst);
    // output layer: dWout^T = h_{D-1}^T dout  ([H][Nop]), dbout, dh = dout Wout
    if (qmc_k_gemm_bf16(m->hbT[D - 1], m->dobT, m->tmp, H, Nop, Bp, m->err, m->stream)) return -1;
    mlp_untranspose<<<nblk((size_t)No * H), 256, 0, m->stream>>>(m->tmp, H, Nop, No, m->grads + m->offW[D]);
    mlp_colsum<<<No, 256, 0, m->stream>>>(m->dof, No, Nop, Bp, m->grads + m->offb[D]);
    if (qmc_k_gemm_bf16(m->dob, m->WbT[D], m->C, Bp, H, Nop, m->err, m->stream)) return -1;
    for (int l = D - 1; l >= 0; --l) {
        mlp_tanh_bwd<<<nblk((size_t)Bp * H), 256, 0, m->stream>>>(m->C, m->hf[l], H, Bp, m->dzb, m->dzbT, m->dz);
        mlp_colsum<<<H, 256, 0, m->stream>>>(m->dz, H, H, Bp, m->grads + m->offb[l]);
        if (l == 0) {
            mlp_layer0_bwd<<<dim3(H, m->nin), 256, 0, m->stream>>>(m->dz, m->x, m->nin, H, Bp, m->grads + m->offW[0]);
        } else {
            // dW_l = dz^T h_{l-1}  ([H][H]); dh_{l-1} = dz W_l
            if (qmc_k_gemm_bf16(m->dzbT, m->hbT[l - 1], m->grads + m->offW[l], H, H, Bp, m->err, m->stream))
                return -1;
            if (qmc_k_gemm_bf16(m->dzb, m->WbT[l], m->C, Bp, H, H, m->err, m->stream)) return -1;
        }
    }
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

// stage a host batch (B rows) padded to Bp rows
int mlp_stage(qmc_mlp *m, const float *x, const float *y, const float *wt, int B, int Bp) {
    if (mlp_ensure_batch(m, Bp)) return -1;
    cudaMemsetAsync(m->x, 0, (size_t)Bp * m->nin * 4, m->stream);
    cudaMemcpyAsync(m->x, x, (size_t)B * m->nin * 4, cudaMemcpyHostToDevice, m->stream);
    if (y) {
        cudaMemsetAsync(m->y, 0, (size_t)Bp * m->No * 4, m->stream);
        cudaMemcpyAsync(m->y, y, (size_t)B * m->No * 4, cudaMemcpyHostToDevice, m->stream);
        std::vector<float> mk(Bp, 0.f);
        for (int b = 0; b < B; ++b) mk[b] = 1.f;
        cudaMemcpyAsync(m->mask, mk.data(), (size_t)Bp * 4, cudaMemcpyHostToDevice, m->stream);
        std::vector<float> w(m->No, 1.f);
        if (wt) w.assign(wt, wt + m->No);
        cudaMemcpyAsync(m->wt, w.data(), (size_t)m->No * 4, cudaMemcpyHostToDevice, m->stream);
        return cudaStreamSynchronize(m->stream) == cudaSuccess ? 0 : -1;   // host vectors go out of scope
    }
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int mlp_check_err(qmc_mlp *m) {
    unsigned e = 0;
    if (cudaMemcpyAsync(&e, m->err, 4, cudaMemcpyDeviceToHost, m->stream) != cudaSuccess) return -1;
    if (cudaStreamSynchronize(m->stream) != cudaSuccess) return -1;
    return e ? -1 : 0;
}

}  // namespace

extern "C" {

int qmc_mlp_create(qmc_mlp **out, int device, int nin, int width, int depth, int nout, uint64_t seed) {
    if (!out || nin < 1 || nin > 64 || width % 128 || width < 128 || width > 256 || depth < 1 || depth > 16 ||
        nout < 1 || nout > 256)
        return QMC_E_INVAL_LOCAL;
    *out = nullptr;
    if (cudaSetDevice(device) != cudaSuccess) return QMC_E_CUDA_LOCAL;
    qmc_mlp *m = new qmc_mlp();
    m->device = device;
    m->nin = nin;
    m->H = width;
    m->D = depth;
    m->No = nout;
    m->Nop = (nout + 15) / 16 * 16;
    m->hf.assign(depth, nullptr);
    m->hb.assign(depth, nullptr);
    m->hbT.assign(depth, nullptr);
    size_t off = 0;
    for (int l = 0; l <= depth; ++l) {
        const size_t fan_in = l == 0 ? nin : width, rows = l == depth ? nout : width;
        m->offW.push_back(off);
        off += rows * fan_in;
        m->offb.push_back(off);
        off += rows;
    }
    m->nparams = off;
    bool bad = cudaStreamCreateWithFlags(&m->stream, cudaStreamNonBlocking) != cudaSuccess;
    bad |= cudaMalloc(&m->params, off * 4) != cudaSuccess;
    bad |= cudaMalloc(&m->grads, off * 4) != cudaSuccess;
    bad |= cudaMalloc(&m->am, off * 4) != cudaSuccess;
    bad |= cudaMalloc(&m->av, off * 4) != cudaSuccess;
    bad |= cudaMalloc(&m->wt, 256 * 4) != cudaSuccess;
    bad |= cudaMalloc(&m->loss, sizeof(double)) != cudaSuccess;
    bad |= cudaMalloc(&m->err, 4) != cudaSuccess;
    m->Wb.assign(depth + 1, nullptr);
    m->WbT.assign(depth + 1, nullptr);
    for (int l = 1; l <= depth; ++l) {
        const size_t Rp = l == depth ? m->Nop : width;
        bad |= cudaMalloc(&m->Wb[l], Rp * width * 2) != cudaSuccess;
        bad |= cudaMalloc(&m->WbT[l], Rp * width * 2) != cudaSuccess;
    }
    if (bad) {
        qmc_mlp_destroy(m);
        return QMC_E_CUDA_LOCAL;
    }
    // uniform(-1/sqrt(fan_in), 1/sqrt(fan_in)) weights, zero biases, from splitmix64
    std::vector<float> p(off, 0.f);
    uint64_t st = seed;
    for (int l = 0; l <= depth; ++l) {
        const size_t fan_in = l == 0 ? nin : width, rows = l == depth ? nout : width;
        const double a = 1.0 / std::sqrt((double)fan_in);
        for (size_t i = 0; i < rows * fan_in; ++i)
            p[m->offW[l] + i] = (float)(a * (2.0 * ((mlp_sm64(st) >> 11) * (1.0 / 9007199254740992.0)) - 1.0));
    }
    cudaMemcpy(m->params, p.data(), off * 4, cudaMemcpyHostToDevice);
    cudaMemset(m->am, 0, off * 4);
    cudaMemset(m->av, 0, off * 4);
    cudaMemset(m->grads, 0, off * 4);
    cudaMemset(m->err, 0, 4);
    if (mlp_sync_weights(m) || cudaStreamSynchronize(m->stream) != cudaSuccess) {
        qmc_mlp_destroy(m);
        return QMC_E_CUDA_LOCAL;
    }
    *out = m;
    return 0;
}

void qmc_mlp_destroy(qmc_mlp *m) {
    if (!m) return;
    cudaSetDevice(m->device);
    if (m->stream) cudaStreamSynchronize(m->stream);
    mlp_free_batch(m);
    cudaFree(m->params);
    cudaFree(m->grads);
    cudaFree(m->am);
    cudaFree(m->av);
    cudaFree(m->wt);
    cudaFree(m->loss);
    cudaFree(m->err);
    for (auto *p : m->Wb) cudaFree(p);
    for (auto *p : m->WbT) cudaFree(p);
    if (m->stream) cudaStreamDestroy(m->stream);
    delete m;
}

int qmc_mlp_num_params(const qmc_mlp *m, size_t *n) {
    if (!m || !n) return QMC_E_INVAL_LOCAL;
    *n = m->nparams;
    return 0;
}

int qmc_mlp_get_params(qmc_mlp *m, float *host, size_t n) {
    if (!m || !host || n != m->nparams) return QMC_E_INVAL_LOCAL;
    cudaSetDevice(m->device);
    if (cudaMemcpyAsync(host, m->params, n * 4, cudaMemcpyDeviceToHost, m->stream) != cudaSuccess ||
        cudaStreamSynchronize(m->stream) != cudaSuccess)
        return QMC_E_CUDA_LOCAL;
    return 0;
}

int qmc_mlp_set_params(qmc_mlp *m, const float *host, size_t n) {
    if (!m || !host || n != m->nparams) return QMC_E_INVAL_LOCAL;
    cudaSetDevice(m->device);
    if (cudaMemcpyAsync(m->params, host, n * 4, cudaMemcpyHostToDevice, m->stream) != cudaSuccess ||
        mlp_sync_weights(m) || cudaStreamSynchronize(m->stream) != cudaSuccess)
        return QMC_E_CUDA_LOCAL;
    return 0;
}

int qmc_mlp_forward(qmc_mlp *m, const float *x, int B, float *y) {
    if (!m || !x || !y || B < 1) return QMC_E_INVAL_LOCAL;
    cudaSetDevice(m->device);
    cudaMemsetAsync(m->err, 0, 4, m->stream);
    const int Bp = (B + 127) / 128 * 128;
    if (mlp_stage(m, x, nullptr, nullptr, B, Bp) || mlp_forward_dev(m, Bp)) return QMC_E_CUDA_LOCAL;
    if (cudaMemcpyAsync(y, m->out, (size_t)B * m->No * 4, cudaMemcpyDeviceToHost, m->stream) != cudaSuccess)
        return QMC_E_CUDA_LOCAL;
    return mlp_check_err(m) ? QMC_E_CUDA_LOCAL : 0;
}

int qmc_mlp_grad(qmc_mlp *m, const float *x, const float *y, const float *wt, int B, float *loss, float *grad) {
    if (!m || !x || !y || B < 1) return QMC_E_INVAL_LOCAL;
    cudaSetDevice(m->device);
    cudaMemsetAsync(m->err, 0, 4, m->stream);
    const int Bp = (B + 127) / 128 * 128;
    if (mlp_stage(m, x, y, wt, B, Bp) || mlp_forward_dev(m, Bp) || mlp_backward_dev(m, Bp, B, m->loss))
        return QMC_E_CUDA_LOCAL;
    double l = 0.0;
    cudaMemcpyAsync(&l, m->loss, sizeof(double), cudaMemcpyDeviceToHost, m->stream);
    if (grad) cudaMemcpyAsync(grad, m->grads, m->nparams * 4, cudaMemcpyDeviceToHost, m->stream);
    if (mlp_check_err(m)) return QMC_E_CUDA_LOCAL;
    if (loss) *loss = (float)l;
    return 0;
}

int qmc_mlp_train(qmc_mlp *m, const float *x, const float *y, const float *wt, int B, int steps, float lr,
                  float *losses) {
    if (!m || !x || !y || B < 1 || steps < 0 || !(lr > 0)) return QMC_E_INVAL_LOCAL;
    cudaSetDevice(m->device);
    cudaMemsetAsync(m->err, 0, 4, m->stream);
    const int Bp = (B + 127) / 128 * 128;
    if (mlp_stage(m, x, y, wt, B, Bp)) return QMC_E_CUDA_LOCAL;
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    // per-step losses stay on the device until the end (no host round trip per step)
    double *hist = nullptr;
    if (cudaMalloc(&hist, (size_t)std::max(steps, 1) * sizeof(double)) != cudaSuccess) return QMC_E_CUDA_LOCAL;
    int rc = 0;
    for (int s = 0; s < steps && !rc; ++s) {
        if (mlp_forward_dev(m, Bp) || mlp_backward_dev(m, Bp, B, hist + s)) {
            rc = QMC_E_CUDA_LOCAL;
            break;
        }
        ++m->t;
        const float c1 = 1.f - std::pow(b1, (float)m->t), c2 = 1.f - std::pow(b2, (float)m->t);
        mlp_adam<<<nblk(m->nparams), 256, 0, m->stream>>>(m->params, m->grads, m->am, m->av, m->nparams, lr, b1,
                                                           b2, eps, c1, c2);
        if (mlp_sync_weights(m)) rc = QMC_E_CUDA_LOCAL;
    }
    if (!rc && losses && steps > 0) {
        std::vector<double> h(steps);
        if (cudaMemcpyAsync(h.data(), hist, steps * sizeof(double), cudaMemcpyDeviceToHost, m->stream) !=
                cudaSuccess ||
            cudaStreamSynchronize(m->stream) != cudaSuccess)
            rc = QMC_E_CUDA_LOCAL;
        for (int s = 0; s < steps && !rc; ++s) losses[s] = (float)h[s];
    }
    cudaStreamSynchronize(m->stream);
    cudaFree(hist);
    if (rc) return rc;
    return mlp_check_err(m) ? QMC_E_CUDA_LOCAL : 0;
}

}  // extern "C"
