// mr3_tc_gemm.cu -- the slice products of the backward pass on the 5th-generation tensor
// cores: C (M x N, FP32, column-major) = A (M x K) B (K x N) with bf16 operands that hold
// small integers exactly, so that every product of a chunk comes out exact in FP32.
//
// Layout: both operands K-major in global memory (A: element (m, k) at A[m lda + k];
// B: element (k, j) at B[j ldb + k]), leading dimensions a multiple of 64 elements.  One CTA
// computes a 128 x 256 tile of C:
//   * one thread loads 64-wide K slabs of A (128 x 64) and B (256 x 64) with TMA
//     (cp.async.bulk.tensor, 128-byte swizzle) into a ring of kStages shared-memory stages;
//   * one thread issues tcgen05.mma (M = 128, N = 256, K = 16, bf16 -> FP32) on each stage,
//     accumulating in tensor memory (256 columns), and frees the stage with
//     tcgen05.commit onto the stage's mbarrier;
//   * after the last slab, the four warps read their 32 accumulator lanes (rows) with
//     tcgen05.ld and store them to C, one column per warp-wide store (128 contiguous bytes).
// Every wait on an mbarrier is bounded; a wait that runs out sets *err and the CTA stops
// issuing work, waits (bounded) for what it issued, frees its tensor memory and returns.
#include <cuda.h>
#include <stdint.h>
#include "mr3_kernels.h"

namespace mr3 {
namespace {

constexpr int kBM = 128, kBN = 256, kBK = 64; // CTA tile; K slab (64 bf16 = 128 bytes)
constexpr int kStages = 4;
constexpr int kAStage = kBM * kBK * 2;        // 16 KiB
constexpr int kBStage = kBN * kBK * 2;        // 32 KiB
constexpr int kStageBytes = kAStage + kBStage;
constexpr int kSmemBytes = kStages * kStageBytes + 1024 /* alignment */ + 256 /* barriers */;
constexpr int kTmemCols = 256;
constexpr long long kWaitLimit = 1ll << 22;   // polls of one mbarrier before giving up

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
                 : "memory");
}

// true once the phase with the given parity has completed; false after kWaitLimit polls
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
    for (long long it = 0; it < kWaitLimit; ++it) {
        uint32_t ok;
        asm volatile("{\n\t.reg .pred p;\n\t"
                     "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                     "selp.u32 %0, 1, 0, p;\n\t}"
                     : "=r"(ok)
                     : "r"(bar), "r"(parity)
                     : "memory");
        if (ok) return true;
    }
    return false;
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap *map, int c0, int c1,
                                            uint32_t bar) {
    asm volatile("cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes"
                 " [%0], [%1, {%2, %3}], [%4];" ::"r"(dst),
                 "l"((unsigned long long)map), "r"(c0), "r"(c1), "r"(bar)
                 : "memory");
}

// Shared-memory matrix descriptor of a K-major tile in the canonical 128-byte-swizzled
// layout (8 rows of 128 bytes per 1024-byte atom): start address, leading byte offset
// (unused by this layout, 16), stride byte offset 1024 between 8-row groups, the fixed
// version bits 0b001 at 46..48, swizzle mode 2 (128 bytes) at 61..63.
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
    uint64_t d = (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)(16 >> 4) << 16;
    d |= (uint64_t)(1024 >> 4) << 32;
    d |= (uint64_t)1 << 46;
    d |= (uint64_t)2 << 61;
    return d;
}

// Instruction descriptor of tcgen05.mma kind::f16: FP32 accumulator (bits 4..5 = 1), A and
// B bf16 (bits 7..9 = 1, 10..12 = 1), both K-major (bits 15, 16 = 0), N >> 3 at 17..22,
// M >> 4 at 24..28.
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(kBN >> 3) << 17) |
                            ((uint32_t)(kBM >> 4) << 24);

__device__ __forceinline__ void mma_bf16(uint32_t tmem, uint64_t adesc, uint64_t bdesc,
                                         uint32_t accumulate) {
    asm volatile("{\n\t.reg .pred p;\n\t"
                 "setp.ne.b32 p, %4, 0;\n\t"
                 "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
                 "l"(adesc), "l"(bdesc), "r"(kIdesc), "r"(accumulate)
                 : "memory");
}

__device__ __forceinline__ void mma_commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
                 : "memory");
}

// C[m, j] (column-major, ldc) = sum_{k0 <= k < k1} A[m, k] B[k, j] for m < M, j < N.  The
// tensor maps cover A as (K inner, M outer) and B as (K inner, N outer), so K slabs past
// the maps' K extent read zeros (k1 may end there; a chunk that ends inside it must end
// on a multiple of 64).
__global__ void __launch_bounds__(128, 1) k_tc_gemm(int M, int N, int k0, int k1,
                                                    const __grid_constant__ CUtensorMap mapA,
                                                    const __grid_constant__ CUtensorMap mapB,
                                                    float *C, int ldc, int *err) {
    extern __shared__ uint8_t smem_raw[];
    __shared__ volatile int s_fail;
    const uint32_t raw = smem_u32(smem_raw);
    const uint32_t base = (raw + 1023u) & ~1023u; // 128-byte swizzle atoms: 1024-byte aligned
    const uint32_t bars = base + kStages * kStageBytes;
    const uint32_t accb = bars + 8u * (2 * kStages);
    const uint32_t tslot = accb + 8u;
    const uint32_t *tslot_ptr = (const uint32_t *)(smem_raw + (tslot - raw));
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int m0 = blockIdx.x * kBM, n0 = blockIdx.y * kBN;
    const int nkt = (k1 - k0 + kBK - 1) / kBK;
    if (threadIdx.x == 0) {
        s_fail = 0;
        for (int s = 0; s < kStages; ++s) {
            mbar_init(bars + 8u * s, 1);             // full: the stage's two loads landed
            mbar_init(bars + 8u * (kStages + s), 1); // empty: the MMAs reading it are done
        }
        mbar_init(accb, 1);                          // the accumulator is complete
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(tslot),
                     "r"(kTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tslot_ptr;

    if (warp == 0 && lane == 0) {
        // ---- producer: K slab kt into stage kt % kStages once the MMAs of slab
        // kt - kStages have released it
        int issued = 0;
        for (int kt = 0; kt < nkt; ++kt) {
            const int s = kt % kStages;
            if (kt >= kStages && !mbar_wait(bars + 8u * (kStages + s), ((kt / kStages) - 1) & 1)) {
                s_fail = 1;
                break;
            }
            if (s_fail) break;
            const uint32_t full = bars + 8u * s;
            const uint32_t sa = base + s * kStageBytes, sb = sa + kAStage;
            mbar_expect_tx(full, kStageBytes);
            tma_load_2d(sa, &mapA, k0 + kt * kBK, m0, full);
            tma_load_2d(sb, &mapB, k0 + kt * kBK, n0, full);
            ++issued;
        }
        if (s_fail) // let the loads in flight land before the CTA goes away
            for (int kt = (issued > kStages ? issued - kStages : 0); kt < issued; ++kt)
                mbar_wait(bars + 8u * (kt % kStages), (kt / kStages) & 1);
    } else if (warp == 1 && lane == 0) {
        // ---- MMA issuer: 4 MMAs of K = 16 per slab, each advancing 32 bytes inside the
        // 128-byte swizzle row; the stage is released when they complete
        for (int kt = 0; kt < nkt; ++kt) {
            const int s = kt % kStages;
            if (!mbar_wait(bars + 8u * s, (kt / kStages) & 1)) {
                s_fail = 1;
                break;
            }
            if (s_fail) break;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t sa = base + s * kStageBytes, sb = sa + kAStage;
#pragma unroll
            for (int kk = 0; kk < kBK / 16; ++kk)
                mma_bf16(tmem, sw128_desc(sa + 32u * kk), sw128_desc(sb + 32u * kk),
                         (kt > 0 || kk > 0) ? 1u : 0u);
            mma_commit(bars + 8u * (kStages + s));
        }
        mma_commit(accb); // arrives once every MMA issued above has completed
    }
    __syncwarp();
    // ---- epilogue: warp w owns accumulator lanes (rows) 32 w .. 32 w + 31
    const bool ready = mbar_wait(accb, 0);
    if (!ready) s_fail = 1;
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const int row = m0 + warp * 32 + lane;
    const uint32_t trow = tmem + ((uint32_t)(warp * 32) << 16);
    if (ready && nkt > 0) {
        for (int c = 0; c < kBN; c += 32) {
            uint32_t v[32];
            asm volatile("tcgen05.ld.sync.aligned.32x32b.x32.b32 "
                         "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
                         "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, "
                         "%30, %31}, [%32];"
                         : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]),
                           "=r"(v[6]), "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]),
                           "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]), "=r"(v[16]),
                           "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]),
                           "=r"(v[22]), "=r"(v[23]), "=r"(v[24]), "=r"(v[25]), "=r"(v[26]),
                           "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
                         : "r"(trow + (uint32_t)c)
                         : "memory");
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            if (row < M) {
#pragma unroll
                for (int j = 0; j < 32; ++j) {
                    const int col = n0 + c + j;
                    if (col < N) C[(size_t)col * ldc + row] = __uint_as_float(v[j]);
                }
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols)
                     : "memory");
    }
    if (threadIdx.x == 0 && s_fail) atomicExch(err, 1);
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *,
                                  const cuuint64_t *, const cuuint64_t *, const cuuint32_t *,
                                  const cuuint32_t *, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_tiled() {
    static EncodeTiledFn fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                             &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (EncodeTiledFn)p;
        else
            cudaGetLastError();
    }
    return fn;
}

// A bf16 matrix with `rows` rows of `inner` contiguous elements (row stride ld elements),
// loaded in boxes of 64 x box_rows with the 128-byte swizzle; out-of-range elements read 0.
bool make_map(CUtensorMap *m, const void *ptr, long long inner, long long rows, long long ld,
              int box_rows) {
    EncodeTiledFn enc = encode_tiled();
    if (!enc) return false;
    const cuuint64_t dims[2] = {(cuuint64_t)inner, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)ld * 2};
    const cuuint32_t box[2] = {(cuuint32_t)kBK, (cuuint32_t)box_rows};
    const cuuint32_t estr[2] = {1, 1};
    return enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void *>(ptr), dims, strides, box,
               estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
               CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

} // namespace

// See mr3_kernels.h.
int tc_gemm_bf16(int M, int N, int K, int k0, int k1, const unsigned short *A, int lda,
                 const unsigned short *B, int ldb, float *C, int ldc, int *err, cudaStream_t s) {
    if (M <= 0 || N <= 0 || k1 <= k0) return 0;
    if ((lda % 64) || (ldb % 64) || (k0 % kBK) || ((uintptr_t)A % 16) || ((uintptr_t)B % 16))
        return -1;
    static bool attr_set = false;
    if (!attr_set) {
        if (cudaFuncSetAttribute(k_tc_gemm, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 kSmemBytes) != cudaSuccess)
            return -1;
        attr_set = true;
    }
    CUtensorMap ma, mb;
    if (!make_map(&ma, A, K, M, lda, kBM) || !make_map(&mb, B, K, N, ldb, kBN)) return -1;
    const dim3 grid((unsigned)((M + kBM - 1) / kBM), (unsigned)((N + kBN - 1) / kBN));
    k_tc_gemm<<<grid, 128, kSmemBytes, s>>>(M, N, k0, k1, ma, mb, C, ldc, err);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

cudaError_t preload_tc_gemm() { return load_kernels(k_tc_gemm); }

} // namespace mr3
