// tc_gemm.cu -- tcgen05 tensor-core GEMM for the reduced-precision path (sm_103a).
//
//   C (FP32, M x N, row-major) <- beta C + alpha sum_t A_t B_t^T
//
// A_t (M x K) and B_t (N x K) are BF16 or FP16, K-major (row-major with K contiguous).  With one
// term this is the plain low-precision product; with three terms (A_hi B_hi + A_hi B_lo +
// A_lo B_hi, where x = x_hi + x_lo is a two-term split of each FP32 operand) it recovers close
// to FP32 products on the tensor cores.  Uses:
//   - the Schur-complement update E <- E - L21 U12 of eq. (3.1) on the FP32 working matrix
//     (alpha = -1, beta = 1), the dominant contraction of GENP;
//   - M = A G for the reduced-precision working matrix (alpha = 1, beta = 0).
//
// Structure (one 128 x 256 output tile per CTA, 4 warps):
//   warp 0 lane 0: TMA producer -- cp.async.bulk.tensor 2-D loads of 128x64 (A) and 256x64 (B)
//                  tiles, 128-byte swizzled, into a 4-stage shared-memory ring (mbarrier
//                  complete_tx); no multicast: every CTA loads its own tiles.
//   warp 1 lane 0: MMA issuer -- tcgen05.mma.cta_group::1.kind::f16, M=128, N=256, K=16, FP32
//                  accumulator in TMEM (256 columns); tcgen05.commit frees each stage.
//   all 4 warps:   epilogue -- tcgen05.ld 32x32b (each warp owns its 32 TMEM lanes = rows),
//                  C <- beta C + alpha acc with bounds checks.
// Every mbarrier wait is bounded by a %globaltimer deadline; on expiry the CTA records
// RMGE_ERR_TIMEOUT in *err, waits (bounded) for its in-flight copies and MMAs, frees its TMEM
// and returns.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "tc_common.cuh"

namespace rmge {
namespace {

using namespace tc;

constexpr int BM = 128, BN = 256, BK = 64, STAGES = 4;
constexpr int A_BYTES = BM * BK * 2;
constexpr int B_BYTES = BN * BK * 2;
constexpr int STAGE_BYTES = A_BYTES + B_BYTES;
constexpr int TMEM_COLS = 256;
constexpr int THREADS = 128;
constexpr unsigned long long kWaitNs = 2000000000ull;  // 2 s
constexpr size_t kSmemBytes = (size_t)STAGES * STAGE_BYTES + 1024 /*align*/ + 256 /*barriers*/;

struct TcParams {
    int M, N, K, terms;
    float alpha, beta;
    float* C;
    int64_t ldc;
    int* err;
    const unsigned long long* mxa;  // FP16 operand scaling: max|A|, max|B| (NULL: unscaled)
    const unsigned long long* mxb;
};

__global__ void __launch_bounds__(THREADS, 1)
tc_gemm_kernel(const __grid_constant__ CUtensorMap tA0, const __grid_constant__ CUtensorMap tA1,
               const __grid_constant__ CUtensorMap tB0, const __grid_constant__ CUtensorMap tB1, TcParams p,
               uint32_t idesc, const int* halt) {
    if (halt != nullptr && *(volatile const int*)halt != 0) return;
    extern __shared__ __align__(16) uint8_t smem_raw[];
    uint8_t* base = reinterpret_cast<uint8_t*>(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint8_t* sA = base;
    uint8_t* sB = base + STAGES * A_BYTES;
    uint64_t* full = reinterpret_cast<uint64_t*>(base + STAGES * STAGE_BYTES);
    uint64_t* empty = full + STAGES;
    uint64_t* tmem_full = empty + STAGES;
    uint32_t* tmem_holder = reinterpret_cast<uint32_t*>(tmem_full + 1);
    __shared__ int aborted;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
    const int nk = (p.K + BK - 1) / BK;
    const int total = nk * p.terms;

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(full + s, 1);
            mbar_init(empty + s, 1);
        }
        mbar_init(tmem_full, 1);
        aborted = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_holder)),
                     "r"(TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tmem_holder;
    const unsigned long long deadline = now_ns() + kWaitNs;

    if (warp == 0 && lane == 0) {
        // TMA producer
        int issued = 0;
        for (int i = 0; i < total; ++i) {
            const int s = i % STAGES;
            const uint32_t ph = (uint32_t)((i / STAGES) & 1);
            if (!mbar_wait(empty + s, ph ^ 1u, deadline)) {
                atomicExch(&aborted, 1);
                break;
            }
            if (*(volatile int*)&aborted) break;
            const int term = i / nk, kb = i % nk;
            const CUtensorMap* ma = (term == 2) ? &tA1 : &tA0;
            const CUtensorMap* mb = (term == 1) ? &tB1 : &tB0;
            mbar_expect_tx(full + s, STAGE_BYTES);
            tma_load_2d(sA + s * A_BYTES, ma, kb * BK, m0, full + s);
            tma_load_2d(sB + s * B_BYTES, mb, kb * BK, n0, full + s);
            ++issued;
        }
        if (*(volatile int*)&aborted) {
            // drain: wait (bounded) for the copies still in flight
            const unsigned long long d2 = now_ns() + kWaitNs;
            for (int i = issued - STAGES < 0 ? 0 : issued - STAGES; i < issued; ++i)
                (void)mbar_wait(full + i % STAGES, (uint32_t)((i / STAGES) & 1), d2);
        }
    } else if (warp == 1 && lane == 0) {
        // MMA issuer
        for (int i = 0; i < total; ++i) {
            const int s = i % STAGES;
            const uint32_t ph = (uint32_t)((i / STAGES) & 1);
            if (!mbar_wait(full + s, ph, deadline)) {
                atomicExch(&aborted, 1);
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t a0 = smem_u32(sA + s * A_BYTES), b0 = smem_u32(sB + s * B_BYTES);
#pragma unroll
            for (int kk = 0; kk < BK / 16; ++kk) {
                mma_f16(tmem, smem_desc(a0 + kk * 32), smem_desc(b0 + kk * 32), idesc,
                        (i > 0 || kk > 0) ? 1u : 0u);
            }
            mma_commit(empty + s);
        }
        mma_commit(tmem_full);  // arrives once every MMA issued above has completed
    }
    __syncwarp();

    // epilogue
    const bool ok = mbar_wait(tmem_full, 0, now_ns() + kWaitNs);
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    __syncwarp();
    if (!ok) atomicExch(&aborted, 1);
    __syncthreads();
    if (!aborted) {
        const float alpha = p.alpha / (pow2_scale(p.mxa) * pow2_scale(p.mxb));
        const int row = m0 + warp * 32 + lane;
        for (int c = 0; c < BN; c += 32) {
            float v[32];
            tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c, v);
            if (row < p.M) {
                float* crow = p.C + (int64_t)row * p.ldc + n0 + c;
                const int lim = p.N - (n0 + c);
                if (lim >= 32 && ((reinterpret_cast<uintptr_t>(crow) & 15) == 0)) {
#pragma unroll
                    for (int j = 0; j < 32; j += 4) {
                        float4 o = make_float4(alpha * v[j], alpha * v[j + 1], alpha * v[j + 2], alpha * v[j + 3]);
                        if (p.beta != 0.0f) {
                            const float4 c4 = *reinterpret_cast<const float4*>(crow + j);
                            o.x = fmaf(p.beta, c4.x, o.x);
                            o.y = fmaf(p.beta, c4.y, o.y);
                            o.z = fmaf(p.beta, c4.z, o.z);
                            o.w = fmaf(p.beta, c4.w, o.w);
                        }
                        *reinterpret_cast<float4*>(crow + j) = o;
                    }
                } else {
                    for (int j = 0; j < 32 && j < lim; ++j) {
                        const float o = alpha * v[j];
                        crow[j] = (p.beta != 0.0f) ? fmaf(p.beta, crow[j], o) : o;
                    }
                }
            }
        }
    } else if (threadIdx.x == 0 && p.err != nullptr) {
        atomicExch(p.err, (int)RMGE_ERR_TIMEOUT);
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
    }
}

// ---------------------------------------------------------------------------------------------
// Two-term split conversions: x = hi + lo with hi = rn(x), lo = rn(x - hi) in the 16-bit type.
// ---------------------------------------------------------------------------------------------
template <typename L>
__device__ __forceinline__ L to_low(float x);
template <>
__device__ __forceinline__ __nv_bfloat16 to_low<__nv_bfloat16>(float x) { return __float2bfloat16_rn(x); }
template <>
__device__ __forceinline__ __half to_low<__half>(float x) { return __float2half_rn(x); }
template <typename L>
__device__ __forceinline__ float from_low(L x);
template <>
__device__ __forceinline__ float from_low<__nv_bfloat16>(__nv_bfloat16 x) { return __bfloat162float(x); }
template <>
__device__ __forceinline__ float from_low<__half>(__half x) { return __half2float(x); }

// dst (rows x cols, K-major, ldd) from src rows x cols (lds); trans: dst[j][i] = src[i][j].
template <typename S, typename L>
__global__ void split_kernel(int64_t rows, int64_t cols, const S* __restrict__ src, int64_t lds, bool trans,
                             float scale0, const unsigned long long* mx, L* __restrict__ hi, L* __restrict__ lo,
                             int64_t ldd) {
    const float scale = scale0 * pow2_scale(mx);
    const int64_t total = rows * cols;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = e / cols, j = e % cols;  // read along source rows
        const float x = (float)src[i * lds + j] * scale;
        const L h = to_low<L>(x);
        const int64_t d = trans ? j * ldd + i : i * ldd + j;
        hi[d] = h;
        if (lo != nullptr) lo[d] = to_low<L>(x - from_low<L>(h));
    }
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (fn == nullptr) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess) {
            (void)cudaGetLastError();
            return nullptr;
        }
        fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    }
    return fn;
}

bool make_map(CUtensorMap* m, const void* ptr, bool bf16, int64_t rows, int64_t k, int64_t ld, int box_rows) {
    auto fn = encode_fn();
    if (fn == nullptr) return false;
    cuuint64_t dims[2] = {(cuuint64_t)k, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)ld * 2};
    cuuint32_t box[2] = {(cuuint32_t)BK, (cuuint32_t)box_rows};
    cuuint32_t estr[2] = {1, 1};
    const CUresult r = fn(m, bf16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 2,
                          const_cast<void*>(ptr), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                          CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

}  // namespace

bool tc_make_map(CUtensorMap* m, const void* ptr, bool bf16, int64_t rows, int64_t k, int64_t ld, int box_rows) {
    return make_map(m, ptr, bf16, rows, k, ld, box_rows);
}

uint32_t tc_idesc(bool bf16) {
    uint32_t d = 0;
    d |= 1u << 4;                        // D format: FP32
    d |= (bf16 ? 1u : 0u) << 7;          // A format: BF16 (1) or FP16 (0)
    d |= (bf16 ? 1u : 0u) << 10;         // B format
    // bits 15/16 = 0: A and B K-major
    d |= (uint32_t)(BN >> 3) << 17;      // N / 8
    d |= (uint32_t)(BM >> 4) << 24;      // M / 16
    return d;
}

template <typename S>
rmge_status tc_split(int64_t rows, int64_t cols, const S* src, int64_t lds, bool trans, float scale,
                     const unsigned long long* mx, bool bf16, void* hi, void* lo, int64_t ldd, cudaStream_t s) {
    int64_t g = (rows * cols + 255) / 256;
    if (g > 152 * 16) g = 152 * 16;
    if (g < 1) g = 1;
    if (bf16)
        split_kernel<S, __nv_bfloat16><<<(unsigned)g, 256, 0, s>>>(rows, cols, src, lds, trans, scale, mx,
                                                                  static_cast<__nv_bfloat16*>(hi),
                                                                  static_cast<__nv_bfloat16*>(lo), ldd);
    else
        split_kernel<S, __half><<<(unsigned)g, 256, 0, s>>>(rows, cols, src, lds, trans, scale, mx,
                                                           static_cast<__half*>(hi), static_cast<__half*>(lo), ldd);
    RMGE_LAUNCH_CHECK();
    return RMGE_OK;
}

rmge_status tc_gemm(int64_t M, int64_t N, int64_t K, int terms, bool bf16, const void* A0, const void* A1, int64_t lda,
                    const void* B0, const void* B1, int64_t ldb, float alpha, float beta, float* C, int64_t ldc,
                    int* err, const int* halt, const unsigned long long* mxa, const unsigned long long* mxb,
                    cudaStream_t s) {
    if (M <= 0 || N <= 0) return RMGE_OK;
    if (K <= 0 || (terms != 1 && terms != 3) || (lda % 8) != 0 || (ldb % 8) != 0 || M > INT32_MAX / 2 ||
        N > INT32_MAX / 2 || K > INT32_MAX / 2)
        return RMGE_ERR_INVALID_ARG;
    if ((((uintptr_t)A0 | (uintptr_t)B0 | (terms == 3 ? ((uintptr_t)A1 | (uintptr_t)B1) : 0)) & 15) != 0)
        return RMGE_ERR_INVALID_ARG;
    CUtensorMap ta0, ta1, tb0, tb1;
    if (!make_map(&ta0, A0, bf16, M, K, lda, BM) || !make_map(&tb0, B0, bf16, N, K, ldb, BN)) return RMGE_ERR_CUDA;
    if (terms == 3) {
        if (!make_map(&ta1, A1, bf16, M, K, lda, BM) || !make_map(&tb1, B1, bf16, N, K, ldb, BN)) return RMGE_ERR_CUDA;
    } else {
        ta1 = ta0;
        tb1 = tb0;
    }
    if (cudaFuncSetAttribute(tc_gemm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemBytes) !=
        cudaSuccess) {
        (void)cudaGetLastError();
        return RMGE_ERR_CUDA;
    }
    TcParams prm{(int)M, (int)N, (int)K, terms, alpha, beta, C, ldc, err, mxa, mxb};
    const dim3 grid((unsigned)((N + BN - 1) / BN), (unsigned)((M + BM - 1) / BM));
    tc_gemm_kernel<<<grid, THREADS, kSmemBytes, s>>>(ta0, ta1, tb0, tb1, prm, tc_idesc(bf16), halt);
    RMGE_LAUNCH_CHECK();
    return RMGE_OK;
}

template rmge_status tc_split<float>(int64_t, int64_t, const float*, int64_t, bool, float, const unsigned long long*,
                                     bool, void*, void*, int64_t, cudaStream_t);
template rmge_status tc_split<double>(int64_t, int64_t, const double*, int64_t, bool, float, const unsigned long long*,
                                      bool, void*, void*, int64_t, cudaStream_t);

}  // namespace rmge
