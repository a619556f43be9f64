// oz_gemm.cu -- FP64 matrix products emulated on the tcgen05 BF16 tensor cores (Ozaki-type splitting).
//
// GB300 executes FP64 only on its DFMA pipe (about 1.2 TFLOP/s) while its BF16 tensor cores run
// about 1.9 PFLOP/s.  An FP64 product C = alpha A B + beta C is rebuilt from exact integer products:
//   - every row i of A gets an exponent ea_i with max_k |A_ik| < 2^ea_i, every column j of B an eb_j;
//   - x = A_ik 2^-ea_i (|x| < 1) is truncated to s base-128 digits, x ~ sign * sum_p d_p 128^-(p+1),
//     0 <= d_p <= 127, and digit plane p is stored as BF16 (exact: integers below 256);
//   - digit products d_p e_q are below 2^14; the d + 1 digit pairs of one diagonal d = p + q share a
//     TMEM accumulator over a K chunk short enough that (d + 1) 127^2 kc < 2^24, so the tensor core's
//     FP32 accumulation of every chunk is exact (kc = 1024, 512, ..., 128 for d = 0 .. 7);
//   - each chunk result (an exact integer) is added, shifted to its weight 128^-(d+2), into a 64-bit
//     fixed-point accumulator per output element (integer work, not FP64): F fractional bits of
//     max|A_i.| max|B_.j| with F = 52 - log2(chunks on diagonal 0 + 1), i.e. 51 bits up to K = 1024;
//   - C_ij = 2^(ea_i + eb_j - F) acc, combined with beta C in FP64 once per element.
// Digit pairs with p + q <= s - 1 are kept.  The first dropped diagonal (p + q = s) is worth about
// (s + 1) 2^(-7s) of max|A_i.| max|B_.j| per term, so s = 8 (36 digit pairs) matches FP64 rounding.
//
// Kernel: one 128 x 128 output tile per CTA, 10 warps.  Warp 8 (one lane) streams 128x64 BF16 tiles
// of A-digit and B-digit planes by TMA into a 6-stage ring; warp 9 (one lane) issues
// tcgen05.mma kind::f16 (M=128, N=128, K=16) into one of two 128-column TMEM accumulators, one
// (diagonal, K chunk) unit at a time; warps 0-7 drain the other accumulator (tcgen05.ld) into their
// fixed-point registers while the next unit accumulates.  All waits are bounded.
#include <cuda_bf16.h>

#include "tc_common.cuh"

namespace rmge {
namespace {

using namespace tc;

constexpr int OBM = 128, OBN = 128, OBK = 64, OSTAGES = 6;
constexpr int OA_BYTES = OBM * OBK * 2;
constexpr int OB_BYTES = OBN * OBK * 2;
constexpr int OSTAGE_BYTES = OA_BYTES + OB_BYTES;
constexpr int OTHREADS = 320;
constexpr int OTMEM = 256;
constexpr unsigned long long kOzWaitNs = 4000000000ull;
constexpr size_t kOzSmem = (size_t)OSTAGES * OSTAGE_BYTES + 1024 + 512;

struct OzParams {
    int M, N, K, s;
    int F;  // fractional bits of the fixed-point accumulator
    int Mp, Np;  // rows per digit plane of A, of B
    const int* ea;
    const int* eb;
    double alpha, beta;
    double* C;
    int64_t ldc;
    int* err;
    const int* halt;
};

// Depth of one exact chunk on diagonal d = p + q: the (d + 1) digit pairs of the diagonal share one
// TMEM accumulator, so (d + 1) 127^2 kc must stay below 2^24 (kc a multiple of the 64-deep K block).
__device__ __forceinline__ int diag_kc(int d) {
    constexpr int kc[8] = {1024, 512, 320, 256, 192, 128, 128, 128};
    return kc[d];
}

__global__ void __launch_bounds__(OTHREADS, 1)
oz_gemm_kernel(const __grid_constant__ CUtensorMap tA, const __grid_constant__ CUtensorMap tB, OzParams p,
               uint32_t idesc) {
    if (p.halt != nullptr && *(volatile const int*)p.halt != 0) return;
    extern __shared__ __align__(16) uint8_t smem_raw[];
    uint8_t* base = reinterpret_cast<uint8_t*>(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint8_t* sA = base;
    uint8_t* sB = base + OSTAGES * OA_BYTES;
    uint64_t* full = reinterpret_cast<uint64_t*>(base + OSTAGES * OSTAGE_BYTES);
    uint64_t* empty = full + OSTAGES;
    uint64_t* tfull = empty + OSTAGES;   // [2]
    uint64_t* tempty = tfull + 2;        // [2]
    uint32_t* tmem_holder = reinterpret_cast<uint32_t*>(tempty + 2);
    __shared__ int aborted;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int m0 = blockIdx.y * OBM, n0 = blockIdx.x * OBN;

    if (threadIdx.x == 0) {
        for (int s = 0; s < OSTAGES; ++s) {
            mbar_init(full + s, 1);
            mbar_init(empty + s, 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(tfull + b, 1);
            mbar_init(tempty + b, 8);
        }
        aborted = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_holder)),
                     "r"(OTMEM)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tmem_holder;
    const unsigned long long deadline = now_ns() + kOzWaitNs;

    if (warp == 8) {
        if (lane == 0) {  // TMA producer: units (d, chunk), then pairs p + q = d, then 64-deep K blocks
            int it = 0;
            for (int d = 0; d < p.s && !*(volatile int*)&aborted; ++d) {
                const int kc = diag_kc(d);
                for (int k0 = 0; k0 < p.K && !*(volatile int*)&aborted; k0 += kc) {
                    const int nkb = ((p.K - k0 < kc ? p.K - k0 : kc) + OBK - 1) / OBK;
                    for (int pa = 0; pa <= d; ++pa) {
                        const int ya = pa * p.Mp + m0, yb = (d - pa) * p.Np + n0;
                        for (int kb = 0; kb < nkb; ++kb, ++it) {
                            const int st = it % OSTAGES;
                            if (!mbar_wait(empty + st, (uint32_t)(((it / OSTAGES) & 1) ^ 1), deadline)) {
                                atomicExch(&aborted, 1);
                                break;
                            }
                            mbar_expect_tx(full + st, OSTAGE_BYTES);
                            tma_load_2d(sA + st * OA_BYTES, &tA, k0 + kb * OBK, ya, full + st);
                            tma_load_2d(sB + st * OB_BYTES, &tB, k0 + kb * OBK, yb, full + st);
                        }
                        if (*(volatile int*)&aborted) break;
                    }
                }
            }
            // drain: the last copies issued must land before the CTA can leave
            const unsigned long long d2 = now_ns() + kOzWaitNs;
            for (int j = it - OSTAGES < 0 ? 0 : it - OSTAGES; j < it; ++j)
                (void)mbar_wait(full + j % OSTAGES, (uint32_t)((j / OSTAGES) & 1), d2);
        }
    } else if (warp == 9) {
        if (lane == 0) {  // MMA issuer: one TMEM accumulator per unit (d, chunk), alternating buffers
            int it = 0, u = 0;
            bool ok = true;
            for (int d = 0; d < p.s && ok; ++d) {
                const int kc = diag_kc(d);
                for (int k0 = 0; k0 < p.K && ok; k0 += kc, ++u) {
                    const int buf = u & 1;
                    if (!mbar_wait(tempty + buf, (uint32_t)(((u >> 1) & 1) ^ 1), deadline)) {
                        atomicExch(&aborted, 1);
                        ok = false;
                        break;
                    }
                    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                    const int nkb = ((p.K - k0 < kc ? p.K - k0 : kc) + OBK - 1) / OBK;
                    for (int pa = 0; pa <= d && ok; ++pa) {
                        for (int kb = 0; kb < nkb; ++kb, ++it) {
                            const int st = it % OSTAGES;
                            if (!mbar_wait(full + st, (uint32_t)((it / OSTAGES) & 1), deadline)) {
                                atomicExch(&aborted, 1);
                                ok = false;
                                break;
                            }
                            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                            const uint32_t a0 = smem_u32(sA + st * OA_BYTES), b0 = smem_u32(sB + st * OB_BYTES);
#pragma unroll
                            for (int kk = 0; kk < OBK / 16; ++kk)
                                mma_f16(tmem + (uint32_t)(buf * 128), smem_desc(a0 + kk * 32), smem_desc(b0 + kk * 32),
                                        idesc, (pa > 0 || kb > 0 || kk > 0) ? 1u : 0u);
                            mma_commit(empty + st);
                        }
                    }
                    mma_commit(tfull + buf);
                }
            }
        }
    } else {
        // epilogue warps 0-7: quadrant (TMEM lanes / tile rows) and column half
        const int quad = warp & 3, half = warp >> 2;
        long long acc[64];  // fixed point: units of 2^-F of max|A_i.| max|B_.j|
#pragma unroll
        for (int j = 0; j < 64; ++j) acc[j] = 0;
        int u = 0;
        bool ok = true;
        for (int d = 0; d < p.s && ok; ++d) {
            const int kc = diag_kc(d);
            const int sh = p.F - 7 * (d + 2);  // chunk value v weighs 2^-(7(d+2)) = 2^(sh - F)
            for (int k0 = 0; k0 < p.K; k0 += kc, ++u) {
                const int buf = u & 1;
                if (!mbar_wait(tfull + buf, (uint32_t)((u >> 1) & 1), deadline)) {
                    atomicExch(&aborted, 1);
                    ok = false;
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                __syncwarp();
                const uint32_t taddr = tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)(buf * 128 + half * 64);
#pragma unroll
                for (int cc = 0; cc < 2; ++cc) {
                    float v[32];
                    tmem_ld32(taddr + cc * 32, v);
#pragma unroll
                    for (int j = 0; j < 32; ++j) {
                        const long long t = __float2ll_rn(v[j]);  // exact: |v| < 2^24 is an integer
                        acc[cc * 32 + j] += (sh >= 0) ? (t << sh) : ((t + (1ll << (-sh - 1))) >> (-sh));
                    }
                }
                asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
                __syncwarp();
                if (lane == 0) mbar_arrive(tempty + buf);
            }
        }
        if (!aborted) {
            const int row = m0 + quad * 32 + lane;
            if (row < p.M) {
                const int er = p.ea[row];
                double* crow = p.C + (int64_t)row * p.ldc;
#pragma unroll
                for (int j = 0; j < 64; ++j) {
                    const int col = n0 + half * 64 + j;
                    if (col < p.N) {
                        const double v = ldexp((double)acc[j], er + p.eb[col] - p.F);
                        crow[col] = (p.beta == 0.0) ? p.alpha * v : fma(p.beta, crow[col], p.alpha * v);
                    }
                }
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (aborted && threadIdx.x == 0 && p.err != nullptr) atomicExch(p.err, (int)RMGE_ERR_TIMEOUT);
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(OTMEM) : "memory");
}

// ---------------------------------------------------------------------------------------------
// Digit planes.  Row (trans = false) or column (trans = true) exponents of the source, then s BF16
// planes of rows_p x kp (K-major, zero padded): plane[p][r][k].
// ---------------------------------------------------------------------------------------------

__device__ __forceinline__ int line_exp(double m) { return (m > 0.0 && isfinite(m)) ? ilogb(m) + 1 : 0; }

// e[r] = smallest integer with max_k |A_rk| < 2^e (0 for an all-zero row): one warp per row.
__global__ void row_exponent_kernel(int64_t rows, int64_t cols, const double* __restrict__ src, int64_t lds,
                                    int* __restrict__ e) {
    const int lane = threadIdx.x & 31;
    const int64_t r = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    if (r >= rows) return;
    double m = 0.0;
    for (int64_t k = lane; k < cols; k += 32) m = fmax(m, fabs(src[r * lds + k]));
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    if (lane == 0) e[r] = line_exp(m);
}

// e[c] = the same for column c: one thread per column, consecutive threads on consecutive columns.
__global__ void col_exponent_kernel(int64_t rows, int64_t cols, const double* __restrict__ src, int64_t lds,
                                    int* __restrict__ e) {
    const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (c >= cols) return;
    double m = 0.0;
    for (int64_t k = 0; k < rows; ++k) m = fmax(m, fabs(src[k * lds + c]));
    e[c] = line_exp(m);
}

// The 7s-bit magnitude |x| 2^(7s), x = v 2^-e, by integer shifts of the FP64 significand.
__device__ __forceinline__ unsigned long long fixed_digits(double v, int e, int s) {
    const unsigned long long bits = (unsigned long long)__double_as_longlong(v);
    const int be = (int)((bits >> 52) & 0x7FF);
    unsigned long long m = bits & 0xFFFFFFFFFFFFFull;
    int ex;
    if (be == 0) {  // zero or subnormal
        if (m == 0) return 0ull;
        ex = -1022 - 52;
    } else {
        m |= 1ull << 52;
        ex = be - 1023 - 52;
    }
    const int sh = ex - e + 7 * s;  // |v| 2^(7s - e) = m 2^sh
    if (sh >= 0) return m << sh;  // |x| < 1 keeps this below 2^(7s) <= 2^56: sh <= 3
    return (-sh >= 64) ? 0ull : (m >> (-sh));
}

__device__ __forceinline__ void store_digits(double v, int er, int s, __nv_bfloat16* dst, int64_t plane) {
    if (!isfinite(v)) {  // a NaN in the leading plane makes every product it enters NaN
        dst[0] = __float2bfloat16_rn(__int_as_float(0x7fc00000));
        for (int q = 1; q < s; ++q) dst[(int64_t)q * plane] = __float2bfloat16_rn(0.0f);
        return;
    }
    const unsigned long long X = fixed_digits(v, er, s);
    const float sg = (v < 0.0) ? -1.0f : 1.0f;
    for (int q = 0; q < s; ++q) {
        const unsigned d = (unsigned)((X >> (7 * (s - 1 - q))) & 127ull);
        dst[(int64_t)q * plane] = __float2bfloat16_rn(sg * (float)d);
    }
}

// Row digits: plane[q][r][k] = digit q of A_rk (rows_p x kp per plane, zero padded).
__global__ void row_digits_kernel(int64_t rows, int64_t cols, const double* __restrict__ src, int64_t lds,
                                  const int* __restrict__ e, int s, int64_t rows_p, int64_t kp,
                                  __nv_bfloat16* __restrict__ planes) {
    const int64_t total = rows_p * kp;
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = idx / kp, k = idx % kp;
        const bool in = r < rows && k < cols;
        store_digits(in ? src[r * lds + k] : 0.0, in ? e[r] : 0, s, planes + idx, total);
    }
}

// Column digits, transposed through shared memory: plane[q][c][k] = digit q of B_kc.
__global__ void col_digits_kernel(int64_t rows, int64_t cols, const double* __restrict__ src, int64_t lds,
                                  const int* __restrict__ e, int s, int64_t cols_p, int64_t kp,
                                  __nv_bfloat16* __restrict__ planes) {
    __shared__ double t[32][33];
    const int64_t k0 = (int64_t)blockIdx.y * 32, c0 = (int64_t)blockIdx.x * 32;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 32 x 8 threads
    for (int i = ty; i < 32; i += 8) {
        const int64_t k = k0 + i, c = c0 + tx;
        t[i][tx] = (k < rows && c < cols) ? src[k * lds + c] : 0.0;
    }
    __syncthreads();
    const int64_t total = cols_p * kp;
    for (int i = ty; i < 32; i += 8) {
        const int64_t c = c0 + i, k = k0 + tx;  // write along k
        if (c < cols_p && k < kp) store_digits(t[tx][i], c < cols ? e[c] : 0, s, planes + c * kp + k, total);
    }
}

unsigned grid_for(int64_t work) {
    int64_t g = (work + 255) / 256;
    if (g > 152 * 16) g = 152 * 16;
    return (unsigned)(g < 1 ? 1 : g);
}

}  // namespace

size_t oz_plane_bytes(int64_t rows, int64_t k, int s) {
    const int64_t rp = (rows + 127) / 128 * 128, kp = (k + 63) / 64 * 64;
    return (size_t)s * (size_t)rp * (size_t)kp * 2;
}

rmge_status oz_gemm(int64_t M, int64_t N, int64_t K, int s, double alpha, const double* A, int64_t lda,
                    const double* B, int64_t ldb, double beta, double* C, int64_t ldc, void* planesA, void* planesB,
                    int* ea, int* eb, int* err, const int* halt, cudaStream_t st) {
    if (M <= 0 || N <= 0) return RMGE_OK;
    if (K <= 0 || s < 1 || s > 8 || M > INT32_MAX / 16 || N > INT32_MAX / 16 || K > INT32_MAX / 2)
        return RMGE_ERR_INVALID_ARG;
    const int64_t Mp = (M + 127) / 128 * 128, Np = (N + 127) / 128 * 128, Kp = (K + 63) / 64 * 64;
    __nv_bfloat16* pa = static_cast<__nv_bfloat16*>(planesA);
    __nv_bfloat16* pb = static_cast<__nv_bfloat16*>(planesB);
    row_exponent_kernel<<<(unsigned)((M * 32 + 255) / 256), 256, 0, st>>>(M, K, A, lda, ea);
    RMGE_LAUNCH_CHECK();
    col_exponent_kernel<<<(unsigned)((N + 255) / 256), 256, 0, st>>>(K, N, B, ldb, eb);
    RMGE_LAUNCH_CHECK();
    row_digits_kernel<<<grid_for(Mp * Kp), 256, 0, st>>>(M, K, A, lda, ea, s, Mp, Kp, pa);
    RMGE_LAUNCH_CHECK();
    col_digits_kernel<<<dim3((unsigned)(Np / 32), (unsigned)(Kp / 32)), 256, 0, st>>>(K, N, B, ldb, eb, s, Np, Kp, pb);
    RMGE_LAUNCH_CHECK();

    CUtensorMap ta, tb;
    if (!tc_make_map(&ta, pa, true, (int64_t)s * Mp, Kp, Kp, OBM) || !tc_make_map(&tb, pb, true, (int64_t)s * Np, Kp, Kp, OBN))
        return RMGE_ERR_CUDA;
    OzParams prm{};
    prm.M = (int)M;
    prm.N = (int)N;
    prm.K = (int)Kp;
    prm.s = s;
    // |acc| < (chunks on diagonal 0 + 1) 2^(F + 10) must stay below 2^62
    int ch0 = (int)((Kp + 1023) / 1024), lg = 0;
    while ((1 << lg) < ch0 + 1) ++lg;
    prm.F = 52 - lg;
    prm.Mp = (int)Mp;
    prm.Np = (int)Np;
    prm.ea = ea;
    prm.eb = eb;
    prm.alpha = alpha;
    prm.beta = beta;
    prm.C = C;
    prm.ldc = ldc;
    prm.err = err;
    prm.halt = halt;
    // idesc: FP32 accumulate, BF16 A and B, both K-major, N = 128, M = 128
    const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(OBN >> 3) << 17) |
                           ((uint32_t)(OBM >> 4) << 24);
    if (cudaFuncSetAttribute(oz_gemm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kOzSmem) != cudaSuccess) {
        (void)cudaGetLastError();
        return RMGE_ERR_CUDA;
    }
    const dim3 grid((unsigned)(Np / OBN), (unsigned)(Mp / OBM));
    oz_gemm_kernel<<<grid, OTHREADS, kOzSmem, st>>>(ta, tb, prm, idesc);
    RMGE_LAUNCH_CHECK();
    return RMGE_OK;
}

}  // namespace rmge
