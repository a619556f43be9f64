// oz_gemm.cu -- FP64 matrix products emulated on the tcgen05 BF16 tensor cores (Ozaki-type splitting).
//
// GB300 executes FP64 only on its DFMA pipe (about 1.2 TFLOP/s) while its BF16 tensor cores run
// about 1.9 PFLOP/s.  An FP64 product C = alpha A B + beta C is rebuilt from exact integer products:
//   - every row i of A gets an exponent ea_i with max_k |A_ik| < 2^ea_i, every column j of B an eb_j;
//   - x = A_ik 2^-ea_i (|x| < 1) is truncated to 8s - 1 bits, X = |x| 2^(8s-1) < 2^(8s-1), and X is
//     written in s balanced base-256 digits, X = sum_p D_p 256^(s-1-p) with -128 <= D_p <= 128 (carries
//     from the low digits keep each digit within half a base; the top digit stays at most 128 because
//     X < 2^(8s-1)), so x ~ sign * sum_p D_p 2^(1 - 8(p+1)); digit plane p holds sign * D_p as BF16
//     (exact: BF16 carries every integer up to 256 in magnitude);
//   - digit products are at most 2^14 in magnitude; the d + 1 digit pairs of one diagonal d = p + q
//     share a TMEM accumulator over a K chunk short enough that (d + 1) 2^14 kc <= 2^24, so the tensor
//     core's FP32 accumulation of every chunk is exact (kc = 1024, 512, 256, 256, 128, 128, 128 for
//     d = 0 .. 6);
//   - each chunk result (an exact integer) is added, shifted to its weight 2^(2 - 8(d+2)), into a 64-bit
//     fixed-point accumulator per output element (integer work, not FP64): F fractional bits of
//     max|A_i.| max|B_.j| with F = 52 - log2(chunks on diagonal 0 + 1), i.e. 51 bits up to K = 1024;
//   - C_ij = 2^(ea_i + eb_j - F) acc, combined with beta C in FP64 once per element.
// Digit pairs with p + q <= s - 1 are kept.  The first dropped diagonal (p + q = s) is worth about
// (s + 1) 2^(-8s) of max|A_i.| max|B_.j| per term, so s = 7 (28 digit pairs, 55 bits per operand)
// matches FP64 rounding.  Balanced digits use all eight bits that BF16 holds exactly; unsigned base-128
// digits needed 8 digits and 36 pairs for the same accuracy.
//
// Kernel: one 128 x 128 output tile per CTA, 18 warps.  Warp 16 (one lane) streams 128x64 BF16 tiles
// of A-digit and B-digit planes by TMA into a 6-stage ring; warp 17 (one lane) issues
// tcgen05.mma kind::f16 (M=128, N=128, K=16) into one of two 128-column TMEM accumulators, one
// (diagonal, K chunk) unit at a time; warps 0-15 drain the other accumulator (tcgen05.ld, 32 columns
// each) into their fixed-point registers while the next unit accumulates, then stage the scaled tile in
// the idle ring and update C one row per warp.  All waits are bounded.
#include <cuda_bf16.h>

#include <algorithm>
#include <climits>

#include "pivot_block.cuh"
#include "tc_common.cuh"

namespace rmge {
namespace {

using namespace tc;

// OBK: the K extent of one TMA box (64 BF16 = one 128-byte swizzle span, also the planes' K padding and
// the update kernel's whole K); OKS: the K depth of one ring stage of the general kernel, two boxes per
// operand, so that each stage feeds 8 MMAs and the per-stage waits and commits are paid half as often.
constexpr int OBM = 128, OBN = 128, OBK = 64, OKS = 128, OSTAGES = 3;
constexpr int OBOX_A = OBM * OBK * 2;   // one 128 x 64 BF16 box, 16 KB
constexpr int OBOX_B = OBN * OBK * 2;
constexpr int OA_BYTES = OBM * OKS * 2;
constexpr int OB_BYTES = OBN * OKS * 2;
constexpr int OSTAGE_BYTES = OA_BYTES + OB_BYTES;
constexpr int OEPI = 16;                    // epilogue warps: 4 TMEM lane quadrants x 4 column groups of 32
constexpr int OTHREADS = (OEPI + 2) * 32;   // + the TMA producer warp and the MMA warp
constexpr int OSTG = OBN + 1;               // row stride (doubles) of the staged output tile
constexpr int OTMEM = 256;
constexpr unsigned long long kOzWaitNs = 4000000000ull;
constexpr size_t kOzSmem = (size_t)OSTAGES * OSTAGE_BYTES + 1024 + 512;
static_assert((size_t)OBM * OSTG * sizeof(double) <= (size_t)OSTAGES * OSTAGE_BYTES, "staged tile must fit the ring");

struct OzParams {
    int M, N, K, s;
    int F;  // fractional bits of the fixed-point accumulator
    int Mp, Np;  // rows per digit plane of A, of B
    int64_t sC;  // elements between the C of successive systems (blockIdx.y); their planes and exponents
                 // follow one another in blocks of s Mp (s Np) plane rows and Mp (Np) exponents
    const int* ea;
    const int* eb;
    double alpha, beta;  // general combine (mode 2): C = beta C + alpha v
    long long alpha_sign;  // modes 0 and 1: alpha = alpha_sign = +-1 is applied to the fixed-point sum
    int mode;              // 0: C = alpha A B; 1: C += alpha A B; 2: general alpha, beta
    double* C;
    int64_t ldc;
    int* err;
    const int* halt;
};

// Depth of one exact chunk on diagonal d = p + q: the (d + 1) digit pairs of the diagonal share one
// TMEM accumulator, so (d + 1) 127^2 kc must stay below 2^24; kc is a multiple of the 64-deep K block
// and divides the 1024-deep super-chunk.  The K loop runs over super-chunks and, inside each, over all
// diagonals, so the digit planes of one super-chunk are re-read for every diagonal while they are still
// in L2 (a diagonal-major order re-fetched plane q from DRAM for every diagonal d >= q).
constexpr int kSuper = 1024;
__device__ __forceinline__ int diag_kc(int d) {
    constexpr int kc[kOzSlices] = {1024, 512, 256, 256, 128, 128, 128};
    return kc[d];
}

// Grouped tile order: bands of kGroupM row blocks, column-major inside a band, so the CTAs resident at
// one time cover a roughly square patch of C (fewer distinct A and B panels per wave).
constexpr int kGroupM = 12;
__device__ __forceinline__ void tile_of(int t, int tm, int tn, int& m, int& n) {
    const int per = kGroupM * tn, g = t / per, first = g * kGroupM;
    const int gm = (tm - first < kGroupM) ? tm - first : kGroupM;
    const int tl = t - g * per;
    m = first + tl % gm;
    n = tl / gm;
}

// a 2^E rounded to the nearest FP64 value (ties to even), assembled from the IEEE-754 fields with
// integer operations only: GB300's FP64 pipe retires 2 operations per clock per SM, so the integer
// -> FP64 conversion and the scaling are kept off it.  Results that would be subnormal or overflow
// take the FP64 route.
__device__ __forceinline__ double fixed_to_double(long long a, int E) {
    const unsigned long long sgn = (unsigned long long)a & 0x8000000000000000ull;
    const unsigned long long m = a < 0 ? 0ull - (unsigned long long)a : (unsigned long long)a;
    if (m == 0) return 0.0;
    // normalise the leading bit to bit 63, keep 53 bits and round the 11 below them to nearest even
    const int lz = __clzll((long long)m);
    const unsigned long long mn = m << lz;
    const unsigned long long keep = mn >> 11, rest = mn & 0x7FFull;
    const unsigned long long q = keep + (unsigned long long)((rest > 0x400ull) | ((rest == 0x400ull) & (keep & 1ull)));
    const int ex = 63 - lz + E + 1023;  // biased exponent before a rounding carry
    if (ex <= 0 || ex >= 2046) return ldexp((double)a, E);
    // q in [2^52, 2^53]: its leading bit adds one to (ex - 1), and a carry to 2^53 one more
    return __longlong_as_double((long long)(sgn | (((unsigned long long)(ex - 1) << 52) + q)));
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
    int tmb, tnb;
    tile_of((int)blockIdx.x, p.Mp / OBM, p.Np / OBN, tmb, tnb);
    const int m0 = tmb * OBM, n0 = tnb * OBN;
    // the system of a batched product: its plane rows start at z s Mp (A) and z s Np (B)
    const int z = (int)blockIdx.y, zra = z * p.s * p.Mp, zrb = z * p.s * p.Np;
    double* const Cz = p.C + (int64_t)z * p.sC;
    const int* const eaz = p.ea + (int64_t)z * p.Mp;
    const int* const ebz = p.eb + (int64_t)z * p.Np;

    if (threadIdx.x == 0) {
        for (int s = 0; s < OSTAGES; ++s) {
            mbar_init(full + s, 1);
            mbar_init(empty + s, 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(tfull + b, 1);
            mbar_init(tempty + b, OEPI);
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

    if (warp == OEPI) {
        if (lane == 0) {  // TMA producer: units (d, chunk), then pairs p + q = d, then 64-deep K blocks
            int it = 0;
            for (int sc = 0; sc < p.K && !*(volatile int*)&aborted; sc += kSuper)
            for (int d = 0; d < p.s && !*(volatile int*)&aborted; ++d) {
                const int kc = diag_kc(d), se = (p.K - sc < kSuper) ? p.K : sc + kSuper;
                for (int k0 = sc; k0 < se && !*(volatile int*)&aborted; k0 += kc) {
                    const int nkb = ((se - k0 < kc ? se - k0 : kc) + OKS - 1) / OKS;
                    for (int pa = 0; pa <= d; ++pa) {
                        const int ya = zra + pa * p.Mp + m0, yb = zrb + (d - pa) * p.Np + n0;
                        for (int kb = 0; kb < nkb; ++kb, ++it) {
                            const int st = it % OSTAGES;
                            if (!mbar_wait_idle(empty + st, (uint32_t)(((it / OSTAGES) & 1) ^ 1), deadline)) {
                                atomicExch(&aborted, 1);
                                break;
                            }
                            // two 64-deep boxes per operand; a box past the padded K reads zeros
                            const int kx = k0 + kb * OKS;
                            mbar_expect_tx(full + st, OSTAGE_BYTES);
                            tma_load_2d(sA + st * OA_BYTES, &tA, kx, ya, full + st);
                            tma_load_2d(sA + st * OA_BYTES + OBOX_A, &tA, kx + OBK, ya, full + st);
                            tma_load_2d(sB + st * OB_BYTES, &tB, kx, yb, full + st);
                            tma_load_2d(sB + st * OB_BYTES + OBOX_B, &tB, kx + OBK, yb, full + st);
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
    } else if (warp == OEPI + 1) {
        if (lane == 0) {  // MMA issuer: one TMEM accumulator per unit (d, chunk), alternating buffers
            int it = 0, u = 0;
            bool ok = true;
            for (int sc = 0; sc < p.K && ok; sc += kSuper)
            for (int d = 0; d < p.s && ok; ++d) {
                const int kc = diag_kc(d), se = (p.K - sc < kSuper) ? p.K : sc + kSuper;
                for (int k0 = sc; k0 < se && ok; k0 += kc, ++u) {
                    const int buf = u & 1;
                    if (!mbar_wait(tempty + buf, (uint32_t)(((u >> 1) & 1) ^ 1), deadline)) {
                        atomicExch(&aborted, 1);
                        ok = false;
                        break;
                    }
                    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                    const int nkb = ((se - k0 < kc ? se - k0 : kc) + OKS - 1) / OKS;
                    for (int pa = 0; pa <= d && ok; ++pa) {
                        for (int kb = 0; kb < nkb; ++kb, ++it) {
                            const int st = it % OSTAGES;
                            if (!mbar_wait(full + st, (uint32_t)((it / OSTAGES) & 1), deadline)) {
                                atomicExch(&aborted, 1);
                                ok = false;
                                break;
                            }
                            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                            // 32-byte K steps inside a swizzled box advance the descriptors' address field by 2
#pragma unroll
                            for (int h = 0; h < OKS / OBK; ++h) {
                                const uint64_t ad = smem_desc(smem_u32(sA + st * OA_BYTES + h * OBOX_A)),
                                               bd = smem_desc(smem_u32(sB + st * OB_BYTES + h * OBOX_B));
#pragma unroll
                                for (int kk = 0; kk < OBK / 16; ++kk)
                                    mma_f16(tmem + (uint32_t)(buf * 128), ad + 2 * kk, bd + 2 * kk, idesc,
                                            (pa > 0 || kb > 0 || h > 0 || kk > 0) ? 1u : 0u);
                            }
                            mma_commit(empty + st);
                        }
                    }
                    mma_commit(tfull + buf);
                }
            }
        }
    } else {
        // epilogue warps 0-15: TMEM lane quadrant (tile rows) and group of 32 columns
        const int quad = warp & 3, cg = warp >> 2;
        long long acc[32];  // fixed point: units of 2^-F of max|A_i.| max|B_.j|
#pragma unroll
        for (int j = 0; j < 32; ++j) acc[j] = 0;
        int u = 0;
        bool ok = true;
        for (int sc = 0; sc < p.K && ok; sc += kSuper)
        for (int d = 0; d < p.s && ok; ++d) {
            const int kc = diag_kc(d), se = (p.K - sc < kSuper) ? p.K : sc + kSuper;
            // chunk value v weighs 2^(2 - 8(d+2)) = 2^(sh - F).  v is an integer of magnitude at most 2^24,
            // converted to int32 (the FP32 -> int64 conversion runs on GB300's narrow FP64 pipe; this one
            // does not).  Right shifts (sh < 0) are done exactly in FP32 (a power-of-two scaling of an
            // integer) and rounded to the nearest integer by the conversion; left shifts in 64-bit integers.
            const int sh = p.F - 8 * d - 14;
            const float rscale = __int_as_float((127 + (sh < 0 ? sh : 0)) << 23);
            const int lsh = sh > 0 ? sh : 0;
            for (int k0 = sc; k0 < se; k0 += kc, ++u) {
                const int buf = u & 1;
                if (!mbar_wait_idle(tfull + buf, (uint32_t)((u >> 1) & 1), deadline)) {
                    atomicExch(&aborted, 1);
                    ok = false;
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                __syncwarp();
                const uint32_t taddr = tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)(buf * 128 + cg * 32);
#pragma unroll
                for (int h = 0; h < 2; ++h) {  // two 16-column loads keep acc + v within the register budget
                    float v[16];
                    tmem_ld16(taddr + h * 16, v);
#pragma unroll
                    for (int j = 0; j < 16; ++j) acc[h * 16 + j] += (long long)__float2int_rn(v[j] * rscale) << lsh;
                }
                asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
                __syncwarp();
                if (lane == 0) mbar_arrive(tempty + buf);
            }
        }
        // The last unit's commit follows every MMA, and every TMA load was consumed by one of them:
        // the ring is idle, and the scaled tile is staged there (128 x OSTG doubles) for row-wise,
        // coalesced read-modify-write of C by the 16 epilogue warps.
        double* stg = reinterpret_cast<double*>(base);
        if (ok && !*(volatile int*)&aborted) {
            const int r = quad * 32 + lane;
            const int er = (m0 + r < p.M) ? eaz[m0 + r] : 0;
#pragma unroll
            for (int j = 0; j < 32; ++j) {
                const int c = cg * 32 + j;
                const int ec = (n0 + c < p.N) ? ebz[n0 + c] : 0;
                stg[r * OSTG + c] = fixed_to_double(p.alpha_sign * acc[j], er + ec - p.F);
            }
        }
        asm volatile("bar.sync 1, %0;" ::"r"(OEPI * 32) : "memory");
        if (!*(volatile int*)&aborted) {
            for (int r = warp; r < OBM; r += OEPI) {
                const int row = m0 + r;
                if (row >= p.M) break;
                double* crow = Cz + (int64_t)row * p.ldc;
#pragma unroll
                for (int q = 0; q < OBN / 32; ++q) {
                    const int c = q * 32 + lane, col = n0 + c;
                    if (col < p.N) {
                        const double v = stg[r * OSTG + c];  // already carries the sign of alpha
                        if (p.mode == 0)
                            crow[col] = v;  // alpha = +-1, beta = 0
                        else if (p.mode == 1)
                            crow[col] += v;  // alpha = +-1, beta = 1 (one FP64 add)
                        else
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
// Products with K <= 64 (GENP's Schur updates: one 64-deep K block).  A persistent CTA walks its
// share of 128 x 64 output tiles in row-major order, so the ND A digit planes of a row block (7 planes:
// 112 KB) are loaded once and stay in shared memory; the B digit planes of each tile stream through a
// 4-stage ring.  With the full ND = 7 digits the 28 digit pairs run in two passes, diagonals d = 0-3 then
// 4-6, each diagonal in its own 64-column TMEM accumulator; the two passes use the two halves of TMEM, so
// one pass's MMAs overlap the drain of the other and the tile's final store.  Per tile the TMA moves 11 B
// planes (88 KB) instead of 28 A and 28 B tiles.  Fewer digits (ND = 4 .. 6) drop the low diagonals:
// ND (ND + 1) / 2 pairs, operands of 8 ND - 1 bits.  (d + 1) 2^14 64 < 2^24 keeps every accumulator exact.
// ---------------------------------------------------------------------------------------------
constexpr int UBM = 128, UBN = 64;
constexpr int UA_PLANE = UBM * OBK * 2;  // 16 KB
constexpr int UB_PLANE = UBN * OBK * 2;  // 8 KB
constexpr int URING = 4;
constexpr size_t kUpdSmem =
    1024 + (size_t)kOzSlices * UA_PLANE + (size_t)URING * UB_PLANE + (size_t)UBM * UBN * 8 + 256;
static_assert(kUpdSmem <= 232448, "update kernel shared memory");

// One chunk per diagonal, K <= 64: |acc| <= sum_d (d + 1) 2^14 64 2^(F + 2 - 8(d + 2)) < 1.01 2^62 at F = 56,
// within a signed 64-bit integer, so the fixed-point sum keeps the 55 bits of the 7-digit operands.  F is
// a compile-time constant here: the epilogue's shifts and scalings are then immediates (the epilogue is
// ALU-bound).
constexpr int kUpdF = 56;

// A drained diagonal d (K <= 64): an integer-valued float with |v| <= (d + 1) 2^20.  For d <= 3 that is at
// most 2^22: adding 1.5 2^23 lands in the binade whose unit is 1 (up to 2^24 inclusive), where the bit
// pattern grows by exactly one per unit, so the pattern minus that of 1.5 2^23 is v.  One FADD and one
// integer subtraction replace the conversion; larger diagonals keep the conversion.
__device__ __forceinline__ int diag_to_int(float v, int d) {
    return d <= 3 ? __float_as_int(v + 12582912.0f) - 0x4B400000 : __float2int_rn(v);
}

struct UpdParams {
    int M, N;            // output rows, columns
    int count;           // systems of a batched update: tile t belongs to system t / tiles
    int64_t sC;          // elements between the systems' C (and pivot blocks D)
    int64_t sFlag;       // ints between the systems' info / halt words
    int F;               // fractional bits of the fixed-point accumulator (kUpdF)
    int Mp, Np;          // rows per digit plane of A, of B
    int tiles_n, tiles;  // column tiles, all tiles
    const int* ea;
    const int* eb;
    long long alpha_sign;
    int mode;
    double alpha, beta;
    double* C;
    int64_t ldc;
    int* err;
    const int* halt;
    // the next pivot block (GENP), factored by CTA 0 after its single tile, which contains the block;
    // D == nullptr: no fused factorization
    double* D;
    int64_t ldd;
    int bd;
    int64_t dk;  // global offset of the block: a breakdown at its step s (1-based) is step dk + s
    int* dinfo;
    int* dhalt;
};

// Barrier over the 16 epilogue warps (named barrier 1).
struct EpiSync {
    __device__ void operator()() const { asm volatile("bar.sync 1, %0;" ::"r"(OEPI * 32) : "memory"); }
};

// Pass P streams B planes q = 0 .. nq(P)-1 and pairs each with the A planes p in [p0, p1], so that p + q
// covers the diagonals 4P .. 4P + nd(P) - 1 (0-3, then 4 .. ND-1); q = 0 opens every diagonal of the pass.
// ND digits per operand keep the diagonals 0 .. ND-1 (ND (ND + 1) / 2 pairs); ND = 4 runs one pass.
template <int ND>
struct UpdDiag {
    static_assert(ND >= 4 && ND <= kOzSlices, "update digits");
    static constexpr int kPasses = ND > 4 ? 2 : 1;
    static __device__ __forceinline__ constexpr int nd(int P) { return P == 0 ? 4 : ND - 4; }
    static __device__ __forceinline__ constexpr int nq(int P) { return P == 0 ? 4 : ND; }
    static __device__ __forceinline__ constexpr int p0(int P, int q) { return P == 0 ? 0 : (q < 4 ? 4 - q : 0); }
    static __device__ __forceinline__ constexpr int p1(int P, int q) { return P == 0 ? 3 - q : ND - 1 - q; }
};

template <int ND>
__global__ void __launch_bounds__(OTHREADS, 1)
oz_update_kernel(const __grid_constant__ CUtensorMap tA, const __grid_constant__ CUtensorMap tB, UpdParams p,
                 uint32_t idesc) {
    using Dg = UpdDiag<ND>;
    if (p.halt != nullptr && *(volatile const int*)p.halt != 0) return;
    extern __shared__ __align__(16) uint8_t smem_raw[];
    uint8_t* base = reinterpret_cast<uint8_t*>(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint8_t* sA = base;
    uint8_t* sB = sA + ND * UA_PLANE;
    double* stg = reinterpret_cast<double*>(sB + URING * UB_PLANE);  // 128 x 64, columns XOR-swizzled by row
    uint64_t* fullA = reinterpret_cast<uint64_t*>(stg + UBM * UBN);
    uint64_t* doneA = fullA + 1;   // the MMAs reading the resident A planes have completed
    uint64_t* mmaEnd = fullA + 2;  // every MMA of the CTA has completed
    uint64_t* fullB = fullA + 3;
    uint64_t* emptyB = fullB + URING;
    uint64_t* tfull = emptyB + URING;  // [2]
    uint64_t* tempty = tfull + 2;      // [2]
    uint32_t* tmem_holder = reinterpret_cast<uint32_t*>(tempty + 2);
    __shared__ int aborted;
    __shared__ double piv_rp;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // With a fused pivot block, CTA 0 takes tile 0 (which holds the block) alone and the other CTAs
    // share the remaining tiles evenly.
    int t0, t1;
    // A batch of systems shares the tiles evenly; the CTA that writes a system's tile 0 then factors that
    // system's pivot block (every pivot block must be done when the launch ends, which is all the next step
    // waits for).
    const int tiles_all = p.tiles * p.count;
    if (p.D != nullptr && gridDim.x > 1 && p.count == 1) {
        t0 = (blockIdx.x == 0) ? 0 : 1 + (int)((long long)(blockIdx.x - 1) * (p.tiles - 1) / (gridDim.x - 1));
        t1 = 1 + (int)((long long)blockIdx.x * (p.tiles - 1) / (gridDim.x - 1));
    } else {
        t0 = (int)((long long)blockIdx.x * tiles_all / gridDim.x);
        t1 = (int)((long long)(blockIdx.x + 1) * tiles_all / gridDim.x);
    }

    if (threadIdx.x == 0) {
        mbar_init(fullA, 1);
        mbar_init(doneA, 1);
        mbar_init(mmaEnd, 1);
        for (int i = 0; i < URING; ++i) {
            mbar_init(fullB + i, 1);
            mbar_init(emptyB + i, 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(tfull + b, 1);
            mbar_init(tempty + b, OEPI);
        }
        aborted = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_holder)),
                     "r"(512)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tmem_holder;
    const unsigned long long deadline = now_ns() + kOzWaitNs;

    if (warp == OEPI) {
        if (lane == 0) {  // TMA producer
            int it = 0, na = 0, cur = -1;
            bool ok = true;
            for (int t = t0; t < t1 && ok; ++t) {
                // row blocks are numbered across the systems (t / tiles_n), so a new system reloads A too
                const int z = t / p.tiles, tl = t - z * p.tiles;
                const int mb = t / p.tiles_n, nb = tl % p.tiles_n, mbz = tl / p.tiles_n;
                if (mb != cur) {
                    if (na > 0 && !mbar_wait_idle(doneA, (uint32_t)((na - 1) & 1), deadline)) {
                        ok = false;
                        break;
                    }
                    mbar_expect_tx(fullA, ND * UA_PLANE);
                    for (int pl = 0; pl < ND; ++pl)
                        tma_load_2d(sA + pl * UA_PLANE, &tA, 0, (z * ND + pl) * p.Mp + mbz * UBM, fullA);
                    ++na;
                    cur = mb;
                }
                for (int P = 0; P < Dg::kPasses && ok; ++P)
                    for (int q = 0; q < Dg::nq(P); ++q, ++it) {
                        const int st = it % URING;
                        if (!mbar_wait_idle(emptyB + st, (uint32_t)(((it / URING) & 1) ^ 1), deadline)) {
                            ok = false;
                            break;
                        }
                        mbar_expect_tx(fullB + st, UB_PLANE);
                        tma_load_2d(sB + st * UB_PLANE, &tB, 0, (z * ND + q) * p.Np + nb * UBN, fullB + st);
                    }
            }
            if (!ok) atomicExch(&aborted, 1);
            // the copies issued last must land before the CTA can leave
            const unsigned long long d2 = now_ns() + kOzWaitNs;
            for (int j = it - URING < 0 ? 0 : it - URING; j < it; ++j)
                (void)mbar_wait(fullB + j % URING, (uint32_t)((j / URING) & 1), d2);
            if (na > 0) (void)mbar_wait(fullA, (uint32_t)((na - 1) & 1), d2);
        }
    } else if (warp == OEPI + 1) {
        if (lane == 0) {  // MMA issuer
            int it = 0, u = 0, na = 0, cur = -1;
            bool ok = true;
            for (int t = t0; t < t1 && ok; ++t) {
                const int mb = t / p.tiles_n;
                if (mb != cur) {
                    if (!mbar_wait(fullA, (uint32_t)(na & 1), deadline)) {
                        ok = false;
                        break;
                    }
                    ++na;
                    cur = mb;
                }
                for (int P = 0; P < Dg::kPasses && ok; ++P, ++u) {
                    const int bank = u & 1;
                    if (!mbar_wait(tempty + bank, (uint32_t)(((u >> 1) & 1) ^ 1), deadline)) {
                        ok = false;
                        break;
                    }
                    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                    for (int q = 0; q < Dg::nq(P); ++q, ++it) {
                        const int st = it % URING;
                        if (!mbar_wait(fullB + st, (uint32_t)((it / URING) & 1), deadline)) {
                            ok = false;
                            break;
                        }
                        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                        const uint64_t bd = smem_desc(smem_u32(sB + st * UB_PLANE));
                        for (int pa = Dg::p0(P, q); pa <= Dg::p1(P, q); ++pa) {
                            const uint64_t ad = smem_desc(smem_u32(sA + pa * UA_PLANE));
                            const uint32_t dcol = tmem + (uint32_t)(bank * 256 + (pa + q - 4 * P) * UBN);
#pragma unroll
                            for (int kk = 0; kk < OBK / 16; ++kk)
                                mma_f16(dcol, ad + 2 * kk, bd + 2 * kk, idesc, (q > 0 || kk > 0) ? 1u : 0u);
                        }
                        mma_commit(emptyB + st);
                    }
                    if (ok) mma_commit(tfull + bank);
                }
                if (ok && (t + 1 == t1 || (t + 1) / p.tiles_n != mb)) mma_commit(doneA);
            }
            if (!ok) atomicExch(&aborted, 1);
            mma_commit(mmaEnd);  // arrives once every MMA issued above has completed
            (void)mbar_wait(mmaEnd, 0u, now_ns() + kOzWaitNs);
        }
    } else {
        // epilogue warps 0-15: TMEM lane quadrant (tile rows) and group of 16 columns.  Every warp runs
        // every tile and both named barriers, also after a timeout (expired waits return at once).
        const int quad = warp & 3, cg = warp >> 2;
        const int r = quad * 32 + lane;
        int u = 0;
        bool ok = true;
        for (int t = t0; t < t1; ++t) {
            const int z = t / p.tiles, tl = t - z * p.tiles;
            const int mb = tl / p.tiles_n, nb = tl % p.tiles_n;
            double* const C = p.C + (int64_t)z * p.sC;
            const int* const ea = p.ea + (int64_t)z * p.Mp;
            const int* const eb = p.eb + (int64_t)z * p.Np;
            if (p.mode != 0 && p.beta != 0.0) {
                // the tile's rows of C into L2 while its MMAs run (one 128-byte line per thread), so that the
                // read-modify-write after the drains waits on L2 rather than on HBM
                const int row = mb * UBM + (threadIdx.x >> 2), col = nb * UBN + (threadIdx.x & 3) * 16;
                if (row < p.M && col < p.N)
                    asm volatile("prefetch.global.L2 [%0];" ::"l"(C + (int64_t)row * p.ldc + col));
            }
            long long acc[16];
#pragma unroll
            for (int j = 0; j < 16; ++j) acc[j] = 0;
#pragma unroll  // P compile-time: the epilogue shifts become immediates
            for (int P = 0; P < Dg::kPasses; ++P, ++u) {
                const int bank = u & 1;
                if (!mbar_wait_idle(tfull + bank, (uint32_t)((u >> 1) & 1), deadline)) {
                    atomicExch(&aborted, 1);
                    ok = false;
                }
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                __syncwarp();
                if (ok) {
                    const uint32_t tq = tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)(bank * 256 + cg * 16);
                    // Diagonals two at a time: v_a 2^8 + v_b is an exact int32 (|v_a| <= 5 2^20 for the first
                    // diagonal of a pair, |v_b| <= 7 2^20), so one 64-bit shift-add serves both.  A diagonal
                    // whose weight is below the fixed point's last bit (sh < 0: diagonal 6) goes alone, rounded.
#pragma unroll
                    for (int sl = 0; sl < Dg::nd(P); sl += 2) {
                        const int d = 4 * P + sl;  // compile-time after unrolling: constant shifts
                        const int sha = kUpdF - 8 * d - 14, shb = sha - 8;
                        if (sl + 1 < Dg::nd(P) && shb >= 0) {
                            float va[16], vb[16];
                            tmem_ld16x2(tq + sl * UBN, tq + (sl + 1) * UBN, va, vb);
#pragma unroll
                            for (int j = 0; j < 16; ++j)
                                acc[j] += (long long)(diag_to_int(va[j], d) * 256 + diag_to_int(vb[j], d + 1)) << shb;
                        } else {
#pragma unroll
                            for (int e = 0; e < 2; ++e) {
                                if (sl + e >= Dg::nd(P)) break;
                                const int sh = sha - 8 * e;
                                const float rscale = __int_as_float((127 + (sh < 0 ? sh : 0)) << 23);
                                const int lsh = sh > 0 ? sh : 0;
                                float v[16];
                                tmem_ld16(tq + (sl + e) * UBN, v);
#pragma unroll
                                for (int j = 0; j < 16; ++j)
                                    acc[j] += (long long)__float2int_rn(v[j] * rscale) << lsh;
                            }
                        }
                    }
                }
                asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
                __syncwarp();
                if (lane == 0) mbar_arrive(tempty + bank);
            }
            if (ok) {
                const int row = mb * UBM + r;
                const int er = (row < p.M) ? ea[row] : 0;
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    const int c = cg * 16 + j, col = nb * UBN + c;
                    const int ec = (col < p.N) ? eb[col] : 0;
                    stg[r * UBN + (c ^ (r & 15))] = fixed_to_double(p.alpha_sign * acc[j], er + ec - kUpdF);
                }
            }
            asm volatile("bar.sync 1, %0;" ::"r"(OEPI * 32) : "memory");
            if (!*(volatile int*)&aborted) {
                // rows warp + 16 i in two groups of four rows: the 8 loads of C of a group are issued before
                // its first add (one memory latency per group instead of one per row)
                constexpr int NR = UBM / OEPI, NG = 4, NH = UBN / 32;
                const bool need_c = p.mode != 0 && p.beta != 0.0;
#pragma unroll
                for (int g0 = 0; g0 < NR; g0 += NG) {
                    double cv[NG][NH];
#pragma unroll
                    for (int i = 0; i < NG; ++i)
#pragma unroll
                        for (int h = 0; h < NH; ++h) {
                            const int row = mb * UBM + warp + OEPI * (g0 + i), col = nb * UBN + h * 32 + lane;
                            cv[i][h] = (need_c && row < p.M && col < p.N) ? C[(int64_t)row * p.ldc + col] : 0.0;
                        }
#pragma unroll
                    for (int i = 0; i < NG; ++i)
#pragma unroll
                        for (int h = 0; h < NH; ++h) {
                            const int rr = warp + OEPI * (g0 + i), c = h * 32 + lane;
                            const int row = mb * UBM + rr, col = nb * UBN + c;
                            if (row < p.M && col < p.N) {
                                const double v = stg[rr * UBN + (c ^ (rr & 15))];
                                double out;
                                if (p.mode == 0)
                                    out = v;
                                else if (p.mode == 1)
                                    out = cv[i][h] + v;
                                else
                                    out = (p.beta == 0.0) ? p.alpha * v : fma(p.beta, cv[i][h], p.alpha * v);
                                C[(int64_t)row * p.ldc + col] = out;
                            }
                        }
                }
            }
            asm volatile("bar.sync 1, %0;" ::"r"(OEPI * 32) : "memory");  // the staging area is reused
            if (p.D != nullptr && tl == 0) {
                // tile 0, just written by these warps, holds the next pivot block: factor it in the staging
                // area while the other CTAs finish the update.  The test is uniform over the 16 warps (the
                // barriers inside must be met by all of them); after a timeout the factorization still
                // runs, over whatever the tile holds, and the launch reports the timeout.
                double* a = stg;
                double* const D = p.D + (int64_t)z * p.sC;
                const int tid = threadIdx.x;
                for (int i = tid >> 6; i < p.bd; i += (OEPI * 32) / 64)
                    if ((tid & 63) < p.bd) a[i * kPivotLds + (tid & 63)] = D[i * p.ldd + (tid & 63)];
                EpiSync{}();
                const int broke = pivot_block_genp<double, OEPI * 32>(a, p.bd, &piv_rp, tid, EpiSync{});
                if (broke != 0) {
                    if (tid == 0) {
                        atomicMin(p.dinfo + (int64_t)z * p.sFlag, (int)(p.dk + broke));
                        atomicExch(p.dhalt + (int64_t)z * p.sFlag, 1);
                    }
                } else {
                    for (int i = tid >> 6; i < p.bd; i += (OEPI * 32) / 64)
                        if ((tid & 63) < p.bd) D[i * p.ldd + (tid & 63)] = a[i * kPivotLds + (tid & 63)];
                }
                EpiSync{}();  // the staging area is reused by the next tile
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (aborted && threadIdx.x == 0 && p.err != nullptr) atomicExch(p.err, (int)RMGE_ERR_TIMEOUT);
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512) : "memory");
}

// ---------------------------------------------------------------------------------------------
// Products with K = 128: the Schur update of two pivot steps at once, E -= [L21_k L21_k+1] [U12_k; U12_k+1]
// (GENP with one step of look-ahead).  A persistent CTA walks its share of 128 x 64 output tiles.
// - The ND B digit planes of a tile (64 columns x 128 K, 16 KB each) sit in ND slots, one per plane; the A
//   planes (128 rows x 128 K, 32 KB) stream through a ring.  Per tile that is ND + ND loads (288 KB at
//   ND = 6) instead of one B load per digit pair.
// - Pairs run A plane by A plane, p = 0 .. ND-1, and within one in descending q, so B plane q is last
//   read by pair (ND-1-q, q): B planes ND-1, ND-2, ... are refilled for the next tile while this one is
//   still multiplying, and the next tile starts with the planes refilled first.
// - Each pair adds into the 64-column TMEM accumulator of its diagonal p + q (ND x 64 <= 448 columns).  The
//   epilogue drains the diagonals, releases TMEM to the next tile's MMAs, then rounds and adds the tile
//   into E while those run, through a half-tile staging area in two rounds.
// (d + 1) 2^14 128 < 2^24 keeps every accumulator exact for d <= 6; the fixed point has F = 55 fractional
// bits (the bound of the K = 64 kernel, doubled).
// ---------------------------------------------------------------------------------------------
constexpr int U2K = 128;                       // K of one launch (two pivot blocks)
constexpr int U2A_SLOT = UBM * U2K * 2;        // 32 KB: one A plane of a row block
constexpr int U2B_SLOT = UBN * U2K * 2;        // 16 KB: one B plane of a column block
constexpr int U2STG = 64 * kPivotLds * 8 > UBM * 32 * 8 ? 64 * kPivotLds * 8 : UBM * 32 * 8;  // half tile, or pivot
constexpr int kUpd2F = 55;
template <int ND>
struct Upd2Cfg {
    static constexpr int kARing = ND == 7 ? 2 : 3;
    static constexpr size_t kSmem =
        1024 + (size_t)kARing * U2A_SLOT + (size_t)ND * U2B_SLOT + (size_t)U2STG + 256;
    static_assert(kSmem <= 232448, "128-deep update kernel shared memory");
};

// |v| <= (d + 1) 2^14 128 for diagonal d of a 128-deep tile: the bit-pattern conversion holds for d <= 1.
__device__ __forceinline__ int diag128_to_int(float v, int d) {
    return d <= 1 ? __float_as_int(v + 12582912.0f) - 0x4B400000 : __float2int_rn(v);
}

template <int ND>
__global__ void __launch_bounds__(OTHREADS, 1)
oz_update128_kernel(const __grid_constant__ CUtensorMap tA, const __grid_constant__ CUtensorMap tB, UpdParams p,
                    uint32_t idesc) {
    static_assert(ND >= 4 && ND <= kOzSlices, "update digits");
    constexpr int AR = Upd2Cfg<ND>::kARing;
    if (p.halt != nullptr && *(volatile const int*)p.halt != 0) return;
    extern __shared__ __align__(16) uint8_t smem_raw[];
    uint8_t* base = reinterpret_cast<uint8_t*>(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint8_t* sA = base;
    uint8_t* sB = sA + AR * U2A_SLOT;
    double* stg = reinterpret_cast<double*>(sB + ND * U2B_SLOT);  // 128 x 32, columns XOR-swizzled by row
    uint64_t* fullA = reinterpret_cast<uint64_t*>(reinterpret_cast<uint8_t*>(stg) + U2STG);  // [AR]
    uint64_t* emptyA = fullA + AR;
    uint64_t* fullB = emptyA + AR;  // [ND]
    uint64_t* emptyB = fullB + ND;
    uint64_t* tfull = emptyB + ND;  // the tile's MMAs have completed
    uint64_t* tempty = tfull + 1;   // the epilogue has drained TMEM
    uint64_t* mmaEnd = tempty + 1;
    uint32_t* tmem_holder = reinterpret_cast<uint32_t*>(mmaEnd + 1);
    __shared__ int aborted;
    __shared__ double piv_rp;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // with a fused pivot block (one system), CTA 0 takes tile 0, which holds it, alone
    const int tiles_all = p.tiles * p.count;
    int t0, t1;
    if (p.D != nullptr && gridDim.x > 1 && p.count == 1) {
        t0 = (blockIdx.x == 0) ? 0 : 1 + (int)((long long)(blockIdx.x - 1) * (p.tiles - 1) / (gridDim.x - 1));
        t1 = 1 + (int)((long long)blockIdx.x * (p.tiles - 1) / (gridDim.x - 1));
    } else {
        t0 = (int)((long long)blockIdx.x * tiles_all / gridDim.x);
        t1 = (int)((long long)(blockIdx.x + 1) * tiles_all / gridDim.x);
    }

    // tiles run down each column block (system z, row block mb, column block nb), so that consecutive tiles
    // of a CTA share their B planes, which then load once per column block
    const int tiles_m = p.tiles / p.tiles_n;
    auto tile_at = [&](int t, int& z, int& mb, int& nb) {
        z = t / p.tiles;
        const int tl = t - z * p.tiles;
        nb = tl / tiles_m;
        mb = tl - nb * tiles_m;
    };
    auto bkey = [&](int t) {
        const int z = t / p.tiles;
        return z * p.tiles_n + (t - z * p.tiles) / tiles_m;
    };
    if (threadIdx.x == 0) {
        for (int i = 0; i < AR; ++i) {
            mbar_init(fullA + i, 1);
            mbar_init(emptyA + i, 1);
        }
        for (int i = 0; i < ND; ++i) {
            mbar_init(fullB + i, 1);
            mbar_init(emptyB + i, 1);
        }
        mbar_init(tfull, 1);
        mbar_init(tempty, OEPI);
        mbar_init(mmaEnd, 1);
        aborted = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_holder)),
                     "r"(512)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tmem_holder;
    const unsigned long long deadline = now_ns() + kOzWaitNs;

    if (warp == OEPI) {
        if (lane == 0) {  // TMA producer, in the MMA warp's order: A_0, B_ND-1 .. B_0, then A_1 .. A_ND-1
            int ia = 0, g = 0;  // A loads; B fills (one per run of tiles in one column block)
            bool ok = true;
            for (int t = t0; t < t1 && ok; ++t) {
                int z, mb, nb;
                tile_at(t, z, mb, nb);
                const bool newB = (t == t0) || bkey(t) != bkey(t - 1);
                for (int pa = 0; pa < ND && ok; ++pa, ++ia) {
                    const int sa = ia % AR;
                    if (!mbar_wait_idle(emptyA + sa, (uint32_t)(((ia / AR) & 1) ^ 1), deadline)) {
                        ok = false;
                        break;
                    }
                    mbar_expect_tx(fullA + sa, U2A_SLOT);
                    const int ya = (z * ND + pa) * p.Mp + mb * UBM;
                    tma_load_2d(sA + sa * U2A_SLOT, &tA, 0, ya, fullA + sa);
                    tma_load_2d(sA + sa * U2A_SLOT + U2A_SLOT / 2, &tA, OBK, ya, fullA + sa);
                    if (pa == 0 && newB)
                        for (int q = ND - 1; q >= 0; --q) {
                            if (!mbar_wait_idle(emptyB + q, (uint32_t)((g & 1) ^ 1), deadline)) {
                                ok = false;
                                break;
                            }
                            mbar_expect_tx(fullB + q, U2B_SLOT);
                            const int yb = (z * ND + q) * p.Np + nb * UBN;
                            tma_load_2d(sB + q * U2B_SLOT, &tB, 0, yb, fullB + q);
                            tma_load_2d(sB + q * U2B_SLOT + U2B_SLOT / 2, &tB, OBK, yb, fullB + q);
                        }
                    if (pa == 0 && newB) ++g;
                }
            }
            if (!ok) atomicExch(&aborted, 1);
            // the copies issued last must land before the CTA can leave
            const unsigned long long d2 = now_ns() + kOzWaitNs;
            for (int j = ia - AR < 0 ? 0 : ia - AR; j < ia; ++j)
                (void)mbar_wait(fullA + j % AR, (uint32_t)((j / AR) & 1), d2);
            if (g > 0)
                for (int q = 0; q < ND; ++q) (void)mbar_wait(fullB + q, (uint32_t)((g - 1) & 1), d2);
        }
    } else if (warp == OEPI + 1) {
        if (lane == 0) {  // MMA issuer
            int ia = 0, u = 0, g = 0;
            bool ok = true;
            for (int t = t0; t < t1 && ok; ++t, ++u) {
                const bool newB = (t == t0) || bkey(t) != bkey(t - 1);
                const bool lastB = (t + 1 == t1) || bkey(t + 1) != bkey(t);
                if (newB) ++g;  // B fill g - 1 serves this tile
                if (!mbar_wait(tempty, (uint32_t)((u & 1) ^ 1), deadline)) {
                    ok = false;
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                for (int pa = 0; pa < ND && ok; ++pa, ++ia) {
                    const int sa = ia % AR;
                    if (!mbar_wait(fullA + sa, (uint32_t)((ia / AR) & 1), deadline)) {
                        ok = false;
                        break;
                    }
                    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                    for (int q = ND - 1 - pa; q >= 0; --q) {
                        if (pa == 0 && newB) {  // the first use of this fill of B plane q
                            if (!mbar_wait(fullB + q, (uint32_t)((g - 1) & 1), deadline)) {
                                ok = false;
                                break;
                            }
                            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                        }
                        const uint32_t dcol = tmem + (uint32_t)((pa + q) * UBN);
#pragma unroll
                        for (int h = 0; h < U2K / OBK; ++h) {
                            const uint64_t ad = smem_desc(smem_u32(sA + sa * U2A_SLOT + h * (U2A_SLOT / 2)));
                            const uint64_t bd = smem_desc(smem_u32(sB + q * U2B_SLOT + h * (U2B_SLOT / 2)));
#pragma unroll
                            for (int kk = 0; kk < OBK / 16; ++kk)
                                mma_f16(dcol, ad + 2 * kk, bd + 2 * kk, idesc, (pa > 0 || h > 0 || kk > 0) ? 1u : 0u);
                        }
                        if (lastB && pa == ND - 1 - q) mma_commit(emptyB + q);  // its last use in this fill
                    }
                    mma_commit(emptyA + sa);
                }
                if (ok) mma_commit(tfull);
            }
            if (!ok) atomicExch(&aborted, 1);
            mma_commit(mmaEnd);  // arrives once every MMA issued above has completed
            (void)mbar_wait(mmaEnd, 0u, now_ns() + kOzWaitNs);
        }
    } else {
        // epilogue warps 0-15: TMEM lane quadrant (tile rows) and group of 16 columns
        const int quad = warp & 3, cg = warp >> 2;
        const int r = quad * 32 + lane;
        int u = 0;
        bool ok = true;
        for (int t = t0; t < t1; ++t, ++u) {
            int z, mb, nb;
            tile_at(t, z, mb, nb);
            const int tl = t - z * p.tiles;
            double* const C = p.C + (int64_t)z * p.sC;
            const int* const ea = p.ea + (int64_t)z * p.Mp;
            const int* const eb = p.eb + (int64_t)z * p.Np;
            const bool need_c = p.mode != 0 && p.beta != 0.0;
            if (need_c) {
                const int row = mb * UBM + (threadIdx.x >> 2), col = nb * UBN + (threadIdx.x & 3) * 16;
                if (row < p.M && col < p.N)
                    asm volatile("prefetch.global.L2 [%0];" ::"l"(C + (int64_t)row * p.ldc + col));
            }
            long long acc[16];
#pragma unroll
            for (int j = 0; j < 16; ++j) acc[j] = 0;
            if (!mbar_wait_idle(tfull, (uint32_t)(u & 1), deadline)) {
                atomicExch(&aborted, 1);
                ok = false;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            __syncwarp();
            if (ok) {
                const uint32_t tq = tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)(cg * 16);
                // diagonals 0 and 1, then 2 and 3, two at a time (v_a 2^8 + v_b is exact in int32 while
                // |v_a| <= 3 2^21), the others one at a time; diagonal 6's weight is below the last bit
#pragma unroll
                for (int d = 0; d < 4; d += 2) {
                    float va[16], vb[16];
                    tmem_ld16x2(tq + d * UBN, tq + (d + 1) * UBN, va, vb);
                    const int shb = kUpd2F - 8 * (d + 1) - 14;
#pragma unroll
                    for (int j = 0; j < 16; ++j)
                        acc[j] += (long long)(diag128_to_int(va[j], d) * 256 + diag128_to_int(vb[j], d + 1)) << shb;
                }
#pragma unroll
                for (int d = 4; d < ND; ++d) {
                    const int sh = kUpd2F - 8 * d - 14;
                    const float rscale = __int_as_float((127 + (sh < 0 ? sh : 0)) << 23);
                    const int lsh = sh > 0 ? sh : 0;
                    float v[16];
                    tmem_ld16(tq + d * UBN, v);
#pragma unroll
                    for (int j = 0; j < 16; ++j) acc[j] += (long long)__float2int_rn(v[j] * rscale) << lsh;
                }
            }
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            __syncwarp();
            if (lane == 0) mbar_arrive(tempty);  // the next tile's MMAs may start
            double dv[16];
            {
                const int row = mb * UBM + r;
                const int er = (row < p.M) ? ea[row] : 0;
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    const int col = nb * UBN + cg * 16 + j;
                    const int ec = (col < p.N) ? eb[col] : 0;
                    dv[j] = fixed_to_double(p.alpha_sign * acc[j], er + ec - kUpd2F);
                }
            }
            // two rounds of 32 columns through the half-tile staging area
#pragma unroll
            for (int half = 0; half < 2; ++half) {
                if (ok && (cg >> 1) == half)
#pragma unroll
                    for (int j = 0; j < 16; ++j) {
                        const int c = (cg & 1) * 16 + j;
                        stg[r * 32 + (c ^ (r & 15))] = dv[j];
                    }
                asm volatile("bar.sync 1, %0;" ::"r"(OEPI * 32) : "memory");
                if (!*(volatile int*)&aborted) {
                    constexpr int NR = UBM / OEPI, NG = 4;
                    const int col = nb * UBN + half * 32 + lane;
#pragma unroll
                    for (int g0 = 0; g0 < NR; g0 += NG) {
                        double cv[NG];
#pragma unroll
                        for (int i = 0; i < NG; ++i) {
                            const int row = mb * UBM + warp + OEPI * (g0 + i);
                            cv[i] = (need_c && row < p.M && col < p.N) ? C[(int64_t)row * p.ldc + col] : 0.0;
                        }
#pragma unroll
                        for (int i = 0; i < NG; ++i) {
                            const int rr = warp + OEPI * (g0 + i);
                            const int row = mb * UBM + rr;
                            if (row < p.M && col < p.N) {
                                const double v = stg[rr * 32 + (lane ^ (rr & 15))];
                                double out;
                                if (p.mode == 0)
                                    out = v;
                                else if (p.mode == 1)
                                    out = cv[i] + v;
                                else
                                    out = (p.beta == 0.0) ? p.alpha * v : fma(p.beta, cv[i], p.alpha * v);
                                C[(int64_t)row * p.ldc + col] = out;
                            }
                        }
                    }
                }
                asm volatile("bar.sync 1, %0;" ::"r"(OEPI * 32) : "memory");  // the staging area is reused
            }
            if (p.D != nullptr && tl == 0) {
                // tile 0 holds the next pivot block: factor it in the staging area (as the 64-deep kernel does)
                double* a = stg;
                double* const D = p.D + (int64_t)z * p.sC;
                const int tid = threadIdx.x;
                for (int i = tid >> 6; i < p.bd; i += (OEPI * 32) / 64)
                    if ((tid & 63) < p.bd) a[i * kPivotLds + (tid & 63)] = D[i * p.ldd + (tid & 63)];
                EpiSync{}();
                const int broke = pivot_block_genp<double, OEPI * 32>(a, p.bd, &piv_rp, tid, EpiSync{});
                if (broke != 0) {
                    if (tid == 0) {
                        atomicMin(p.dinfo + (int64_t)z * p.sFlag, (int)(p.dk + broke));
                        atomicExch(p.dhalt + (int64_t)z * p.sFlag, 1);
                    }
                } else {
                    for (int i = tid >> 6; i < p.bd; i += (OEPI * 32) / 64)
                        if ((tid & 63) < p.bd) D[i * p.ldd + (tid & 63)] = a[i * kPivotLds + (tid & 63)];
                }
                EpiSync{}();
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (aborted && threadIdx.x == 0 && p.err != nullptr) atomicExch(p.err, (int)RMGE_ERR_TIMEOUT);
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512) : "memory");
}

// ---------------------------------------------------------------------------------------------
// Digit planes.  Row (trans = false) or column (trans = true) exponents of the source, then s BF16
// planes of rows_p x kp (K-major, zero padded): plane[p][r][k].
// ---------------------------------------------------------------------------------------------

// Exact per-k balancing of a product A B (used for GENP's Schur updates, where column k of L scales
// like 1 / u_kk and row k of U like u_kk): column k of A is taken as A_.k 2^t_k and row k of B as
// 2^-t_k B_k., which leaves A B unchanged.  t_k = floor((log2 max|B_k.| - log2 max|A_.k|) / 2) brings
// both maxima to about their geometric mean, so the per-row / per-column digit scaling below no longer
// pairs a large column of A with a large row of B.  kmaxA, kmaxB hold the FP64 bit patterns of those
// maxima; NULL means no balancing.
__device__ __forceinline__ int bal_shift(const unsigned long long* kmaxA, const unsigned long long* kmaxB, int64_t k) {
    if (kmaxA == nullptr) return 0;
    const double a = __longlong_as_double((long long)kmaxA[k]), b = __longlong_as_double((long long)kmaxB[k]);
    if (!(a > 0.0) || !(b > 0.0) || !isfinite(a) || !isfinite(b)) return 0;
    return (ilogb(b) - ilogb(a)) >> 1;
}

// Exponent of one entry, q + 1 for |x| in [2^q, 2^(q+1)), shifted by the balancing; INT_MIN for zero
// or non-finite entries (which store_digits handles on its own).
__device__ __forceinline__ int entry_exp(double x, int t) {
    return (x != 0.0 && isfinite(x)) ? ilogb(x) + 1 + t : INT_MIN;
}

// e[r] = smallest integer with max_k |A_rk 2^t_k| < 2^e (0 for an all-zero row): one warp per row.
// blockIdx.y: the system of a batch (BatchOff strides); the same below for every digit kernel.
struct BatchOff {
    int64_t src;   // elements between the systems' source matrices
    int64_t kmax;  // slots between their per-k maxima
    int64_t e;     // ints between their exponent vectors
    int64_t pl;    // elements between their digit-plane blocks
};

__global__ void row_exponent_kernel(int64_t rows, int64_t cols, const double* __restrict__ src, int64_t lds,
                                    const unsigned long long* __restrict__ kmaxA,
                                    const unsigned long long* __restrict__ kmaxB, int* __restrict__ e, BatchOff bo) {
    const int lane = threadIdx.x & 31;
    const int64_t r = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    if (r >= rows) return;
    src += blockIdx.y * bo.src;
    e += blockIdx.y * bo.e;
    if (kmaxA != nullptr) {
        kmaxA += blockIdx.y * bo.kmax;
        kmaxB += blockIdx.y * bo.kmax;
    }
    int m = INT_MIN;
    for (int64_t k = lane; k < cols; k += 32) m = max(m, entry_exp(src[r * lds + k], bal_shift(kmaxA, kmaxB, k)));
    for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
    if (lane == 0) e[r] = (m == INT_MIN) ? 0 : m;
}

// e[c] = the same for column c of B 2^-t_k: 32 columns per block (consecutive threads on consecutive
// columns), rows split over 8 thread groups and reduced in shared memory.
__global__ void col_exponent_kernel(int64_t rows, int64_t cols, const double* __restrict__ src, int64_t lds,
                                    const unsigned long long* __restrict__ kmaxA,
                                    const unsigned long long* __restrict__ kmaxB, int* __restrict__ e, BatchOff bo) {
    __shared__ int part[8][32];
    src += blockIdx.y * bo.src;
    e += blockIdx.y * bo.e;
    if (kmaxA != nullptr) {
        kmaxA += blockIdx.y * bo.kmax;
        kmaxB += blockIdx.y * bo.kmax;
    }
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    const int64_t c = (int64_t)blockIdx.x * 32 + tx;
    int m = INT_MIN;
    if (c < cols)
        for (int64_t k = ty; k < rows; k += 8) m = max(m, entry_exp(src[k * lds + c], -bal_shift(kmaxA, kmaxB, k)));
    part[ty][tx] = m;
    __syncthreads();
    if (ty == 0 && c < cols) {
#pragma unroll
        for (int g = 1; g < 8; ++g) m = max(m, part[g][tx]);
        e[c] = (m == INT_MIN) ? 0 : m;
    }
}

// The (8s - 1)-bit magnitude |x| 2^(8s-1), x = v 2^-e (|x| < 1), by integer shifts of the FP64 significand.
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
    const int sh = ex - e + 8 * s - 1;  // |v| 2^(8s - 1 - e) = m 2^sh
    if (sh >= 0) return m << sh;  // |x| < 1 keeps this below 2^(8s-1) <= 2^55: sh <= 2
    return (-sh >= 64) ? 0ull : (m >> (-sh));
}

// The s balanced base-256 digits of X < 2^(8s-1), most significant first: the low digits are brought
// into [-128, 127] by carrying into the next digit up, which leaves the top digit in [0, 128].
__device__ __forceinline__ void store_digits(double v, int er, int s, __nv_bfloat16* dst, int64_t plane) {
    if (!isfinite(v)) {  // a NaN in the leading plane makes every product it enters NaN
        dst[0] = __float2bfloat16_rn(__int_as_float(0x7fc00000));
        for (int q = 1; q < s; ++q) dst[(int64_t)q * plane] = __float2bfloat16_rn(0.0f);
        return;
    }
    const unsigned long long X = fixed_digits(v, er, s);
    const float sg = (v < 0.0) ? -1.0f : 1.0f;
    int carry = 0;
    for (int q = s - 1; q >= 0; --q) {
        int d = (int)((X >> (8 * (s - 1 - q))) & 255ull) + carry;
        carry = 0;
        if (q > 0 && d >= 128) {
            d -= 256;
            carry = 1;
        }
        dst[(int64_t)q * plane] = __float2bfloat16_rn(sg * (float)d);
    }
}

// Row digits: plane[q][r][k] = digit q of A_rk 2^t_k (rows_p x kp per plane, zero padded).
__global__ void row_digits_kernel(int64_t rows, int64_t cols, const double* __restrict__ src, int64_t lds,
                                  const int* __restrict__ e, const unsigned long long* __restrict__ kmaxA,
                                  const unsigned long long* __restrict__ kmaxB, int s, int64_t rows_p, int64_t kp,
                                  __nv_bfloat16* __restrict__ planes, BatchOff bo) {
    const int64_t total = rows_p * kp;
    src += blockIdx.y * bo.src;
    e += blockIdx.y * bo.e;
    planes += blockIdx.y * bo.pl;
    if (kmaxA != nullptr) {
        kmaxA += blockIdx.y * bo.kmax;
        kmaxB += blockIdx.y * bo.kmax;
    }
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = idx / kp, k = idx % kp;
        const bool in = r < rows && k < cols;
        store_digits(in ? src[r * lds + k] : 0.0, in ? e[r] - bal_shift(kmaxA, kmaxB, k) : 0, s, planes + idx, total);
    }
}

// Column digits, transposed through shared memory: plane[q][c][k] = digit q of 2^-t_k B_kc.
__global__ void col_digits_kernel(int64_t rows, int64_t cols, const double* __restrict__ src, int64_t lds,
                                  const int* __restrict__ e, const unsigned long long* __restrict__ kmaxA,
                                  const unsigned long long* __restrict__ kmaxB, int s, int64_t cols_p, int64_t kp,
                                  __nv_bfloat16* __restrict__ planes, BatchOff bo) {
    __shared__ double t[32][33];
    const int64_t k0 = (int64_t)blockIdx.y * 32, c0 = (int64_t)blockIdx.x * 32;
    src += blockIdx.z * bo.src;  // the system index is blockIdx.z here (y runs over k blocks)
    e += blockIdx.z * bo.e;
    planes += blockIdx.z * bo.pl;
    if (kmaxA != nullptr) {
        kmaxA += blockIdx.z * bo.kmax;
        kmaxB += blockIdx.z * bo.kmax;
    }
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 32 x 8 threads
    for (int i = ty; i < 32; i += 8) {
        const int64_t k = k0 + i, c = c0 + tx;
        t[i][tx] = (k < rows && c < cols) ? src[k * lds + c] : 0.0;
    }
    __syncthreads();
    const int64_t total = cols_p * kp;
    for (int i = ty; i < 32; i += 8) {
        const int64_t c = c0 + i, k = k0 + tx;  // write along k
        if (c < cols_p && k < kp)
            store_digits(t[tx][i], (c < cols && k < rows) ? e[c] + bal_shift(kmaxA, kmaxB, k) : 0, s, planes + c * kp + k,
                         total);
    }
}

// K <= KW (KW = 64: one K block; 128: two pivot blocks): the exponent and the digits of a row in one pass,
// one warp per padded row (lane l holds k = l + 32 i).
template <int KW>
__device__ void row_prep(int64_t bid, int64_t rows, int cols, const double* __restrict__ src, int64_t lds,
                         const unsigned long long* __restrict__ kmaxA, const unsigned long long* __restrict__ kmaxB,
                         int s, int64_t rows_p, int* __restrict__ e, __nv_bfloat16* __restrict__ planes) {
    constexpr int NV = KW / 32;
    const int lane = threadIdx.x & 31;
    const int64_t r = (bid * (int64_t)blockDim.x + threadIdx.x) >> 5;
    if (r >= rows_p) return;
    const bool live = r < rows;
    double v[NV];
    int t[NV];
    int m = INT_MIN;
#pragma unroll
    for (int i = 0; i < NV; ++i) {
        const int k = lane + 32 * i;
        v[i] = (live && k < cols) ? src[r * lds + k] : 0.0;
        t[i] = (k < cols) ? bal_shift(kmaxA, kmaxB, k) : 0;
        m = max(m, entry_exp(v[i], t[i]));
    }
    for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
    const int er = (m == INT_MIN) ? 0 : m;
    if (lane == 0 && live) e[r] = er;
    const int64_t total = rows_p * KW;
#pragma unroll
    for (int i = 0; i < NV; ++i) store_digits(v[i], er - t[i], s, planes + r * KW + lane + 32 * i, total);
}

// K <= KW: the exponent and the (transposed) digits of 32 columns per block; 256 threads = 32 columns x
// 8 row groups for the exponent, then consecutive threads along k for the digit stores.
template <int KW>
__device__ void col_prep(int64_t bid, int rows, int64_t cols, const double* __restrict__ src, int64_t lds,
                         const unsigned long long* __restrict__ kmaxA, const unsigned long long* __restrict__ kmaxB,
                         int s, int64_t cols_p, int* __restrict__ e, __nv_bfloat16* __restrict__ planes) {
    __shared__ double t[KW][33];
    __shared__ int part[8][32];
    __shared__ int tk[KW];
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    const int64_t c0 = bid * 32, c = c0 + tx;
    for (int i = threadIdx.x; i < KW; i += 256) tk[i] = (i < rows) ? bal_shift(kmaxA, kmaxB, i) : 0;
    for (int i = ty; i < KW; i += 8) t[i][tx] = (i < rows && c < cols) ? src[(int64_t)i * lds + c] : 0.0;
    __syncthreads();
    int m = INT_MIN;
    for (int i = ty; i < rows; i += 8) m = max(m, entry_exp(t[i][tx], -tk[i]));
    part[ty][tx] = m;
    __syncthreads();
    if (ty == 0) {
#pragma unroll
        for (int g = 1; g < 8; ++g) m = max(m, part[g][tx]);
        part[0][tx] = (m == INT_MIN) ? 0 : m;
        if (c < cols) e[c] = part[0][tx];
    }
    __syncthreads();
    const int64_t total = cols_p * KW;
    for (int idx = threadIdx.x; idx < 32 * KW; idx += 256) {
        const int cl = idx / KW, k = idx % KW;
        if (c0 + cl < cols_p)
            store_digits(t[k][cl], (c0 + cl < cols && k < rows) ? part[0][cl] + tk[k] : 0, s,
                         planes + (c0 + cl) * KW + k, total);
    }
}

// Both operands of a K <= KW product in one launch: blocks [0, row_blocks) prepare the rows of A, the
// rest the columns of B (one launch instead of four per GENP step).
template <int KW>
__global__ void prep_kernel(int64_t row_blocks, int64_t M, int64_t N, int K, const double* __restrict__ A,
                            int64_t lda, const double* __restrict__ B, int64_t ldb,
                            const unsigned long long* __restrict__ kmaxA,
                            const unsigned long long* __restrict__ kmaxB, int s, int64_t Mp, int64_t Np,
                            int* __restrict__ ea, int* __restrict__ eb, __nv_bfloat16* __restrict__ pa,
                            __nv_bfloat16* __restrict__ pb, BatchOff boA, BatchOff boB) {
    const int64_t z = blockIdx.y;
    A += z * boA.src;
    B += z * boB.src;
    ea += z * boA.e;
    eb += z * boB.e;
    pa += z * boA.pl;
    pb += z * boB.pl;
    if (kmaxA != nullptr) {
        kmaxA += z * boA.kmax;
        kmaxB += z * boA.kmax;
    }
    if ((int64_t)blockIdx.x < row_blocks)
        row_prep<KW>(blockIdx.x, M, K, A, lda, kmaxA, kmaxB, s, Mp, ea, pa);
    else
        col_prep<KW>((int64_t)blockIdx.x - row_blocks, K, N, B, ldb, kmaxA, kmaxB, s, Np, eb, pb);
}

unsigned grid_for(int64_t work) {
    int64_t g = (work + 255) / 256;
    if (g > 152 * 16) g = 152 * 16;
    return (unsigned)(g < 1 ? 1 : g);
}

// Multiprocessors of the current device (persistent grids), cached per device.
int sm_count() {
    static int cached[64] = {0};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 152;
    if (cached[dev] == 0) {
        int v = 0;
        if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v <= 0) v = 152;
        cached[dev] = v;
    }
    return cached[dev];
}

}  // namespace

size_t oz_plane_bytes(int64_t rows, int64_t k, int s) {
    const int64_t rp = (rows + 127) / 128 * 128, kp = (k + 63) / 64 * 64;
    return (size_t)s * (size_t)rp * (size_t)kp * 2;
}

template <int ND>
rmge_status launch_update(const CUtensorMap& ta, const CUtensorMap& tb, const UpdParams& u, uint32_t idesc, int grid,
                          cudaStream_t st) {
    if (cudaFuncSetAttribute(oz_update_kernel<ND>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kUpdSmem) !=
        cudaSuccess) {
        (void)cudaGetLastError();
        return RMGE_ERR_CUDA;
    }
    oz_update_kernel<ND><<<grid, OTHREADS, kUpdSmem, st>>>(ta, tb, u, idesc);
    RMGE_LAUNCH_CHECK();
    return RMGE_OK;
}

template <int ND>
rmge_status launch_update128(const CUtensorMap& ta, const CUtensorMap& tb, const UpdParams& u, uint32_t idesc,
                             int grid, cudaStream_t st) {
    constexpr size_t smem = Upd2Cfg<ND>::kSmem;
    if (cudaFuncSetAttribute(oz_update128_kernel<ND>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
        cudaSuccess) {
        (void)cudaGetLastError();
        return RMGE_ERR_CUDA;
    }
    oz_update128_kernel<ND><<<grid, OTHREADS, smem, st>>>(ta, tb, u, idesc);
    RMGE_LAUNCH_CHECK();
    return RMGE_OK;
}

rmge_status oz_gemm(int64_t M, int64_t N, int64_t K, int s, double alpha, const double* A, int64_t lda,
                    const double* B, int64_t ldb, double beta, double* C, int64_t ldc, void* planesA, void* planesB,
                    int* ea, int* eb, const unsigned long long* kmaxA, const unsigned long long* kmaxB, int* err,
                    const int* halt, cudaStream_t st, const OzFuse* fuse, const OzBatch& bt) {
    if ((kmaxA == nullptr) != (kmaxB == nullptr)) return RMGE_ERR_INVALID_ARG;
    if (bt.count < 1 || bt.count > 65535) return RMGE_ERR_INVALID_ARG;
    if (M <= 0 || N <= 0) return RMGE_OK;
    if (K <= 0 || s < 1 || s > kOzSlices || M > INT32_MAX / 16 || N > INT32_MAX / 16 || K > INT32_MAX / 2)
        return RMGE_ERR_INVALID_ARG;
    const int64_t Mp = (M + 127) / 128 * 128, Np = (N + 127) / 128 * 128, Kp = (K + 63) / 64 * 64;
    // the fused pivot block needs the persistent update kernel and must lie in its first tile
    if (fuse != nullptr && (Kp != OBK || s < 4 || fuse->D == nullptr || fuse->b < 1 || fuse->b > UBN ||
                            fuse->b > M || fuse->b > N || fuse->info == nullptr || fuse->halt == nullptr))
        return RMGE_ERR_INVALID_ARG;
    __nv_bfloat16* pa = static_cast<__nv_bfloat16*>(planesA);
    __nv_bfloat16* pb = static_cast<__nv_bfloat16*>(planesB);
    // per-system offsets of a batch: sources, per-k maxima, exponents, digit-plane blocks
    const unsigned nz = (unsigned)bt.count;
    const BatchOff boA{bt.sA, bt.sK, Mp, (int64_t)s * Mp * Kp}, boB{bt.sB, bt.sK, Np, (int64_t)s * Np * Kp};
    if (Kp == OBK) {
        const int64_t row_blocks = (Mp * 32 + 255) / 256, col_blocks = Np / 32;
        prep_kernel<64><<<dim3((unsigned)(row_blocks + col_blocks), nz), 256, 0, st>>>(
            row_blocks, M, N, (int)K, A, lda, B, ldb, kmaxA, kmaxB, s, Mp, Np, ea, eb, pa, pb, boA, boB);
        RMGE_LAUNCH_CHECK();
    } else {
        row_exponent_kernel<<<dim3((unsigned)((M * 32 + 255) / 256), nz), 256, 0, st>>>(M, K, A, lda, kmaxA, kmaxB,
                                                                                       ea, boA);
        RMGE_LAUNCH_CHECK();
        col_exponent_kernel<<<dim3((unsigned)((N + 31) / 32), nz), 256, 0, st>>>(K, N, B, ldb, kmaxA, kmaxB, eb, boB);
        RMGE_LAUNCH_CHECK();
        row_digits_kernel<<<dim3(grid_for(Mp * Kp), nz), 256, 0, st>>>(M, K, A, lda, ea, kmaxA, kmaxB, s, Mp, Kp, pa,
                                                                       boA);
        RMGE_LAUNCH_CHECK();
        col_digits_kernel<<<dim3((unsigned)(Np / 32), (unsigned)(Kp / 32), nz), 256, 0, st>>>(
            K, N, B, ldb, eb, kmaxA, kmaxB, s, Np, Kp, pb, boB);
        RMGE_LAUNCH_CHECK();
    }

    const bool unit_alpha = (alpha == 1.0 || alpha == -1.0);
    const int mode = (unit_alpha && beta == 0.0) ? 0 : (unit_alpha && beta == 1.0) ? 1 : 2;
    const long long alpha_sign = (mode < 2 && alpha < 0.0) ? -1 : 1;
    const double alpha_g = (mode < 2) ? 1.0 : alpha;

    if (Kp == OBK && s >= 4) {  // one K block: the persistent update kernel
        CUtensorMap ta, tb;
        if (!tc_make_map(&ta, pa, true, (int64_t)bt.count * s * Mp, Kp, Kp, UBM) ||
            !tc_make_map(&tb, pb, true, (int64_t)bt.count * s * Np, Kp, Kp, UBN))
            return RMGE_ERR_CUDA;
        UpdParams u{};
        u.M = (int)M;
        u.N = (int)N;
        u.count = bt.count;
        u.sC = bt.sC;
        u.sFlag = bt.sFlag;
        u.F = kUpdF;
        u.Mp = (int)Mp;
        u.Np = (int)Np;
        u.tiles_n = (int)((N + UBN - 1) / UBN);
        u.tiles = (int)((M + UBM - 1) / UBM) * u.tiles_n;
        u.ea = ea;
        u.eb = eb;
        u.alpha_sign = alpha_sign;
        u.mode = mode;
        u.alpha = alpha_g;
        u.beta = beta;
        u.C = C;
        u.ldc = ldc;
        u.err = err;
        u.halt = bt.count == 1 ? halt : nullptr;  // a batch keeps going past one system's breakdown
        if (fuse != nullptr) {
            u.D = fuse->D;
            u.ldd = fuse->ldd;
            u.bd = fuse->b;
            u.dk = fuse->k;
            u.dinfo = fuse->info;
            u.dhalt = fuse->halt;
        }
        // idesc: FP32 accumulate, BF16 A and B, both K-major, N = 64, M = 128
        const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(UBN >> 3) << 17) |
                               ((uint32_t)(UBM >> 4) << 24);
        const int64_t all = (int64_t)u.tiles * bt.count;
        const int grid = all < sm_count() ? (int)all : sm_count();
        // GENP's balanced updates (per-k maxima given) are the ones rmge_launch_timing records
        const int64_t tk = kmaxA == nullptr ? -1
                                            : timing_begin(RMGE_TIMED_UPDATE, st, (double)(s * (s + 1) / 2) * 2.0 *
                                                                                      (double)M * (double)N * (double)K *
                                                                                      (double)bt.count);
        rmge_status rc;
        switch (s) {
            case 4: rc = launch_update<4>(ta, tb, u, idesc, grid, st); break;
            case 5: rc = launch_update<5>(ta, tb, u, idesc, grid, st); break;
            case 6: rc = launch_update<6>(ta, tb, u, idesc, grid, st); break;
            default: rc = launch_update<7>(ta, tb, u, idesc, grid, st); break;
        }
        timing_end(tk, st);
        return rc;
    }

    // |acc| < (chunks on diagonal 0 + 1) 2^(F + 10) must stay below 2^62
    int ch0 = (int)((Kp + 1023) / 1024), lg = 0;
    while ((1 << lg) < ch0 + 1) ++lg;
    CUtensorMap ta, tb;
    if (!tc_make_map(&ta, pa, true, (int64_t)bt.count * s * Mp, Kp, Kp, OBM) ||
        !tc_make_map(&tb, pb, true, (int64_t)bt.count * s * Np, Kp, Kp, OBN))
        return RMGE_ERR_CUDA;
    OzParams prm{};
    prm.M = (int)M;
    prm.N = (int)N;
    prm.K = (int)Kp;
    prm.s = s;
    prm.F = 52 - lg;
    prm.Mp = (int)Mp;
    prm.Np = (int)Np;
    prm.ea = ea;
    prm.eb = eb;
    prm.mode = mode;
    prm.alpha_sign = alpha_sign;
    prm.alpha = alpha_g;
    prm.beta = beta;
    prm.C = C;
    prm.ldc = ldc;
    prm.sC = bt.sC;
    prm.err = err;
    prm.halt = bt.count == 1 ? halt : nullptr;
    // idesc: FP32 accumulate, BF16 A and B, both K-major, N = 128, M = 128
    const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(OBN >> 3) << 17) |
                           ((uint32_t)(OBM >> 4) << 24);
    if (cudaFuncSetAttribute(oz_gemm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kOzSmem) != cudaSuccess) {
        (void)cudaGetLastError();
        return RMGE_ERR_CUDA;
    }
    oz_gemm_kernel<<<dim3((unsigned)((Np / OBN) * (Mp / OBM)), nz), OTHREADS, kOzSmem, st>>>(ta, tb, prm, idesc);
    RMGE_LAUNCH_CHECK();
    return RMGE_OK;
}

rmge_status oz_update128(int64_t M, int64_t N, int s, const double* A, int64_t lda, const double* B, int64_t ldb,
                         double* C, int64_t ldc, void* planesA, void* planesB, int* ea, int* eb,
                         const unsigned long long* kmaxA, const unsigned long long* kmaxB, int* err, const int* halt,
                         cudaStream_t st, const OzFuse* fuse, const OzBatch& bt) {
    if (bt.count < 1 || bt.count > 65535 || s < 4 || s > kOzSlices || (kmaxA == nullptr) != (kmaxB == nullptr))
        return RMGE_ERR_INVALID_ARG;
    if (fuse != nullptr && (fuse->D == nullptr || fuse->b < 1 || fuse->b > UBN || fuse->b > M || fuse->b > N ||
                            fuse->info == nullptr || fuse->halt == nullptr))
        return RMGE_ERR_INVALID_ARG;
    if (M <= 0 || N <= 0) return RMGE_OK;
    if (M > INT32_MAX / 16 || N > INT32_MAX / 16) return RMGE_ERR_INVALID_ARG;
    constexpr int64_t K = U2K, Kp = U2K;
    const int64_t Mp = (M + 127) / 128 * 128, Np = (N + 127) / 128 * 128;
    __nv_bfloat16* pa = static_cast<__nv_bfloat16*>(planesA);
    __nv_bfloat16* pb = static_cast<__nv_bfloat16*>(planesB);
    const unsigned nz = (unsigned)bt.count;
    const BatchOff boA{bt.sA, bt.sK, Mp, (int64_t)s * Mp * Kp}, boB{bt.sB, bt.sK, Np, (int64_t)s * Np * Kp};
    {
        const int64_t row_blocks = (Mp * 32 + 255) / 256, col_blocks = Np / 32;
        prep_kernel<U2K><<<dim3((unsigned)(row_blocks + col_blocks), nz), 256, 0, st>>>(
            row_blocks, M, N, (int)K, A, lda, B, ldb, kmaxA, kmaxB, s, Mp, Np, ea, eb, pa, pb, boA, boB);
        RMGE_LAUNCH_CHECK();
    }
    CUtensorMap ta, tb;
    if (!tc_make_map(&ta, pa, true, (int64_t)bt.count * s * Mp, Kp, Kp, UBM) ||
        !tc_make_map(&tb, pb, true, (int64_t)bt.count * s * Np, Kp, Kp, UBN))
        return RMGE_ERR_CUDA;
    UpdParams u{};
    u.M = (int)M;
    u.N = (int)N;
    u.count = bt.count;
    u.sC = bt.sC;
    u.sFlag = bt.sFlag;
    u.F = kUpd2F;
    u.Mp = (int)Mp;
    u.Np = (int)Np;
    u.tiles_n = (int)((N + UBN - 1) / UBN);
    u.tiles = (int)((M + UBM - 1) / UBM) * u.tiles_n;
    u.ea = ea;
    u.eb = eb;
    u.alpha_sign = -1;  // E - A B: mode 1 (alpha = -1, beta = 1)
    u.mode = 1;
    u.alpha = 1.0;
    u.beta = 1.0;
    u.C = C;
    u.ldc = ldc;
    u.err = err;
    u.halt = bt.count == 1 ? halt : nullptr;
    if (fuse != nullptr) {
        u.D = fuse->D;
        u.ldd = fuse->ldd;
        u.bd = fuse->b;
        u.dk = fuse->k;
        u.dinfo = fuse->info;
        u.dhalt = fuse->halt;
    }
    // idesc: FP32 accumulate, BF16 A and B, both K-major, N = 64, M = 128
    const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(UBN >> 3) << 17) |
                           ((uint32_t)(UBM >> 4) << 24);
    const int64_t all = (int64_t)u.tiles * bt.count;
    const int grid = all < sm_count() ? (int)all : sm_count();
    const int64_t tk = timing_begin(RMGE_TIMED_UPDATE128, st, (double)(s * (s + 1) / 2) * 2.0 * (double)M *
                                                                  (double)N * (double)K * (double)bt.count);
    rmge_status rc;
    switch (s) {
        case 4: rc = launch_update128<4>(ta, tb, u, idesc, grid, st); break;
        case 5: rc = launch_update128<5>(ta, tb, u, idesc, grid, st); break;
        case 6: rc = launch_update128<6>(ta, tb, u, idesc, grid, st); break;
        default: rc = launch_update128<7>(ta, tb, u, idesc, grid, st); break;
    }
    timing_end(tk, st);
    return rc;
}

}  // namespace rmge
