// trsv.cu -- triangular solves with the packed GENP factors, one launch per solve.
//
// The solves of Fact 4.1 (L z = b, U y = z) and of the adjoint (U^T p = g, L^T q = p) are
// blocked into TB-row blocks and KC-column blocks of the right-hand sides.  Each CTA owns one
// (row block, column block) and runs left-looking: it subtracts the contributions of the
// already-solved row blocks as they complete, then solves its diagonal block in shared memory.
// Completion is published per (row block, column block) with a release store of an epoch value;
// consumers acquire it.  CTAs take a ticket from an atomic counter at start and derive their
// block from it, so a CTA only ever waits for CTAs that took earlier tickets and are therefore
// already running: no co-residency assumption, no deadlock.  The last CTA to finish resets the
// counter, so consecutive solves on one stream need no re-initialisation.  Every wait is bounded
// (DevState::spin_limit polls, set per call); on expiry the CTA records RMGE_ERR_TIMEOUT in
// DevState::error and all waiting CTAs return without writing.
//
// The factor is read once from HBM per column block; FP64 runs on the DFMA pipe (2 FP64 operations per
// clock per SM on GB300).  The chain of row blocks is bound by the latency of each link (flag hand-off,
// the product with the block just solved, the diagonal substitution) more than by its FP64 work: one
// right-hand side takes nearly as long as sixteen.  So narrow column blocks (KC = 2) give more
// independent chains; the diagonal block is row-scaled by reciprocals formed before the CTA starts
// waiting, so that the substitution is one DFMA and one warp shuffle per step (one warp per column, no
// block-wide barriers), in two phases of 32 steps so that no step issues a DFMA whose lanes are all
// idle; one thread fences before the release.  Measured per 64-row block at n = 4096: flag hand-off
// 0.5 us, the product with the block just solved 2.8 to 3 us (64 x 64 x 2 FMAs: the FP64 throughput of
// one SM; two interleaved chains were no faster), the substitution 5.6 us (7.2 us before the two
// phases; 64 dependent DFMA + shuffle steps), release 0.5 to 0.8 us.
// An explicit inverse of the diagonal block (formed off the chain) replaces the substitution by a
// product but loses about u kappa of the block, which GENP's factors can make large; refined once
// with its residual it is accurate again but three block products cost more than the substitution.
#include "kernels.cuh"

namespace rmge {
namespace {

constexpr int TB = kTrsvRows;
constexpr int KC = kTrsvCols;
constexpr int NT = TB * KC;  // one thread per (row, column) of the block

// Coefficient (i, t) of the triangular matrix of `kind`, read from the packed factors.
template <typename T>
__device__ __forceinline__ T coef(int kind, const T* LU, int64_t ld, int64_t i, int64_t t) {
    return (kind <= 1) ? LU[i * ld + t] : LU[t * ld + i];
}

// The last CTA to finish re-arms the ticket counters for the next solve on the stream.
__device__ __forceinline__ void finish_ticket(DevState* st) {
    if (atomicAdd(&st->done, 1u) == gridDim.x - 1) {
        st->ticket = 0u;
        st->done = 0u;
        __threadfence();
    }
}

template <typename T>
__global__ void __launch_bounds__(NT) trsv_kernel(int kind, int64_t n, int64_t nrhs, const T* __restrict__ LU,
                                                  int64_t ld, T* B, int64_t ldb, DevState* st, int* flags,
                                                  int epoch, const int* skip, Zb zb) {
    extern __shared__ __align__(16) unsigned char trsv_smem[];
    // a batch's systems (blockIdx.z) each have their own factors, right-hand sides, ticket counter and flags
    skip = zws(skip, zb.ws);
    st = zws(st, zb.ws);
    flags = zws(flags, zb.ws);
    LU = zmat(LU, zb.m0);
    B = zmat(B, zb.m1);
    T (*cs)[TB + 1] = reinterpret_cast<T (*)[TB + 1]>(trsv_smem);  // off-diagonal coefficient tile
    T (*cd)[TB + 1] = cs + TB;                                     // diagonal block
    __shared__ T ys[TB][KC];
    __shared__ T rd[TB];  // reciprocals of the diagonal (non-unit kinds)
    __shared__ int my_ticket;
    __shared__ int failed;
    if (skip != nullptr && *(volatile const int*)skip != 0) return;

    const int tid = threadIdx.x;
    const int r = tid / KC, c = tid % KC;
    const int64_t nblk = (n + TB - 1) / TB;
    const int64_t ncb = (nrhs + KC - 1) / KC;
    if (tid == 0) {
        my_ticket = (int)atomicAdd(&st->ticket, 1u);
        failed = 0;
    }
    __syncthreads();
    const int64_t q = my_ticket / ncb, cb = my_ticket % ncb;
    const bool forward = (kind == 0 || kind == 2);
    const bool unit = (kind == 0 || kind == 3);
    const int64_t rb = forward ? q : nblk - 1 - q;
    const int64_t r0 = rb * TB, c0 = cb * KC;
    const int64_t gr = r0 + r, gc = c0 + c;
    const bool live = (gr < n) && (gc < nrhs);

    T acc = live ? B[gr * ldb + gc] : T(0);

    // The diagonal block's coefficients do not depend on other blocks: stage them first.
    for (int e = tid; e < TB * TB; e += NT) {
        int i, t;
        if (kind <= 1) { i = e / TB; t = e % TB; }   // rows of LU: contiguous along t
        else           { t = e / TB; i = e % TB; }   // transposed: contiguous along i
        const int64_t gi = r0 + i, gt = r0 + t;
        cd[i][t] = (gi < n && gt < n) ? coef(kind, LU, ld, gi, gt) : ((i == t) ? T(1) : T(0));
    }
    __syncthreads();
    if (!unit && tid < TB) rd[tid] = T(1) / cd[tid][tid];
    __syncthreads();
    // Non-unit kinds: row i of the block is divided by its diagonal entry, so the substitution below
    // runs on a unit triangle and its chain of dependent steps carries no multiplication by 1 / u_ii.
    if (!unit)
        for (int e = tid; e < TB * TB; e += NT) {
            const int i = e / TB, t = e % TB;
            if (t != i) cd[i][t] *= rd[i];
        }

    constexpr int CPT = TB * TB / NT;  // coefficients per thread per tile
    for (int64_t qq = 0; qq < q; ++qq) {
        const int64_t sb = forward ? qq : nblk - 1 - qq;
        const int64_t s0 = sb * TB;
        // coefficient tile (rows r0.., columns s0..): fetched before waiting, it is final already
        T cr[CPT];
#pragma unroll
        for (int u = 0; u < CPT; ++u) {
            const int e = tid + u * NT;
            int i, t;
            if (kind <= 1) { i = e / TB; t = e % TB; }
            else           { t = e / TB; i = e % TB; }
            const int64_t gi = r0 + i, gt = s0 + t;
            cr[u] = (gi < n && gt < n) ? coef(kind, LU, ld, gi, gt) : T(0);
        }
        if (tid == 0) {
            const int* f = flags + sb * ncb + cb;
            const long long limit = *(volatile const long long*)&st->spin_limit;
            long long spins = 0;
            while (ld_acquire(f) != epoch) {
                if (*(volatile int*)&st->error != 0) { failed = 1; break; }
                if (++spins > limit) {
                    atomicExch(&st->error, (int)RMGE_ERR_TIMEOUT);
                    failed = 1;
                    break;
                }
                __nanosleep(64);
            }
        }
        __syncthreads();
        if (failed) {
            if (tid == 0) finish_ticket(st);
            return;
        }
#pragma unroll
        for (int u = 0; u < CPT; ++u) {
            const int e = tid + u * NT;
            int i, t;
            if (kind <= 1) { i = e / TB; t = e % TB; }
            else           { t = e / TB; i = e % TB; }
            cs[i][t] = cr[u];
        }
        {
            const int64_t gt = s0 + r;
            ys[r][c] = (gt < n && gc < nrhs) ? ldcg(B + gt * ldb + gc) : T(0);
        }
        __syncthreads();
#pragma unroll 8
        for (int t = 0; t < TB; ++t) acc = fma(-cs[r][t], ys[t][c], acc);
        __syncthreads();
    }

    // diagonal block: column-oriented substitution inside the (row-scaled, unit) block, one warp per
    // column (lane l holds rows l and l + 32), stepping by warp shuffles instead of block-wide barriers
    static_assert(TB == 64, "two rows per lane");
    ys[r][c] = unit ? acc : acc * rd[r];  // the row scaling of the right-hand side
    __syncthreads();
    const int warp = tid >> 5, lane = tid & 31;
    if (warp < KC) {
        const int col = warp;
        T x0 = ys[lane][col], x1 = ys[lane + 32][col];
        // Two phases of 32 steps.  While the rows of one half are being finalised, every row of the other
        // half is still pending (one unpredicated DFMA); once that half is done, the loop touches only the
        // other register, so no step issues a DFMA with all lanes idle.
        if (forward) {
#pragma unroll 8
            for (int p = 0; p < 32; ++p) {
                const T y = __shfl_sync(0xffffffffu, x0, p);  // final: unit diagonal
                if (lane > p) x0 = fma(-cd[lane][p], y, x0);
                x1 = fma(-cd[lane + 32][p], y, x1);
            }
#pragma unroll 8
            for (int p = 32; p < TB; ++p) {
                const T y = __shfl_sync(0xffffffffu, x1, p - 32);
                if (lane + 32 > p) x1 = fma(-cd[lane + 32][p], y, x1);
            }
        } else {
#pragma unroll 8
            for (int p = TB - 1; p >= 32; --p) {
                const T y = __shfl_sync(0xffffffffu, x1, p - 32);
                if (lane + 32 < p) x1 = fma(-cd[lane + 32][p], y, x1);
                x0 = fma(-cd[lane][p], y, x0);
            }
#pragma unroll 8
            for (int p = 31; p >= 0; --p) {
                const T y = __shfl_sync(0xffffffffu, x0, p);
                if (lane < p) x0 = fma(-cd[lane][p], y, x0);
            }
        }
        const int64_t gcol = c0 + col;
        if (gcol < nrhs) {
            if (r0 + lane < n) B[(r0 + lane) * ldb + gcol] = x0;
            if (r0 + lane + 32 < n) B[(r0 + lane + 32) * ldb + gcol] = x1;
        }
    }
    // the block's results are published by one release after the barrier (the barrier orders the
    // other threads' stores before thread 0's fence)
    __syncthreads();
    if (tid == 0) {
        __threadfence();
        st_release(flags + rb * ncb + cb, epoch);
        finish_ticket(st);
    }
}

}  // namespace

template <typename T>
rmge_status trsv(int kind, int64_t n, int64_t nrhs, const T* LU, int64_t ldlu, T* B, int64_t ldb, DevState* st,
                 int* flags, int epoch, const int* skip, cudaStream_t s, const Zb& zb) {
    const int64_t nblk = (n + TB - 1) / TB;
    const int64_t ncb = (nrhs + KC - 1) / KC;
    const int64_t grid = nblk * ncb;
    const size_t smem = 2 * (size_t)TB * (TB + 1) * sizeof(T);
    if (cudaFuncSetAttribute(trsv_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) {
        (void)cudaGetLastError();
        return RMGE_ERR_CUDA;
    }
    // CTAs of a batch take tickets from their own system's counter and wait only for that system's earlier
    // tickets, which are running already: systems do not wait for one another
    trsv_kernel<T><<<dim3((unsigned)grid, 1, (unsigned)zb.count), NT, smem, s>>>(kind, n, nrhs, LU, ldlu, B, ldb, st,
                                                                               flags, epoch, skip, zb);
    RMGE_LAUNCH_CHECK();
    return RMGE_OK;
}

template rmge_status trsv<double>(int, int64_t, int64_t, const double*, int64_t, double*, int64_t, DevState*, int*,
                                  int, const int*, cudaStream_t, const Zb&);
template rmge_status trsv<float>(int, int64_t, int64_t, const float*, int64_t, float*, int64_t, DevState*, int*, int,
                                 const int*, cudaStream_t, const Zb&);

}  // namespace rmge
