// genp.cu -- blocked Gaussian elimination with no pivoting (Sec. 3).
//
// One step of eq. (3.1) with a pivot block B of nb = kNb columns at offset k:
//   1. one CTA factors B = L11 U11 by unblocked GENP in shared memory (no pivot search: the only
//      branch is the breakdown test of Cor. 3.1).  In the FP64, FP32 and emulated-FP64 forms only
//      the first block has a launch of its own (diag_factor): every later block is the top-left tile
//      of the previous step's Schur update, and the CTA that computes that tile factors it in the same
//      launch (gemm_update_fused, oz_update).  The 16-bit tensor-core forms launch diag_factor per step.
//   2. panel_apply: row tiles of D become D B^{-1}-rows  L21 = A21 U11^{-1}  (each row of L21
//      depends on its own row of A21 only -- the row-parallel elimination that GENP allows and
//      partial pivoting does not), and column tiles of C become U12 = L11^{-1} A12, both by
//      substitution against the factored pivot block.
//   3. the Schur complement E <- E - L21 U12 (gemm).
// By Sec. 3 every blocking reaches the same Schur complements, so the packed L\U equals that of
// unblocked GENP up to rounding.  A zero or non-finite pivot records the 1-based step in
// DevState::info (atomicMin, first step wins) and raises DevState::halt, after which every later
// kernel of the factorization returns at once.
#include <climits>

#include "kernels.cuh"
#include "pivot_block.cuh"

namespace rmge {
namespace {

constexpr int NB = kNb;
constexpr int LDS = NB + 1;  // padded shared-memory row

template <typename T>
__device__ __forceinline__ bool finite_nonzero(T v) {
    return v != T(0) && isfinite(v);
}

// One CTA factors the pivot block in shared memory (pivot_block_genp, 256 threads).
struct CtaSync {
    __device__ void operator()() const { __syncthreads(); }
};

// blockIdx.y (here and in the kernels below): the system of a batch of equal-size factorizations, whose
// matrices lie sM elements apart and whose control blocks follow one another.
template <typename T>
__global__ void __launch_bounds__(256) diag_factor_kernel(int64_t k, int b, T* __restrict__ M, int64_t ldm,
                                                          DevState* st, int64_t sM) {
    __shared__ T a[NB * kPivotLds];
    __shared__ T rp;
    M += blockIdx.y * sM;
    st += blockIdx.y;
    if (*(volatile int*)&st->halt) return;
    const int tid = threadIdx.x;
    T* blk = M + k * ldm + k;
    for (int i = tid >> 6; i < b; i += 4)
        if ((tid & 63) < b) a[i * kPivotLds + (tid & 63)] = blk[i * ldm + (tid & 63)];
    __syncthreads();
    const int broke = pivot_block_genp<T, 256>(a, b, &rp, tid, CtaSync{});
    if (broke != 0) {
        if (tid == 0) {
            atomicMin(&st->info, (int)(k + broke));
            atomicExch(&st->halt, 1);
        }
        return;
    }
    for (int i = tid >> 6; i < b; i += 4)
        if ((tid & 63) < b) blk[i * ldm + (tid & 63)] = a[i * kPivotLds + (tid & 63)];
}

// Panel of pivot step k by substitution against the factored pivot block (in shared memory):
//   row tiles (blockIdx.x < row_tiles):  L21 = A21 U11^{-1}, row by row (x U11 = a);
//   column tiles:                         U12 = L11^{-1} A12, column by column (L11 x = a).
// PT rows (columns) per CTA, 16 lanes per row (column); the substitution of one row (column) is
// sequential over the b pivot columns, held in registers and stepped by 16-lane shuffles.  With kmax != NULL the
// kernel also leaves, for the balancing of the emulated Schur update, max_i |L21_ik| in kmax[k] and
// max_j |U12_kj| in kmax[uoff + k] (FP64 bit patterns of the finite maxima, merged by atomicMax into
// zeroed slots).
template <typename T, int PT>
__global__ void __launch_bounds__(256) panel_apply_kernel(int64_t k, int b, int64_t rest, int row_tiles,
                                                          T* __restrict__ M, int64_t ldm, const DevState* st,
                                                          unsigned long long* kmax, int64_t sM, int64_t sK,
                                                          int uoff) {
    static_assert(PT * 16 == 256, "16 lanes per row or column");
    __shared__ T dd[NB][LDS];
    __shared__ T tile[PT][LDS];  // row tile: tile[r][t]; column tile stored transposed: tile[c][t]
    __shared__ T rdiag[NB];      // 1 / u_jj, once per CTA (FP64 division is costly on GB300's FP64 pipe)
    M += blockIdx.y * sM;
    st += blockIdx.y;
    if (kmax != nullptr) kmax += blockIdx.y * sK;
    if (*(volatile const int*)&st->halt) return;
    const int tid = threadIdx.x;
    const bool is_row = (int)blockIdx.x < row_tiles;
    const int64_t t0 = (int64_t)(is_row ? blockIdx.x : blockIdx.x - row_tiles) * PT;
    const int64_t base = k + b + t0;  // first row (row tile) or column (column tile) of this tile
    const int cnt = (int)((rest - t0) < PT ? (rest - t0) : PT);
    for (int e = tid; e < b * b; e += blockDim.x) dd[e / b][e % b] = M[(k + e / b) * ldm + k + e % b];
    __syncthreads();
    if (is_row && tid < b) rdiag[tid] = T(1) / dd[tid][tid];
    if (is_row) {
        for (int e = tid; e < PT * NB; e += blockDim.x) {
            const int r = e / NB, t = e % NB;
            tile[r][t] = (r < cnt && t < b) ? M[(base + r) * ldm + k + t] : T(0);
        }
    } else {
        for (int e = tid; e < PT * NB; e += blockDim.x) {
            const int t = e / PT, c = e % PT;  // consecutive threads: consecutive columns of a row
            tile[c][t] = (c < cnt && t < b) ? M[(k + t) * ldm + base + c] : T(0);
        }
    }
    __syncthreads();
    // Row tiles solve x U11 = a as x U' = a D^{-1} with U11 = U' D (D its diagonal, U' unit): the
    // columns of U11 and the entries of a are scaled first, so every step of the substitution below is
    // a single DFMA on its dependency chain (GB300's FP64 latency is long).
    if (is_row)
        for (int e = tid; e < NB * NB; e += blockDim.x) {
            const int j = e / NB, t = e % NB;
            if (j < t && t < b) dd[j][t] *= rdiag[t];
        }
    const int q = tid >> 4, lane = tid & 15;  // row (column) q of the tile, lane within it
    // lane holds entries lane + 16 kk of its row (column); entry j is broadcast by its owner lane
    T x[NB / 16];
#pragma unroll
    for (int kk = 0; kk < NB / 16; ++kk) {
        const int t = lane + 16 * kk;
        x[kk] = (t < b) ? (is_row ? tile[q][t] * rdiag[t] : tile[q][t]) : T(0);
    }
    __syncthreads();
#pragma unroll
    for (int jj = 0; jj < NB / 16; ++jj)
        for (int jl = 0; jl < 16; ++jl) {
            const int j = 16 * jj + jl;
            if (j >= b) break;  // uniform
            const T xj = __shfl_sync(0xffffffffu, x[jj], jl, 16);
#pragma unroll
            for (int kk = jj; kk < NB / 16; ++kk) {
                const int t = lane + 16 * kk;
                if (t > j && t < b) x[kk] = fma(-xj, is_row ? dd[j][t] : dd[t][j], x[kk]);
            }
        }
#pragma unroll
    for (int kk = 0; kk < NB / 16; ++kk) {
        const int t = lane + 16 * kk;
        if (t < b) tile[q][t] = x[kk];
    }
    __syncthreads();
    if (kmax != nullptr && tid < b) {  // column tid of this tile's L21 rows, or row tid of its U12 columns
        unsigned long long m = 0ull;
        for (int r = 0; r < cnt; ++r) {
            const unsigned long long v = abs_bits((double)tile[r][tid]);
            if (v < 0x7ff0000000000000ull && v > m) m = v;  // finite entries only
        }
        if (m != 0ull) atomicMax(kmax + (is_row ? 0 : uoff) + tid, m);
    }
    if (is_row) {
        for (int e = tid; e < PT * NB; e += blockDim.x) {
            const int r = e / NB, jj = e % NB;
            if (r < cnt && jj < b) M[(base + r) * ldm + k + jj] = tile[r][jj];
        }
    } else {
        for (int e = tid; e < PT * NB; e += blockDim.x) {
            const int i = e / PT, c = e % PT;
            if (c < cnt && i < b) M[(k + i) * ldm + base + c] = tile[c][i];
        }
    }
}

template <typename T>
__global__ void maxabs_kernel(int64_t rows, int64_t cols, const T* __restrict__ P, int64_t ldp, bool upper_only,
                              unsigned long long* out, int64_t sP, int64_t sOut) {
    unsigned long long best = 0;
    P += blockIdx.y * sP;
    out += blockIdx.y * sOut;
    const int64_t total = rows * cols;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = e / cols, j = e % cols;
        if (upper_only && j < i) continue;
        const unsigned long long v = abs_bits((double)P[i * ldp + j]);
        best = v > best ? v : best;
    }
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long other = __shfl_xor_sync(0xffffffffu, best, o);
        best = other > best ? other : best;
    }
    if ((threadIdx.x & 31) == 0 && best != 0) atomicMax(out, best);
}

__global__ void finish_kernel(DevState* st, int32_t* info, double* growth) {
    st += blockIdx.x;
    if (info) info += blockIdx.x;
    if (growth) growth += blockIdx.x;
    const int v = st->info;
    if (info) *info = (v == INT_MAX) ? 0 : v;
    if (growth) {
        const double mu = __longlong_as_double((long long)st->maxabs_u);
        const double mm = __longlong_as_double((long long)st->maxabs_m);
        *growth = (v != INT_MAX) ? __longlong_as_double(0x7ff8000000000000LL) : mu / mm;
    }
}

}  // namespace

template <typename T>
rmge_status maxabs(int64_t rows, int64_t cols, const T* P, int64_t ldp, bool upper_only, unsigned long long* out_bits,
                   cudaStream_t s) {
    const int64_t total = rows * cols;
    int64_t g = (total + 255) / 256;
    if (g > 152 * 8) g = 152 * 8;
    if (g < 1) g = 1;
    maxabs_kernel<T><<<(unsigned)g, 256, 0, s>>>(rows, cols, P, ldp, upper_only, out_bits, 0, 0);
    RMGE_LAUNCH_CHECK();
    return RMGE_OK;
}

template <typename T>
rmge_status genp_factor(int64_t n, T* M, int64_t ldm, DevState* st, cudaStream_t s) {
    constexpr int PT = 16;
    RMGE_TRY(maxabs<T>(n, n, M, ldm, false, &st->maxabs_m, s));
    for (int64_t k = 0; k < n; k += NB) {
        const int b = (int)((n - k) < NB ? (n - k) : NB);
        if (k == 0) {  // every later pivot block is factored inside the previous step's update launch
            diag_factor_kernel<T><<<1, 256, 0, s>>>(k, b, M, ldm, st, 0);
            RMGE_LAUNCH_CHECK();
        }
        const int64_t rest = n - k - b;
        if (rest <= 0) break;
        const int tiles = (int)((rest + PT - 1) / PT);
        panel_apply_kernel<T, PT><<<2 * tiles, 256, 0, s>>>(k, b, rest, tiles, M, ldm, st, nullptr, 0, 0, 0);
        RMGE_LAUNCH_CHECK();
        RMGE_TRY(gemm_update_fused<T>(rest, rest, b, M + (k + b) * ldm + k, ldm, M + k * ldm + k + b, ldm,
                                      M + (k + b) * ldm + (k + b), ldm, &st->halt, (int)(rest < NB ? rest : NB),
                                      k + b, &st->info, &st->halt, s));
    }
    RMGE_TRY(maxabs<T>(n, n, M, ldm, true, &st->maxabs_u, s));
    return RMGE_OK;
}

// FP32 working matrix with the Schur-complement update on the tensor cores: the same pivot-block
// steps, with L21 and U12 converted to K-major 16-bit operands (two-term splits for three-pass
// products) and E <- E - L21 U12 done by tc_gemm.
rmge_status genp_factor_tc(int64_t n, float* M, int64_t ldm, DevState* st, const TcUpdate& tc,
                           cudaStream_t s) {
    constexpr int PT = 16;
    RMGE_TRY(maxabs<float>(n, n, M, ldm, false, &st->maxabs_m, s));
    int64_t step = 0;
    for (int64_t k = 0; k < n; k += NB, ++step) {
        const int b = (int)((n - k) < NB ? (n - k) : NB);
        diag_factor_kernel<float><<<1, 256, 0, s>>>(k, b, M, ldm, st, 0);
        RMGE_LAUNCH_CHECK();
        const int64_t rest = n - k - b;
        if (rest <= 0) break;
        const int tiles = (int)((rest + PT - 1) / PT);
        panel_apply_kernel<float, PT><<<2 * tiles, 256, 0, s>>>(k, b, rest, tiles, M, ldm, st, nullptr, 0, 0, 0);
        RMGE_LAUNCH_CHECK();
        const float* L21 = M + (k + b) * ldm + k;
        const float* U12 = M + k * ldm + k + b;
        unsigned long long* mxa = tc.scale ? tc.mx + 2 * step : nullptr;
        unsigned long long* mxb = tc.scale ? tc.mx + 2 * step + 1 : nullptr;
        if (tc.scale) {
            RMGE_TRY(maxabs<float>(rest, b, L21, ldm, false, mxa, s));
            RMGE_TRY(maxabs<float>(b, rest, U12, ldm, false, mxb, s));
        }
        RMGE_TRY(tc_split<float>(rest, b, L21, ldm, false, 1.0f, mxa, tc.bf16, tc.a_hi,
                                 tc.terms == 3 ? tc.a_lo : nullptr, tc.ldk, s));
        RMGE_TRY(tc_split<float>(b, rest, U12, ldm, true, 1.0f, mxb, tc.bf16, tc.b_hi,
                                 tc.terms == 3 ? tc.b_lo : nullptr, tc.ldk, s));
        RMGE_TRY(tc_gemm(rest, rest, b, tc.terms, tc.bf16, tc.a_hi, tc.a_lo, tc.ldk, tc.b_hi, tc.b_lo, tc.ldk, -1.0f,
                         1.0f, M + (k + b) * ldm + (k + b), ldm, &st->error, &st->halt, mxa, mxb, s));
    }
    RMGE_TRY(maxabs<float>(n, n, M, ldm, true, &st->maxabs_u, s));
    return RMGE_OK;
}

// The Schur update E <- E - L21 U12 as an emulated FP64 product.  Column k of L21 carries 1 / u_kk and
// row k of U12 carries u_kk, so the pair is first balanced by an exact power of two per k, from the
// per-k maxima that the panel kernel leaves; without it the per-row scaling of L21 and per-column
// scaling of U12 pair the large column of a small pivot with the large rows of other pivots and the
// update loses most of its relative accuracy.
//
// Pivot steps go in pairs (k, k + 1), with one step of look-ahead (the Schur complements are the same for
// any blocking, Sec. 3):
//   1. the panel of step k (L21, U12 and their per-k maxima);
//   2. step k's update of block column k + 1 only, whose launch also factors pivot block k + 1 (the CTA
//      holding it takes that tile alone), and of block row k + 1 only;
//   3. the panel of step k + 1;
//   4. one 128-deep update of the rest by both steps, E -= [L21_k L21_k+1] [U12_k; U12_k+1], whose
//      launch also factors pivot block k + 2.
// The trailing matrix is read and written once per pair instead of once per step: the emulated update is
// bound by that read-modify-write and the digit drains, not by its MMAs.  Steps whose trailing matrix is
// smaller than 4096 rows go unpaired: one 64-deep update that also factors the next pivot block.
rmge_status genp_factor_oz(int64_t n, double* M, int64_t ldm, DevState* st, const OzUpdate& oz, cudaStream_t s,
                           int count, int64_t sM, int digits) {
    constexpr int PT = 16;
    constexpr int64_t kPairRest = 4096;
    const unsigned nz = (unsigned)count;
    const int64_t sK = oz_kmax_per_system(n);
    constexpr int64_t kStateUll = sizeof(DevState) / sizeof(unsigned long long);
    constexpr int64_t kStateInt = sizeof(DevState) / sizeof(int);
    // growth numerator and denominator go to each system's control block
    {
        int64_t g = (n * n + 255) / 256;
        if (g > 152 * 8) g = 152 * 8;
        maxabs_kernel<double><<<dim3((unsigned)g, nz), 256, 0, s>>>(n, n, M, ldm, false, &st->maxabs_m, sM, kStateUll);
        RMGE_LAUNCH_CHECK();
    }
    OzBatch bt;
    bt.count = count;
    bt.sA = bt.sB = bt.sC = sM;
    bt.sK = sK;
    bt.sFlag = kStateInt;
    // maxima of step j: L21 columns at kmax + 256 (j / 2) + 64 (j % 2), U12 rows 128 slots further
    auto panel = [&](int64_t k, int b, int64_t rest, unsigned long long* kmL) -> rmge_status {
        const int tiles = (int)((rest + PT - 1) / PT);
        panel_apply_kernel<double, PT><<<dim3(2 * tiles, nz), 256, 0, s>>>(k, b, rest, tiles, M, ldm, st, kmL, sM,
                                                                           sK, 128);
        RMGE_LAUNCH_CHECK();
        return RMGE_OK;
    };
    diag_factor_kernel<double><<<dim3(1, nz), 256, 0, s>>>(0, (int)(n < NB ? n : NB), M, ldm, st, sM);
    RMGE_LAUNCH_CHECK();
    int64_t step = 0;
    for (int64_t k = 0; k < n;) {
        const int b = (int)((n - k) < NB ? (n - k) : NB);
        const int64_t rest = n - k - b;
        if (rest <= 0) break;
        unsigned long long* kmL = oz.kmax + 256 * (step / 2) + 64 * (step % 2);  // zeroed with the state
        RMGE_TRY(panel(k, b, rest, kmL));
        const double* L21 = M + (k + b) * ldm + k;
        const double* U12 = M + k * ldm + k + b;
        double* E = M + (k + b) * ldm + (k + b);
        // Pairing exposes the factorization of pivot block k + 1 (about 70 us on one SM) in the thin strip update,
        // and saves about a third of the Schur updates' time (128 x 64 tiles of 2 steps in 12 us instead of
        // 2 x 9.3 us): it pays once the trailing matrix has more than about 2^24 entries.  The test looks at one
        // system only, so that a system of a batch is factored exactly as it is alone.
        if (step % 2 != 0 || rest < kPairRest) {  // an unpaired step: one 64-deep update, next pivot fused
            const OzFuse next{E, ldm, (int)(rest < NB ? rest : NB), k + b, &st->info, &st->halt};
            RMGE_TRY(oz_gemm(rest, rest, b, digits, -1.0, L21, ldm, U12, ldm, 1.0, E, ldm, oz.planesA, oz.planesB,
                             oz.ea, oz.eb, kmL, kmL + 128, &st->error, &st->halt, s, &next, bt));
            k += b;
            ++step;
            continue;
        }
        // b == NB here.  Step k's update of block column k + 1 (factoring pivot block k + 1) and block row k + 1.
        const OzFuse next{E, ldm, NB, k + b, &st->info, &st->halt};
        RMGE_TRY(oz_gemm(rest, NB, b, digits, -1.0, L21, ldm, U12, ldm, 1.0, E, ldm, oz.planesA, oz.planesB, oz.ea,
                         oz.eb, kmL, kmL + 128, &st->error, &st->halt, s, &next, bt));
        RMGE_TRY(oz_gemm(NB, rest - NB, b, digits, -1.0, L21, ldm, U12 + NB, ldm, 1.0, E + NB, ldm, oz.planesA,
                         oz.planesB, oz.ea, oz.eb, kmL, kmL + 128, &st->error, &st->halt, s, nullptr, bt));
        // step k + 1's panel, then both steps' update of the rest in one 128-deep product
        const int64_t k1 = k + NB, rest1 = rest - NB;
        RMGE_TRY(panel(k1, NB, rest1, kmL + 64));
        double* E2 = M + (k1 + NB) * ldm + k1 + NB;
        const OzFuse next2{E2, ldm, (int)(rest1 < NB ? rest1 : NB), k1 + NB, &st->info, &st->halt};
        RMGE_TRY(oz_update128(rest1, rest1, digits, M + (k1 + NB) * ldm + k, ldm, M + k * ldm + k1 + NB, ldm, E2, ldm,
                              oz.planesA, oz.planesB, oz.ea, oz.eb, kmL, kmL + 128, &st->error, &st->halt, s, &next2,
                              bt));
        k += 2 * NB;
        step += 2;
    }
    {
        int64_t g = (n * n + 255) / 256;
        if (g > 152 * 8) g = 152 * 8;
        maxabs_kernel<double><<<dim3((unsigned)g, nz), 256, 0, s>>>(n, n, M, ldm, true, &st->maxabs_u, sM, kStateUll);
        RMGE_LAUNCH_CHECK();
    }
    return RMGE_OK;
}

rmge_status genp_finish(DevState* st, int32_t* info, double* growth, cudaStream_t s, int count) {
    finish_kernel<<<count, 1, 0, s>>>(st, info, growth);
    RMGE_LAUNCH_CHECK();
    return RMGE_OK;
}

template rmge_status genp_factor<double>(int64_t, double*, int64_t, DevState*, cudaStream_t);
template rmge_status genp_factor<float>(int64_t, float*, int64_t, DevState*, cudaStream_t);
template rmge_status maxabs<double>(int64_t, int64_t, const double*, int64_t, bool, unsigned long long*, cudaStream_t);
template rmge_status maxabs<float>(int64_t, int64_t, const float*, int64_t, bool, unsigned long long*, cudaStream_t);

}  // namespace rmge
