// genp.cu -- blocked Gaussian elimination with no pivoting (Sec. 3).
//
// One step of eq. (3.1) with a pivot block B of nb = kNb columns at offset k:
//   1. diag_factor: one CTA factors B = L11 U11 by unblocked GENP in shared memory (no pivot
//      search: the only branch is the breakdown test of Cor. 3.1), then forms U11^{-1} and
//      L11^{-1} in shared memory and writes them to the workspace.
//   2. panel_apply: row tiles of D become D B^{-1}-rows  L21 = A21 U11^{-1}  (each row of L21
//      depends on its own row of A21 only -- the row-parallel elimination that GENP allows and
//      partial pivoting does not), and column tiles of C become U12 = L11^{-1} A12.
//   3. the Schur complement E <- E - L21 U12 (gemm).
// By Sec. 3 every blocking reaches the same Schur complements, so the packed L\U equals that of
// unblocked GENP up to rounding.  A zero or non-finite pivot records the 1-based step in
// DevState::info (atomicMin, first step wins) and raises DevState::halt, after which every later
// kernel of the factorization returns at once.
#include <climits>

#include "kernels.cuh"

namespace rmge {
namespace {

constexpr int NB = kNb;
constexpr int LDS = NB + 1;  // padded shared-memory row

template <typename T>
__device__ __forceinline__ bool finite_nonzero(T v) {
    return v != T(0) && isfinite(v);
}

// Dynamic shared memory: a[NB][LDS], ui[NB][LDS], li[NB][LDS].
template <typename T>
__global__ void __launch_bounds__(256) diag_factor_kernel(int64_t k, int b, T* __restrict__ M, int64_t ldm,
                                                          DevState* st, T* __restrict__ inv) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* a = reinterpret_cast<T*>(smem_raw);
    T* ui = a + NB * LDS;
    T* li = ui + NB * LDS;
    __shared__ int broke;
    if (*(volatile int*)&st->halt) return;
    const int tid = threadIdx.x;
    T* blk = M + k * ldm + k;
    for (int e = tid; e < NB * NB; e += blockDim.x) {
        const int i = e / NB, j = e % NB;
        a[i * LDS + j] = (i < b && j < b) ? blk[i * ldm + j] : (i == j ? T(1) : T(0));
    }
    if (tid == 0) broke = 0;
    __syncthreads();

    // Unblocked GENP of the pivot block: step s is eq. (3.1) with a 1 x 1 pivot block.
    for (int s = 0; s < b; ++s) {
        const T piv = a[s * LDS + s];
        if (!finite_nonzero(piv)) {
            if (tid == 0) {
                atomicMin(&st->info, (int)(k + s + 1));
                atomicExch(&st->halt, 1);
                broke = 1;
            }
            break;  // uniform: every thread read the same pivot
        }
        for (int i = s + 1 + tid; i < b; i += blockDim.x) a[i * LDS + s] /= piv;
        __syncthreads();
        const int w = b - s - 1;
        for (int e = tid; e < w * w; e += blockDim.x) {
            const int i = s + 1 + e / w, j = s + 1 + e % w;
            a[i * LDS + j] = fma(-a[i * LDS + s], a[s * LDS + j], a[i * LDS + j]);
        }
        __syncthreads();
    }
    __syncthreads();
    if (broke) return;

    for (int e = tid; e < b * b; e += blockDim.x) {
        const int i = e / b, j = e % b;
        blk[i * ldm + j] = a[i * LDS + j];
    }

    // Triangular inverses, NB steps; threads 0..127 build U^{-1} bottom-up row by row, threads
    // 128..255 build L^{-1} top-down, two threads per column splitting each dot product.
    // Padding rows/columns (>= b) of a hold the identity, so the inverses are block-identity there.
    for (int e = tid; e < NB * NB; e += blockDim.x) {
        ui[(e / NB) * LDS + e % NB] = T(0);
        li[(e / NB) * LDS + e % NB] = T(0);
    }
    __syncthreads();
    const bool upper = tid < 128;
    const int lt = upper ? tid : tid - 128;
    const int j = lt >> 1, half = lt & 1;
    for (int step = 0; step < NB; ++step) {
        T sum = T(0);
        if (upper) {
            const int i = NB - 1 - step;  // row of U^{-1} being formed; rows > i are final
            if (j >= i) {
                for (int t = i + 1 + half; t <= j; t += 2) sum = fma(a[i * LDS + t], ui[t * LDS + j], sum);
            }
            sum += __shfl_xor_sync(0xffffffffu, sum, 1);
            if (j >= i && half == 0) ui[i * LDS + j] = ((i == j ? T(1) : T(0)) - sum) / a[i * LDS + i];
        } else {
            const int i = step;  // row of L^{-1} being formed; rows < i are final
            if (j <= i) {
                for (int t = j + half; t < i; t += 2) sum = fma(a[i * LDS + t], li[t * LDS + j], sum);
            }
            sum += __shfl_xor_sync(0xffffffffu, sum, 1);
            if (j <= i && half == 0) li[i * LDS + j] = (i == j ? T(1) : T(0)) - sum;
        }
        __syncthreads();
    }
    for (int e = tid; e < NB * NB; e += blockDim.x) {
        const int i = e / NB, jj = e % NB;
        inv[e] = ui[i * LDS + jj];
        inv[NB * NB + e] = li[i * LDS + jj];
    }
}

// Row tiles (blockIdx.x < row_tiles): L21[rows] = A21[rows] * U11^{-1}.
// Column tiles: U12[:, cols] = L11^{-1} * A12[:, cols].  PT rows/columns per CTA.
template <typename T, int PT>
__global__ void __launch_bounds__(256) panel_apply_kernel(int64_t k, int b, int64_t rest, int row_tiles,
                                                          T* __restrict__ M, int64_t ldm, const DevState* st,
                                                          const T* __restrict__ inv) {
    __shared__ T iv[NB][LDS];
    __shared__ T tile[PT][LDS];  // row tile: tile[r][t]; column tile stored transposed: tile[c][t]
    if (*(volatile const int*)&st->halt) return;
    const int tid = threadIdx.x;
    const bool is_row = (int)blockIdx.x < row_tiles;
    const int64_t t0 = (int64_t)(is_row ? blockIdx.x : blockIdx.x - row_tiles) * PT;
    const int64_t base = k + b + t0;  // first row (row tile) or column (column tile) of this tile
    const int cnt = (int)((rest - t0) < PT ? (rest - t0) : PT);
    const T* src_inv = inv + (is_row ? 0 : NB * NB);
    for (int e = tid; e < NB * NB; e += blockDim.x) iv[e / NB][e % NB] = src_inv[e];
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
    // each thread: outputs (r, j) with e = tid + q*256 over PT*NB outputs
    constexpr int PER = PT * NB / 256;
    T out[PER];
#pragma unroll
    for (int q = 0; q < PER; ++q) {
        const int e = tid + q * 256;
        T sum = T(0);
        if (is_row) {  // L21[r][j] = sum_{t <= j} A21[r][t] Uinv[t][j]
            const int r = e / NB, jj = e % NB;
            for (int t = 0; t <= jj; ++t) sum = fma(tile[r][t], iv[t][jj], sum);
        } else {  // U12[i][c] = sum_{t <= i} Linv[i][t] A12[t][c]
            const int i = e / PT, c = e % PT;
            for (int t = 0; t <= i; ++t) sum = fma(iv[i][t], tile[c][t], sum);
        }
        out[q] = sum;
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < PER; ++q) {
        const int e = tid + q * 256;
        if (is_row) {
            const int r = e / NB, jj = e % NB;
            if (r < cnt && jj < b) M[(base + r) * ldm + k + jj] = out[q];
        } else {
            const int i = e / PT, c = e % PT;
            if (c < cnt && i < b) M[(k + i) * ldm + base + c] = out[q];
        }
    }
}

template <typename T>
__global__ void maxabs_kernel(int64_t rows, int64_t cols, const T* __restrict__ P, int64_t ldp, bool upper_only,
                              unsigned long long* out) {
    unsigned long long best = 0;
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
    maxabs_kernel<T><<<(unsigned)g, 256, 0, s>>>(rows, cols, P, ldp, upper_only, out_bits);
    RMGE_LAUNCH_CHECK();
    return RMGE_OK;
}

template <typename T>
rmge_status genp_factor(int64_t n, T* M, int64_t ldm, DevState* st, T* inv, cudaStream_t s) {
    constexpr int PT = 16;
    const size_t smem = 3 * NB * LDS * sizeof(T);
    // The attribute belongs to the current device's context; setting it is cheap and idempotent.
    if (cudaFuncSetAttribute(diag_factor_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
        cudaSuccess) {
        (void)cudaGetLastError();
        return RMGE_ERR_CUDA;
    }
    RMGE_TRY(maxabs<T>(n, n, M, ldm, false, &st->maxabs_m, s));
    for (int64_t k = 0; k < n; k += NB) {
        const int b = (int)((n - k) < NB ? (n - k) : NB);
        diag_factor_kernel<T><<<1, 256, smem, s>>>(k, b, M, ldm, st, inv);
        RMGE_LAUNCH_CHECK();
        const int64_t rest = n - k - b;
        if (rest <= 0) break;
        const int tiles = (int)((rest + PT - 1) / PT);
        panel_apply_kernel<T, PT><<<2 * tiles, 256, 0, s>>>(k, b, rest, tiles, M, ldm, st, inv);
        RMGE_LAUNCH_CHECK();
        RMGE_TRY(gemm<T>(false, rest, rest, b, T(-1), M + (k + b) * ldm + k, ldm, M + k * ldm + k + b, ldm, T(1),
                         M + (k + b) * ldm + (k + b), ldm, &st->halt, s));
    }
    RMGE_TRY(maxabs<T>(n, n, M, ldm, true, &st->maxabs_u, s));
    return RMGE_OK;
}

rmge_status genp_finish(DevState* st, int32_t* info, double* growth, cudaStream_t s) {
    finish_kernel<<<1, 1, 0, s>>>(st, info, growth);
    RMGE_LAUNCH_CHECK();
    return RMGE_OK;
}

template rmge_status genp_factor<double>(int64_t, double*, int64_t, DevState*, double*, cudaStream_t);
template rmge_status genp_factor<float>(int64_t, float*, int64_t, DevState*, float*, cudaStream_t);
template rmge_status maxabs<double>(int64_t, int64_t, const double*, int64_t, bool, unsigned long long*, cudaStream_t);
template rmge_status maxabs<float>(int64_t, int64_t, const float*, int64_t, bool, unsigned long long*, cudaStream_t);

}  // namespace rmge
