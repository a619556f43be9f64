// lowrank.cu -- randomized low-rank approximation (Sec. 6, Algorithm 6.1).
//
//   B = A H            (m x l; H an n x l Gaussian, or the n x l leading block of a random circulant,
//                       Sec. 7.2, applied by FFT row correlation truncated to l outputs)
//   Q = Q(B)           orthonormal columns sharing B's range: CholeskyQR2 (two passes of
//                       W = Q^T Q = R^T R, Q <- Q R^{-1}), R with a positive diagonal, so Q is the unique
//                       thin QR factor of a full-rank B
//   Z = Q^T A          (l x n), so that A ~ Q Z = Q Q^T A (rank <= l)
//
// The paper's algorithm needs any orthonormal basis of range(A H); CholeskyQR2 replaces Householder
// QR because on the GPU it is two Gram products (HBM-bound over the tall B) and two row-parallel
// triangular solves instead of l sequential reflections.  It needs B well-conditioned enough for the
// first Cholesky (kappa(B) well below 1e8), which holds for l equal to the numerical rank, the
// paper's setting; a non-positive Cholesky pivot is reported (info > 0) and the solve stops.
// FP64 throughout (the DFMA pipe).
#include "kernels.cuh"

namespace rmge {
namespace {

constexpr int kGramRows = 64;  // rows of Q per CTA of the Gram kernel (33 KB of shared memory)
constexpr int kMaxL = kLowRankMaxL;

// W (l x l) += Q_chunk^T Q_chunk over a chunk of rows, with FP64 atomics into the zeroed W.
__global__ void __launch_bounds__(256) gram_kernel(int64_t m, int l, const double* __restrict__ Q, int64_t ldq,
                                                   double* __restrict__ W, const int* halt) {
    __shared__ double q[kGramRows][kMaxL + 1];
    if (halt != nullptr && *(volatile const int*)halt != 0) return;
    const int64_t r0 = (int64_t)blockIdx.x * kGramRows;
    const int rows = (int)((m - r0) < kGramRows ? (m - r0) : kGramRows);
    for (int e = threadIdx.x; e < kGramRows * l; e += blockDim.x) {
        const int i = e / l, j = e % l;
        q[i][j] = (i < rows) ? Q[(r0 + i) * ldq + j] : 0.0;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < l * l; e += blockDim.x) {
        const int a = e / l, b = e % l;
        if (b < a) continue;  // symmetric: the upper triangle, mirrored below
        double acc = 0.0;
        for (int i = 0; i < rows; ++i) acc = fma(q[i][a], q[i][b], acc);
        atomicAdd(&W[a * l + b], acc);
        if (b != a) atomicAdd(&W[b * l + a], acc);
    }
}

// One CTA: W = R^T R (upper R, positive diagonal) by the column-oriented Cholesky; rinv[j] = 1 / R_jj.
// A pivot that is not positive beyond rounding (R_jj^2 <= 64 u W_jj, or non-finite) records
// info = j + 1 and raises the halt flag.
__global__ void __launch_bounds__(kMaxL) chol_kernel(int l, const double* __restrict__ W, double* __restrict__ R,
                                                     double* __restrict__ rinv, int* info, int* halt) {
    __shared__ double r[kMaxL][kMaxL + 1];
    __shared__ int bad;
    const int c = threadIdx.x;
    if (*(volatile const int*)halt != 0) return;
    if (c == 0) bad = 0;
    for (int i = 0; i < l; ++i)
        if (c < l) r[i][c] = W[i * l + c];
    __syncthreads();
    for (int j = 0; j < l; ++j) {
        // the pivot: R_jj^2 = W_jj - sum_{k<j} R_kj^2 (rows k < j of column j are final)
        if (c == j) {
            double d = r[j][j];
            for (int k = 0; k < j; ++k) d = fma(-r[k][j], r[k][j], d);
            // a pivot below 64 u of its Gram entry means B has numerical rank below l
            if (!(d > 64.0 * 1.1102230246251565e-16 * W[j * l + j]) || !isfinite(d)) {
                bad = j + 1;
            } else {
                r[j][j] = sqrt(d);
            }
        }
        __syncthreads();
        if (bad != 0) break;
        // row j: R_jc = (W_jc - sum_{k<j} R_kj R_kc) / R_jj for c > j
        if (c > j && c < l) {
            double v = r[j][c];
            for (int k = 0; k < j; ++k) v = fma(-r[k][j], r[k][c], v);
            r[j][c] = v / r[j][j];
        }
        __syncthreads();
    }
    if (bad != 0) {
        if (c == 0) {
            *info = bad;
            *halt = 1;
        }
        return;
    }
    if (c < l) {
        for (int i = 0; i < l; ++i) R[i * l + c] = (i <= c) ? r[i][c] : 0.0;
        rinv[c] = 1.0 / r[c][c];
    }
}

// Q <- Q R^{-1} row by row (y R = x, forward substitution over the columns), one warp per row; lane t
// holds entries t and t + 32.
__global__ void __launch_bounds__(256) right_solve_kernel(int64_t m, int l, double* __restrict__ Q, int64_t ldq,
                                                          const double* __restrict__ R,
                                                          const double* __restrict__ rinv, const int* halt) {
    __shared__ double r[kMaxL][kMaxL + 1];
    __shared__ double ri[kMaxL];
    if (*(volatile const int*)halt != 0) return;
    for (int e = threadIdx.x; e < l * l; e += blockDim.x) r[e / l][e % l] = R[e];
    for (int e = threadIdx.x; e < l; e += blockDim.x) ri[e] = rinv[e];
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int64_t row = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (row >= m) return;
    double* q = Q + row * ldq;
    double x0 = (lane < l) ? q[lane] : 0.0, x1 = (lane + 32 < l) ? q[lane + 32] : 0.0;
    for (int j = 0; j < l; ++j) {
        const double xj = __shfl_sync(0xffffffffu, (j < 32) ? x0 : x1, j & 31);
        const double yj = xj * ri[j];
        if (lane == (j & 31)) {
            if (j < 32) x0 = yj;
            else x1 = yj;
        }
        if (lane > j && lane < l) x0 = fma(-yj, r[j][lane], x0);
        if (lane + 32 > j && lane + 32 < l) x1 = fma(-yj, r[j][lane + 32], x1);
    }
    if (lane < l) q[lane] = x0;
    if (lane + 32 < l) q[lane + 32] = x1;
}

__global__ void zero_kernel(int64_t count, double* p) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x)
        p[i] = 0.0;
}

__global__ void lowrank_state_kernel(int* info, int* halt) {
    *info = 0;
    *halt = 0;
}

__global__ void copy_info_kernel(const int* src, int32_t* dst) { *dst = *src; }

}  // namespace

size_t lowrank_workspace_bytes(int64_t n, int l, bool fft) {
    size_t b = 256;                                             // info, halt
    b += (size_t)(3 * l * l + l) * sizeof(double);              // W, R, (spare), rinv
    b = (b + 255) / 256 * 256;
    if (fft) b += (size_t)(n / 2 + 1) * sizeof(double2);        // twiddles
    return (b + 255) / 256 * 256;
}

rmge_status lowrank_basis(int kind, int64_t m, int64_t n, int l, const double* A, int64_t lda, const double* H,
                          double* Q, int64_t ldq, int32_t* info, void* ws, cudaStream_t s) {
    char* base = static_cast<char*>(ws);
    int* dinfo = reinterpret_cast<int*>(base);
    int* halt = dinfo + 1;
    double* W = reinterpret_cast<double*>(base + 256);
    double* R = W + l * l;
    double* rinv = R + 2 * l * l;
    const size_t head = (256 + (size_t)(3 * l * l + l) * sizeof(double) + 255) / 256 * 256;
    double2* tw = reinterpret_cast<double2*>(base + head);
    lowrank_state_kernel<<<1, 1, 0, s>>>(dinfo, halt);
    RMGE_LAUNCH_CHECK();
    // B = A H into Q
    if (kind == 0)
        RMGE_TRY(gemm<double>(false, m, l, n, 1.0, A, lda, H, l, 0.0, Q, ldq, nullptr, s));
    else
        RMGE_TRY(circulant_apply_rows_block(m, n, l, A, lda, H, tw, Q, ldq, s));
    // CholeskyQR2
    for (int pass = 0; pass < 2; ++pass) {
        zero_kernel<<<(unsigned)((l * l + 255) / 256), 256, 0, s>>>((int64_t)l * l, W);
        RMGE_LAUNCH_CHECK();
        gram_kernel<<<(unsigned)((m + kGramRows - 1) / kGramRows), 256, 0, s>>>(m, l, Q, ldq, W, halt);
        RMGE_LAUNCH_CHECK();
        chol_kernel<<<1, kMaxL, 0, s>>>(l, W, R, rinv, dinfo, halt);
        RMGE_LAUNCH_CHECK();
        right_solve_kernel<<<(unsigned)((m * 32 + 255) / 256), 256, 0, s>>>(m, l, Q, ldq, R, rinv, halt);
        RMGE_LAUNCH_CHECK();
    }
    if (info != nullptr) {
        copy_info_kernel<<<1, 1, 0, s>>>(dinfo, info);
        RMGE_LAUNCH_CHECK();
    }
    return RMGE_OK;
}

rmge_status lowrank_project(int64_t m, int64_t n, int l, const double* Q, int64_t ldq, const double* A, int64_t lda,
                            double* Z, int64_t ldz, cudaStream_t s) {
    return gemm<double>(true, l, n, m, 1.0, Q, ldq, A, lda, 0.0, Z, ldz, nullptr, s);
}

}  // namespace rmge
