// gemm.cu -- register-tiled SIMT GEMM on the FMA pipes: C = alpha op(A) B + beta C.
//
// Used for the FP64 path, where GB300's FP64 runs only on the DFMA pipe (about 2 DFMA per
// clock per SM; the FP64 tensor path measures slower), so the kernel's job is to keep that pipe
// issuing: each thread owns a TM x TN register tile and does TM*TN FMAs per TM + TN shared-memory
// loads, the next K slice is prefetched into registers while the current one is consumed, and
// the tile size is chosen so that every SM gets several tiles.  The same template serves FP32
// (RMGE_F32 working matrices and skinny products).
//
// Roles on the path: M = A G (Fact 4.1; 2n^3 - n^2 flops), the Schur-complement update
// E <- E - (D B^-1)(B^-1 C) of eq. (3.1) in the blocked GENP, X = G Y, R = B - A X and the
// adjoint product G^T dX.
#include "kernels.cuh"

namespace rmge {
namespace {

// Thread (tx, ty) owns rows ty + i*RY and columns tx + j*RX of the CTA tile (i < TM, j < TN), so
// a warp's shared-memory reads are broadcasts (A) or consecutive words (B), and its global
// stores are consecutive along a row.
template <typename T, typename SA, typename SB, int BM, int BN, int BK, int TM, int TN, bool TA>
__global__ void __launch_bounds__((BM / TM) * (BN / TN))
gemm_kernel(int64_t M, int64_t N, int64_t K, T alpha, const SA* __restrict__ A, int64_t lda,
            const SB* __restrict__ B, int64_t ldb, T beta, T* __restrict__ C, int64_t ldc, const int* halt) {
    constexpr int RX = BN / TN;  // threads along a row of the tile
    constexpr int RY = BM / TM;
    constexpr int NT = RX * RY;
    if (halt != nullptr && *(volatile const int*)halt != 0) return;

    __shared__ T As[2][BK][BM + 1];
    __shared__ T Bs[2][BK][BN];

    const int tid = threadIdx.x;
    const int tx = tid % RX, ty = tid / RX;
    const int64_t m0 = (int64_t)blockIdx.y * BM, n0 = (int64_t)blockIdx.x * BN;

    T acc[TM][TN];
#pragma unroll
    for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) acc[i][j] = T(0);

    constexpr int A_PER = (BM * BK + NT - 1) / NT;
    constexpr int B_PER = (BK * BN + NT - 1) / NT;
    T ra[A_PER], rb[B_PER];

    auto load_tiles = [&](int64_t k0) {
#pragma unroll
        for (int r = 0; r < A_PER; ++r) {
            const int e = tid + r * NT;
            T v = T(0);
            if (e < BM * BK) {
                int m, k;
                if (TA) { k = e / BM; m = e % BM; }
                else    { m = e / BK; k = e % BK; }
                const int64_t gm = m0 + m, gk = k0 + k;
                if (gm < M && gk < K) v = (T)(TA ? A[gk * lda + gm] : A[gm * lda + gk]);
            }
            ra[r] = v;
        }
#pragma unroll
        for (int r = 0; r < B_PER; ++r) {
            const int e = tid + r * NT;
            T v = T(0);
            if (e < BK * BN) {
                const int k = e / BN, nn = e % BN;
                const int64_t gk = k0 + k, gn = n0 + nn;
                if (gk < K && gn < N) v = (T)B[gk * ldb + gn];
            }
            rb[r] = v;
        }
    };
    auto store_tiles = [&](int buf) {
#pragma unroll
        for (int r = 0; r < A_PER; ++r) {
            const int e = tid + r * NT;
            if (e < BM * BK) {
                int m, k;
                if (TA) { k = e / BM; m = e % BM; }
                else    { m = e / BK; k = e % BK; }
                As[buf][k][m] = ra[r];
            }
        }
#pragma unroll
        for (int r = 0; r < B_PER; ++r) {
            const int e = tid + r * NT;
            if (e < BK * BN) Bs[buf][e / BN][e % BN] = rb[r];
        }
    };

    const int64_t ktiles = (K + BK - 1) / BK;
    if (ktiles > 0) {
        load_tiles(0);
        store_tiles(0);
    }
    __syncthreads();
    for (int64_t kt = 0; kt < ktiles; ++kt) {
        const int buf = (int)(kt & 1);
        if (kt + 1 < ktiles) load_tiles((kt + 1) * BK);  // prefetch into registers
#pragma unroll
        for (int k = 0; k < BK; ++k) {
            T a[TM], b[TN];
#pragma unroll
            for (int i = 0; i < TM; ++i) a[i] = As[buf][k][ty + i * RY];
#pragma unroll
            for (int j = 0; j < TN; ++j) b[j] = Bs[buf][k][tx + j * RX];
#pragma unroll
            for (int i = 0; i < TM; ++i)
#pragma unroll
                for (int j = 0; j < TN; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
        }
        if (kt + 1 < ktiles) store_tiles(buf ^ 1);
        __syncthreads();
    }

#pragma unroll
    for (int i = 0; i < TM; ++i) {
        const int64_t gm = m0 + ty + i * RY;
        if (gm >= M) continue;
#pragma unroll
        for (int j = 0; j < TN; ++j) {
            const int64_t gn = n0 + tx + j * RX;
            if (gn >= N) continue;
            T* c = C + gm * ldc + gn;
            const T v = alpha * acc[i][j];
            *c = (beta == T(0)) ? v : fma(beta, *c, v);
        }
    }
}

template <typename T, typename SA, typename SB, int BM, int BN, int BK, int TM, int TN>
rmge_status launch(bool ta, int64_t M, int64_t N, int64_t K, T alpha, const SA* A, int64_t lda, const SB* B,
                   int64_t ldb, T beta, T* C, int64_t ldc, const int* halt, cudaStream_t s) {
    const dim3 grid((unsigned)((N + BN - 1) / BN), (unsigned)((M + BM - 1) / BM));
    const int threads = (BM / TM) * (BN / TN);
    if (ta)
        gemm_kernel<T, SA, SB, BM, BN, BK, TM, TN, true><<<grid, threads, 0, s>>>(M, N, K, alpha, A, lda, B, ldb,
                                                                                 beta, C, ldc, halt);
    else
        gemm_kernel<T, SA, SB, BM, BN, BK, TM, TN, false><<<grid, threads, 0, s>>>(M, N, K, alpha, A, lda, B, ldb,
                                                                                  beta, C, ldc, halt);
    RMGE_LAUNCH_CHECK();
    return RMGE_OK;
}

constexpr int64_t kSMs = 152;

template <typename T, typename SA, typename SB>
rmge_status gemm_any(bool trans_a, int64_t M, int64_t N, int64_t K, T alpha, const SA* A, int64_t lda, const SB* B,
                     int64_t ldb, T beta, T* C, int64_t ldc, const int* halt, cudaStream_t s) {
    if (M <= 0 || N <= 0) return RMGE_OK;
    // One output per thread: the FMA pipe, not shared memory, bounds these on GB300.
    if (N <= 8)
        return launch<T, SA, SB, 16, 8, 64, 1, 1>(trans_a, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, halt, s);
    if (N <= 16)
        return launch<T, SA, SB, 16, 16, 32, 1, 1>(trans_a, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, halt, s);
    // Square-ish: the largest tile that still gives every SM several tiles.
    if constexpr (sizeof(T) == 4) {
        const int64_t t128 = ((M + 127) / 128) * ((N + 127) / 128);
        if (t128 >= 4 * kSMs)
            return launch<T, SA, SB, 128, 128, 16, 8, 8>(trans_a, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, halt,
                                                         s);
    }
    const int64_t t64 = ((M + 63) / 64) * ((N + 63) / 64);
    if (t64 >= 2 * kSMs)
        return launch<T, SA, SB, 64, 64, 16, 4, 4>(trans_a, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, halt, s);
    return launch<T, SA, SB, 32, 32, 16, 2, 2>(trans_a, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, halt, s);
}

}  // namespace

template <typename T>
rmge_status gemm(bool trans_a, int64_t M, int64_t N, int64_t K, T alpha, const T* A, int64_t lda, const T* B,
                 int64_t ldb, T beta, T* C, int64_t ldc, const int* halt, cudaStream_t s) {
    return gemm_any<T, T, T>(trans_a, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, halt, s);
}

rmge_status gemm_f64a_f32(int64_t M, int64_t N, int64_t K, const double* A, int64_t lda, const float* B, int64_t ldb,
                          float* C, int64_t ldc, cudaStream_t s) {
    return gemm_any<float, double, float>(false, M, N, K, 1.0f, A, lda, B, ldb, 0.0f, C, ldc, nullptr, s);
}

template rmge_status gemm<double>(bool, int64_t, int64_t, int64_t, double, const double*, int64_t, const double*,
                                  int64_t, double, double*, int64_t, const int*, cudaStream_t);
template rmge_status gemm<float>(bool, int64_t, int64_t, int64_t, float, const float*, int64_t, const float*,
                                 int64_t, float, float*, int64_t, const int*, cudaStream_t);

}  // namespace rmge
