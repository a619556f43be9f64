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
#include "pivot_block.cuh"

namespace rmge {
namespace {

struct CtaBarrier {
    __device__ void operator()() const { __syncthreads(); }
};

// Thread (tx, ty) owns rows ty + i*RY and columns tx + j*RX of the CTA tile (i < TM, j < TN), so
// a warp's shared-memory reads are broadcasts (A) or consecutive words (B), and its global
// stores are consecutive along a row.
//
// FUSE (GENP's trailing update, 64 x 64 tiles): tile (0, 0) of C holds the whole pivot block of the
// next step, and its CTA factors that block once the tile is written (pivot_block_genp in the tile
// staging area), while the other CTAs finish the update; a breakdown records its global step in
// fz.info and raises fz.halt.
template <typename T>
struct PivotFuse {
    T* D;        // the next pivot block: C's top-left corner, C's leading dimension
    int b;       // its order, <= 64
    int64_t k;   // its global offset (a breakdown at its step s is step k + s)
    int* info;
    int* halt;
};

template <typename T, typename SA, typename SB, int BM, int BN, int BK, int TM, int TN, bool TA, bool FUSE>
__global__ void __launch_bounds__((BM / TM) * (BN / TN))
gemm_kernel(int64_t M, int64_t N, int64_t K, T alpha, const SA* __restrict__ A, int64_t lda,
            const SB* __restrict__ B, int64_t ldb, T beta, T* __restrict__ C, int64_t ldc, const int* halt,
            PivotFuse<T> fz, Zb zb) {
    constexpr int RX = BN / TN;  // threads along a row of the tile
    constexpr int RY = BM / TM;
    constexpr int NT = RX * RY;
    halt = zws(halt, zb.ws);
    if (halt != nullptr && *(volatile const int*)halt != 0) return;
    A = zmat(A, zb.m0);
    B = zmat(B, zb.m1);
    C = zmat(C, zb.m2);

    // the two double-buffered tiles, carved from one array (the fused pivot block reuses it whole)
    constexpr int kTileBytes = (int)sizeof(T) * (2 * BK * (BM + 1) + 2 * BK * BN);
    __shared__ __align__(16) unsigned char tiles[kTileBytes];
    T (*As)[BK][BM + 1] = reinterpret_cast<T (*)[BK][BM + 1]>(tiles);
    T (*Bs)[BK][BN] = reinterpret_cast<T (*)[BK][BN]>(tiles + sizeof(T) * 2 * BK * (BM + 1));
    static_assert(!FUSE || (BM == 64 && BN == 64 && NT == 256 && kTileBytes >= (int)sizeof(T) * 64 * 64),
                  "the fused pivot block is one 64 x 64 tile, staged in the tile buffers");

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
    if constexpr (FUSE) {
        if (blockIdx.x == 0 && blockIdx.y == 0) {
            __shared__ T piv_rp;
            T* a = reinterpret_cast<T*>(tiles);  // 64 x 64 at row stride 64
            __syncthreads();      // the tile's stores to C are visible to the whole CTA
            for (int e = tid; e < 64 * 64; e += NT) {
                const int i = e / 64, j = e % 64;
                if (i < fz.b && j < fz.b) a[e] = fz.D[i * ldc + j];
            }
            __syncthreads();
            const int broke = pivot_block_genp<T, NT, CtaBarrier, 64>(a, fz.b, &piv_rp, tid, CtaBarrier{});
            if (broke != 0) {
                if (tid == 0) {
                    atomicMin(fz.info, (int)(fz.k + broke));
                    atomicExch(fz.halt, 1);
                }
            } else {
                for (int e = tid; e < 64 * 64; e += NT) {
                    const int i = e / 64, j = e % 64;
                    if (i < fz.b && j < fz.b) fz.D[i * ldc + j] = a[e];
                }
            }
        }
    }
}

// Products with at most four columns (one to four right-hand sides, op(A) = A): one warp per row of A,
// its lanes striding along the row (coalesced reads), NC partial sums per lane in two interleaved chains,
// reduced by shuffles.  A register-tiled kernel would issue FMAs for its padded columns as well: 7 of 8 of
// them for one right-hand side.
template <typename T, typename SA, typename SB, int NC>
__global__ void __launch_bounds__(256) gemv_kernel(int64_t M, int64_t K, T alpha, const SA* __restrict__ A,
                                                   int64_t lda, const SB* __restrict__ B, int64_t ldb, T beta,
                                                   T* __restrict__ C, int64_t ldc, const int* halt, Zb zb) {
    halt = zws(halt, zb.ws);
    if (halt != nullptr && *(volatile const int*)halt != 0) return;
    A = zmat(A, zb.m0);
    B = zmat(B, zb.m1);
    C = zmat(C, zb.m2);
    const int lane = threadIdx.x & 31;
    const int64_t m = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;  // one row per warp: uniform
    if (m >= M) return;
    const SA* a = A + m * lda;
    T acc[NC], acc2[NC];
#pragma unroll
    for (int j = 0; j < NC; ++j) acc[j] = acc2[j] = T(0);
    int64_t k = lane;
#pragma unroll 4
    for (; k + 32 < K; k += 64) {
        const T a0 = (T)a[k], a1 = (T)a[k + 32];
#pragma unroll
        for (int j = 0; j < NC; ++j) {
            acc[j] = fma(a0, (T)B[k * ldb + j], acc[j]);
            acc2[j] = fma(a1, (T)B[(k + 32) * ldb + j], acc2[j]);
        }
    }
    if (k < K) {
        const T a0 = (T)a[k];
#pragma unroll
        for (int j = 0; j < NC; ++j) acc[j] = fma(a0, (T)B[k * ldb + j], acc[j]);
    }
#pragma unroll
    for (int j = 0; j < NC; ++j) {
        T v = acc[j] + acc2[j];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        acc[j] = v;
    }
    if (lane == 0)
#pragma unroll
        for (int j = 0; j < NC; ++j) {
            T* c = C + m * ldc + j;
            const T v = alpha * acc[j];
            *c = (beta == T(0)) ? v : fma(beta, *c, v);
        }
}

// The same products with op(A) = A^T (the adjoint's G^T dX and A^T dB): column m of A is row m of op(A),
// so a lane takes one column (consecutive lanes on consecutive columns: coalesced rows of A) and the 8
// warps of a block split the rows of A, their partial sums reduced in shared memory.
template <typename T, typename SA, typename SB, int NC>
__global__ void __launch_bounds__(256) gemv_t_kernel(int64_t M, int64_t K, T alpha, const SA* __restrict__ A,
                                                     int64_t lda, const SB* __restrict__ B, int64_t ldb, T beta,
                                                     T* __restrict__ C, int64_t ldc, const int* halt, Zb zb) {
    __shared__ T part[8][NC][32];
    halt = zws(halt, zb.ws);
    if (halt != nullptr && *(volatile const int*)halt != 0) return;
    A = zmat(A, zb.m0);
    B = zmat(B, zb.m1);
    C = zmat(C, zb.m2);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t m = (int64_t)blockIdx.x * 32 + lane;
    const int64_t k0 = K * w / 8, k1 = K * (w + 1) / 8;
    T acc[NC], acc2[NC];
#pragma unroll
    for (int j = 0; j < NC; ++j) acc[j] = acc2[j] = T(0);
    if (m < M) {
        int64_t k = k0;
#pragma unroll 4
        for (; k + 1 < k1; k += 2) {
            const T a0 = (T)A[k * lda + m], a1 = (T)A[(k + 1) * lda + m];
#pragma unroll
            for (int j = 0; j < NC; ++j) {
                acc[j] = fma(a0, (T)B[k * ldb + j], acc[j]);
                acc2[j] = fma(a1, (T)B[(k + 1) * ldb + j], acc2[j]);
            }
        }
        if (k < k1) {
            const T a0 = (T)A[k * lda + m];
#pragma unroll
            for (int j = 0; j < NC; ++j) acc[j] = fma(a0, (T)B[k * ldb + j], acc[j]);
        }
    }
#pragma unroll
    for (int j = 0; j < NC; ++j) part[w][j][lane] = acc[j] + acc2[j];
    __syncthreads();
    if (w < NC && m < M) {
        const int j = w;
        T v = part[0][j][lane];
#pragma unroll
        for (int g = 1; g < 8; ++g) v += part[g][j][lane];
        T* c = C + m * ldc + j;
        const T av = alpha * v;
        *c = (beta == T(0)) ? av : fma(beta, *c, av);
    }
}

template <typename T, typename SA, typename SB, int NC>
rmge_status launch_gemv_t(int64_t M, int64_t K, T alpha, const SA* A, int64_t lda, const SB* B, int64_t ldb, T beta,
                          T* C, int64_t ldc, const int* halt, cudaStream_t s, const Zb& zb) {
    const int64_t blocks = (M + 31) / 32;
    gemv_t_kernel<T, SA, SB, NC><<<dim3((unsigned)blocks, 1, zb.count), 256, 0, s>>>(M, K, alpha, A, lda, B, ldb,
                                                                                    beta, C, ldc, halt, zb);
    RMGE_LAUNCH_CHECK();
    return RMGE_OK;
}

template <typename T, typename SA, typename SB, int NC>
rmge_status launch_gemv(int64_t M, int64_t K, T alpha, const SA* A, int64_t lda, const SB* B, int64_t ldb, T beta,
                        T* C, int64_t ldc, const int* halt, cudaStream_t s, const Zb& zb) {
    const int64_t blocks = (M + 7) / 8;  // 8 warps (rows) per block
    gemv_kernel<T, SA, SB, NC><<<dim3((unsigned)blocks, 1, zb.count), 256, 0, s>>>(M, K, alpha, A, lda, B, ldb, beta,
                                                                                  C, ldc, halt, zb);
    RMGE_LAUNCH_CHECK();
    return RMGE_OK;
}

template <typename T, typename SA, typename SB, int BM, int BN, int BK, int TM, int TN>
rmge_status launch(bool ta, int64_t M, int64_t N, int64_t K, T alpha, const SA* A, int64_t lda, const SB* B,
                   int64_t ldb, T beta, T* C, int64_t ldc, const int* halt, cudaStream_t s, const Zb& zb) {
    const dim3 grid((unsigned)((N + BN - 1) / BN), (unsigned)((M + BM - 1) / BM), (unsigned)zb.count);
    const int threads = (BM / TM) * (BN / TN);
    if (ta)
        gemm_kernel<T, SA, SB, BM, BN, BK, TM, TN, true, false><<<grid, threads, 0, s>>>(
            M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, halt, PivotFuse<T>{}, zb);
    else
        gemm_kernel<T, SA, SB, BM, BN, BK, TM, TN, false, false><<<grid, threads, 0, s>>>(
            M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, halt, PivotFuse<T>{}, zb);
    RMGE_LAUNCH_CHECK();
    return RMGE_OK;
}

constexpr int64_t kSMs = 152;

template <typename T, typename SA, typename SB>
rmge_status gemm_any(bool trans_a, int64_t M, int64_t N, int64_t K, T alpha, const SA* A, int64_t lda, const SB* B,
                     int64_t ldb, T beta, T* C, int64_t ldc, const int* halt, cudaStream_t s, const Zb& zb = Zb{}) {
    if (M <= 0 || N <= 0) return RMGE_OK;
    if (trans_a && N <= 4) {
        switch (N) {
            case 1: return launch_gemv_t<T, SA, SB, 1>(M, K, alpha, A, lda, B, ldb, beta, C, ldc, halt, s, zb);
            case 2: return launch_gemv_t<T, SA, SB, 2>(M, K, alpha, A, lda, B, ldb, beta, C, ldc, halt, s, zb);
            case 3: return launch_gemv_t<T, SA, SB, 3>(M, K, alpha, A, lda, B, ldb, beta, C, ldc, halt, s, zb);
            default: return launch_gemv_t<T, SA, SB, 4>(M, K, alpha, A, lda, B, ldb, beta, C, ldc, halt, s, zb);
        }
    }
    if (!trans_a && N <= 4) {
        switch (N) {
            case 1: return launch_gemv<T, SA, SB, 1>(M, K, alpha, A, lda, B, ldb, beta, C, ldc, halt, s, zb);
            case 2: return launch_gemv<T, SA, SB, 2>(M, K, alpha, A, lda, B, ldb, beta, C, ldc, halt, s, zb);
            case 3: return launch_gemv<T, SA, SB, 3>(M, K, alpha, A, lda, B, ldb, beta, C, ldc, halt, s, zb);
            default: return launch_gemv<T, SA, SB, 4>(M, K, alpha, A, lda, B, ldb, beta, C, ldc, halt, s, zb);
        }
    }
    // One output per thread: the FMA pipe, not shared memory, bounds these on GB300.  (4-row tiles, which
    // spread M = 4096 x 16 columns more evenly over the 152 SMs than 256 tiles of 16 rows, measured slower.)
    if (N <= 8)
        return launch<T, SA, SB, 16, 8, 64, 1, 1>(trans_a, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, halt, s, zb);
    if (N <= 16)
        return launch<T, SA, SB, 16, 16, 32, 1, 1>(trans_a, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, halt, s, zb);
    // Square-ish: the largest tile that still gives every SM several tiles.
    if constexpr (sizeof(T) == 4) {
        const int64_t t128 = ((M + 127) / 128) * ((N + 127) / 128);
        if (t128 >= 4 * kSMs)
            return launch<T, SA, SB, 128, 128, 16, 8, 8>(trans_a, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, halt,
                                                         s, zb);
    }
    const int64_t t64 = ((M + 63) / 64) * ((N + 63) / 64);
    if (t64 >= 2 * kSMs)
        return launch<T, SA, SB, 64, 64, 16, 4, 4>(trans_a, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, halt, s, zb);
    return launch<T, SA, SB, 32, 32, 16, 2, 2>(trans_a, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, halt, s, zb);
}

}  // namespace

template <typename T>
rmge_status gemm(bool trans_a, int64_t M, int64_t N, int64_t K, T alpha, const T* A, int64_t lda, const T* B,
                 int64_t ldb, T beta, T* C, int64_t ldc, const int* halt, cudaStream_t s, const Zb& zb) {
    return gemm_any<T, T, T>(trans_a, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, halt, s, zb);
}

template <typename T>
rmge_status gemm_update_fused(int64_t M, int64_t N, int64_t K, const T* A, int64_t lda, const T* B, int64_t ldb, T* C,
                              int64_t ldc, const int* halt, int b, int64_t k, int* info, int* halt_w, cudaStream_t s) {
    if (b < 1 || b > 64 || b > M || b > N || info == nullptr || halt_w == nullptr) return RMGE_ERR_INVALID_ARG;
    const dim3 grid((unsigned)((N + 63) / 64), (unsigned)((M + 63) / 64));
    gemm_kernel<T, T, T, 64, 64, 16, 4, 4, false, true><<<grid, 256, 0, s>>>(
        M, N, K, T(-1), A, lda, B, ldb, T(1), C, ldc, halt, PivotFuse<T>{C, b, k, info, halt_w}, Zb{});
    RMGE_LAUNCH_CHECK();
    return RMGE_OK;
}
template rmge_status gemm_update_fused<double>(int64_t, int64_t, int64_t, const double*, int64_t, const double*,
                                               int64_t, double*, int64_t, const int*, int, int64_t, int*, int*,
                                               cudaStream_t);
template rmge_status gemm_update_fused<float>(int64_t, int64_t, int64_t, const float*, int64_t, const float*, int64_t,
                                              float*, int64_t, const int*, int, int64_t, int*, int*, cudaStream_t);

rmge_status gemm_f64a_f32(int64_t M, int64_t N, int64_t K, const double* A, int64_t lda, const float* B, int64_t ldb,
                          float* C, int64_t ldc, cudaStream_t s) {
    return gemm_any<float, double, float>(false, M, N, K, 1.0f, A, lda, B, ldb, 0.0f, C, ldc, nullptr, s);
}

template rmge_status gemm<double>(bool, int64_t, int64_t, int64_t, double, const double*, int64_t, const double*,
                                  int64_t, double, double*, int64_t, const int*, cudaStream_t, const Zb&);
template rmge_status gemm<float>(bool, int64_t, int64_t, int64_t, float, const float*, int64_t, const float*,
                                 int64_t, float, float*, int64_t, const int*, cudaStream_t, const Zb&);

}  // namespace rmge
