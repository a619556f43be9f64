// batched.cu -- thousands of independent randomized GENP solves of uneven size in one persistent launch.
//
// Each system i (size n_i, one right-hand side) runs the whole method inside one CTA:
//   G_i  = FP32 Gaussian multiplier (Def. 4.1), Philox stream (seed, subsequence i)
//   M_i  = A_i G_i                       (Fact 4.1; A_i FP64, rounded to FP32 on load)
//   M_i  = L U  by blocked GENP           (eq. (3.1), 32-column pivot blocks, FP32)
//   x_i  = G_i U^{-1} L^{-1} b_i          (Fact 4.1)
//   sweeps of r = b - A x (FP64), x += G U^{-1} L^{-1} r, until the normwise backward error is
//   below tol (Sec. 1.2, Sec. 7.1); once a sweep fails to halve the error, the remaining sweeps are
//   right-preconditioned GMRES cycles (FP64 basis, FP32 products with A and the preconditioner
//   G U^{-1} L^{-1}; the residual of every sweep stays FP64); when those
//   stall too, a fresh multiplier is drawn (up to three draws), and a system that no FP32 draw can
//   refine is factored in FP64 in the same CTA (its A G and GENP on the DFMA pipe; the first such
//   system of a launch shares the rows of its A G with the CTAs that pass between two systems)
// CTAs are persistent: each takes the next system from a queue ordered by decreasing n (longest
// first), so uneven sizes balance across the SMs.  The queue counter re-arms itself when the last
// CTA finishes, so the launch can be captured once in a CUDA graph and replayed.  Per-CTA scratch
// (G, M and vectors, sized for the largest system) lives in the caller's workspace.  The tile size
// and thread count are template parameters chosen by the host-side autotuner.
#include <climits>

#include "kernels.cuh"

namespace rmge {
namespace {

struct BatchArgs {
    int64_t count;
    const int32_t* n;          // sizes
    const int64_t* offA;       // element offset of A_i (n_i x n_i, row-major, ld n_i)
    const int64_t* offv;       // element offset of b_i, x_i
    const int32_t* order;      // processing order (decreasing n)
    const double* A;
    const double* b;
    double* x;
    int32_t* info;             // per system: 0 or first breakdown step
    double* berr;              // per system: final backward error
    int32_t* sweeps;           // per system: refinement sweeps
    uint64_t seed;
    int max_sweeps;
    double tol;
    float* scratch;            // per CTA: G (nmax^2), M (nmax^2), y, t (nmax each) floats
    double* dscratch;          // per CTA: r (nmax) doubles
    int64_t nmax;
    unsigned int* queue;       // [0] next system, [1] finished CTAs, [2] CTAs working on a system
    struct HelpJob* help;      // the shared FP64 product of a fallback system (in the zeroed queue head)
    long long spin_limit;      // polls of the bounded waits around the shared product
};

// A system that falls back to FP64 factors posts its product M = A G here, split into blocks of TILE
// rows.  CTAs between two systems (and CTAs whose queue ran dry, while others still work) take blocks
// from `next` and count them in `done`; the owner takes blocks too, then waits for `done`.  One job per
// launch: `claimed` is never released, so no CTA can mistake a later job's fields for this one's.
struct HelpJob {
    unsigned int claimed;  // set once by the owner (atomicCAS)
    int ready;             // release-stored 1 once the fields below are valid
    unsigned int next;     // next block to take (can run past `blocks`)
    int done;              // finished blocks
    int n, blocks;
    const double* A;
    const float* G;
    double* M;
};

// ---------------------------------------------------------------------------------------------
// Philox4x32-10 (same stream definition as gen.cu's FP32 Gaussian multipliers)
// ---------------------------------------------------------------------------------------------
__device__ __forceinline__ uint4 philox(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t hi_a = __umulhi(0xD2511F53u, c.x), lo_a = 0xD2511F53u * c.x;
        const uint32_t hi_b = __umulhi(0xCD9E8D57u, c.z), lo_b = 0xCD9E8D57u * c.z;
        c = make_uint4(hi_b ^ c.y ^ k0, lo_b, hi_a ^ c.w ^ k1, lo_a);
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return c;
}

template <int T>
__device__ void gen_gaussian_f32(int64_t count, uint64_t seed, uint64_t subseq, float* out) {
    for (int64_t p = threadIdx.x; p < (count + 1) / 2; p += T) {
        const uint4 x = philox(make_uint4((uint32_t)p, (uint32_t)(p >> 32), (uint32_t)subseq, (uint32_t)(subseq >> 32)),
                               (uint32_t)seed, (uint32_t)(seed >> 32));
        const float u1 = (float)((x.x >> 8) + 1u) * 0x1p-24f;
        const float u2 = (float)(x.z >> 8) * 0x1p-24f;
        const float r = sqrtf(-2.0f * logf(u1));
        float sn, cs;
        sincospif(2.0f * u2, &sn, &cs);
        out[2 * p] = r * cs;
        if (2 * p + 1 < count) out[2 * p + 1] = r * sn;
    }
}

// ---------------------------------------------------------------------------------------------
// CTA-wide FP32 GEMM: C (M x N, ldc) = alpha A B + beta C, A (M x K) of type SA, B (K x N) FP32.
// TILE x TILE output tiles, each thread an (TILE/RT) x (TILE/RT) micro-tile, RT = sqrt(T).
// ---------------------------------------------------------------------------------------------
template <int T, int TILE, typename SA, typename E>
__device__ void cta_gemm(int M, int N, int K, const SA* __restrict__ A, int lda, const float* __restrict__ B, int ldb,
                         E* __restrict__ C, int ldc, E alpha, E beta, E* smem) {
    constexpr int BK = 16;
    constexpr int RT = (T == 256) ? 16 : 32;  // threads per tile row
    constexpr int RY = T / RT;
    constexpr int TM = TILE / RY, TN = TILE / RT;
    E* As = smem;                  // [BK][TILE]
    E* Bs = smem + BK * TILE;      // [BK][TILE]
    const int tx = threadIdx.x % RT, ty = threadIdx.x / RT;
    for (int t0 = 0; t0 < ((M + TILE - 1) / TILE) * ((N + TILE - 1) / TILE); ++t0) {
        const int tm = t0 / ((N + TILE - 1) / TILE), tn = t0 % ((N + TILE - 1) / TILE);
        const int m0 = tm * TILE, n0 = tn * TILE;
        E acc[TM][TN];
#pragma unroll
        for (int i = 0; i < TM; ++i)
#pragma unroll
            for (int j = 0; j < TN; ++j) acc[i][j] = E(0);
        for (int k0 = 0; k0 < K; k0 += BK) {
            for (int e = threadIdx.x; e < TILE * BK; e += T) {
                const int m = e / BK, kk = e % BK;
                const int gm = m0 + m, gk = k0 + kk;
                As[kk * TILE + m] = (gm < M && gk < K) ? (E)A[(int64_t)gm * lda + gk] : E(0);
                const int kb = e / TILE, nn = e % TILE;
                const int gkb = k0 + kb, gn = n0 + nn;
                Bs[kb * TILE + nn] = (gkb < K && gn < N) ? (E)B[(int64_t)gkb * ldb + gn] : E(0);
            }
            __syncthreads();
#pragma unroll
            for (int kk = 0; kk < BK; ++kk) {
                E a[TM], bb[TN];
#pragma unroll
                for (int i = 0; i < TM; ++i) a[i] = As[kk * TILE + ty + i * RY];
#pragma unroll
                for (int j = 0; j < TN; ++j) bb[j] = Bs[kk * TILE + tx + j * RT];
#pragma unroll
                for (int i = 0; i < TM; ++i)
#pragma unroll
                    for (int j = 0; j < TN; ++j) acc[i][j] = fma(a[i], bb[j], acc[i][j]);
            }
            __syncthreads();
        }
#pragma unroll
        for (int i = 0; i < TM; ++i) {
            const int gm = m0 + ty + i * RY;
            if (gm >= M) continue;
#pragma unroll
            for (int j = 0; j < TN; ++j) {
                const int gn = n0 + tx + j * RT;
                if (gn >= N) continue;
                E* c = C + (int64_t)gm * ldc + gn;
                *c = (beta == E(0)) ? alpha * acc[i][j] : fma(beta, *c, alpha * acc[i][j]);
            }
        }
    }
    __syncthreads();
}

// C -= A B with all operands of type E (the Schur-complement update inside cta_genp).
template <int T, int TILE, typename E>
__device__ void cta_gemm_same(int M, int N, int K, const E* __restrict__ A, int lda, const E* __restrict__ B, int ldb,
                              E* __restrict__ C, int ldc, E* smem) {
    constexpr int BK = 16;
    constexpr int RT = (T == 256) ? 16 : 32;
    constexpr int RY = T / RT;
    constexpr int TM = TILE / RY, TN = TILE / RT;
    E* As = smem;
    E* Bs = smem + BK * TILE;
    const int tx = threadIdx.x % RT, ty = threadIdx.x / RT;
    const int tn_count = (N + TILE - 1) / TILE;
    for (int t0 = 0; t0 < ((M + TILE - 1) / TILE) * tn_count; ++t0) {
        const int m0 = (t0 / tn_count) * TILE, n0 = (t0 % tn_count) * TILE;
        E acc[TM][TN];
#pragma unroll
        for (int i = 0; i < TM; ++i)
#pragma unroll
            for (int j = 0; j < TN; ++j) acc[i][j] = E(0);
        for (int k0 = 0; k0 < K; k0 += BK) {
            for (int e = threadIdx.x; e < TILE * BK; e += T) {
                const int m = e / BK, kk = e % BK;
                As[kk * TILE + m] = (m0 + m < M && k0 + kk < K) ? A[(int64_t)(m0 + m) * lda + k0 + kk] : E(0);
                const int kb = e / TILE, nn = e % TILE;
                Bs[kb * TILE + nn] = (k0 + kb < K && n0 + nn < N) ? B[(int64_t)(k0 + kb) * ldb + n0 + nn] : E(0);
            }
            __syncthreads();
#pragma unroll
            for (int kk = 0; kk < BK; ++kk) {
                E a[TM], bb[TN];
#pragma unroll
                for (int i = 0; i < TM; ++i) a[i] = As[kk * TILE + ty + i * RY];
#pragma unroll
                for (int j = 0; j < TN; ++j) bb[j] = Bs[kk * TILE + tx + j * RT];
#pragma unroll
                for (int i = 0; i < TM; ++i)
#pragma unroll
                    for (int j = 0; j < TN; ++j) acc[i][j] = fma(a[i], bb[j], acc[i][j]);
            }
            __syncthreads();
        }
#pragma unroll
        for (int i = 0; i < TM; ++i) {
            const int gm = m0 + ty + i * RY;
            if (gm >= M) continue;
#pragma unroll
            for (int j = 0; j < TN; ++j) {
                const int gn = n0 + tx + j * RT;
                if (gn < N) C[(int64_t)gm * ldc + gn] -= acc[i][j];
            }
        }
    }
    __syncthreads();
}

// ---------------------------------------------------------------------------------------------
// CTA-wide blocked GENP of M (n x n, ld n) with 32-column pivot blocks; returns 0 or the first
// breakdown step.
// ---------------------------------------------------------------------------------------------
constexpr int PB = 32;

template <int T, int TILE, typename E>
__device__ int cta_genp(int n, E* M, E* smem, int* flag) {
    E* d = smem;  // [PB][PB + 1] pivot block
    for (int k = 0; k < n; k += PB) {
        const int b = min(PB, n - k);
        for (int e = threadIdx.x; e < b * b; e += T) d[(e / b) * (PB + 1) + e % b] = M[(int64_t)(k + e / b) * n + k + e % b];
        if (threadIdx.x == 0) *flag = 0;
        __syncthreads();
        for (int s = 0; s < b; ++s) {
            const E piv = d[s * (PB + 1) + s];
            if (piv == E(0) || !isfinite(piv)) {
                __syncthreads();
                return k + s + 1;
            }
            for (int i = s + 1 + threadIdx.x; i < b; i += T) d[i * (PB + 1) + s] /= piv;
            __syncthreads();
            const int w = b - s - 1;
            for (int e = threadIdx.x; e < w * w; e += T) {
                const int i = s + 1 + e / w, j = s + 1 + e % w;
                d[i * (PB + 1) + j] = fma(-d[i * (PB + 1) + s], d[s * (PB + 1) + j], d[i * (PB + 1) + j]);
            }
            __syncthreads();
        }
        for (int e = threadIdx.x; e < b * b; e += T) M[(int64_t)(k + e / b) * n + k + e % b] = d[(e / b) * (PB + 1) + e % b];
        const int rest = n - k - b;
        if (rest > 0) {
            // L21 rows: x U11 = a, one thread per row; U12 columns: L11 x = a, one thread per column
            for (int q = threadIdx.x; q < 2 * rest; q += T) {
                if (q < rest) {
                    E* row = M + (int64_t)(k + b + q) * n + k;
                    for (int j = 0; j < b; ++j) {
                        E v = row[j];
                        for (int t = 0; t < j; ++t) v = fma(-row[t], d[t * (PB + 1) + j], v);
                        row[j] = v / d[j * (PB + 1) + j];
                    }
                } else {
                    E* col = M + (int64_t)k * n + k + b + (q - rest);
                    for (int i = 0; i < b; ++i) {
                        E v = col[(int64_t)i * n];
                        for (int t = 0; t < i; ++t) v = fma(-d[i * (PB + 1) + t], col[(int64_t)t * n], v);
                        col[(int64_t)i * n] = v;
                    }
                }
            }
            __syncthreads();
            cta_gemm_same<T, TILE, E>(rest, rest, b, M + (int64_t)(k + b) * n + k, n, M + (int64_t)k * n + k + b, n,
                                      M + (int64_t)(k + b) * n + k + b, n, smem + PB * (PB + 1));
        }
    }
    return 0;
}

// In-place y <- U^{-1} L^{-1} y (FP32 vector, n), warp 0 solving 32-row diagonal blocks, all threads
// updating the rows below (above) with the solved block.
// FP32 factors: each lane first loads its row of the 32 x 32 diagonal block into registers, so the
// dependent shuffle chain does not wait on a global load at every step.
template <int T, typename E>
__device__ void cta_lu_solve(int n, const E* M, E* y) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    constexpr bool kRegRow = sizeof(E) == 4;
    for (int k = 0; k < n; k += 32) {  // L z = y
        const int b = min(32, n - k);
        if (warp == 0) {
            E v = lane < b ? y[k + lane] : E(0);
            if constexpr (kRegRow) {
                E row[32];
#pragma unroll
                for (int j = 0; j < 32; ++j) row[j] = (lane < b && j < lane) ? M[(int64_t)(k + lane) * n + k + j] : E(0);
#pragma unroll
                for (int j = 0; j < 32; ++j) {
                    const E zj = __shfl_sync(0xffffffffu, v, j);
                    v = fma(-row[j], zj, v);  // row[j] = 0 for j >= lane
                }
            } else {
                for (int j = 0; j < b; ++j) {
                    const E zj = __shfl_sync(0xffffffffu, v, j);
                    if (lane > j && lane < b) v = fma(-M[(int64_t)(k + lane) * n + k + j], zj, v);
                }
            }
            if (lane < b) y[k + lane] = v;
        }
        __syncthreads();
        for (int i = k + b + threadIdx.x; i < n; i += T) {
            E v = y[i];
            for (int j = 0; j < b; ++j) v = fma(-M[(int64_t)i * n + k + j], y[k + j], v);
            y[i] = v;
        }
        __syncthreads();
    }
    for (int k = ((n - 1) / 32) * 32; k >= 0; k -= 32) {  // U x = z
        const int b = min(32, n - k);
        if (warp == 0) {
            E v = lane < b ? y[k + lane] : E(0);
            if constexpr (kRegRow) {
                E row[32];
#pragma unroll
                for (int j = 0; j < 32; ++j) row[j] = (lane < b && j >= lane && j < b) ? M[(int64_t)(k + lane) * n + k + j] : E(0);
#pragma unroll
                for (int j = 31; j >= 0; --j) {
                    if (j < b) {  // uniform
                        if (lane == j) v = v / row[j];
                        const E xj = __shfl_sync(0xffffffffu, v, j);
                        if (lane < j) v = fma(-row[j], xj, v);
                    }
                }
            } else {
                for (int j = b - 1; j >= 0; --j) {
                    if (lane == j) v = v / M[(int64_t)(k + j) * n + k + j];
                    const E xj = __shfl_sync(0xffffffffu, v, j);
                    if (lane < j) v = fma(-M[(int64_t)(k + lane) * n + k + j], xj, v);
                }
            }
            if (lane < b) y[k + lane] = v;
        }
        __syncthreads();
        for (int i = threadIdx.x; i < k; i += T) {
            E v = y[i];
            for (int j = 0; j < b; ++j) v = fma(-M[(int64_t)i * n + k + j], y[k + j], v);
            y[i] = v;
        }
        __syncthreads();
    }
}

// out (FP32 or FP64, accumulate or assign) = G v, one warp per row
template <int T, typename E>
__device__ void cta_gemv(int n, const float* G, const E* v, double* out, bool accumulate) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int i = warp; i < n; i += T / 32) {
        E s = E(0);
        for (int j = lane; j < n; j += 32) s = fma((E)G[(int64_t)i * n + j], v[j], s);
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) out[i] = accumulate ? out[i] + (double)s : (double)s;
    }
    __syncthreads();
}

// CTA-wide sum of one double per thread; every thread gets the total.
template <int T>
__device__ double cta_sum(double v, double* red) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    double t = 0.0;
    for (int w = 0; w < T / 32; ++w) t += red[w];
    __syncthreads();
    return t;
}

constexpr int GM = 16;  // restart length of the per-system GMRES cycles

// CTA-wide maximum of one non-negative FP64 bit pattern per thread (integer compares: GB300's FP64
// pipe is narrow and slow to answer); every thread gets the total.
template <int T>
__device__ unsigned long long cta_max_bits(unsigned long long v, unsigned long long* redb) {
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long u = __shfl_xor_sync(0xffffffffu, v, o);
        v = u > v ? u : v;
    }
    if ((threadIdx.x & 31) == 0) redb[threadIdx.x >> 5] = v;
    __syncthreads();
    unsigned long long t = 0ull;
    for (int w = 0; w < T / 32; ++w) t = redb[w] > t ? redb[w] : t;
    __syncthreads();
    return t;
}

// r = b - A x in FP64 (the residual of every sweep) with its maximum, and, when with_norm, the largest
// absolute row sum of A.  Each warp takes four rows at a time so that four independent FMA chains
// hide the FP64 latency.
template <int T>
__device__ void cta_residual(int n, const double* A, const double* b, const double* x, double* r, bool with_norm,
                             unsigned long long* rmax_bits, unsigned long long* amax_bits, unsigned long long* redb) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    unsigned long long rb = 0ull, ab = 0ull;
    for (int i0 = warp * 4; i0 < n; i0 += (T / 32) * 4) {
        double sacc[4], as[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            sacc[q] = (lane == 0 && i0 + q < n) ? b[i0 + q] : 0.0;  // b enters the warp sum once
            as[q] = 0.0;
        }
        for (int j = lane; j < n; j += 32) {
            const double xj = x[j];
#pragma unroll
            for (int q = 0; q < 4; ++q)
                if (i0 + q < n) {
                    const double aij = A[(int64_t)(i0 + q) * n + j];
                    sacc[q] = fma(-aij, xj, sacc[q]);
                    if (with_norm) as[q] += fabs(aij);
                }
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            for (int o = 16; o > 0; o >>= 1) {
                sacc[q] += __shfl_xor_sync(0xffffffffu, sacc[q], o);
                if (with_norm) as[q] += __shfl_xor_sync(0xffffffffu, as[q], o);
            }
            if (i0 + q < n) {
                if (lane == 0) r[i0 + q] = sacc[q];
                const unsigned long long v = abs_bits(sacc[q]), w = abs_bits(as[q]);
                rb = v > rb ? v : rb;
                ab = w > ab ? w : ab;
            }
        }
    }
    *rmax_bits = cta_max_bits<T>(rb, redb);
    *amax_bits = with_norm ? cta_max_bits<T>(ab, redb) : 0ull;
}

template <int T>
__device__ double cta_max_abs(int n, const double* v, unsigned long long* redb) {
    unsigned long long m = 0ull;
    for (int i = threadIdx.x; i < n; i += T) {
        const unsigned long long u = abs_bits(v[i]);
        m = u > m ? u : m;
    }
    return __longlong_as_double((long long)cta_max_bits<T>(m, redb));
}

// z (FP64) = G U^{-1} L^{-1} v with the FP32 factors: the preconditioner P of Fact 4.1.
template <int T>
__device__ void cta_precond(int n, const float* M, const float* G, const double* v, float* y, double* z) {
    for (int i = threadIdx.x; i < n; i += T) y[i] = (float)v[i];
    __syncthreads();
    cta_lu_solve<T, float>(n, M, y);
    cta_gemv<T, float>(n, G, y, z, false);
}

// One right-preconditioned GMRES(GM) cycle on A d = r (r in rz on entry), x += P V y, with the
// Krylov basis, orthogonalisation and rotations in FP64 and the products A z in FP32 against A32, an
// FP32 copy of A: GMRES-based refinement only needs the correction to a modest relative accuracy
// while the residual of every sweep stays in FP64 (a lower-precision Krylov product, as in the
// five-precision GMRES-IR analysis of Amestoy, Buttari, Higham, L'Excellent, Mary and Vieuble).
// V: (GM + 1) x n doubles of scratch; rz is reused as the preconditioned vector; z32: n floats.
template <int T>
__device__ void cta_gmres_cycle(int n, const float* A32, const float* M, const float* G, double* x, double* rz,
                                double* V, float* y, float* z32, double* red) {
    __shared__ double H[(GM + 1) * GM], cs[GM], sn[GM], g[GM + 1], hs[GM + 1], ys[GM];
    __shared__ double redm[T / 32][GM];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    double acc = 0.0;
    for (int i = threadIdx.x; i < n; i += T) acc = fma(rz[i], rz[i], acc);
    const double beta = sqrt(cta_sum<T>(acc, red));
    if (!(beta > 0.0) || !isfinite(beta)) return;
    for (int i = threadIdx.x; i < n; i += T) V[i] = rz[i] / beta;
    if (threadIdx.x == 0) {
        g[0] = beta;
        for (int i = 1; i <= GM; ++i) g[i] = 0.0;
        for (int i = 0; i < (GM + 1) * GM; ++i) H[i] = 0.0;
    }
    __syncthreads();
    int m = GM;
    for (int j = 0; j < GM; ++j) {
        double* vj = V + (int64_t)j * n;
        double* w = V + (int64_t)(j + 1) * n;
        cta_precond<T>(n, M, G, vj, y, rz);  // rz = P v_j (FP32 values held in doubles)
        for (int i = threadIdx.x; i < n; i += T) z32[i] = (float)rz[i];
        __syncthreads();
        for (int i0 = warp * 4; i0 < n; i0 += (T / 32) * 4) {  // w = A z, four rows per warp at a time
            float sv[4] = {0.0f, 0.0f, 0.0f, 0.0f};
            for (int k = lane; k < n; k += 32) {
                const float zk = z32[k];
#pragma unroll
                for (int q = 0; q < 4; ++q)
                    if (i0 + q < n) sv[q] = fmaf(A32[(int64_t)(i0 + q) * n + k], zk, sv[q]);
            }
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                for (int o = 16; o > 0; o >>= 1) sv[q] += __shfl_xor_sync(0xffffffffu, sv[q], o);
                if (lane == 0 && i0 + q < n) w[i0 + q] = (double)sv[q];
            }
        }
        __syncthreads();
        for (int pass = 0; pass < 2; ++pass) {  // classical Gram-Schmidt, twice
            // the j + 1 dot products in groups of LB: one reduction round per group instead of per product
            constexpr int LB = (T >= 1024) ? 4 : GM;  // 1024-thread CTAs have 64 registers per thread
            for (int l0 = 0; l0 <= j; l0 += LB) {
                double d[LB];
#pragma unroll
                for (int l = 0; l < LB; ++l) d[l] = 0.0;
                for (int i = threadIdx.x; i < n; i += T) {
                    const double wi = w[i];
#pragma unroll
                    for (int l = 0; l < LB; ++l)
                        if (l0 + l <= j) d[l] = fma(V[(int64_t)(l0 + l) * n + i], wi, d[l]);
                }
#pragma unroll
                for (int l = 0; l < LB; ++l)
                    if (l0 + l <= j) {
                        for (int o = 16; o > 0; o >>= 1) d[l] += __shfl_xor_sync(0xffffffffu, d[l], o);
                        if (lane == 0) redm[warp][l0 + l] = d[l];
                    }
            }
            __syncthreads();
            if (threadIdx.x <= j) {
                double t = 0.0;
                for (int w2 = 0; w2 < T / 32; ++w2) t += redm[w2][threadIdx.x];
                hs[threadIdx.x] = t;
                H[threadIdx.x * GM + j] += t;
            }
            __syncthreads();
            for (int i = threadIdx.x; i < n; i += T) {
                double v = w[i];
                for (int l = 0; l <= j; ++l) v = fma(-hs[l], V[(int64_t)l * n + i], v);
                w[i] = v;
            }
            __syncthreads();
        }
        acc = 0.0;
        for (int i = threadIdx.x; i < n; i += T) acc = fma(w[i], w[i], acc);
        const double h = sqrt(cta_sum<T>(acc, red));
        const double inv = h > 0.0 ? 1.0 / h : 0.0;
        for (int i = threadIdx.x; i < n; i += T) w[i] *= inv;
        if (threadIdx.x == 0) {
            H[(j + 1) * GM + j] = h;
            for (int i = 0; i < j; ++i) {  // previous rotations on column j
                const double a0 = H[i * GM + j], b0 = H[(i + 1) * GM + j];
                H[i * GM + j] = cs[i] * a0 + sn[i] * b0;
                H[(i + 1) * GM + j] = -sn[i] * a0 + cs[i] * b0;
            }
            const double a0 = H[j * GM + j], b0 = H[(j + 1) * GM + j];
            const double rr = hypot(a0, b0);
            cs[j] = rr > 0.0 ? a0 / rr : 1.0;
            sn[j] = rr > 0.0 ? b0 / rr : 0.0;
            H[j * GM + j] = rr;
            H[(j + 1) * GM + j] = 0.0;
            g[j + 1] = -sn[j] * g[j];
            g[j] = cs[j] * g[j];
        }
        __syncthreads();
        if (h == 0.0) {  // the Krylov space is exhausted: the solution lies in V_(j+1)
            m = j + 1;
            break;
        }
    }
    if (threadIdx.x == 0) {  // y = H^{-1} g
        for (int i = m - 1; i >= 0; --i) {
            double sacc = g[i];
            for (int t = i + 1; t < m; ++t) sacc = fma(-H[i * GM + t], ys[t], sacc);
            ys[i] = H[i * GM + i] != 0.0 ? sacc / H[i * GM + i] : 0.0;
        }
    }
    __syncthreads();
    // u = V y (into the first basis vector's slot), x += P u
    for (int i = threadIdx.x; i < n; i += T) {
        double u = 0.0;
        for (int l = 0; l < m; ++l) u = fma(ys[l], V[(int64_t)l * n + i], u);
        V[i] = u;
    }
    __syncthreads();
    cta_precond<T>(n, M, G, V, y, rz);
    for (int i = threadIdx.x; i < n; i += T) x[i] += rz[i];
    __syncthreads();
}

// Take blocks of the posted FP64 product while any remain: rows [TILE blk, TILE blk + TILE) of M = A G.
// Every thread of the CTA calls this; blk_s is a shared slot.  Nothing in here waits on another CTA.
template <int T, int TILE>
__device__ void help_pass(HelpJob* h, double* smem_d, int* blk_s) {
    for (;;) {
        if (threadIdx.x == 0) {
            int blk = -1;
            if (ld_acquire(&h->ready) == 1 && *(volatile unsigned int*)&h->next < (unsigned int)h->blocks) {
                const unsigned int q = atomicAdd(&h->next, 1u);
                if (q < (unsigned int)h->blocks) blk = (int)q;
            }
            *blk_s = blk;
        }
        __syncthreads();
        const int blk = *blk_s;
        __syncthreads();
        if (blk < 0) return;
        const int n = h->n, r0 = blk * TILE, rows = min(TILE, n - r0);
        cta_gemm<T, TILE, double, double>(rows, n, n, h->A + (int64_t)r0 * n, n, h->G, n, h->M + (int64_t)r0 * n, n,
                                          1.0, 0.0, smem_d);
        __threadfence();  // every thread's rows of M before the count (cta_gemm ends with a barrier)
        __syncthreads();
        if (threadIdx.x == 0) atomicAdd(&h->done, 1);
    }
}

// 256-thread CTAs are held to 80 registers so that three fit on an SM: the refinement's FP64 loops are
// latency-bound and gain more from the third CTA than they lose to a few spilled registers (measured:
// 178 against 215 ms for the 4096-system batch at two CTAs per SM).
template <int T, int TILE>
__global__ void __launch_bounds__(T, T >= 1024 ? 1 : 3) batched_kernel(BatchArgs a) {
    extern __shared__ __align__(16) float smem[];
    __shared__ int sys_s, flag, stop_s, blk_s, job_s;
    __shared__ double red[T / 32];
    __shared__ unsigned long long redb[T / 32];
    // per CTA: G (nmax^2 floats), M (nmax^2 doubles: FP32 factors, or FP64 ones on the fallback), y
    float* G = a.scratch + (int64_t)blockIdx.x * (3 * a.nmax * a.nmax + 2 * a.nmax);
    float* M = G + a.nmax * a.nmax;
    double* M64 = reinterpret_cast<double*>(M);
    float* y = M + 2 * a.nmax * a.nmax;
    float* z32 = y + a.nmax;
    float* A32 = M + a.nmax * a.nmax;  // FP32 copy of A for the Krylov products (M's FP64 half is free then)
    double* r = a.dscratch + (int64_t)blockIdx.x * a.nmax * (GM + 2);
    double* V = r + a.nmax;
    double* smem_d = reinterpret_cast<double*>(smem);
    bool stranded = false;  // a helper CTA timed out on this CTA's product: its scratch may still be written
    for (;;) {
        help_pass<T, TILE>(a.help, smem_d, &blk_s);  // a fallback system's FP64 product comes first
        if (threadIdx.x == 0) {
            const unsigned int q = atomicAdd(&a.queue[0], 1u);
            sys_s = (q < (unsigned int)a.count) ? a.order[q] : -1;
            if (sys_s >= 0) atomicAdd(&a.queue[2], 1u);
        }
        __syncthreads();
        const int sys = sys_s;
        __syncthreads();
        if (sys < 0) {
            // The queue is empty: keep taking blocks while other CTAs still work on systems (one of them
            // may yet post its product).  Bounded: past spin_limit polls the CTA simply leaves.
            for (long long polls = 0; polls < a.spin_limit; ++polls) {
                help_pass<T, TILE>(a.help, smem_d, &blk_s);
                if (threadIdx.x == 0) stop_s = (*(volatile unsigned int*)&a.queue[2] == 0u) ? 1 : 0;
                __syncthreads();
                const int quit = stop_s;
                __syncthreads();
                if (quit) break;
                __nanosleep(1000);
            }
            break;
        }
        const int n = a.n[sys];
        const double* A = a.A + a.offA[sys];
        const double* b = a.b + a.offv[sys];
        double* x = a.x + a.offv[sys];

        // Up to kDraws multipliers: a draw whose FP32 factors cannot be refined (GENP growth times
        // kappa(A G) too large, or a zero pivot) is replaced by a fresh Gaussian G from another
        // subsequence -- the method's guarantees hold with probability close to 1 per draw (Sec. 4).
        constexpr int kDraws = 3;
        int info = 0, total_sweeps = 0;
        for (int64_t e = threadIdx.x; e < (int64_t)n * n; e += T) A32[e] = (float)A[e];
        const double bmax = cta_max_abs<T>(n, b, redb);  // also orders the A32 stores before their use
        double eta = __longlong_as_double(0x7ff0000000000000LL);
        bool done = false;
        for (int draw = 0; draw < kDraws && !done; ++draw) {
            gen_gaussian_f32<T>((int64_t)n * n, a.seed, (uint64_t)sys + (uint64_t)draw * (uint64_t)a.count, G);
            __syncthreads();
            cta_gemm<T, TILE, double, float>(n, n, n, A, n, G, n, M, n, 1.0f, 0.0f, smem);
            info = cta_genp<T, TILE, float>(n, M, smem, &flag);
            if (info != 0) continue;
            // x = G U^{-1} L^{-1} b
            for (int i = threadIdx.x; i < n; i += T) y[i] = (float)b[i];
            __syncthreads();
            cta_lu_solve<T, float>(n, M, y);
            cta_gemv<T, float>(n, G, y, x, false);
            // sweeps: r = b - A x in FP64, eta = ||r|| / (||A|| ||x|| + ||b||); the correction is
            // x += G U^{-1} L^{-1} r while that at least halves eta, then preconditioned GMRES cycles in
            // FP64; a GMRES cycle that fails to halve eta ends this draw.
            double norm_a = 0.0, eta_prev = 0.0;
            bool krylov = false;
            for (int sw = 0;; ++sw, ++total_sweeps) {
                unsigned long long rbits, abits;
                cta_residual<T>(n, A, b, x, r, sw == 0, &rbits, &abits, redb);
                const double xmax = cta_max_abs<T>(n, x, redb);
                if (threadIdx.x == 0) {
                    const double rm = __longlong_as_double((long long)rbits), xm = xmax, bm = bmax;
                    if (sw == 0) norm_a = __longlong_as_double((long long)abits);
                    const double den = norm_a * xm + bm;
                    double e = den > 0.0 ? rm / den : 0.0;
                    if (!isfinite(e) || !isfinite(xm)) e = __longlong_as_double(0x7ff0000000000000LL);
                    red[0] = e;
                    int st = 0;  // 0 continue classical, 1 continue GMRES, 2 converged, 3 give up this draw
                    if (e <= a.tol) st = 2;
                    else if (sw >= a.max_sweeps || !isfinite(e)) st = 3;
                    else if (sw > 0 && !(e <= 0.5 * eta_prev)) st = krylov ? 3 : 1;
                    else st = krylov ? 1 : 0;
                    stop_s = st;
                }
                __syncthreads();
                const double e = red[0];
                const int st = stop_s;
                __syncthreads();
                eta = e;  // the report matches the x left behind
                if (st == 2) {
                    done = true;
                    eta = e;
                    break;
                }
                if (st == 3) break;
                krylov = (st == 1);
                eta_prev = e;
                if (krylov) {
                    cta_gmres_cycle<T>(n, A32, M, G, x, r, V, y, z32, red);
                } else {
                    for (int i = threadIdx.x; i < n; i += T) y[i] = (float)r[i];
                    __syncthreads();
                    cta_lu_solve<T, float>(n, M, y);
                    cta_gemv<T, float>(n, G, y, x, true);
                }
            }
        }
        if (!done) {
            // FP64 fallback: M = A G and its GENP in FP64 (first multiplier), classical FP64 sweeps.  The
            // product (n^3 FMAs on the DFMA pipe) is posted as row blocks for the other CTAs to share,
            // unless another system already holds this launch's job slot.
            double* y64 = V;
            gen_gaussian_f32<T>((int64_t)n * n, a.seed, (uint64_t)sys, G);
            __threadfence();  // G before the job is published
            __syncthreads();
            HelpJob* h = a.help;
            if (threadIdx.x == 0) {
                job_s = 0;
                if (n > TILE && atomicCAS(&h->claimed, 0u, 1u) == 0u) {
                    h->n = n;
                    h->blocks = (n + TILE - 1) / TILE;
                    h->A = A;
                    h->G = G;
                    h->M = M64;
                    __threadfence();
                    st_release(&h->ready, 1);
                    job_s = 1;
                }
            }
            __syncthreads();
            const bool shared = job_s != 0;
            if (shared) {
                help_pass<T, TILE>(h, smem_d, &blk_s);
                if (threadIdx.x == 0) {
                    // A block is at most TILE n^2 FMAs (under a second at n = 4096 with three CTAs on the
                    // SM's DFMA pipe); the default bound, about a minute of 1 us polls, only ends a real fault.
                    long long spins = 0;
                    stop_s = 0;
                    while (ld_acquire(&h->done) < h->blocks) {
                        if (++spins > 16 * a.spin_limit) { stop_s = 1; break; }
                        __nanosleep(1000);
                    }
                }
                __syncthreads();
                stranded = stop_s != 0;
                __threadfence();  // the helpers' rows of M are read below
            } else {
                cta_gemm<T, TILE, double, double>(n, n, n, A, n, G, n, M64, n, 1.0, 0.0, smem_d);
            }
            info = stranded ? -1 : cta_genp<T, TILE, double>(n, M64, smem_d, &flag);
            if (info == 0) {
                for (int i = threadIdx.x; i < n; i += T) y64[i] = b[i];
                __syncthreads();
                cta_lu_solve<T, double>(n, M64, y64);
                cta_gemv<T, double>(n, G, y64, x, false);
                double eta_prev = 0.0, norm_a = 0.0;
                for (int sw = 0;; ++sw, ++total_sweeps) {
                    unsigned long long rbits, abits;
                    cta_residual<T>(n, A, b, x, r, sw == 0, &rbits, &abits, redb);
                    const double xmax = cta_max_abs<T>(n, x, redb);
                    if (threadIdx.x == 0) {
                        const double rm = __longlong_as_double((long long)rbits), xm = xmax, bm = bmax;
                        if (sw == 0) norm_a = __longlong_as_double((long long)abits);
                        const double den = norm_a * xm + bm;
                        double e = den > 0.0 ? rm / den : 0.0;
                        if (!isfinite(e) || !isfinite(xm)) e = __longlong_as_double(0x7ff0000000000000LL);
                        red[0] = e;
                        stop_s = (e <= a.tol) ? 2
                                 : (sw >= a.max_sweeps || !isfinite(e) || (sw > 0 && !(e <= 0.5 * eta_prev))) ? 3
                                                                                                            : 0;
                    }
                    __syncthreads();
                    const double e = red[0];
                    const int st = stop_s;
                    __syncthreads();
                    eta = e;
                    eta_prev = e;
                    if (st == 2) done = true;
                    if (st != 0) break;
                    for (int i = threadIdx.x; i < n; i += T) y64[i] = r[i];
                    __syncthreads();
                    cta_lu_solve<T, double>(n, M64, y64);
                    cta_gemv<T, double>(n, G, y64, x, true);
                }
            }
        }
        if (!done && info != 0)
            for (int i = threadIdx.x; i < n; i += T) x[i] = __longlong_as_double(0x7ff8000000000000LL);
        if (threadIdx.x == 0) {
            a.info[sys] = done ? 0 : info;
            a.berr[sys] = (!done && info != 0) ? __longlong_as_double(0x7ff8000000000000LL) : eta;
            a.sweeps[sys] = total_sweeps;
            atomicSub(&a.queue[2], 1u);
        }
        __syncthreads();
        if (stranded) break;  // never reached in practice: leave the scratch to the late helper
    }
    // the last CTA to leave re-arms the queue for the next launch (or graph replay)
    if (threadIdx.x == 0) {
        __threadfence();
        if (atomicAdd(&a.queue[1], 1u) == gridDim.x - 1) {
            a.queue[0] = 0u;
            a.queue[1] = 0u;
            a.queue[2] = 0u;
            a.help->claimed = 0u;
            a.help->ready = 0;
            a.help->next = 0u;
            a.help->done = 0;
            __threadfence();
        }
    }
}

template <int T, int TILE>
rmge_status launch_batched(const BatchArgs& a, int ctas, cudaStream_t s) {
    const size_t smem = (size_t)(2 * 16 * TILE + PB * (PB + 1)) * sizeof(double);  // FP32 or FP64 tiles
    if (cudaFuncSetAttribute(batched_kernel<T, TILE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
        cudaSuccess) {
        (void)cudaGetLastError();
        return RMGE_ERR_CUDA;
    }
    batched_kernel<T, TILE><<<ctas, T, smem, s>>>(a);
    RMGE_LAUNCH_CHECK();
    return RMGE_OK;
}

}  // namespace

static_assert(64 + sizeof(HelpJob) <= 256, "the job slot lives in the zeroed queue head");
// queue words 0..2 at bytes 0..11, the status word at byte 32, the job slot from byte 64

// RMGE_ERR_TIMEOUT if a system's wait for its shared product gave up (info -1), else RMGE_OK, into *slot
// (the queue head) and *out (may be NULL).
__global__ void batched_status_kernel(int64_t count, const int32_t* info, int* slot, int32_t* out) {
    __shared__ int bad;
    if (threadIdx.x == 0) bad = 0;
    __syncthreads();
    for (int64_t i = threadIdx.x; i < count; i += blockDim.x)
        if (info[i] == -1) bad = 1;
    __syncthreads();
    if (threadIdx.x == 0) {
        const int st = bad ? (int)RMGE_ERR_TIMEOUT : (int)RMGE_OK;
        *slot = st;
        if (out != nullptr) *out = st;
    }
}

size_t batched_scratch_bytes(int64_t nmax, int ctas) {
    return align256((size_t)ctas * (size_t)(3 * nmax * nmax + 2 * nmax) * sizeof(float)) +
           align256((size_t)ctas * (size_t)nmax * (GM + 2) * sizeof(double)) + 256;
}

rmge_status batched_solve(int64_t count, const int32_t* n, const int64_t* offA, const int64_t* offv,
                          const int32_t* order, const double* A, const double* b, double* x, int32_t* info,
                          double* berr, int32_t* sweeps, uint64_t seed, int max_sweeps, double tol, int64_t nmax,
                          int config, int ctas, long long spin_limit, void* ws, cudaStream_t s) {
    char* base = static_cast<char*>(ws);
    BatchArgs a{};
    a.spin_limit = spin_limit;
    a.count = count;
    a.n = n;
    a.offA = offA;
    a.offv = offv;
    a.order = order;
    a.A = A;
    a.b = b;
    a.x = x;
    a.info = info;
    a.berr = berr;
    a.sweeps = sweeps;
    a.seed = seed;
    a.max_sweeps = max_sweeps;
    a.tol = tol;
    a.nmax = nmax;
    a.queue = reinterpret_cast<unsigned int*>(base);
    a.help = reinterpret_cast<HelpJob*>(base + 64);  // inside the 256 bytes the caller zeroes per launch
    a.scratch = reinterpret_cast<float*>(base + 256);
    a.dscratch = reinterpret_cast<double*>(base + 256 +
                                           align256((size_t)ctas * (size_t)(3 * nmax * nmax + 2 * nmax) * sizeof(float)));
    switch (config) {
        case 0: return launch_batched<256, 32>(a, ctas, s);
        case 1: return launch_batched<256, 64>(a, ctas, s);
        case 2: return launch_batched<1024, 64>(a, ctas, s);
        default: return RMGE_ERR_INVALID_ARG;
    }
}

rmge_status batched_status(int64_t count, const int32_t* info, void* ws, int32_t* out, cudaStream_t s) {
    batched_status_kernel<<<1, 256, 0, s>>>(count, info, reinterpret_cast<int*>(static_cast<char*>(ws) + 32), out);
    RMGE_LAUNCH_CHECK();
    return RMGE_OK;
}

}  // namespace rmge
