/*
 * rmge_oracle.c -- plain, slow, obviously-correct CPU FP64 oracle for the
 * randomized-multiplier GENP solve of Pan, Qian and Yan, "Random multipliers
 * numerically stabilize Gaussian and block Gaussian elimination"
 * (arXiv:1406.5802).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may call, link or
 * load this file; only the test-suite, the smoke check and the CPU-baseline
 * leg of the benchmark do.  It shares no code, header, table or constant with
 * the CUDA library: everything here is written from the paper's definitions.
 *
 * Conventions: row-major, leading dimension = number of columns, FP64.
 * Loops are written in the order the definitions state them; OpenMP only
 * distributes independent rows over threads (each row is still computed by
 * one thread in the same order, so results do not depend on the thread count).
 *
 * Parity pins for every function live in tests/test_oracle_*.py.  The only
 * function without a pin is none; the paper's Table 7.16 (condition numbers of
 * Gaussian matrices) is not reproduced here at all.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_PI 3.14159265358979323846264338327950288

/* ------------------------------------------------------------------------ */
/* Threads                                                                  */
/* ------------------------------------------------------------------------ */
static int orc_threads = 1;

void orc_set_threads(int t) { orc_threads = t < 1 ? 1 : t; }

int orc_get_threads(void) { return orc_threads; }

/* ------------------------------------------------------------------------ */
/* Philox4x32-10 counter-based generator.                                   */
/* Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy as 1, 2,   */
/* 3", SC'11: ten rounds of S-box = two 32x32->64 multiplies with the       */
/* published multipliers, key schedule bumped by the published Weyl         */
/* constants.  The paper (Sec. 7) draws with MATLAB randn and prescribes no */
/* generator; this counter-based one is written from its publication.      */
/* ------------------------------------------------------------------------ */
static void philox_round(uint32_t c[4], const uint32_t k[2]) {
    const uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c[0];
    const uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c[2];
    const uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    const uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t n0 = hi1 ^ c[1] ^ k[0];
    uint32_t n1 = lo1;
    uint32_t n2 = hi0 ^ c[3] ^ k[1];
    uint32_t n3 = lo0;
    c[0] = n0; c[1] = n1; c[2] = n2; c[3] = n3;
}

void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
    uint32_t c[4] = {ctr[0], ctr[1], ctr[2], ctr[3]};
    uint32_t k[2] = {key[0], key[1]};
    for (int r = 0; r < 10; ++r) {
        philox_round(c, k);
        k[0] += 0x9E3779B9u;
        k[1] += 0xBB67AE85u;
    }
    memcpy(out, c, sizeof c);
}

/* One Philox block for the pair index p of stream (seed, subsequence). */
static void draw_block(uint64_t p, uint64_t seed, uint64_t subseq, uint32_t x[4]) {
    uint32_t ctr[4] = {(uint32_t)p, (uint32_t)(p >> 32), (uint32_t)subseq, (uint32_t)(subseq >> 32)};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    orc_philox4x32_10(ctr, key, x);
}

/* 53-bit integer from two 32-bit words: all of hi, the top 21 bits of lo. */
static uint64_t bits53(uint32_t hi, uint32_t lo) {
    return ((uint64_t)hi << 21) | (uint64_t)(lo >> 11);
}

/*
 * Standard Gaussian entries (Def. 4.1: i.i.d., mean 0, variance 1) by the
 * Box-Muller transform (Box & Muller 1958).  Entry e uses Philox block
 * p = e/2: u1 = (m1+1)/2^53 in (0,1], u2 = m2/2^53 in [0,1),
 * r = sqrt(-2 ln u1); entry 2p is r cos(2 pi u2), entry 2p+1 is r sin(2 pi u2).
 */
void orc_gaussian(int64_t count, uint64_t seed, uint64_t subseq, double* out) {
    const double two_m53 = 1.0 / 9007199254740992.0;
    for (int64_t e = 0; e < count; e += 2) {
        uint32_t x[4];
        draw_block((uint64_t)(e / 2), seed, subseq, x);
        const double u1 = (double)(bits53(x[0], x[1]) + 1) * two_m53;
        const double u2 = (double)bits53(x[2], x[3]) * two_m53;
        const double r = sqrt(-2.0 * log(u1));
        out[e] = r * cos(2.0 * ORC_PI * u2);
        if (e + 1 < count) out[e + 1] = r * sin(2.0 * ORC_PI * u2);
    }
}

/*
 * FP32 Gaussian entries for the reduced-precision multipliers: the same Box-Muller pair in
 * single precision from 24-bit uniforms u1 = ((x0 >> 8) + 1) / 2^24, u2 = (x2 >> 8) / 2^24 of
 * Philox block e/2.
 */
void orc_gaussian_f32(int64_t count, uint64_t seed, uint64_t subseq, float* out) {
    const float two_m24 = 1.0f / 16777216.0f;
    for (int64_t e = 0; e < count; e += 2) {
        uint32_t x[4];
        draw_block((uint64_t)(e / 2), seed, subseq, x);
        const float u1 = (float)((x[0] >> 8) + 1u) * two_m24;
        const float u2 = (float)(x[2] >> 8) * two_m24;
        const float r = sqrtf(-2.0f * logf(u1));
        out[e] = r * cosf(2.0f * (float)ORC_PI * u2);
        if (e + 1 < count) out[e + 1] = r * sinf(2.0f * (float)ORC_PI * u2);
    }
}

/*
 * Uniform entries in [-1, 1) (Ex. 5.1 draws the first column of a real
 * circulant uniformly from [-1, 1]).  Entry e uses Philox block e/2; word
 * pair (x0,x1) feeds even entries, (x2,x3) odd ones; value 2m/2^53 - 1.
 */
void orc_uniform_pm1(int64_t count, uint64_t seed, uint64_t subseq, double* out) {
    const double two_m53 = 1.0 / 9007199254740992.0;
    for (int64_t e = 0; e < count; e += 2) {
        uint32_t x[4];
        draw_block((uint64_t)(e / 2), seed, subseq, x);
        out[e] = 2.0 * ((double)bits53(x[0], x[1]) * two_m53) - 1.0;
        if (e + 1 < count) out[e + 1] = 2.0 * ((double)bits53(x[2], x[3]) * two_m53) - 1.0;
    }
}

/*
 * Uniform phases in [0, 1): the same stream layout, value m/2^53.
 */
void orc_uniform01(int64_t count, uint64_t seed, uint64_t subseq, double* out) {
    const double two_m53 = 1.0 / 9007199254740992.0;
    for (int64_t e = 0; e < count; e += 2) {
        uint32_t x[4];
        draw_block((uint64_t)(e / 2), seed, subseq, x);
        out[e] = (double)bits53(x[0], x[1]) * two_m53;
        if (e + 1 < count) out[e + 1] = (double)bits53(x[2], x[3]) * two_m53;
    }
}

/*
 * Spectrum of a random unitary circulant (Ex. 5.2): u_j = exp(2 pi phi_j sqrt(-1)) with phi_j
 * uniform in [0, 1).  The draw is made Hermitian-symmetric (u_{n-j} = conj(u_j), u_0 and u_{n/2}
 * real), so that c = Omega^{-1} u is real and C a real orthogonal matrix: phi_0 .. phi_{n/2} are
 * entries 0 .. n/2 of the phase stream, u_0 = +1 if phi_0 < 1/2 else -1, likewise u_{n/2}
 * (n even).
 */
void orc_unitary_spectrum(int64_t n, uint64_t seed, uint64_t subseq, double* ur, double* ui) {
    const int64_t h = n / 2;
    double* phi = (double*)malloc(sizeof(double) * (size_t)(h + 1));
    orc_uniform01(h + 1, seed, subseq, phi);
    ur[0] = (phi[0] < 0.5) ? 1.0 : -1.0;
    ui[0] = 0.0;
    for (int64_t j = 1; j < h; ++j) {
        ur[j] = cos(2.0 * ORC_PI * phi[j]);
        ui[j] = sin(2.0 * ORC_PI * phi[j]);
        ur[n - j] = ur[j];
        ui[n - j] = -ui[j];
    }
    ur[h] = (phi[h] < 0.5) ? 1.0 : -1.0;
    ui[h] = 0.0;
    free(phi);
}

/* ------------------------------------------------------------------------ */
/* Dense products and the circulant multiplier                              */
/* ------------------------------------------------------------------------ */

/* C (m x n) = A (m x k) * B (k x n), the definition sum_t a_it b_tj. */
void orc_matmul(int64_t m, int64_t k, int64_t n, const double* A, const double* B, double* C) {
#pragma omp parallel for num_threads(orc_threads) schedule(static)
    for (int64_t i = 0; i < m; ++i) {
        double* c = C + i * n;
        for (int64_t j = 0; j < n; ++j) c[j] = 0.0;
        for (int64_t t = 0; t < k; ++t) {
            const double a = A[i * k + t];
            const double* b = B + t * n;
            for (int64_t j = 0; j < n; ++j) c[j] += a * b[j];
        }
    }
}

/* Circulant C = (c_{(i-j) mod n}) defined by its first column (Sec. 5). */
void orc_circulant_dense(int64_t n, const double* c, double* C) {
    for (int64_t i = 0; i < n; ++i)
        for (int64_t j = 0; j < n; ++j) C[i * n + j] = c[((i - j) % n + n) % n];
}

/*
 * Toeplitz multiplier T (n x n) = the leading n x n block of the 2n x 2n circulant with first
 * column c2 (length 2n): T_ij = c2[(i - j) mod 2n] (the paper's Toeplitz multipliers are leading
 * submatrices of random circulant matrices, Sec. 7.2).
 */
void orc_toeplitz_dense(int64_t n, const double* c2, double* T) {
    const int64_t N = 2 * n;
    for (int64_t i = 0; i < n; ++i)
        for (int64_t j = 0; j < n; ++j) T[i * n + j] = c2[((i - j) % N + N) % N];
}

/*
 * Selected rows of A H for a multiplier that is the leading n x n block of an N x N circulant with first
 * column c (N = n: the circulant of Sec. 5; N = 2n: the Toeplitz multiplier above), straight from the
 * entries H_kj = c[(k - j) mod N]:  out_ij = sum_{k < n} a_ik c[(k - j) mod N], for the r rows of A given
 * (r x n).  For checking A H at sizes where the dense H does not fit in memory.
 */
void orc_circulant_rows(int64_t n, int64_t N, int64_t r, const double* A, const double* c, double* out) {
#pragma omp parallel for num_threads(orc_threads) schedule(static)
    for (int64_t i = 0; i < r; ++i)
        for (int64_t j = 0; j < n; ++j) {
            double s = 0.0;
            for (int64_t k = 0; k < n; ++k) s += A[i * n + k] * c[((k - j) % N + N) % N];
            out[i * n + j] = s;
        }
}

/*
 * Plain O(n^2) DFT y_f = sum_t x_t w^{f t}, w = exp(sign * 2 pi i / n).
 * With sign = +1 this is the matrix Omega of Sec. 5 applied to x.
 */
void orc_dft(int64_t n, const double* xr, const double* xi, double* yr, double* yi, int sign) {
    for (int64_t f = 0; f < n; ++f) {
        double sr = 0.0, si = 0.0;
        for (int64_t t = 0; t < n; ++t) {
            const double ang = (double)sign * 2.0 * ORC_PI * (double)((f * t) % n) / (double)n;
            const double wr = cos(ang), wi = sin(ang);
            sr += xr[t] * wr - xi[t] * wi;
            si += xr[t] * wi + xi[t] * wr;
        }
        yr[f] = sr;
        yi[f] = si;
    }
}

/*
 * First column of the random unitary circulant of Ex. 5.2: c = Omega^{-1} u = (1/n) Omega^H u for the
 * Hermitian-symmetric spectrum of orc_unitary_spectrum, by the plain inverse DFT.  c is real; cim
 * receives the imaginary parts left by rounding.
 */
void orc_unitary_circulant_column(int64_t n, uint64_t seed, uint64_t subseq, double* c, double* cim) {
    double* ur = (double*)malloc(sizeof(double) * (size_t)n);
    double* ui = (double*)malloc(sizeof(double) * (size_t)n);
    orc_unitary_spectrum(n, seed, subseq, ur, ui);
    orc_dft(n, ur, ui, c, cim, -1);
    for (int64_t t = 0; t < n; ++t) {
        c[t] /= (double)n;
        cim[t] /= (double)n;
    }
    free(ur);
    free(ui);
}

/* ------------------------------------------------------------------------ */
/* GENP: Gaussian elimination with no pivoting (Sec. 3)                     */
/* ------------------------------------------------------------------------ */

/*
 * In-place unblocked right-looking GENP: eq. (3.1) with a 1x1 pivot block,
 * applied recursively to the Schur complement (Sec. 3, "if k = 1 at all
 * recursive steps ... defines GENP").  On return M holds the unit lower
 * factor below the diagonal and U on and above it.  Returns 0, or the
 * 1-based step s whose pivot is zero or not finite (Cor. 3.1: a zero pivot
 * appears exactly when a leading block is singular); M is then left as it
 * was after step s-1.
 */
int orc_genp(int64_t n, double* M) {
    for (int64_t s = 0; s < n; ++s) {
        const double piv = M[s * n + s];
        if (piv == 0.0 || !isfinite(piv)) return (int)(s + 1);
#pragma omp parallel for num_threads(orc_threads) schedule(static)
        for (int64_t i = s + 1; i < n; ++i) {
            const double l = M[i * n + s] / piv;
            M[i * n + s] = l;
            for (int64_t j = s + 1; j < n; ++j) M[i * n + j] -= l * M[s * n + j];
        }
    }
    return 0;
}

/*
 * Blocked GENP with pivot blocks of size nb (eq. (3.1) with k = nb): factor
 * the leading nb x nb block B by orc_genp, form D B^{-1} (rows of the lower
 * factor) and B^{-1} C (rows of the upper factor) by substitution, and
 * replace E by the Schur complement E - (D B^{-1})(L_B^{-1} C).  Used only to
 * pin the statement of Sec. 3 that any blocking yields the same Schur
 * complements, hence the same L and U.
 */
int orc_genp_blocked(int64_t n, int64_t nb, double* M) {
    for (int64_t k = 0; k < n; k += nb) {
        const int64_t b = (n - k < nb) ? n - k : nb;
        /* factor the diagonal block in place (unblocked GENP on a b x b view) */
        for (int64_t s = k; s < k + b; ++s) {
            const double piv = M[s * n + s];
            if (piv == 0.0 || !isfinite(piv)) return (int)(s + 1);
            for (int64_t i = s + 1; i < k + b; ++i) {
                const double l = M[i * n + s] / piv;
                M[i * n + s] = l;
                for (int64_t j = s + 1; j < k + b; ++j) M[i * n + j] -= l * M[s * n + j];
            }
        }
        /* U12 = L11^{-1} A12: forward substitution down each column j */
        for (int64_t j = k + b; j < n; ++j)
            for (int64_t i = k; i < k + b; ++i)
                for (int64_t t = k; t < i; ++t) M[i * n + j] -= M[i * n + t] * M[t * n + j];
        /* L21 = A21 U11^{-1}: substitution along each row i */
        for (int64_t i = k + b; i < n; ++i)
            for (int64_t j = k; j < k + b; ++j) {
                double v = M[i * n + j];
                for (int64_t t = k; t < j; ++t) v -= M[i * n + t] * M[t * n + j];
                M[i * n + j] = v / M[j * n + j];
            }
        /* Schur complement E <- E - L21 U12 */
#pragma omp parallel for num_threads(orc_threads) schedule(static)
        for (int64_t i = k + b; i < n; ++i)
            for (int64_t t = k; t < k + b; ++t) {
                const double l = M[i * n + t];
                for (int64_t j = k + b; j < n; ++j) M[i * n + j] -= l * M[t * n + j];
            }
    }
    return 0;
}

/*
 * GEPP, the customary partial-pivoting baseline the paper compares against
 * (Sec. 1, Table 7.2).  At step s the pivot row is the first row i >= s with
 * the largest |M[i][s]|; rows are swapped explicitly and piv[s] records i.
 * Returns 0, or the 1-based step whose whole column is zero.
 */
int orc_gepp(int64_t n, double* M, int64_t* piv) {
    for (int64_t s = 0; s < n; ++s) {
        int64_t p = s;
        double best = fabs(M[s * n + s]);
        for (int64_t i = s + 1; i < n; ++i)
            if (fabs(M[i * n + s]) > best) { best = fabs(M[i * n + s]); p = i; }
        piv[s] = p;
        if (best == 0.0 || !isfinite(best)) return (int)(s + 1);
        if (p != s)
            for (int64_t j = 0; j < n; ++j) {
                double t = M[s * n + j]; M[s * n + j] = M[p * n + j]; M[p * n + j] = t;
            }
        const double pv = M[s * n + s];
#pragma omp parallel for num_threads(orc_threads) schedule(static)
        for (int64_t i = s + 1; i < n; ++i) {
            const double l = M[i * n + s] / pv;
            M[i * n + s] = l;
            for (int64_t j = s + 1; j < n; ++j) M[i * n + j] -= l * M[s * n + j];
        }
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Triangular solves with packed L\U factors, k right-hand sides            */
/* ------------------------------------------------------------------------ */

/* B (n x k) <- U^{-1} L^{-1} B, L unit lower and U upper packed in LU. */
void orc_lu_solve(int64_t n, int64_t k, const double* LU, double* B) {
    for (int64_t i = 0; i < n; ++i)              /* L z = b, top to bottom */
        for (int64_t t = 0; t < i; ++t) {
            const double l = LU[i * n + t];
            for (int64_t c = 0; c < k; ++c) B[i * k + c] -= l * B[t * k + c];
        }
    for (int64_t i = n - 1; i >= 0; --i) {       /* U y = z, bottom to top */
        for (int64_t t = i + 1; t < n; ++t) {
            const double u = LU[i * n + t];
            for (int64_t c = 0; c < k; ++c) B[i * k + c] -= u * B[t * k + c];
        }
        for (int64_t c = 0; c < k; ++c) B[i * k + c] /= LU[i * n + i];
    }
}

/* B <- U^{-T} ... transposed solve:  B <- L^{-T} U^{-T} B  (A^T x = b with A = L U). */
void orc_lu_solve_transposed(int64_t n, int64_t k, const double* LU, double* B) {
    for (int64_t i = 0; i < n; ++i) {            /* U^T p = b: U^T is lower */
        for (int64_t t = 0; t < i; ++t) {
            const double u = LU[t * n + i];
            for (int64_t c = 0; c < k; ++c) B[i * k + c] -= u * B[t * k + c];
        }
        for (int64_t c = 0; c < k; ++c) B[i * k + c] /= LU[i * n + i];
    }
    for (int64_t i = n - 1; i >= 0; --i)         /* L^T q = p: L^T is unit upper */
        for (int64_t t = i + 1; t < n; ++t) {
            const double l = LU[t * n + i];
            for (int64_t c = 0; c < k; ++c) B[i * k + c] -= l * B[t * k + c];
        }
}

/* Solve with GEPP factors: apply the recorded row swaps to B, then L, U. */
void orc_gepp_solve(int64_t n, int64_t k, const double* LU, const int64_t* piv, double* B) {
    for (int64_t s = 0; s < n; ++s)
        if (piv[s] != s)
            for (int64_t c = 0; c < k; ++c) {
                double t = B[s * k + c]; B[s * k + c] = B[piv[s] * k + c]; B[piv[s] * k + c] = t;
            }
    orc_lu_solve(n, k, LU, B);
}

/* ------------------------------------------------------------------------ */
/* Residuals and backward error                                             */
/* ------------------------------------------------------------------------ */

/*
 * R = B - A X with each entry accumulated by the compensated dot product
 * Dot2 of Ogita, Rump and Oishi (SIAM J. Sci. Comput. 26, 2005): TwoProduct
 * by fma, TwoSum by Knuth's branch-free form, so the residual is as accurate
 * as if computed in twice the working precision and then rounded.
 */
void orc_residual(int64_t n, int64_t k, const double* A, const double* X, const double* B, double* R) {
#pragma omp parallel for num_threads(orc_threads) schedule(static)
    for (int64_t i = 0; i < n; ++i)
        for (int64_t c = 0; c < k; ++c) {
            double s = B[i * k + c], err = 0.0;
            for (int64_t t = 0; t < n; ++t) {
                const double p = -A[i * n + t] * X[t * k + c];
                const double pe = fma(-A[i * n + t], X[t * k + c], -p);
                const double s2 = s + p;
                const double z = s2 - s;
                const double se = (s - (s2 - z)) + (p - z);
                s = s2;
                err += pe + se;
            }
            R[i * k + c] = s + err;
        }
}

/* ||A||_inf = max_i sum_j |a_ij| */
double orc_norm_inf(int64_t m, int64_t n, const double* A) {
    double best = 0.0;
    for (int64_t i = 0; i < m; ++i) {
        double s = 0.0;
        for (int64_t j = 0; j < n; ++j) s += fabs(A[i * n + j]);
        if (s > best || isnan(s)) best = s;
    }
    return best;
}

/*
 * Normwise backward error, per right-hand side column c:
 *   eta_c = ||b_c - A x_c||_inf / (||A||_inf ||x_c||_inf + ||b_c||_inf),
 * returned as the max over columns (Rigal-Gaches normwise backward error, the
 * quantity the accuracy target is stated in).  NaN/Inf anywhere -> +Inf.
 */
double orc_backward_error(int64_t n, int64_t k, const double* A, const double* X, const double* B) {
    double* R = (double*)malloc(sizeof(double) * (size_t)(n * k));
    if (!R) return INFINITY;
    orc_residual(n, k, A, X, B, R);
    const double an = orc_norm_inf(n, n, A);
    double eta = 0.0;
    for (int64_t c = 0; c < k; ++c) {
        double rn = 0.0, xn = 0.0, bn = 0.0;
        for (int64_t i = 0; i < n; ++i) {
            rn = fmax(rn, fabs(R[i * k + c]));
            xn = fmax(xn, fabs(X[i * k + c]));
            bn = fmax(bn, fabs(B[i * k + c]));
            if (!isfinite(R[i * k + c]) || !isfinite(X[i * k + c])) { free(R); return INFINITY; }
        }
        const double den = an * xn + bn;
        const double e = den > 0.0 ? rn / den : (rn > 0.0 ? INFINITY : 0.0);
        if (e > eta) eta = e;
    }
    free(R);
    return eta;
}

/* Relative residual ||A y - b||_2 / ||b||_2 per column, max over columns (Sec. 7.1's metric). */
double orc_relative_residual(int64_t n, int64_t k, const double* A, const double* X, const double* B) {
    double* R = (double*)malloc(sizeof(double) * (size_t)(n * k));
    if (!R) return INFINITY;
    orc_residual(n, k, A, X, B, R);
    double worst = 0.0;
    for (int64_t c = 0; c < k; ++c) {
        double rn = 0.0, bn = 0.0;
        for (int64_t i = 0; i < n; ++i) { rn += R[i * k + c] * R[i * k + c]; bn += B[i * k + c] * B[i * k + c]; }
        const double v = sqrt(rn) / sqrt(bn);
        if (!(v <= worst)) worst = v;
    }
    free(R);
    return worst;
}

/* Growth rho = max |U_ij| / max |M_ij| (the pivot-growth check of Thm 3.2 / Remark 3.2). */
double orc_growth(int64_t n, const double* M, const double* LU) {
    double mm = 0.0, um = 0.0;
    for (int64_t i = 0; i < n; ++i)
        for (int64_t j = 0; j < n; ++j) {
            mm = fmax(mm, fabs(M[i * n + j]));
            if (j >= i) um = fmax(um, fabs(LU[i * n + j]));
        }
    return mm > 0.0 ? um / mm : INFINITY;
}

/* ------------------------------------------------------------------------ */
/* The randomized GENP solve (Fact 4.1 with F = I, H = G)                   */
/* ------------------------------------------------------------------------ */

/*
 * Multiplier kinds: 0 dense Gaussian H (n x n); 1, 2, 3 circulant H given by its first column (n);
 * 4, 5 Toeplitz H given by the first column of the 2n x 2n circulant it is the leading block of.
 * The dense matrix of H, for the products below.
 */
void orc_multiplier_dense(int kind, int64_t n, const double* H, double* D) {
    if (kind == 0)
        memcpy(D, H, sizeof(double) * (size_t)(n * n));
    else if (kind <= 3)
        orc_circulant_dense(n, H, D);
    else
        orc_toeplitz_dense(n, H, D);
}

static void apply_H(int kind, int64_t n, int64_t k, const double* H, const double* Y, double* X) {
    double* D = (double*)malloc(sizeof(double) * (size_t)(n * n));
    orc_multiplier_dense(kind, n, H, D);
    orc_matmul(n, n, k, D, Y, X);
    free(D);
}

/* M = A H (post-multiplication, Fact 4.1), with the dense matrix of a structured H. */
void orc_apply_multiplier(int kind, int64_t n, const double* A, const double* H, double* M) {
    double* D = (double*)malloc(sizeof(double) * (size_t)(n * n));
    orc_multiplier_dense(kind, n, H, D);
    orc_matmul(n, n, n, A, D, M);
    free(D);
}

/*
 * One refinement sweep (Sec. 1.2, Sec. 7.1): R = B - A X (compensated),
 * D = H U^{-1} L^{-1} R, X <- X + D.
 */
void orc_refine_step(int kind, int64_t n, int64_t k, const double* A, const double* LU, const double* H,
                     const double* B, double* X) {
    double* R = (double*)malloc(sizeof(double) * (size_t)(n * k));
    double* D = (double*)malloc(sizeof(double) * (size_t)(n * k));
    orc_residual(n, k, A, X, B, R);
    orc_lu_solve(n, k, LU, R);
    apply_H(kind, n, k, H, R, D);
    for (int64_t i = 0; i < n * k; ++i) X[i] += D[i];
    free(R);
    free(D);
}

/*
 * Full randomized GENP solve of A X = B (Fact 4.1, post-multiplication):
 * M = A H; GENP M = L U; Y = U^{-1} L^{-1} B; X = H Y; then refinement sweeps
 * until the normwise backward error is <= be_tol or max_iters sweeps ran.
 * LU (n x n) receives the factors; berr[0..max_iters] the backward error
 * after 0, 1, ... sweeps (entries past the last sweep are left untouched).
 * Returns the GENP info (0 = ok); *iters = sweeps performed.
 */
int orc_rmge_solve(int kind, int64_t n, int64_t k, const double* A, const double* H, const double* B,
                   double* X, double* LU, int max_iters, double be_tol, double* berr, int* iters) {
    orc_apply_multiplier(kind, n, A, H, LU);
    const int info = orc_genp(n, LU);
    *iters = 0;
    if (info != 0) return info;
    double* Y = (double*)malloc(sizeof(double) * (size_t)(n * k));
    memcpy(Y, B, sizeof(double) * (size_t)(n * k));
    orc_lu_solve(n, k, LU, Y);
    apply_H(kind, n, k, H, Y, X);
    free(Y);
    double be = orc_backward_error(n, k, A, X, B);
    berr[0] = be;
    int it = 0;
    while (it < max_iters && !(be <= be_tol)) {
        orc_refine_step(kind, n, k, A, LU, H, B, X);
        be = orc_backward_error(n, k, A, X, B);
        ++it;
        berr[it] = be;
    }
    *iters = it;
    return 0;
}

/* D (n x n) = the dense matrix of a multiplier, or the identity when kind < 0 (one-sided forms). */
static void multiplier_or_identity(int kind, int64_t n, const double* H, double* D) {
    if (kind < 0) {
        memset(D, 0, sizeof(double) * (size_t)(n * n));
        for (int64_t i = 0; i < n; ++i) D[i * n + i] = 1.0;
    } else {
        orc_multiplier_dense(kind, n, H, D);
    }
}

/*
 * Two-sided randomized GENP solve (Fact 4.1: A^{-1} = H (F A H)^{-1} F, so F A H y = F b and x = H y):
 * M = F A H, GENP M = L U, X = H U^{-1} L^{-1} F B, then refinement sweeps
 * X <- X + H U^{-1} L^{-1} F (B - A X) until the backward error is <= be_tol or max_iters sweeps ran.
 * kindF < 0 means F = I (post-multiplication only), kindH < 0 means H = I (pre-multiplication only).
 * Outputs as for orc_rmge_solve.
 */
int orc_rmge_solve_two_sided(int kindF, const double* F, int kindH, const double* H, int64_t n, int64_t k,
                             const double* A, const double* B, double* X, double* LU, int max_iters, double be_tol,
                             double* berr, int* iters) {
    double* DF = (double*)malloc(sizeof(double) * (size_t)(n * n));
    double* DH = (double*)malloc(sizeof(double) * (size_t)(n * n));
    double* T = (double*)malloc(sizeof(double) * (size_t)(n * n));
    double* V = (double*)malloc(sizeof(double) * (size_t)(n * k));
    double* Y = (double*)malloc(sizeof(double) * (size_t)(n * k));
    multiplier_or_identity(kindF, n, F, DF);
    multiplier_or_identity(kindH, n, H, DH);
    orc_matmul(n, n, n, A, DH, T);   /* A H */
    orc_matmul(n, n, n, DF, T, LU);  /* F A H */
    const int info = orc_genp(n, LU);
    *iters = 0;
    if (info == 0) {
        /* X = H U^{-1} L^{-1} F B */
        orc_matmul(n, n, k, DF, B, Y);
        orc_lu_solve(n, k, LU, Y);
        orc_matmul(n, n, k, DH, Y, X);
        double be = orc_backward_error(n, k, A, X, B);
        berr[0] = be;
        int it = 0;
        while (it < max_iters && !(be <= be_tol)) {
            orc_residual(n, k, A, X, B, V);
            orc_matmul(n, n, k, DF, V, Y);
            orc_lu_solve(n, k, LU, Y);
            orc_matmul(n, n, k, DH, Y, V);
            for (int64_t i = 0; i < n * k; ++i) X[i] += V[i];
            be = orc_backward_error(n, k, A, X, B);
            ++it;
            berr[it] = be;
        }
        *iters = it;
    }
    free(DF);
    free(DH);
    free(T);
    free(V);
    free(Y);
    return info;
}

/* ------------------------------------------------------------------------ */
/* Low-rank approximation (Sec. 6, Algorithm 6.1)                           */
/* ------------------------------------------------------------------------ */

/*
 * Thin Householder QR of B (m x l, m >= l): B = Q R, Q (m x l) with orthonormal columns, R (l x l)
 * upper triangular.  Column j is reflected by I - 2 v v^T / v^T v with v = x - alpha e_1,
 * alpha = -sign(x_1) ||x||; Q is the product of the reflections applied to the first l columns of
 * the identity.  Finally each j with R_jj < 0 has row j of R and column j of Q negated, so that
 * diag(R) >= 0 and the factorization of a full-rank B is unique.
 */
void orc_qr(int64_t m, int64_t l, const double* B, double* Q, double* R) {
    double* W = (double*)malloc(sizeof(double) * (size_t)(m * l));
    double* V = (double*)malloc(sizeof(double) * (size_t)(m * l));  /* reflection j in column j, rows j.. */
    memcpy(W, B, sizeof(double) * (size_t)(m * l));
    memset(V, 0, sizeof(double) * (size_t)(m * l));
    for (int64_t j = 0; j < l; ++j) {
        double nx = 0.0;
        for (int64_t i = j; i < m; ++i) nx += W[i * l + j] * W[i * l + j];
        nx = sqrt(nx);
        const double x1 = W[j * l + j];
        const double alpha = (x1 >= 0.0) ? -nx : nx;
        double vv = 0.0;
        for (int64_t i = j; i < m; ++i) {
            const double v = W[i * l + j] - ((i == j) ? alpha : 0.0);
            V[i * l + j] = v;
            vv += v * v;
        }
        if (vv > 0.0) {
            for (int64_t c = j; c < l; ++c) {
                double d = 0.0;
                for (int64_t i = j; i < m; ++i) d += V[i * l + j] * W[i * l + c];
                const double f = 2.0 * d / vv;
                for (int64_t i = j; i < m; ++i) W[i * l + c] -= f * V[i * l + j];
            }
        }
        /* keep v^T v with the reflection for forming Q */
        V[j * l + j] = (vv > 0.0) ? V[j * l + j] : 0.0;
        W[j * l + j] = (vv > 0.0) ? W[j * l + j] : x1;
        for (int64_t c = 0; c < l; ++c) R[j * l + c] = (c >= j) ? W[j * l + c] : 0.0;
    }
    /* Q = H_0 H_1 ... H_{l-1} [I_l; 0]: apply the reflections in reverse order */
    for (int64_t i = 0; i < m; ++i)
        for (int64_t c = 0; c < l; ++c) Q[i * l + c] = (i == c) ? 1.0 : 0.0;
    for (int64_t j = l - 1; j >= 0; --j) {
        double vv = 0.0;
        for (int64_t i = j; i < m; ++i) vv += V[i * l + j] * V[i * l + j];
        if (vv == 0.0) continue;
        for (int64_t c = 0; c < l; ++c) {
            double d = 0.0;
            for (int64_t i = j; i < m; ++i) d += V[i * l + j] * Q[i * l + c];
            const double f = 2.0 * d / vv;
            for (int64_t i = j; i < m; ++i) Q[i * l + c] -= f * V[i * l + j];
        }
    }
    for (int64_t j = 0; j < l; ++j) {
        if (R[j * l + j] < 0.0) {
            for (int64_t c = 0; c < l; ++c) R[j * l + c] = -R[j * l + c];
            for (int64_t i = 0; i < m; ++i) Q[i * l + j] = -Q[i * l + j];
        }
    }
    free(W);
    free(V);
}

/*
 * The n x l multiplier of Algorithm 6.1 as a dense matrix: kind 0, H itself (n x l); kinds 1, 2, 3,
 * the n x l leading block of the n x n circulant with first column c = H (Sec. 7.2's Toeplitz
 * multipliers: the maximal leading submatrices of random circulants), D_ij = c_{(i - j) mod n}.
 */
void orc_lowrank_multiplier_dense(int kind, int64_t n, int64_t l, const double* H, double* D) {
    for (int64_t i = 0; i < n; ++i)
        for (int64_t j = 0; j < l; ++j) D[i * l + j] = (kind == 0) ? H[i * l + j] : H[((i - j) % n + n) % n];
}

/*
 * Algorithm 6.1 (low-rank approximation, after Halko, Martinsson and Tropp): B = A H (m x l),
 * Q = Q(B) by orc_qr (orthonormal columns sharing B's range), Z = Q^T A (l x n); Q Z = Q Q^T A has
 * rank at most l and approximates A.
 */
void orc_lowrank(int kind, int64_t m, int64_t n, int64_t l, const double* A, const double* H, double* Q, double* Z) {
    double* D = (double*)malloc(sizeof(double) * (size_t)(n * l));
    double* B = (double*)malloc(sizeof(double) * (size_t)(m * l));
    double* R = (double*)malloc(sizeof(double) * (size_t)(l * l));
    orc_lowrank_multiplier_dense(kind, n, l, H, D);
    orc_matmul(m, n, l, A, D, B);
    orc_qr(m, l, B, Q, R);
    for (int64_t i = 0; i < l; ++i)
        for (int64_t j = 0; j < n; ++j) {
            double z = 0.0;
            for (int64_t t = 0; t < m; ++t) z += Q[t * l + i] * A[t * n + j];
            Z[i * n + j] = z;
        }
    free(D);
    free(B);
    free(R);
}

/*
 * Reference gradient of a loss L(X) with X = A^{-1} B, given Wbar = dL/dX:
 * dB = A^{-T} Wbar by GEPP on A^T (independent of the GENP factors),
 * dA = -dB X^T.  (The paper has no gradients; this is the adjoint of the
 * linear solve the paper's method computes.)
 */
int orc_solve_adjoint_gepp(int64_t n, int64_t k, const double* A, const double* X, const double* Wbar,
                           double* dB, double* dA) {
    double* AT = (double*)malloc(sizeof(double) * (size_t)(n * n));
    int64_t* piv = (int64_t*)malloc(sizeof(int64_t) * (size_t)n);
    for (int64_t i = 0; i < n; ++i)
        for (int64_t j = 0; j < n; ++j) AT[j * n + i] = A[i * n + j];
    const int info = orc_gepp(n, AT, piv);
    if (info == 0) {
        memcpy(dB, Wbar, sizeof(double) * (size_t)(n * k));
        orc_gepp_solve(n, k, AT, piv, dB);
#pragma omp parallel for num_threads(orc_threads) schedule(static)
        for (int64_t i = 0; i < n; ++i)
            for (int64_t j = 0; j < n; ++j) {
                double s = 0.0;
                for (int64_t c = 0; c < k; ++c) s += dB[i * k + c] * X[j * k + c];
                dA[i * n + j] = -s;
            }
    }
    free(AT);
    free(piv);
    return info;
}

/* ------------------------------------------------------------------------ */
/* Complex GENP (Theorem 5.2 concerns the complex DFT matrix)               */
/* ------------------------------------------------------------------------ */

/* In-place complex GENP on (re, im); pivots written to (pr, pi). */
int orc_genp_complex(int64_t n, double* re, double* im, double* pr, double* pi) {
    for (int64_t s = 0; s < n; ++s) {
        const double a = re[s * n + s], b = im[s * n + s];
        pr[s] = a;
        pi[s] = b;
        if ((a == 0.0 && b == 0.0) || !isfinite(a) || !isfinite(b)) return (int)(s + 1);
        const double d = a * a + b * b;
        for (int64_t i = s + 1; i < n; ++i) {
            const double xr = re[i * n + s], xi = im[i * n + s];
            const double lr = (xr * a + xi * b) / d, li = (xi * a - xr * b) / d;
            re[i * n + s] = lr;
            im[i * n + s] = li;
            for (int64_t j = s + 1; j < n; ++j) {
                const double ur = re[s * n + j], ui = im[s * n + j];
                re[i * n + j] -= lr * ur - li * ui;
                im[i * n + j] -= lr * ui + li * ur;
            }
        }
    }
    return 0;
}
