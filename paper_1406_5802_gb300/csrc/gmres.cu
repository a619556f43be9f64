// gmres.cu -- FGMRES cycles used as refinement sweeps for reduced-precision factors.
//
// Residual correction (Sec. 1.2, Sec. 7.1) with factors of A G computed in FP32/BF16/FP16 converges
// only while the factorization error times kappa(A G) stays below one; for the Gaussian multiplier
// kappa(A G) grows like kappa(A) n, so at large n that bound fails.  Each sweep then solves the
// correction equation A d = r by right-preconditioned flexible GMRES in FP64 (GMRES-based
// iterative refinement; Carson and Higham, SIAM J. Sci. Comput. 2017/2018) with the preconditioner
// P = G U^{-1} L^{-1} of Fact 4.1 applied in the factor precision.  All k right-hand sides run
// side by side, each with its own Krylov basis (V, Z: vector v, row r, column c at
// [v][r * k + c]), its own Hessenberg matrix H[c][i][j] (i <= m, j < m) and Givens rotations.
// Orthogonalisation is classical Gram-Schmidt applied twice.  Every kernel skips its work once
// DevState::stop is set; the steps of a cycle also stop once its residual estimate has fallen by
// kInnerTol for every column, and the correction uses the steps taken.
#include "kernels.cuh"

namespace rmge {
namespace {

constexpr int RT = 1024;  // threads of the per-column reduction kernels
// A cycle ends early once every column's FGMRES residual estimate has fallen by this factor: the outer
// sweep then recomputes the residual in FP64 and starts a new cycle if the target is not met.
constexpr double kInnerTol = 1e-6;

__device__ __forceinline__ bool stopped(const int* skip) { return skip != nullptr && *(volatile const int*)skip != 0; }

// Deterministic block sum of one value per thread (RT threads).
__device__ double block_sum(double v, double* red) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) red[w] = v;
    __syncthreads();
    double t = 0.0;
    if (w == 0) {
        t = (l < RT / 32) ? red[l] : 0.0;
        for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    }
    __syncthreads();
    if (threadIdx.x == 0) red[0] = t;
    __syncthreads();
    const double s = red[0];
    __syncthreads();
    return s;
}

// One CTA per column c: nrm = ||src[:, c]||_2; dst[:, c] = src[:, c] / nrm (0 if nrm == 0).
// start: nrm -> beta[c], g[c] = (beta, 0, ...); else nrm -> H[c][j+1][j].
__global__ void __launch_bounds__(RT) norm_scale_kernel(int64_t n, int64_t k, int m, const double* __restrict__ src,
                                                        double* __restrict__ dst, bool start, int j,
                                                        double* __restrict__ H, double* __restrict__ g,
                                                        double* __restrict__ beta, const int* skip) {
    __shared__ double red[RT / 32];
    if (stopped(skip)) return;
    const int64_t c = blockIdx.x;
    double acc = 0.0;
    for (int64_t r = threadIdx.x; r < n; r += RT) {
        const double v = src[r * k + c];
        acc = fma(v, v, acc);
    }
    const double nrm = sqrt(block_sum(acc, red));
    const double inv = nrm > 0.0 ? 1.0 / nrm : 0.0;
    for (int64_t r = threadIdx.x; r < n; r += RT) dst[r * k + c] = src[r * k + c] * inv;
    if (threadIdx.x == 0) {
        if (start) {
            g[c * (m + 1)] = nrm;
            for (int i = 1; i <= m; ++i) g[c * (m + 1) + i] = 0.0;
            beta[c] = nrm;
        } else {
            H[(c * (m + 1) + (j + 1)) * m + j] = nrm;
        }
    }
}

// CTA (l, c): h = <V_l[:, c], W[:, c]>; hc[c][l] = h; H[c][l][j] (+)= h.
__global__ void __launch_bounds__(RT) dots_kernel(int64_t n, int64_t k, int m, int j, const double* __restrict__ V,
                                                  const double* __restrict__ W, double* __restrict__ hc,
                                                  double* __restrict__ H, bool accumulate, const int* skip) {
    __shared__ double red[RT / 32];
    if (stopped(skip)) return;
    const int l = blockIdx.x;
    const int64_t c = blockIdx.y;
    const double* v = V + (int64_t)l * n * k;
    double acc = 0.0;
    for (int64_t r = threadIdx.x; r < n; r += RT) acc = fma(v[r * k + c], W[r * k + c], acc);
    const double h = block_sum(acc, red);
    if (threadIdx.x == 0) {
        hc[c * (m + 1) + l] = h;
        double* hp = H + (c * (m + 1) + l) * m + j;
        *hp = accumulate ? *hp + h : h;
    }
}

// W[r][c] -= sum_{l <= j} V_l[r][c] hc[c][l]
__global__ void axpy_kernel(int64_t n, int64_t k, int m, int j, const double* __restrict__ V,
                            const double* __restrict__ hc, double* __restrict__ W, const int* skip) {
    if (stopped(skip)) return;
    const int64_t total = n * k;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t c = e % k;
        double w = W[e];
        for (int l = 0; l <= j; ++l) w = fma(-V[(int64_t)l * total + e], hc[c * (m + 1) + l], w);
        W[e] = w;
    }
}

// Columns strided over one CTA: rotate column j of H by the previous rotations, form rotation j so that
// H[j+1][j] becomes 0, and rotate g.  ctl[1] <- j + 1 (steps taken); once every column's residual
// estimate |g_{j+1}| is within kInnerTol of its starting norm, ctl[0] <- 1 ends the cycle early.
__global__ void __launch_bounds__(128) givens_kernel(int64_t k, int m, int j, double* __restrict__ H,
                                                     double* __restrict__ cs, double* __restrict__ sn,
                                                     double* __restrict__ g, const double* __restrict__ beta,
                                                     int* ctl) {
    __shared__ int open_cols;
    if (stopped(ctl)) return;
    if (threadIdx.x == 0) open_cols = 0;
    __syncthreads();
    for (int64_t c = threadIdx.x; c < k; c += blockDim.x) {
        double* h = H + c * (m + 1) * m;
        for (int i = 0; i < j; ++i) {
            const double a = h[i * m + j], b = h[(i + 1) * m + j];
            const double cc = cs[c * m + i], ss = sn[c * m + i];
            h[i * m + j] = cc * a + ss * b;
            h[(i + 1) * m + j] = -ss * a + cc * b;
        }
        const double a = h[j * m + j], b = h[(j + 1) * m + j];
        const double r = hypot(a, b);
        double cc = 1.0, ss = 0.0;
        if (r > 0.0) {
            cc = a / r;
            ss = b / r;
        }
        cs[c * m + j] = cc;
        sn[c * m + j] = ss;
        h[j * m + j] = r;
        h[(j + 1) * m + j] = 0.0;
        double* gc = g + c * (m + 1);
        const double g0 = gc[j];
        gc[j] = cc * g0;
        gc[j + 1] = -ss * g0;
        if (!(fabs(gc[j + 1]) <= kInnerTol * beta[c])) atomicAdd(&open_cols, 1);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        ctl[1] = j + 1;
        if (open_cols == 0) ctl[0] = 1;
    }
}

// One thread per column: y = H(0:j, 0:j)^{-1} g(0:j) by back substitution (zero pivot -> 0), j = ctl[1]
// the steps the cycle took.
__global__ void backsolve_kernel(int64_t k, int m, const double* __restrict__ H, const double* __restrict__ g,
                                 double* __restrict__ y, const int* ctl, const int* skip) {
    if (stopped(skip)) return;
    const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (c >= k) return;
    const int steps = ctl[1];
    const double* h = H + c * (m + 1) * m;
    for (int i = steps - 1; i >= 0; --i) {
        double s = g[c * (m + 1) + i];
        for (int t = i + 1; t < steps; ++t) s = fma(-h[i * m + t], y[c * m + t], s);
        const double d = h[i * m + i];
        y[c * m + i] = d != 0.0 ? s / d : 0.0;
    }
}

// X[r][c] += sum_{i < ctl[1]} Z_i[r][c] y[c][i]
__global__ void update_kernel(int64_t n, int64_t k, int m, const double* __restrict__ Z, const double* __restrict__ y,
                              double* __restrict__ X, int64_t ldx, const int* ctl, const int* skip) {
    if (stopped(skip)) return;
    const int steps = ctl[1];
    const int64_t total = n * k;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = e / k, c = e % k;
        double s = 0.0;
        for (int i = 0; i < steps; ++i) s = fma(Z[(int64_t)i * total + e], y[c * m + i], s);
        X[r * ldx + c] += s;
    }
}

// The cycle's own skip flag starts as the sweep's (stop || not in the Krylov phase); givens_kernel raises it
// once the cycle has converged.
__global__ void cycle_begin_kernel(const int* skip, int* ctl) {
    ctl[0] = (skip != nullptr && *(volatile const int*)skip != 0) ? 1 : 0;
    ctl[1] = 0;
}

unsigned grid_for(int64_t work) {
    int64_t g = (work + 255) / 256;
    if (g > 152 * 8) g = 152 * 8;
    return (unsigned)(g < 1 ? 1 : g);
}

}  // namespace

size_t gmres_bytes(int64_t n, int64_t k, int m) {
    const size_t vec = (size_t)n * (size_t)k * sizeof(double);
    const size_t small = (size_t)k * (size_t)((m + 1) * m + 3 * m + 3 * (m + 1) + 1) * sizeof(double);
    return (size_t)(2 * m + 2) * vec + small + 256;
}

rmge_status gmres_cycle(int64_t n, int64_t k, int m, const double* A, int64_t lda, bool trans_a, const double* R,
                        double* X, int64_t ldx, double* buf, const GmresPrecond& P, int epoch0, const int* skip,
                        cudaStream_t s) {
    const int64_t vec = n * k;
    double* V = buf;                          // (m + 1) vectors
    double* Z = V + (int64_t)(m + 1) * vec;   // m vectors
    double* W = Z + (int64_t)m * vec;         // 1 vector
    double* H = W + vec;                      // k (m + 1) m
    double* hc = H + k * (m + 1) * m;         // k (m + 1)
    double* cs = hc + k * (m + 1);            // k m
    double* sn = cs + k * m;                  // k m
    double* g = sn + k * m;                   // k (m + 1)
    double* y = g + k * (m + 1);              // k m
    double* beta = y + k * m;                 // k
    int* ctl = reinterpret_cast<int*>(beta + k);  // the cycle's skip flag, steps taken

    cycle_begin_kernel<<<1, 1, 0, s>>>(skip, ctl);
    RMGE_LAUNCH_CHECK();
    norm_scale_kernel<<<(unsigned)k, RT, 0, s>>>(n, k, m, R, V, true, 0, H, g, beta, ctl);
    RMGE_LAUNCH_CHECK();
    for (int j = 0; j < m; ++j) {
        double* vj = V + (int64_t)j * vec;
        double* zj = Z + (int64_t)j * vec;
        // z_j = P v_j in the factor precision, widened to FP64
        RMGE_TRY(P.apply(P.ctx, vj, zj, epoch0 + 2 * j, ctl, s));
        // w = op(A) z_j in FP64
        RMGE_TRY(gemm<double>(trans_a, n, k, n, 1.0, A, lda, zj, k, 0.0, W, k, ctl, s));
        // classical Gram-Schmidt, twice
        for (int pass = 0; pass < 2; ++pass) {
            dots_kernel<<<dim3((unsigned)(j + 1), (unsigned)k), RT, 0, s>>>(n, k, m, j, V, W, hc, H, pass == 1,
                                                                           ctl);
            RMGE_LAUNCH_CHECK();
            axpy_kernel<<<grid_for(vec), 256, 0, s>>>(n, k, m, j, V, hc, W, ctl);
            RMGE_LAUNCH_CHECK();
        }
        norm_scale_kernel<<<(unsigned)k, RT, 0, s>>>(n, k, m, W, V + (int64_t)(j + 1) * vec, false, j, H, g, beta,
                                                     ctl);
        RMGE_LAUNCH_CHECK();
        givens_kernel<<<1, 128, 0, s>>>(k, m, j, H, cs, sn, g, beta, ctl);
        RMGE_LAUNCH_CHECK();
    }
    backsolve_kernel<<<(unsigned)((k + 127) / 128), 128, 0, s>>>(k, m, H, g, y, ctl, skip);
    RMGE_LAUNCH_CHECK();
    update_kernel<<<grid_for(vec), 256, 0, s>>>(n, k, m, Z, y, X, ldx, ctl, skip);
    RMGE_LAUNCH_CHECK();
    return RMGE_OK;
}

}  // namespace rmge
