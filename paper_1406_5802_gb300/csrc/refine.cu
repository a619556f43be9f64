// refine.cu -- residual-correction support kernels (Sec. 1.2, Sec. 7.1) and small utilities:
// control-block initialisation, ||A||_inf, column maxima and the normwise backward error with
// the stopping test, the FP64 update X += D, and dA = -dB X^T for the adjoint.
#include <climits>

#include "kernels.cuh"

namespace rmge {
namespace {

__global__ void state_init_kernel(DevState* st, int* flags, int64_t nflags, double* colred, int ncolred,
                                  double* berr_out, int nberr, long long spin_limit, Zb zb) {
    st = zws(st, zb.ws);
    flags = zws(flags, zb.ws);
    colred = zws(colred, zb.ws);
    berr_out = zmat(berr_out, zb.m0);
    const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    if (tid == 0) {
        st->info = INT_MAX;
        st->halt = 0;
        st->stop = 0;
        st->sweeps = 0;
        st->error = 0;
        st->maxabs_m = 0;
        st->maxabs_u = 0;
        st->norm_a = 0.0;
        st->berr_prev = __longlong_as_double(0x7ff0000000000000LL);
        st->berr_last = __longlong_as_double(0x7ff0000000000000LL);
        st->krylov = 0;
        st->krylov_start = 0;
        st->skip_cls = 0;
        st->skip_kry = 1;
        st->nonfinite = 0;
        st->status = 0;
        st->spin_limit = spin_limit;
    }
    if (tid == 0) {
        st->ticket = 0u;
        st->done = 0u;
    }
    for (int64_t i = tid; i < nflags; i += stride) flags[i] = 0;
    for (int64_t i = tid; i < ncolred; i += stride) colred[i] = 0.0;
    for (int64_t i = tid; i < nberr; i += stride) berr_out[i] = -1.0;
}

// count consecutive control blocks reset as state_init resets one (no solve flags or berr), and nzero
// 64-bit words of scratch cleared.
__global__ void states_init_kernel(DevState* st, int count, unsigned long long* zero, int64_t nzero,
                                   long long spin_limit) {
    const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t z = tid; z < count; z += stride) {
        DevState* d = st + z;
        d->info = INT_MAX;
        d->halt = 0;
        d->stop = 0;
        d->sweeps = 0;
        d->error = 0;
        d->maxabs_m = 0;
        d->maxabs_u = 0;
        d->norm_a = 0.0;
        d->berr_prev = __longlong_as_double(0x7ff0000000000000LL);
        d->berr_last = __longlong_as_double(0x7ff0000000000000LL);
        d->ticket = 0u;
        d->done = 0u;
        d->spin_limit = spin_limit;
        d->krylov = 0;
        d->krylov_start = 0;
        d->skip_cls = 0;
        d->skip_kry = 1;
        d->nonfinite = 0;
        d->status = 0;
    }
    for (int64_t i = tid; i < nzero; i += stride) zero[i] = 0ull;
}

// One warp per row: ||A||_inf = max_i sum_j |a_ij|.
__global__ void row_abs_sums_kernel(int64_t n, const double* __restrict__ A, int64_t lda, DevState* st, Zb zb) {
    A = zmat(A, zb.m0);
    st = zws(st, zb.ws);
    const int lane = threadIdx.x & 31;
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    unsigned long long best = 0;
    for (int64_t i = warp; i < n; i += nwarps) {
        double s = 0.0;
        for (int64_t j = lane; j < n; j += 32) s += fabs(A[i * lda + j]);
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        const unsigned long long b = abs_bits(s);
        best = b > best ? b : best;
    }
    if (lane == 0 && best != 0) atomicMax(reinterpret_cast<unsigned long long*>(&st->norm_a), best);
}

template <typename Tin, typename Tout>
__global__ void copy_kernel(int64_t rows, int64_t cols, const Tin* __restrict__ src, int64_t lds, Tout* __restrict__ dst,
                            int64_t ldd, const int* skip, Zb zb) {
    skip = zws(skip, zb.ws);
    if (skip != nullptr && *(volatile const int*)skip != 0) return;
    src = zmat(src, zb.m0);
    dst = zmat(dst, zb.m1);
    const int64_t total = rows * cols;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = e / cols, j = e % cols;
        dst[i * ldd + j] = (Tout)src[i * lds + j];
    }
}

template <typename T>
__global__ void add_kernel(int64_t rows, int64_t cols, const T* __restrict__ D, int64_t ldd, double* __restrict__ X,
                           int64_t ldx, const int* skip, Zb zb) {
    skip = zws(skip, zb.ws);
    if (skip != nullptr && *(volatile const int*)skip != 0) return;
    D = zmat(D, zb.m0);
    X = zmat(X, zb.m1);
    const int64_t total = rows * cols;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = e / cols, j = e % cols;
        X[i * ldx + j] += (double)D[i * ldd + j];
    }
}

// colred layout (as ull bits of non-negative doubles): [0,k) max|r|, [k,2k) max|x|, [2k,3k) max|b|.
__global__ void colmax_kernel(int64_t n, int64_t k, const double* __restrict__ R, int64_t ldr,
                              const double* __restrict__ X, int64_t ldx, const double* __restrict__ B, int64_t ldb,
                              const DevState* st, unsigned long long* colred, Zb zb) {
    st = zws(st, zb.ws);
    if (*(volatile const int*)&st->stop != 0) return;
    colred = zws(colred, zb.ws);
    R = zmat(R, zb.m0);
    X = zmat(X, zb.m1);
    B = zmat(B, zb.m2);
    const int64_t total = n * k;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = e / k, j = e % k;
        const unsigned long long r = abs_bits(R[i * ldr + j]);
        const unsigned long long x = abs_bits(X[i * ldx + j]);
        const unsigned long long b = abs_bits(B[i * ldb + j]);
        // NaN bit patterns exceed +Inf's, so a NaN anywhere surfaces in the maxima
        if (r) atomicMax(colred + j, r);
        if (x) atomicMax(colred + k + j, x);
        if (b) atomicMax(colred + 2 * k + j, b);
    }
}

// eta = max_c max|r_c| / (||A||_inf max|x_c| + max|b_c|); stopping test; clears colred.
// hybrid (reduced-precision factors): the sweeps are classical corrections while each at least halves
// eta, then FGMRES cycles, which stop once a cycle fails to halve eta against two sweeps back; without
// hybrid that last test applies from the start.
__global__ void decide_kernel(int64_t k, DevState* st, unsigned long long* colred, int sweep, double tol,
                              int max_iters, double* berr_out, bool hybrid, Zb zb) {
    st = zws(st, zb.ws);
    if (st->stop != 0) return;
    colred = zws(colred, zb.ws);
    berr_out = zmat(berr_out, zb.m3);
    double eta = 0.0;
    bool bad = false;
    for (int64_t j = 0; j < k; ++j) {
        const double rn = __longlong_as_double((long long)colred[j]);
        const double xn = __longlong_as_double((long long)colred[k + j]);
        const double bn = __longlong_as_double((long long)colred[2 * k + j]);
        colred[j] = colred[k + j] = colred[2 * k + j] = 0ull;
        if (!isfinite(rn) || !isfinite(xn)) { bad = true; continue; }
        const double den = st->norm_a * xn + bn;
        const double e = den > 0.0 ? rn / den : (rn > 0.0 ? __longlong_as_double(0x7ff0000000000000LL) : 0.0);
        eta = e > eta ? e : eta;
    }
    if (bad || !isfinite(st->norm_a)) eta = __longlong_as_double(0x7ff0000000000000LL);
    if (berr_out) berr_out[sweep] = eta;
    st->sweeps = sweep;
    bool stagnated;
    if (!hybrid) {
        stagnated = sweep >= 2 && !(eta <= 0.5 * st->berr_prev);
    } else if (st->krylov == 0) {
        stagnated = false;
        if (sweep >= 1 && !(eta <= 0.5 * st->berr_last)) {
            st->krylov = 1;
            st->krylov_start = sweep;
        }
    } else {
        stagnated = sweep - st->krylov_start >= 2 && !(eta <= 0.5 * st->berr_prev);
    }
    if (eta <= tol || sweep >= max_iters || stagnated || !isfinite(eta)) st->stop = 1;
    st->skip_cls = (st->stop != 0 || st->krylov != 0) ? 1 : 0;
    st->skip_kry = (st->stop != 0 || st->krylov == 0) ? 1 : 0;
    st->berr_prev = st->berr_last;
    st->berr_last = eta;
}

__global__ void refine_finish_kernel(const DevState* st, int32_t* iters, Zb zb) {
    st = zws(st, zb.ws);
    iters = zmat(iters, zb.m0);
    if (iters) *iters = st->sweeps;
}

// Flags an Inf or NaN anywhere in P (rows x cols).
template <typename T>
__global__ void nonfinite_scan_kernel(int64_t rows, int64_t cols, const T* __restrict__ P, int64_t ldp, DevState* st) {
    bool bad = false;
    const int64_t total = rows * cols;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x)
        if (!isfinite(P[(e / cols) * ldp + e % cols])) bad = true;
    if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicExch(&st->nonfinite, 1);
}

// The call's outcome (rmge_options.status): a bounded wait that gave up first, then a breakdown, then a
// non-finite result, then growth above growth_tol (factorizations) or a backward error above be_tol
// (refinement).
__global__ void status_kernel(DevState* st, int what, double growth_tol, double be_tol, int32_t* out) {
    int s = RMGE_OK;
    if (st->error != 0) {
        s = st->error;
    } else if (what == kStatusFactor) {
        const double mu = __longlong_as_double((long long)st->maxabs_u);
        const double mm = __longlong_as_double((long long)st->maxabs_m);
        const double growth = mu / mm;
        if (st->info != INT_MAX) s = RMGE_ERR_BREAKDOWN;
        else if (!isfinite(mu) || !isfinite(mm)) s = RMGE_ERR_NONFINITE;
        else if (growth_tol > 0.0 && !(growth <= growth_tol)) s = RMGE_ERR_GROWTH;
    } else if (what == kStatusSolve) {
        if (st->nonfinite != 0) s = RMGE_ERR_NONFINITE;
    } else {
        if (!isfinite(st->berr_last)) s = RMGE_ERR_NONFINITE;
        else if (!(st->berr_last <= be_tol)) s = RMGE_ERR_NOT_CONVERGED;
    }
    st->status = s;
    if (out != nullptr) *out = s;
}

__global__ void outer_neg_kernel(int64_t n, int64_t k, const double* __restrict__ dB, int64_t lddb,
                                 const double* __restrict__ X, int64_t ldx, double* __restrict__ dA, int64_t ldda,
                                 Zb zb) {
    dB = zmat(dB, zb.m0);
    X = zmat(X, zb.m1);
    dA = zmat(dA, zb.m2);
    // one CTA per row of dA; the row's dB entries are broadcast from registers
    const int64_t i = blockIdx.x;
    double b[16];
    const int kk = (int)(k < 16 ? k : 16);
    for (int c = 0; c < kk; ++c) b[c] = dB[i * lddb + c];
    for (int64_t j = threadIdx.x; j < n; j += blockDim.x) {
        double s = 0.0;
        for (int c = 0; c < kk; ++c) s = fma(b[c], X[j * ldx + c], s);
        for (int64_t c = 16; c < k; ++c) s = fma(dB[i * lddb + c], X[j * ldx + c], s);
        dA[i * ldda + j] = -s;
    }
}

// ||A^T||_inf = max_j sum_i |a_ij|: one thread per column (consecutive threads, consecutive columns).
__global__ void col_abs_sums_kernel(int64_t n, const double* __restrict__ A, int64_t lda, DevState* st, Zb zb) {
    A = zmat(A, zb.m0);
    st = zws(st, zb.ws);
    unsigned long long best = 0;
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x) {
        double s = 0.0;
        for (int64_t i = 0; i < n; ++i) s += fabs(A[i * lda + j]);
        const unsigned long long b = abs_bits(s);
        best = b > best ? b : best;
    }
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long other = __shfl_xor_sync(0xffffffffu, best, o);
        best = other > best ? other : best;
    }
    if ((threadIdx.x & 31) == 0 && best != 0) atomicMax(reinterpret_cast<unsigned long long*>(&st->norm_a), best);
}

unsigned grid_for(int64_t work, int threads) {
    int64_t g = (work + threads - 1) / threads;
    if (g > 152 * 8) g = 152 * 8;
    return (unsigned)(g < 1 ? 1 : g);
}

}  // namespace

rmge_status state_init(DevState* st, int* flags, int64_t nflags, double* colred, int ncolred, double* berr_out,
                       int nberr, cudaStream_t s, long long spin_limit, const Zb& zb) {
    int64_t work = nflags > ncolred ? nflags : ncolred;
    if (work < 64) work = 64;
    state_init_kernel<<<dim3(grid_for(work, 256), 1, zb.count), 256, 0, s>>>(st, flags, nflags, colred, ncolred,
                                                                           berr_out, berr_out ? nberr : 0,
                                                                           spin_limit, zb);
    RMGE_LAUNCH_CHECK();
    return RMGE_OK;
}

rmge_status states_init(DevState* st, int count, unsigned long long* zero, int64_t nzero, cudaStream_t s,
                        long long spin_limit) {
    const int64_t work = nzero > count ? nzero : count;
    states_init_kernel<<<grid_for(work < 64 ? 64 : work, 256), 256, 0, s>>>(st, count, zero, nzero, spin_limit);
    RMGE_LAUNCH_CHECK();
    return RMGE_OK;
}

rmge_status abs_sums_max(int64_t n, const double* A, int64_t lda, bool transposed, DevState* st, cudaStream_t s,
                         const Zb& zb) {
    if (transposed)
        col_abs_sums_kernel<<<dim3((unsigned)((n + 127) / 128), 1, zb.count), 128, 0, s>>>(n, A, lda, st, zb);
    else
        row_abs_sums_kernel<<<dim3(grid_for(n * 32, 256), 1, zb.count), 256, 0, s>>>(n, A, lda, st, zb);
    RMGE_LAUNCH_CHECK();
    return RMGE_OK;
}

template <typename Tin, typename Tout>
rmge_status copy_matrix(int64_t rows, int64_t cols, const Tin* src, int64_t lds, Tout* dst, int64_t ldd,
                        const int* skip, cudaStream_t s, const Zb& zb) {
    copy_kernel<Tin, Tout><<<dim3(grid_for(rows * cols, 256), 1, zb.count), 256, 0, s>>>(rows, cols, src, lds, dst,
                                                                                        ldd, skip, zb);
    RMGE_LAUNCH_CHECK();
    return RMGE_OK;
}

template <typename T>
rmge_status add_update(int64_t rows, int64_t cols, const T* D, int64_t ldd, double* X, int64_t ldx, const int* skip,
                       cudaStream_t s, const Zb& zb) {
    add_kernel<T><<<dim3(grid_for(rows * cols, 256), 1, zb.count), 256, 0, s>>>(rows, cols, D, ldd, X, ldx, skip,
                                                                                zb);
    RMGE_LAUNCH_CHECK();
    return RMGE_OK;
}

// Batched: R, X, B are the launcher's arrays 0-2 and berr_out its array 3.
rmge_status backward_error(int64_t n, int64_t k, const double* R, int64_t ldr, const double* X, int64_t ldx,
                           const double* B, int64_t ldb, DevState* st, double* colred, int sweep, double be_tol,
                           int max_iters, double* berr_out, cudaStream_t s, bool hybrid, const Zb& zb) {
    unsigned long long* cr = reinterpret_cast<unsigned long long*>(colred);
    colmax_kernel<<<dim3(grid_for(n * k, 256), 1, zb.count), 256, 0, s>>>(n, k, R, ldr, X, ldx, B, ldb, st, cr, zb);
    RMGE_LAUNCH_CHECK();
    decide_kernel<<<dim3(1, 1, zb.count), 1, 0, s>>>(k, st, cr, sweep, be_tol, max_iters, berr_out, hybrid, zb);
    RMGE_LAUNCH_CHECK();
    return RMGE_OK;
}

rmge_status refine_finish(DevState* st, int max_iters, double* berr_out, int32_t* iters, cudaStream_t s,
                          const Zb& zb) {
    (void)max_iters;
    (void)berr_out;
    refine_finish_kernel<<<dim3(1, 1, zb.count), 1, 0, s>>>(st, iters, zb);
    RMGE_LAUNCH_CHECK();
    return RMGE_OK;
}

template <typename T>
rmge_status nonfinite_scan(int64_t rows, int64_t cols, const T* P, int64_t ldp, DevState* st, cudaStream_t s) {
    nonfinite_scan_kernel<T><<<grid_for(rows * cols, 256), 256, 0, s>>>(rows, cols, P, ldp, st);
    RMGE_LAUNCH_CHECK();
    return RMGE_OK;
}

rmge_status write_status(DevState* st, int what, double growth_tol, double be_tol, int32_t* out, cudaStream_t s) {
    status_kernel<<<1, 1, 0, s>>>(st, what, growth_tol, be_tol, out);
    RMGE_LAUNCH_CHECK();
    return RMGE_OK;
}

rmge_status outer_neg(int64_t n, int64_t k, const double* dB, int64_t lddb, const double* X, int64_t ldx, double* dA,
                      int64_t ldda, cudaStream_t s, const Zb& zb) {
    outer_neg_kernel<<<dim3((unsigned)n, 1, zb.count), 256, 0, s>>>(n, k, dB, lddb, X, ldx, dA, ldda, zb);
    RMGE_LAUNCH_CHECK();
    return RMGE_OK;
}

template rmge_status copy_matrix<double, double>(int64_t, int64_t, const double*, int64_t, double*, int64_t,
                                                 const int*, cudaStream_t, const Zb&);
template rmge_status copy_matrix<double, float>(int64_t, int64_t, const double*, int64_t, float*, int64_t, const int*,
                                                cudaStream_t, const Zb&);
template rmge_status copy_matrix<float, double>(int64_t, int64_t, const float*, int64_t, double*, int64_t, const int*,
                                                cudaStream_t, const Zb&);
template rmge_status add_update<double>(int64_t, int64_t, const double*, int64_t, double*, int64_t, const int*,
                                        cudaStream_t, const Zb&);
template rmge_status nonfinite_scan<double>(int64_t, int64_t, const double*, int64_t, DevState*, cudaStream_t);
template rmge_status nonfinite_scan<float>(int64_t, int64_t, const float*, int64_t, DevState*, cudaStream_t);
template rmge_status add_update<float>(int64_t, int64_t, const float*, int64_t, double*, int64_t, const int*,
                                       cudaStream_t, const Zb&);

}  // namespace rmge
