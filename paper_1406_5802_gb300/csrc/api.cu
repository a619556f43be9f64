// api.cu -- the extern "C" entry points of librmge (declared and documented in include/rmge.h).
//
// Each entry point validates its arguments, carves its scratch out of the caller's workspace,
// and enqueues the kernels of one step of the method on the caller's stream.
#include <climits>
#include <cstring>

#include "kernels.cuh"

namespace rmge {

std::atomic<unsigned long long> g_launches{0};

namespace {

bool valid_kind(rmge_mult_kind k) { return (int)k >= (int)RMGE_GAUSSIAN && (int)k <= (int)RMGE_TOEPLITZ_UNIFORM; }
bool valid_prec(rmge_prec p) { return (int)p >= (int)RMGE_F64 && (int)p <= (int)RMGE_F64X_TC; }
bool is_tc(rmge_prec p) { return (int)p >= (int)RMGE_BF16_TC && (int)p <= (int)RMGE_F16X3_TC; }
// RMGE_F64X_TC keeps FP64 data everywhere; only the engine of A G and of the Schur updates differs.
rmge_prec data_prec(rmge_prec p) { return p == RMGE_F64X_TC ? RMGE_F64 : p; }
bool tc_bf16(rmge_prec p) { return p == RMGE_BF16_TC || p == RMGE_BF16X3_TC; }
int tc_terms(rmge_prec p) { return (p == RMGE_BF16X3_TC || p == RMGE_F16X3_TC) ? 3 : 1; }
int64_t tc_ldk(int64_t n) { return (n + 63) / 64 * 64; }
// the FFT kinds: circulants (transform length n) and Toeplitz multipliers (the leading n x n block of a
// 2n x 2n circulant, transform length 2n)
bool is_circ(rmge_mult_kind k) { return k != RMGE_GAUSSIAN; }
bool is_toeplitz(rmge_mult_kind k) { return k == RMGE_TOEPLITZ_GAUSSIAN || k == RMGE_TOEPLITZ_UNIFORM; }
int64_t fft_len(rmge_mult_kind k, int64_t n) { return is_toeplitz(k) ? 2 * n : n; }
bool pow2(int64_t n) { return n > 0 && (n & (n - 1)) == 0; }
// one real transform of length N = 2^p, 4 <= N <= 16384, per CTA (fft.cu)
bool circ_ok(rmge_mult_kind k, int64_t n) { return pow2(n) && fft_len(k, n) >= 4 && fft_len(k, n) <= 16384; }
size_t elem(rmge_prec p) { return data_prec(p) == RMGE_F64 ? 8 : 4; }

int64_t nflags_for(int64_t n, int64_t nrhs) {
    return ((n + kTrsvRows - 1) / kTrsvRows) * ((nrhs + kTrsvCols - 1) / kTrsvCols);
}

struct Ws {
    DevState* st;
    int* flags;
    double* colred;
    double* R;
    double* Y;
    double* D;
    double2* tw;
    void* tc;                  // 16-bit operand buffers: A hi, A lo, B hi, B lo, each n x tc_ldk(n)
    double* gm;                // FGMRES work
    unsigned long long* tcmx;  // FP16 scaling slots
    char* oz;                  // digit planes and exponents of the emulated FP64 products
    long long spin;            // spin limit of the bounded waits (rmge_options.spin_limit)
    int gm_m;                  // FGMRES restart length (rmge_options.gmres_m)
};

// rmge_options with the defaults filled in (the calls without _ex use these).
struct Opts {
    double growth_tol = 0.0;
    long long spin = kSpinLimit;
    int gm_m = kGmresM;
    bool sync = false;
    int32_t* status = nullptr;
    int digits = kOzSlices;   // balanced base-256 digits of the emulated A G
    int fdigits = kOzSlices;  // ... of the emulated Schur updates
    bool report() const { return sync || status != nullptr; }
};

bool opts_of(const rmge_options* o, Opts* out) {
    *out = Opts{};
    if (o == nullptr) return true;
    if (!(o->growth_tol >= 0.0) || o->spin_limit < 0 || o->gmres_m < 1 || o->gmres_m > kMaxGmresM ||
        o->apply_digits < 1 || o->apply_digits > kOzSlices || o->factor_digits < 4 || o->factor_digits > kOzSlices)
        return false;
    out->digits = o->apply_digits;
    out->fdigits = o->factor_digits;
    out->growth_tol = o->growth_tol;
    out->spin = o->spin_limit;
    out->gm_m = o->gmres_m;
    out->sync = o->sync != 0;
    out->status = o->status;
    return true;
}

// full = false: the call needs no tensor-core operand buffers and no FGMRES work (solves, adjoint),
// which sit at the end of the layout.
rmge_status carve(void* ws, size_t ws_bytes, int64_t n, int64_t nrhs, rmge_mult_kind kind, rmge_prec prec, Ws* out,
                  bool full = true, const Opts& o = Opts{}) {
    if (ws == nullptr || ((uintptr_t)ws & 255) != 0) return RMGE_ERR_WORKSPACE;
    const WsLayout L = ws_layout(n, nrhs, kind, prec, o.gm_m);
    out->spin = o.spin;
    out->gm_m = o.gm_m;
    if (ws_bytes < (full ? L.total : L.tcmx)) return RMGE_ERR_WORKSPACE;
    char* b = static_cast<char*>(ws);
    out->st = reinterpret_cast<DevState*>(b + L.state);
    out->flags = reinterpret_cast<int*>(b + L.flags);
    out->colred = reinterpret_cast<double*>(b + L.colred);
    out->R = reinterpret_cast<double*>(b + L.R);
    out->Y = reinterpret_cast<double*>(b + L.Y);
    out->D = reinterpret_cast<double*>(b + L.D);
    out->tw = reinterpret_cast<double2*>(b + L.fft);
    out->tc = is_tc(prec) ? b + L.tc : nullptr;
    out->tcmx = (full && is_tc(prec)) ? reinterpret_cast<unsigned long long*>(b + L.tcmx) : nullptr;
    out->gm = (full && data_prec(prec) != RMGE_F64) ? reinterpret_cast<double*>(b + L.gm) : nullptr;
    out->oz = (full && prec == RMGE_F64X_TC) ? b + L.oz : nullptr;
    if (!full) out->tc = nullptr;
    return RMGE_OK;
}

// The call's outcome into o.status and, with o.sync, synchronise and return it (rmge_options).
rmge_status finish_call(const Ws& w, int what, const Opts& o, double be_tol, cudaStream_t s) {
    if (!o.report()) return RMGE_OK;
    RMGE_TRY(write_status(w.st, what, o.growth_tol, be_tol, o.status, s));
    if (!o.sync) return RMGE_OK;
    int h = RMGE_OK;
    if (cudaMemcpyAsync(&h, &w.st->status, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) {
        (void)cudaGetLastError();
        return RMGE_ERR_CUDA;
    }
    return (rmge_status)h;
}

// Digit planes (A side, B side) and line exponents of the emulated FP64 products, in w.oz.
OzUpdate oz_buffers(const Ws& w, int64_t n) {
    const size_t pb = oz_plane_bytes(n, n, kOzSlices);
    OzUpdate o{};
    o.planesA = w.oz;
    o.planesB = w.oz + pb;
    o.ea = reinterpret_cast<int*>(w.oz + 2 * pb);
    o.eb = o.ea + n + 128;
    o.kmax = reinterpret_cast<unsigned long long*>(w.oz + 2 * pb + 2 * sizeof(int) * (size_t)(n + 128));
    return o;
}

// 128 per-k maxima slots per 64-wide pivot-block step of the emulated-update GENP.
size_t oz_kmax_slots(int64_t n) { return (size_t)oz_kmax_per_system(n); }

bool check_dims(int64_t n, int64_t nrhs) { return n >= 1 && n <= RMGE_MAX_N && nrhs >= 1 && nrhs <= RMGE_MAX_N; }

// d = op(G) y for the multiplier of `kind`; y, d are n x k (FP64, or FP32 for reduced precisions
// with a dense G).  accumulate: d += op(G) y.
rmge_status apply_g_cols(rmge_mult_kind kind, rmge_prec prec, int64_t n, int64_t k, const void* G, bool transpose,
                         const void* y, int64_t ldy, void* d, int64_t ldd, bool accumulate, const int* skip,
                         const Ws& w, cudaStream_t s) {
    if (is_circ(kind))
        return circulant_apply_cols(n, fft_len(kind, n), k, static_cast<const double*>(G), w.tw, transpose,
                                    static_cast<const double*>(y), ldy, static_cast<double*>(d), ldd, accumulate, skip,
                                    s);
    if (prec == RMGE_F64)
        return gemm<double>(transpose, n, k, n, 1.0, static_cast<const double*>(G), n, static_cast<const double*>(y),
                            ldy, accumulate ? 1.0 : 0.0, static_cast<double*>(d), ldd, skip, s);
    return gemm<float>(transpose, n, k, n, 1.0f, static_cast<const float*>(G), n, static_cast<const float*>(y), ldy,
                       accumulate ? 1.0f : 0.0f, static_cast<float*>(d), ldd, skip, s);
}

// In-place y <- U^{-1} L^{-1} y (transposed: L^{-T} U^{-T} y) with the factor type of prec.
rmge_status lu_solve(rmge_prec prec, bool transposed, int64_t n, int64_t k, const void* LU, int64_t ldlu, void* y,
                     int64_t ldy, const Ws& w, int epoch, const int* skip, cudaStream_t s) {
    const int k1 = transposed ? 2 : 0, k2 = transposed ? 3 : 1;
    if (prec == RMGE_F64) {
        RMGE_TRY(trsv<double>(k1, n, k, static_cast<const double*>(LU), ldlu, static_cast<double*>(y), ldy, w.st,
                              w.flags, epoch, skip, s));
        return trsv<double>(k2, n, k, static_cast<const double*>(LU), ldlu, static_cast<double*>(y), ldy, w.st,
                            w.flags, epoch + 1, skip, s);
    }
    RMGE_TRY(trsv<float>(k1, n, k, static_cast<const float*>(LU), ldlu, static_cast<float*>(y), ldy, w.st, w.flags,
                         epoch, skip, s));
    return trsv<float>(k2, n, k, static_cast<const float*>(LU), ldlu, static_cast<float*>(y), ldy, w.st, w.flags,
                       epoch + 1, skip, s);
}

// X (+)= G U^{-1} L^{-1} V for FP64 V (n x k, ldv), using w.Y (and w.D) as scratch; with trans,
// X (+)= L^{-T} U^{-T} G^T V (the same approximate inverse for the transposed system).
rmge_status correction(rmge_mult_kind kind, rmge_prec prec, int64_t n, int64_t k, const void* LU, int64_t ldlu,
                       const void* G, const double* V, int64_t ldv, double* X, int64_t ldx, bool accumulate,
                       const Ws& w, int epoch, const int* skip, cudaStream_t s, bool trans = false) {
    const bool low = prec != RMGE_F64;
    if (trans) {
        // z = G^T v first (FP64 for FP64 factors or a circulant G, else FP32), then U^T, L^T solves
        if (!low) {
            RMGE_TRY(apply_g_cols(kind, prec, n, k, G, true, V, ldv, w.Y, k, false, skip, w, s));
            RMGE_TRY(lu_solve(prec, true, n, k, LU, ldlu, w.Y, k, w, epoch, skip, s));
            if (accumulate) return add_update<double>(n, k, w.Y, k, X, ldx, skip, s);
            return copy_matrix<double, double>(n, k, w.Y, k, X, ldx, skip, s);
        }
        float* zf = reinterpret_cast<float*>(w.Y);
        if (is_circ(kind)) {
            RMGE_TRY(apply_g_cols(kind, RMGE_F64, n, k, G, true, V, ldv, w.D, k, false, skip, w, s));
            RMGE_TRY(copy_matrix<double, float>(n, k, w.D, k, zf, k, skip, s));
        } else {
            float* vf = reinterpret_cast<float*>(w.D);
            RMGE_TRY(copy_matrix<double, float>(n, k, V, ldv, vf, k, skip, s));
            RMGE_TRY(apply_g_cols(kind, prec, n, k, G, true, vf, k, zf, k, false, skip, w, s));
        }
        RMGE_TRY(lu_solve(prec, true, n, k, LU, ldlu, zf, k, w, epoch, skip, s));
        if (accumulate) return add_update<float>(n, k, zf, k, X, ldx, skip, s);
        return copy_matrix<float, double>(n, k, zf, k, X, ldx, skip, s);
    }
    if (!low || is_circ(kind)) {
        if (!low) {
            RMGE_TRY(copy_matrix<double, double>(n, k, V, ldv, w.Y, k, skip, s));
            RMGE_TRY(lu_solve(prec, false, n, k, LU, ldlu, w.Y, k, w, epoch, skip, s));
            return apply_g_cols(kind, prec, n, k, G, false, w.Y, k, X, ldx, accumulate, skip, w, s);
        }
        // reduced-precision factors with a circulant G: solve in FP32, widen, apply C in FP64
        float* yf = reinterpret_cast<float*>(w.Y);
        RMGE_TRY(copy_matrix<double, float>(n, k, V, ldv, yf, k, skip, s));
        RMGE_TRY(lu_solve(prec, false, n, k, LU, ldlu, yf, k, w, epoch, skip, s));
        RMGE_TRY(copy_matrix<float, double>(n, k, yf, k, w.D, k, skip, s));
        return apply_g_cols(kind, RMGE_F64, n, k, G, false, w.D, k, X, ldx, accumulate, skip, w, s);
    }
    float* yf = reinterpret_cast<float*>(w.Y);
    float* df = reinterpret_cast<float*>(w.D);
    RMGE_TRY(copy_matrix<double, float>(n, k, V, ldv, yf, k, skip, s));
    RMGE_TRY(lu_solve(prec, false, n, k, LU, ldlu, yf, k, w, epoch, skip, s));
    RMGE_TRY(apply_g_cols(kind, prec, n, k, G, false, yf, k, df, k, false, skip, w, s));
    if (accumulate) return add_update<float>(n, k, df, k, X, ldx, skip, s);
    return copy_matrix<float, double>(n, k, df, k, X, ldx, skip, s);
}

struct PrecondCtx {
    rmge_mult_kind kind;
    rmge_prec prec;
    int64_t n, k;
    const void* LU;
    int64_t ldlu;
    const void* G;
    const Ws* w;
    bool trans;
};

// z = G U^{-1} L^{-1} v (the preconditioner of the FGMRES sweeps; transposed for A^T), factor
// precision inside.
rmge_status precond_apply(const void* ctx, const double* v, double* z, int epoch, const int* skip, cudaStream_t s) {
    const PrecondCtx* c = static_cast<const PrecondCtx*>(ctx);
    return correction(c->kind, c->prec, c->n, c->k, c->LU, c->ldlu, c->G, v, c->k, z, c->k, false, *c->w, epoch, skip,
                      s, c->trans);
}

// Refinement sweeps for A X = B (trans = false) or A^T X = B (trans = true); see rmge_refine.
rmge_status refine_loop(rmge_mult_kind kind, rmge_prec prec, bool trans, int64_t n, int64_t nrhs, const double* A,
                        int64_t lda, const void* LU, int64_t ldlu, const void* G, const double* B, int64_t ldb,
                        double* X, int64_t ldx, int32_t max_iters, double be_tol, double* berr, int32_t* iters,
                        const Ws& w, int epoch0, cudaStream_t s) {
    RMGE_TRY(state_init(w.st, w.flags, nflags_for(n, nrhs), w.colred, (int)(3 * nrhs), berr, max_iters + 1, s,
                        w.spin));
    RMGE_TRY(abs_sums_max(n, A, lda, trans, w.st, s));
    const int* stop = &w.st->stop;
    const PrecondCtx pctx{kind, prec, n, nrhs, LU, ldlu, G, &w, trans};
    const GmresPrecond pre{precond_apply, &pctx};
    for (int it = 0; it <= max_iters; ++it) {
        // R = B - op(A) X in FP64, then the backward error and the stopping test
        RMGE_TRY(copy_matrix<double, double>(n, nrhs, B, ldb, w.R, nrhs, stop, s));
        RMGE_TRY(gemm<double>(trans, n, nrhs, n, -1.0, A, lda, X, ldx, 1.0, w.R, nrhs, stop, s));
        const bool hybrid = prec != RMGE_F64;
        RMGE_TRY(backward_error(n, nrhs, w.R, nrhs, X, ldx, B, ldb, w.st, w.colred, it, be_tol, max_iters, berr, s,
                                hybrid));
        if (it == max_iters) break;
        const int epoch = epoch0 + 2 * w.gm_m * it;
        if (!hybrid) {
            // X <- X + G U^{-1} L^{-1} R  (transposed: L^{-T} U^{-T} G^T R)
            RMGE_TRY(correction(kind, prec, n, nrhs, LU, ldlu, G, w.R, nrhs, X, ldx, true, w, epoch, stop, s, trans));
        } else {
            // the same classical correction with the reduced-precision factors while it halves the backward
            // error; after that X <- X + d, op(A) d = R solved by one preconditioned FGMRES cycle in FP64.
            // decide_kernel sets the two skip flags, so exactly one of the two runs.
            RMGE_TRY(correction(kind, prec, n, nrhs, LU, ldlu, G, w.R, nrhs, X, ldx, true, w, epoch, &w.st->skip_cls,
                                s, trans));
            RMGE_TRY(gmres_cycle(n, nrhs, w.gm_m, A, lda, trans, w.R, X, ldx, w.gm, pre, epoch, &w.st->skip_kry,
                                 s));
        }
    }
    return refine_finish(w.st, max_iters, berr, iters, s);
}

// ---- uniform batches of the solve, the refinement and the adjoint (FP64 factors, dense Gaussian G) ---------
// Every system has its own workspace block (the single-system layout), ws bytes after the previous one, so
// each workspace array advances by ws / sizeof(element); user arrays advance by their own strides.

struct Bt {
    int count;
    int64_t ws;  // bytes between the systems' workspace blocks
    int64_t lu, g;
    int64_t wd() const { return ws / (int64_t)sizeof(double); }
};

Zb zb3(const Bt& bt, int64_t m0, int64_t m1, int64_t m2 = 0, int64_t m3 = 0) {
    Zb z;
    z.count = bt.count;
    z.m0 = m0;
    z.m1 = m1;
    z.m2 = m2;
    z.m3 = m3;
    z.ws = bt.ws;
    return z;
}

// X (+)= G U^{-1} L^{-1} V (trans: X (+)= L^{-T} U^{-T} G^T V) for every system; V and X advance by sV, sX.
rmge_status correction_z(const Bt& bt, int64_t n, int64_t k, const double* LU, int64_t ldlu, const double* G,
                         const double* V, int64_t ldv, int64_t sV, double* X, int64_t ldx, int64_t sX,
                         bool accumulate, const Ws& w, int epoch, const int* skip, cudaStream_t s, bool trans) {
    const int64_t wd = bt.wd();
    if (trans) {
        RMGE_TRY(gemm<double>(true, n, k, n, 1.0, G, n, V, ldv, 0.0, w.Y, k, skip, s, zb3(bt, bt.g, sV, wd)));
        RMGE_TRY(trsv<double>(2, n, k, LU, ldlu, w.Y, k, w.st, w.flags, epoch, skip, s, zb3(bt, bt.lu, wd)));
        RMGE_TRY(trsv<double>(3, n, k, LU, ldlu, w.Y, k, w.st, w.flags, epoch + 1, skip, s, zb3(bt, bt.lu, wd)));
        if (accumulate) return add_update<double>(n, k, w.Y, k, X, ldx, skip, s, zb3(bt, wd, sX));
        return copy_matrix<double, double>(n, k, w.Y, k, X, ldx, skip, s, zb3(bt, wd, sX));
    }
    RMGE_TRY(copy_matrix<double, double>(n, k, V, ldv, w.Y, k, skip, s, zb3(bt, sV, wd)));
    RMGE_TRY(trsv<double>(0, n, k, LU, ldlu, w.Y, k, w.st, w.flags, epoch, skip, s, zb3(bt, bt.lu, wd)));
    RMGE_TRY(trsv<double>(1, n, k, LU, ldlu, w.Y, k, w.st, w.flags, epoch + 1, skip, s, zb3(bt, bt.lu, wd)));
    return gemm<double>(false, n, k, n, 1.0, G, n, w.Y, k, accumulate ? 1.0 : 0.0, X, ldx, skip, s,
                        zb3(bt, bt.g, wd, sX));
}

// Classical FP64 refinement sweeps of every system (see rmge_refine); berr and iters advance by
// max_iters + 1 and 1 entries.
rmge_status refine_loop_z(const Bt& bt, bool trans, int64_t n, int64_t nrhs, const double* A, int64_t lda,
                          int64_t sA, const double* LU, int64_t ldlu, const double* G, const double* B, int64_t ldb,
                          int64_t sB, double* X, int64_t ldx, int64_t sX, int32_t max_iters, double be_tol,
                          double* berr, int32_t* iters, const Ws& w, int epoch0, cudaStream_t s) {
    const int64_t wd = bt.wd(), sb = max_iters + 1;
    RMGE_TRY(state_init(w.st, w.flags, nflags_for(n, nrhs), w.colred, (int)(3 * nrhs), berr, max_iters + 1, s,
                        w.spin, zb3(bt, sb, 0)));
    RMGE_TRY(abs_sums_max(n, A, lda, trans, w.st, s, zb3(bt, sA, 0)));
    const int* stop = &w.st->stop;
    for (int it = 0; it <= max_iters; ++it) {
        RMGE_TRY(copy_matrix<double, double>(n, nrhs, B, ldb, w.R, nrhs, stop, s, zb3(bt, sB, wd)));
        RMGE_TRY(gemm<double>(trans, n, nrhs, n, -1.0, A, lda, X, ldx, 1.0, w.R, nrhs, stop, s, zb3(bt, sA, sX, wd)));
        RMGE_TRY(backward_error(n, nrhs, w.R, nrhs, X, ldx, B, ldb, w.st, w.colred, it, be_tol, max_iters, berr, s,
                                false, zb3(bt, wd, sX, sB, sb)));
        if (it == max_iters) break;
        RMGE_TRY(correction_z(bt, n, nrhs, LU, ldlu, G, w.R, nrhs, wd, X, ldx, sX, true, w, epoch0 + 2 * it, stop, s,
                              trans));
    }
    return refine_finish(w.st, max_iters, berr, iters, s, zb3(bt, 1, 0));
}

// The common argument checks of the three uniform-batch calls; fills bt and carves system 0's workspace.
rmge_status uniform_setup(int64_t count, int64_t n, int64_t nrhs, rmge_prec prec, const void* LU, int64_t ldlu,
                          int64_t sLU, const void* G, int64_t sG, void* ws, size_t ws_bytes, Bt* bt, Ws* w) {
    if (count < 1 || count > 65535 || !check_dims(n, nrhs) || !valid_prec(prec) || LU == nullptr || G == nullptr ||
        ldlu < n || sLU < (n - 1) * ldlu + n || sG < n * n)
        return RMGE_ERR_INVALID_ARG;
    if (data_prec(prec) != RMGE_F64) return RMGE_ERR_UNSUPPORTED;
    const size_t per = ws_layout(n, nrhs, RMGE_GAUSSIAN, RMGE_F64).total;
    if (ws == nullptr || ((uintptr_t)ws & 255) != 0 || ws_bytes / (size_t)count < per) return RMGE_ERR_WORKSPACE;
    bt->count = (int)count;
    bt->ws = (int64_t)per;
    bt->lu = sLU;
    bt->g = sG;
    return carve(ws, per, n, nrhs, RMGE_GAUSSIAN, RMGE_F64, w);
}

bool mat_ok(const void* P, int64_t n, int64_t cols, int64_t ld, int64_t stride) {
    return P != nullptr && ld >= cols && stride >= (n - 1) * ld + cols;
}

// ---- two-sided forms (Fact 4.1: A^{-1} = H (F A H)^{-1} F), FP64 data ------------------------------------

// The layout kind whose workspace serves both multipliers: the longer FFT wins.
rmge_mult_kind layout_kind(const void* F, rmge_mult_kind kF, const void* H, rmge_mult_kind kH) {
    if ((F != nullptr && is_toeplitz(kF)) || (H != nullptr && is_toeplitz(kH))) return RMGE_TOEPLITZ_GAUSSIAN;
    if ((F != nullptr && is_circ(kF)) || (H != nullptr && is_circ(kH))) return RMGE_CIRCULANT_GAUSSIAN;
    return RMGE_GAUSSIAN;
}

// d (+)= P y for a multiplier P (FP64 or FFT kind), or d (+)= y when P is the identity (NULL); n x k.
rmge_status apply_side(rmge_mult_kind kind, const void* P, int64_t n, int64_t k, const double* y, int64_t ldy,
                       double* d, int64_t ldd, bool accumulate, const int* skip, const Ws& w, cudaStream_t s) {
    if (P == nullptr)
        return accumulate ? add_update<double>(n, k, y, ldy, d, ldd, skip, s)
                          : copy_matrix<double, double>(n, k, y, ldy, d, ldd, skip, s);
    return apply_g_cols(kind, RMGE_F64, n, k, P, false, y, ldy, d, ldd, accumulate, skip, w, s);
}

// X (+)= H U^{-1} L^{-1} F V with FP64 factors, w.Y as scratch.
rmge_status two_sided_correction(rmge_mult_kind kF, const void* F, rmge_mult_kind kH, const void* H, int64_t n,
                                 int64_t k, const void* LU, int64_t ldlu, const double* V, int64_t ldv, double* X,
                                 int64_t ldx, bool accumulate, const Ws& w, int epoch, const int* skip,
                                 cudaStream_t s) {
    RMGE_TRY(apply_side(kF, F, n, k, V, ldv, w.Y, k, false, skip, w, s));
    RMGE_TRY(lu_solve(RMGE_F64, false, n, k, LU, ldlu, w.Y, k, w, epoch, skip, s));
    return apply_side(kH, H, n, k, w.Y, k, X, ldx, accumulate, skip, w, s);
}

// M = A H (FP64 data; emulated on the tensor cores for RMGE_F64X_TC and a dense H).
rmge_status right_multiply(rmge_mult_kind kH, const void* H, rmge_prec prec, int64_t n, const double* A, int64_t lda,
                           double* M, int64_t ldm, const Ws& w, cudaStream_t s) {
    if (is_circ(kH))
        return circulant_apply_rows(n, fft_len(kH, n), A, lda, static_cast<const double*>(H), w.tw, M, ldm, false, s);
    if (prec == RMGE_F64X_TC) {
        const OzUpdate oz = oz_buffers(w, n);
        return oz_gemm(n, n, n, kOzSlices, 1.0, A, lda, static_cast<const double*>(H), n, 0.0, M, ldm, oz.planesA,
                       oz.planesB, oz.ea, oz.eb, nullptr, nullptr, &w.st->error, nullptr, s);
    }
    return gemm<double>(false, n, n, n, 1.0, A, lda, static_cast<const double*>(H), n, 0.0, M, ldm, nullptr, s);
}

// M = F A: the columns of A convolved with F's first column for the FFT kinds, else a product.
rmge_status left_multiply(rmge_mult_kind kF, const void* F, rmge_prec prec, int64_t n, const double* A, int64_t lda,
                          double* M, int64_t ldm, const Ws& w, cudaStream_t s) {
    if (is_circ(kF))
        return circulant_apply_cols(n, fft_len(kF, n), n, static_cast<const double*>(F), w.tw, false, A, lda, M, ldm,
                                    false, nullptr, s);
    if (prec == RMGE_F64X_TC) {
        const OzUpdate oz = oz_buffers(w, n);
        return oz_gemm(n, n, n, kOzSlices, 1.0, static_cast<const double*>(F), n, A, lda, 0.0, M, ldm, oz.planesA,
                       oz.planesB, oz.ea, oz.eb, nullptr, nullptr, &w.st->error, nullptr, s);
    }
    return gemm<double>(false, n, n, n, 1.0, static_cast<const double*>(F), n, A, lda, 0.0, M, ldm, nullptr, s);
}

bool two_sided_ok(rmge_mult_kind kF, const void* F, rmge_mult_kind kH, const void* H, int64_t n, rmge_prec prec,
                  rmge_status* why) {
    *why = RMGE_ERR_INVALID_ARG;
    if (!valid_kind(kF) || !valid_kind(kH) || !valid_prec(prec)) return false;
    *why = RMGE_ERR_UNSUPPORTED;
    if (data_prec(prec) != RMGE_F64) return false;
    if (F != nullptr && is_circ(kF) && !circ_ok(kF, n)) return false;
    if (H != nullptr && is_circ(kH) && !circ_ok(kH, n)) return false;
    return true;
}

}  // namespace

WsLayout ws_layout(int64_t n, int64_t nrhs, rmge_mult_kind kind, rmge_prec prec, int gmres_m) {
    WsLayout L{};
    size_t off = 0;
    L.state = off;
    off = align256(off + sizeof(DevState));
    L.flags = off;
    off = align256(off + sizeof(int) * (size_t)nflags_for(n, nrhs));
    L.rowsum = off;
    L.colred = off;
    off = align256(off + 3 * sizeof(double) * (size_t)nrhs);
    L.R = off;
    off = align256(off + sizeof(double) * (size_t)(n * nrhs));
    L.Y = off;
    off = align256(off + sizeof(double) * (size_t)(n * nrhs));
    L.D = off;
    off = align256(off + sizeof(double) * (size_t)(n * nrhs));
    L.fft = off;
    if (is_circ(kind)) off = align256(off + sizeof(double2) * (size_t)(fft_len(kind, n) / 2 + 1));
    L.tcmx = off;
    if (is_tc(prec)) off = align256(off + sizeof(unsigned long long) * (size_t)(2 * (n / kNb + 2)));
    L.tc = off;
    if (is_tc(prec)) off = align256(off + 4 * 2 * (size_t)n * (size_t)tc_ldk(n));
    L.gm = off;
    if (data_prec(prec) != RMGE_F64) off = align256(off + gmres_bytes(n, nrhs, gmres_m));
    L.oz = off;
    if (prec == RMGE_F64X_TC)
        off = align256(off + 2 * oz_plane_bytes(n, n, kOzSlices) + 2 * sizeof(int) * (size_t)(n + 128) +
                       oz_kmax_slots(n) * sizeof(unsigned long long));
    L.total = off;
    return L;
}

}  // namespace rmge

using namespace rmge;

extern "C" {

unsigned long long rmge_kernel_launches(void) { return g_launches.load(std::memory_order_relaxed); }

const char* rmge_status_string(rmge_status s) {
    switch (s) {
        case RMGE_OK: return "ok";
        case RMGE_ERR_INVALID_ARG: return "invalid argument";
        case RMGE_ERR_BREAKDOWN: return "GENP breakdown (zero or non-finite pivot)";
        case RMGE_ERR_GROWTH: return "growth above threshold";
        case RMGE_ERR_NOT_CONVERGED: return "refinement did not converge";
        case RMGE_ERR_CUDA: return "CUDA launch or copy failed";
        case RMGE_ERR_TIMEOUT: return "bounded device wait expired";
        case RMGE_ERR_WORKSPACE: return "workspace missing, too small or misaligned";
        case RMGE_ERR_UNSUPPORTED: return "unsupported request (e.g. a circulant n that is not a power of two)";
        case RMGE_ERR_NONFINITE: return "non-finite values in the result";
    }
    return "unknown status";
}

size_t rmge_multiplier_bytes(rmge_mult_kind kind, int64_t n, rmge_prec prec) {
    if (!valid_kind(kind) || !valid_prec(prec) || n < 1 || n > RMGE_MAX_N) return 0;
    if (is_circ(kind)) return circ_ok(kind, n) ? 3 * sizeof(double) * (size_t)fft_len(kind, n) : 0;
    return (size_t)n * (size_t)n * elem(prec);
}

size_t rmge_solve_workspace_size(int64_t n, int64_t nrhs, rmge_mult_kind kind, rmge_prec prec) {
    if (!valid_kind(kind) || !valid_prec(prec) || !check_dims(n, nrhs)) return 0;
    if (is_circ(kind) && !circ_ok(kind, n)) return 0;
    return ws_layout(n, nrhs, kind, prec).tcmx;
}

size_t rmge_workspace_size(int64_t n, int64_t nrhs, rmge_mult_kind kind, rmge_prec prec) {
    return rmge_workspace_size_ex(n, nrhs, kind, prec, nullptr);
}

void rmge_options_init(rmge_options* opts) {
    if (opts == nullptr) return;
    const Opts d{};
    opts->growth_tol = d.growth_tol;
    opts->spin_limit = d.spin;
    opts->gmres_m = d.gm_m;
    opts->apply_digits = d.digits;
    opts->factor_digits = d.fdigits;
    opts->sync = 0;
    opts->status = nullptr;
}

size_t rmge_workspace_size_ex(int64_t n, int64_t nrhs, rmge_mult_kind kind, rmge_prec prec, const rmge_options* opts) {
    Opts o;
    if (!opts_of(opts, &o) || !valid_kind(kind) || !valid_prec(prec) || !check_dims(n, nrhs)) return 0;
    if (is_circ(kind) && !circ_ok(kind, n)) return 0;
    return ws_layout(n, nrhs, kind, prec, o.gm_m).total;
}

rmge_status rmge_make_multiplier(rmge_mult_kind kind, int64_t n, uint64_t seed, uint64_t subsequence, rmge_prec prec,
                                 void* G, rmge_stream_t stream) {
    if (!valid_kind(kind) || !valid_prec(prec) || n < 1 || n > RMGE_MAX_N || G == nullptr)
        return RMGE_ERR_INVALID_ARG;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    if (kind == RMGE_GAUSSIAN) {
        if (data_prec(prec) == RMGE_F64) return launch_gaussian(n * n, seed, subsequence, static_cast<double*>(G), s);
        return launch_gaussian(n * n, seed, subsequence, static_cast<float*>(G), s);
    }
    if (!circ_ok(kind, n)) return RMGE_ERR_UNSUPPORTED;
    if (((uintptr_t)G & 15) != 0) return RMGE_ERR_INVALID_ARG;
    double* g = static_cast<double*>(G);
    const int64_t N = fft_len(kind, n);
    if (kind == RMGE_CIRCULANT_UNITARY) {
        // Ex. 5.2: the unit spectrum is drawn, c = Omega^{-1} u follows; the twiddle table lives in c's
        // slot until the inverse transform overwrites it (the CTA reads the table first)
        RMGE_TRY(launch_unitary_spectrum(N, seed, subsequence, reinterpret_cast<double2*>(g + N), s));
        return circulant_from_spectrum(N, g, reinterpret_cast<double2*>(g), s);
    }
    if (kind == RMGE_CIRCULANT_GAUSSIAN || kind == RMGE_TOEPLITZ_GAUSSIAN)
        RMGE_TRY(launch_gaussian(N, seed, subsequence, g, s));
    else
        RMGE_TRY(launch_uniform_pm1(N, seed, subsequence, g, s));
    // The spectrum's twiddle table lives in the third block of G until the FFT overwrites it:
    // u occupies G[N .. 3N) as N double2 and the table needs N/2 double2 -- use the tail half.
    // The FFT reads the table into shared memory before writing u, so the overlap is safe.
    return circulant_spectrum(N, g, reinterpret_cast<double2*>(g + 2 * N), s);
}

rmge_status rmge_apply_multiplier(rmge_mult_kind kind, int64_t n, const double* A, int64_t lda, const void* G, void* M,
                                  int64_t ldm, rmge_prec prec, void* ws, size_t ws_bytes, rmge_stream_t stream) {
    return rmge_apply_multiplier_ex(kind, n, A, lda, G, M, ldm, prec, nullptr, ws, ws_bytes, stream);
}

rmge_status rmge_apply_multiplier_ex(rmge_mult_kind kind, int64_t n, const double* A, int64_t lda, const void* G,
                                     void* M, int64_t ldm, rmge_prec prec, const rmge_options* opts, void* ws,
                                     size_t ws_bytes, rmge_stream_t stream) {
    Opts o;
    if (!opts_of(opts, &o) || !valid_kind(kind) || !valid_prec(prec) || !check_dims(n, 1) || A == nullptr ||
        G == nullptr || M == nullptr || lda < n || ldm < n)
        return RMGE_ERR_INVALID_ARG;
    if (is_circ(kind) && !circ_ok(kind, n)) return RMGE_ERR_UNSUPPORTED;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    Ws w{};
    RMGE_TRY(carve(ws, ws_bytes, n, 1, kind, prec, &w));
    if (is_circ(kind))
        return circulant_apply_rows(n, fft_len(kind, n), A, lda, static_cast<const double*>(G), w.tw, M, ldm,
                                    data_prec(prec) != RMGE_F64, s);
    if (prec == RMGE_F64X_TC) {
        const OzUpdate oz = oz_buffers(w, n);
        return oz_gemm(n, n, n, o.digits, 1.0, A, lda, static_cast<const double*>(G), n, 0.0, static_cast<double*>(M),
                       ldm, oz.planesA, oz.planesB, oz.ea, oz.eb, nullptr, nullptr, &w.st->error, nullptr, s);
    }
    if (prec == RMGE_F64)
        return gemm<double>(false, n, n, n, 1.0, A, lda, static_cast<const double*>(G), n, 0.0,
                            static_cast<double*>(M), ldm, nullptr, s);
    if (prec == RMGE_F32)
        return gemm_f64a_f32(n, n, n, A, lda, static_cast<const float*>(G), n, static_cast<float*>(M), ldm, s);
    // tensor cores: A (rows, K-major) and G^T (K-major) as 16-bit terms, then M = A G in FP32
    const int64_t ldk = tc_ldk(n);
    const size_t plane = (size_t)n * (size_t)ldk * 2;
    char* buf = static_cast<char*>(w.tc);
    const bool bf = tc_bf16(prec);
    const int terms = tc_terms(prec);
    unsigned long long* mxa = bf ? nullptr : w.tcmx;
    unsigned long long* mxb = bf ? nullptr : w.tcmx + 1;
    if (!bf) {
        RMGE_TRY(state_init(w.st, w.flags, 0, reinterpret_cast<double*>(w.tcmx), 2, nullptr, 0, s));
        RMGE_TRY(maxabs<double>(n, n, A, lda, false, mxa, s));
        RMGE_TRY(maxabs<float>(n, n, static_cast<const float*>(G), n, false, mxb, s));
    }
    RMGE_TRY(tc_split<double>(n, n, A, lda, false, 1.0f, mxa, bf, buf, terms == 3 ? buf + plane : nullptr, ldk, s));
    RMGE_TRY(tc_split<float>(n, n, static_cast<const float*>(G), n, true, 1.0f, mxb, bf, buf + 2 * plane,
                             terms == 3 ? buf + 3 * plane : nullptr, ldk, s));
    return tc_gemm(n, n, n, terms, bf, buf, buf + plane, ldk, buf + 2 * plane, buf + 3 * plane, ldk, 1.0f, 0.0f,
                   static_cast<float*>(M), ldm, &w.st->error, nullptr, mxa, mxb, s);
}

rmge_status rmge_factor(int64_t n, void* M, int64_t ldm, rmge_prec prec, int32_t* info, double* growth, void* ws,
                        size_t ws_bytes, rmge_stream_t stream) {
    return rmge_factor_ex(n, M, ldm, prec, info, growth, nullptr, ws, ws_bytes, stream);
}

rmge_status rmge_factor_ex(int64_t n, void* M, int64_t ldm, rmge_prec prec, int32_t* info, double* growth,
                           const rmge_options* opts, void* ws, size_t ws_bytes, rmge_stream_t stream) {
    Opts o;
    if (!opts_of(opts, &o) || !valid_prec(prec) || !check_dims(n, 1) || M == nullptr || ldm < n)
        return RMGE_ERR_INVALID_ARG;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    Ws w{};
    RMGE_TRY(carve(ws, ws_bytes, n, 1, RMGE_GAUSSIAN, prec, &w, true, o));
    RMGE_TRY(state_init(w.st, w.flags, 0, w.colred, 0, nullptr, 0, s, w.spin));
    if (prec == RMGE_F64)
        RMGE_TRY(genp_factor<double>(n, static_cast<double*>(M), ldm, w.st, s));
    else if (prec == RMGE_F64X_TC) {
        const OzUpdate oz = oz_buffers(w, n);
        RMGE_TRY(state_init(w.st, w.flags, 0, reinterpret_cast<double*>(oz.kmax), (int)oz_kmax_slots(n), nullptr, 0, s,
                            w.spin));
        RMGE_TRY(genp_factor_oz(n, static_cast<double*>(M), ldm, w.st, oz, s, 1, 0, o.fdigits));
    }
    else if (prec == RMGE_F32)
        RMGE_TRY(genp_factor<float>(n, static_cast<float*>(M), ldm, w.st, s));
    else {
        const int64_t ldk = kNb;
        const size_t plane = (size_t)n * (size_t)ldk * 2;
        char* buf = static_cast<char*>(w.tc);
        TcUpdate tc{tc_terms(prec), tc_bf16(prec), !tc_bf16(prec), buf, buf + plane, buf + 2 * plane,
                    buf + 3 * plane, ldk, w.tcmx};
        if (tc.scale)
            RMGE_TRY(state_init(w.st, w.flags, 0, reinterpret_cast<double*>(w.tcmx), (int)(2 * (n / kNb + 2)),
                                nullptr, 0, s, w.spin));
        RMGE_TRY(genp_factor_tc(n, static_cast<float*>(M), ldm, w.st, tc, s));
    }
    RMGE_TRY(genp_finish(w.st, info, growth, s));
    return finish_call(w, kStatusFactor, o, 0.0, s);
}

rmge_status rmge_solve(rmge_mult_kind kind, int64_t n, int64_t nrhs, const void* LU, int64_t ldlu, const void* G,
                       const double* B, int64_t ldb, double* X, int64_t ldx, rmge_prec prec, void* ws, size_t ws_bytes,
                       rmge_stream_t stream) {
    return rmge_solve_ex(kind, n, nrhs, LU, ldlu, G, B, ldb, X, ldx, prec, nullptr, ws, ws_bytes, stream);
}

rmge_status rmge_solve_ex(rmge_mult_kind kind, int64_t n, int64_t nrhs, const void* LU, int64_t ldlu, const void* G,
                          const double* B, int64_t ldb, double* X, int64_t ldx, rmge_prec prec,
                          const rmge_options* opts, void* ws, size_t ws_bytes, rmge_stream_t stream) {
    Opts o;
    if (!opts_of(opts, &o) || !valid_kind(kind) || !valid_prec(prec) || !check_dims(n, nrhs) || LU == nullptr ||
        G == nullptr || B == nullptr || X == nullptr || ldlu < n || ldb < nrhs || ldx < nrhs)
        return RMGE_ERR_INVALID_ARG;
    if (is_circ(kind) && !circ_ok(kind, n)) return RMGE_ERR_UNSUPPORTED;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    Ws w{};
    RMGE_TRY(carve(ws, ws_bytes, n, nrhs, kind, prec, &w, false, o));
    RMGE_TRY(state_init(w.st, w.flags, nflags_for(n, nrhs), w.colred, 0, nullptr, 0, s, w.spin));
    RMGE_TRY(correction(kind, data_prec(prec), n, nrhs, LU, ldlu, G, B, ldb, X, ldx, false, w, 1, nullptr, s));
    if (o.report()) RMGE_TRY(nonfinite_scan<double>(n, nrhs, X, ldx, w.st, s));
    return finish_call(w, kStatusSolve, o, 0.0, s);
}

rmge_status rmge_refine(rmge_mult_kind kind, int64_t n, int64_t nrhs, const double* A, int64_t lda, const void* LU,
                        int64_t ldlu, const void* G, const double* B, int64_t ldb, double* X, int64_t ldx,
                        rmge_prec prec, int32_t max_iters, double be_tol, double* berr, int32_t* iters, void* ws,
                        size_t ws_bytes, rmge_stream_t stream) {
    return rmge_refine_ex(kind, n, nrhs, A, lda, LU, ldlu, G, B, ldb, X, ldx, prec, max_iters, be_tol, berr, iters,
                          nullptr, ws, ws_bytes, stream);
}

rmge_status rmge_refine_ex(rmge_mult_kind kind, int64_t n, int64_t nrhs, const double* A, int64_t lda, const void* LU,
                           int64_t ldlu, const void* G, const double* B, int64_t ldb, double* X, int64_t ldx,
                           rmge_prec prec, int32_t max_iters, double be_tol, double* berr, int32_t* iters,
                           const rmge_options* opts, void* ws, size_t ws_bytes, rmge_stream_t stream) {
    Opts o;
    if (!opts_of(opts, &o) || !valid_kind(kind) || !valid_prec(prec) || !check_dims(n, nrhs) || A == nullptr ||
        LU == nullptr || G == nullptr || B == nullptr || X == nullptr || lda < n || ldlu < n || ldb < nrhs ||
        ldx < nrhs || max_iters < 0 || max_iters > kMaxSweeps || !(be_tol >= 0.0))
        return RMGE_ERR_INVALID_ARG;
    if (is_circ(kind) && !circ_ok(kind, n)) return RMGE_ERR_UNSUPPORTED;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    Ws w{};
    RMGE_TRY(carve(ws, ws_bytes, n, nrhs, kind, prec, &w, true, o));
    RMGE_TRY(refine_loop(kind, data_prec(prec), false, n, nrhs, A, lda, LU, ldlu, G, B, ldb, X, ldx, max_iters, be_tol,
                         berr, iters, w, 1, s));
    return finish_call(w, kStatusRefine, o, be_tol, s);
}

rmge_status rmge_solve_backward(rmge_mult_kind kind, int64_t n, int64_t nrhs, const double* A, int64_t lda,
                                const void* LU, int64_t ldlu, const void* G, const double* X, int64_t ldx,
                                const double* dX, int64_t lddx, double* dB, int64_t lddb, double* dA, int64_t ldda,
                                rmge_prec prec, int32_t max_iters, double be_tol, double* berr, int32_t* iters,
                                void* ws, size_t ws_bytes, rmge_stream_t stream) {
    if (!valid_kind(kind) || !valid_prec(prec) || !check_dims(n, nrhs) || LU == nullptr || G == nullptr ||
        dX == nullptr || dB == nullptr || ldlu < n || lddx < nrhs || lddb < nrhs ||
        (dA != nullptr && (X == nullptr || ldda < n || ldx < nrhs)) || max_iters < 0 || max_iters > kMaxSweeps ||
        (max_iters > 0 && (A == nullptr || lda < n)) || !(be_tol >= 0.0))
        return RMGE_ERR_INVALID_ARG;
    if (is_circ(kind) && !circ_ok(kind, n)) return RMGE_ERR_UNSUPPORTED;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    Ws w{};
    RMGE_TRY(carve(ws, ws_bytes, n, nrhs, kind, prec, &w, max_iters > 0));
    prec = data_prec(prec);
    RMGE_TRY(state_init(w.st, w.flags, nflags_for(n, nrhs), w.colred, 0, nullptr, 0, s));
    // dB = A^{-T} dX ~= L^{-T} U^{-T} G^T dX
    RMGE_TRY(correction(kind, prec, n, nrhs, LU, ldlu, G, dX, lddx, dB, lddb, false, w, 1, nullptr, s, true));
    if (max_iters > 0)
        RMGE_TRY(refine_loop(kind, prec, true, n, nrhs, A, lda, LU, ldlu, G, dX, lddx, dB, lddb, max_iters, be_tol,
                             berr, iters, w, 3, s));
    if (dA != nullptr) return outer_neg(n, nrhs, dB, lddb, X, ldx, dA, ldda, s);
    return RMGE_OK;
}

size_t rmge_workspace_size_two_sided(int64_t n, int64_t nrhs, rmge_mult_kind kindF, rmge_mult_kind kindH,
                                     rmge_prec prec) {
    rmge_status why;
    const int present = 1;  // both sides are sized as present
    const void* P = &present;
    if (!check_dims(n, nrhs) || !two_sided_ok(kindF, P, kindH, P, n, prec, &why)) return 0;
    return ws_layout(n, nrhs, layout_kind(P, kindF, P, kindH), prec).total;
}

rmge_status rmge_apply_two_sided(rmge_mult_kind kindF, const void* F, rmge_mult_kind kindH, const void* H, int64_t n,
                                 const double* A, int64_t lda, double* M, int64_t ldm, double* T, int64_t ldt,
                                 rmge_prec prec, void* ws, size_t ws_bytes, rmge_stream_t stream) {
    rmge_status why;
    if (!check_dims(n, 1) || A == nullptr || M == nullptr || lda < n || ldm < n ||
        (F != nullptr && H != nullptr && (T == nullptr || ldt < n)))
        return RMGE_ERR_INVALID_ARG;
    if (!two_sided_ok(kindF, F, kindH, H, n, prec, &why)) return why;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    Ws w{};
    RMGE_TRY(carve(ws, ws_bytes, n, 1, layout_kind(F, kindF, H, kindH), prec, &w));
    if (F == nullptr && H == nullptr) return copy_matrix<double, double>(n, n, A, lda, M, ldm, nullptr, s);
    if (F == nullptr) return right_multiply(kindH, H, prec, n, A, lda, M, ldm, w, s);
    if (H == nullptr) return left_multiply(kindF, F, prec, n, A, lda, M, ldm, w, s);
    RMGE_TRY(right_multiply(kindH, H, prec, n, A, lda, T, ldt, w, s));
    return left_multiply(kindF, F, prec, n, T, ldt, M, ldm, w, s);
}

rmge_status rmge_solve_two_sided(rmge_mult_kind kindF, const void* F, rmge_mult_kind kindH, const void* H, int64_t n,
                                 int64_t nrhs, const void* LU, int64_t ldlu, const double* B, int64_t ldb, double* X,
                                 int64_t ldx, rmge_prec prec, void* ws, size_t ws_bytes, rmge_stream_t stream) {
    rmge_status why;
    if (!check_dims(n, nrhs) || LU == nullptr || B == nullptr || X == nullptr || ldlu < n || ldb < nrhs ||
        ldx < nrhs)
        return RMGE_ERR_INVALID_ARG;
    if (!two_sided_ok(kindF, F, kindH, H, n, prec, &why)) return why;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    Ws w{};
    RMGE_TRY(carve(ws, ws_bytes, n, nrhs, layout_kind(F, kindF, H, kindH), prec, &w, false));
    RMGE_TRY(state_init(w.st, w.flags, nflags_for(n, nrhs), w.colred, 0, nullptr, 0, s));
    return two_sided_correction(kindF, F, kindH, H, n, nrhs, LU, ldlu, B, ldb, X, ldx, false, w, 1, nullptr, s);
}

rmge_status rmge_refine_two_sided(rmge_mult_kind kindF, const void* F, rmge_mult_kind kindH, const void* H, int64_t n,
                                  int64_t nrhs, const double* A, int64_t lda, const void* LU, int64_t ldlu,
                                  const double* B, int64_t ldb, double* X, int64_t ldx, rmge_prec prec,
                                  int32_t max_iters, double be_tol, double* berr, int32_t* iters, void* ws,
                                  size_t ws_bytes, rmge_stream_t stream) {
    rmge_status why;
    if (!check_dims(n, nrhs) || A == nullptr || LU == nullptr || B == nullptr || X == nullptr || lda < n ||
        ldlu < n || ldb < nrhs || ldx < nrhs || max_iters < 0 || max_iters > kMaxSweeps || !(be_tol >= 0.0))
        return RMGE_ERR_INVALID_ARG;
    if (!two_sided_ok(kindF, F, kindH, H, n, prec, &why)) return why;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    Ws w{};
    RMGE_TRY(carve(ws, ws_bytes, n, nrhs, layout_kind(F, kindF, H, kindH), prec, &w));
    RMGE_TRY(state_init(w.st, w.flags, nflags_for(n, nrhs), w.colred, (int)(3 * nrhs), berr, max_iters + 1, s));
    RMGE_TRY(abs_sums_max(n, A, lda, false, w.st, s));
    const int* stop = &w.st->stop;
    for (int it = 0; it <= max_iters; ++it) {
        // R = B - A X in FP64, the backward error and the stopping test (Sec. 1.2, Sec. 7.1)
        RMGE_TRY(copy_matrix<double, double>(n, nrhs, B, ldb, w.R, nrhs, stop, s));
        RMGE_TRY(gemm<double>(false, n, nrhs, n, -1.0, A, lda, X, ldx, 1.0, w.R, nrhs, stop, s));
        RMGE_TRY(backward_error(n, nrhs, w.R, nrhs, X, ldx, B, ldb, w.st, w.colred, it, be_tol, max_iters, berr, s));
        if (it == max_iters) break;
        // X <- X + H U^{-1} L^{-1} F R
        RMGE_TRY(two_sided_correction(kindF, F, kindH, H, n, nrhs, LU, ldlu, w.R, nrhs, X, ldx, true, w, 3 + 2 * it,
                                      stop, s));
    }
    return refine_finish(w.st, max_iters, berr, iters, s);
}

// ---- low-rank approximation (Sec. 6, Algorithm 6.1) ------------------------------------------------

static bool lowrank_args_ok(rmge_mult_kind kind, int64_t m, int64_t n, int32_t l) {
    if ((int)kind < (int)RMGE_GAUSSIAN || (int)kind > (int)RMGE_CIRCULANT_UNITARY) return false;
    if (m < 1 || n < 1 || m > RMGE_MAX_N || n > RMGE_MAX_N || l < 1 || l > kLowRankMaxL || l > m || l > n) return false;
    return kind == RMGE_GAUSSIAN || circ_ok(kind, n);
}

size_t rmge_lowrank_workspace_size(rmge_mult_kind kind, int64_t m, int64_t n, int32_t l) {
    if (!lowrank_args_ok(kind, m, n, l)) return 0;
    return lowrank_workspace_bytes(n, l, kind != RMGE_GAUSSIAN);
}

rmge_status rmge_lowrank_multiplier(rmge_mult_kind kind, int64_t n, int32_t l, uint64_t seed, uint64_t subsequence,
                                    double* H, rmge_stream_t stream) {
    if (!lowrank_args_ok(kind, n, n, l) || H == nullptr) return RMGE_ERR_INVALID_ARG;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    if (kind == RMGE_GAUSSIAN) return launch_gaussian(n * (int64_t)l, seed, subsequence, H, s);
    return rmge_make_multiplier(kind, n, seed, subsequence, RMGE_F64, H, stream);
}

rmge_status rmge_lowrank_basis(rmge_mult_kind kind, int64_t m, int64_t n, int32_t l, const double* A, int64_t lda,
                               const double* H, double* Q, int64_t ldq, int32_t* info, void* ws, size_t ws_bytes,
                               rmge_stream_t stream) {
    if (!lowrank_args_ok(kind, m, n, l) || A == nullptr || H == nullptr || Q == nullptr || lda < n || ldq < l)
        return RMGE_ERR_INVALID_ARG;
    if (ws == nullptr || ((uintptr_t)ws & 255) != 0 || ws_bytes < lowrank_workspace_bytes(n, l, kind != RMGE_GAUSSIAN))
        return RMGE_ERR_WORKSPACE;
    if (kind != RMGE_GAUSSIAN && ((uintptr_t)H & 15) != 0) return RMGE_ERR_INVALID_ARG;
    return lowrank_basis((int)kind, m, n, l, A, lda, H, Q, ldq, info, ws, reinterpret_cast<cudaStream_t>(stream));
}

rmge_status rmge_lowrank_project(int64_t m, int64_t n, int32_t l, const double* Q, int64_t ldq, const double* A,
                                 int64_t lda, double* Z, int64_t ldz, rmge_stream_t stream) {
    if (!lowrank_args_ok(RMGE_GAUSSIAN, m, n, l) || Q == nullptr || A == nullptr || Z == nullptr || ldq < l ||
        lda < n || ldz < n)
        return RMGE_ERR_INVALID_ARG;
    return lowrank_project(m, n, l, Q, ldq, A, lda, Z, ldz, reinterpret_cast<cudaStream_t>(stream));
}

// ---- uniform batches (emulated FP64): count systems of order n, one launch per kernel and step -------------

struct UniLayout {
    size_t states, kmax, ea, eb, planesA, planesB, total;
    int64_t Mp, Kp, steps;
};

static UniLayout uni_layout(int64_t count, int64_t n) {
    UniLayout L{};
    L.Mp = (n + 127) / 128 * 128;
    L.Kp = (n + 63) / 64 * 64;
    L.steps = (n + kNb - 1) / kNb;
    size_t off = 0;
    L.states = off;
    off = align256(off + sizeof(DevState) * (size_t)count);
    L.kmax = off;
    off = align256(off + sizeof(unsigned long long) * (size_t)oz_kmax_per_system(n) * (size_t)count);
    L.ea = off;
    off = align256(off + sizeof(int) * (size_t)L.Mp * (size_t)count);
    L.eb = off;
    off = align256(off + sizeof(int) * (size_t)L.Mp * (size_t)count);
    const size_t plane = (size_t)kOzSlices * (size_t)L.Mp * (size_t)L.Kp * 2 * (size_t)count;
    L.planesA = off;
    off = align256(off + plane);
    L.planesB = off;
    off = align256(off + plane);
    L.total = off;
    return L;
}

static bool uni_args_ok(int64_t count, int64_t n) {
    return count >= 1 && count <= 65535 && n >= 1 && n <= RMGE_MAX_N;
}

static bool uni_stride_ok(int64_t n, int64_t ld, int64_t stride) {
    return ld >= n && stride >= (n - 1) * ld + n;
}

size_t rmge_batched_uniform_workspace_size(int64_t count, int64_t n, rmge_prec prec) {
    if (!uni_args_ok(count, n) || prec != RMGE_F64X_TC) return 0;
    return uni_layout(count, n).total;
}

rmge_status rmge_apply_multiplier_batched(int64_t count, int64_t n, const double* A, int64_t lda, int64_t strideA,
                                          const double* G, int64_t strideG, double* M, int64_t ldm, int64_t strideM,
                                          rmge_prec prec, const rmge_options* opts, void* ws, size_t ws_bytes,
                                          rmge_stream_t stream) {
    Opts o;
    if (!opts_of(opts, &o) || !uni_args_ok(count, n) || !valid_prec(prec) || A == nullptr || G == nullptr ||
        M == nullptr || !uni_stride_ok(n, lda, strideA) || !uni_stride_ok(n, n, strideG) ||
        !uni_stride_ok(n, ldm, strideM))
        return RMGE_ERR_INVALID_ARG;
    if (prec != RMGE_F64X_TC) return RMGE_ERR_UNSUPPORTED;
    const UniLayout L = uni_layout(count, n);
    if (ws == nullptr || ((uintptr_t)ws & 255) != 0 || ws_bytes < L.total) return RMGE_ERR_WORKSPACE;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    char* b = static_cast<char*>(ws);
    DevState* st = reinterpret_cast<DevState*>(b + L.states);
    RMGE_TRY(states_init(st, (int)count, nullptr, 0, s, o.spin));
    OzBatch bt;
    bt.count = (int)count;
    bt.sA = strideA;
    bt.sB = strideG;
    bt.sC = strideM;
    return oz_gemm(n, n, n, o.digits, 1.0, A, lda, G, n, 0.0, M, ldm, b + L.planesA, b + L.planesB,
                   reinterpret_cast<int*>(b + L.ea), reinterpret_cast<int*>(b + L.eb), nullptr, nullptr, &st->error,
                   nullptr, s, nullptr, bt);
}

rmge_status rmge_factor_batched(int64_t count, int64_t n, double* M, int64_t ldm, int64_t strideM, rmge_prec prec,
                                int32_t* info, double* growth, const rmge_options* opts, void* ws, size_t ws_bytes,
                                rmge_stream_t stream) {
    Opts o;
    if (!opts_of(opts, &o) || !uni_args_ok(count, n) || !valid_prec(prec) || M == nullptr || info == nullptr ||
        !uni_stride_ok(n, ldm, strideM))
        return RMGE_ERR_INVALID_ARG;
    if (prec != RMGE_F64X_TC) return RMGE_ERR_UNSUPPORTED;
    const UniLayout L = uni_layout(count, n);
    if (ws == nullptr || ((uintptr_t)ws & 255) != 0 || ws_bytes < L.total) return RMGE_ERR_WORKSPACE;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    char* b = static_cast<char*>(ws);
    DevState* st = reinterpret_cast<DevState*>(b + L.states);
    OzUpdate oz{};
    oz.planesA = b + L.planesA;
    oz.planesB = b + L.planesB;
    oz.ea = reinterpret_cast<int*>(b + L.ea);
    oz.eb = reinterpret_cast<int*>(b + L.eb);
    oz.kmax = reinterpret_cast<unsigned long long*>(b + L.kmax);
    RMGE_TRY(states_init(st, (int)count, oz.kmax, oz_kmax_per_system(n) * count, s));
    RMGE_TRY(genp_factor_oz(n, M, ldm, st, oz, s, (int)count, strideM, o.fdigits));
    return genp_finish(st, info, growth, s, (int)count);
}

size_t rmge_uniform_solve_workspace_size(int64_t count, int64_t n, int64_t nrhs, rmge_prec prec) {
    if (count < 1 || count > 65535 || !check_dims(n, nrhs) || !valid_prec(prec) || data_prec(prec) != RMGE_F64)
        return 0;
    return (size_t)count * ws_layout(n, nrhs, RMGE_GAUSSIAN, RMGE_F64).total;
}

rmge_status rmge_solve_uniform_batched(int64_t count, int64_t n, int64_t nrhs, const double* LU, int64_t ldlu,
                                       int64_t strideLU, const double* G, int64_t strideG, const double* B,
                                       int64_t ldb, int64_t strideB, double* X, int64_t ldx, int64_t strideX,
                                       rmge_prec prec, void* ws, size_t ws_bytes, rmge_stream_t stream) {
    Bt bt{};
    Ws w{};
    if (!mat_ok(B, n, nrhs, ldb, strideB) || !mat_ok(X, n, nrhs, ldx, strideX)) return RMGE_ERR_INVALID_ARG;
    RMGE_TRY(uniform_setup(count, n, nrhs, prec, LU, ldlu, strideLU, G, strideG, ws, ws_bytes, &bt, &w));
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    RMGE_TRY(state_init(w.st, w.flags, nflags_for(n, nrhs), w.colred, 0, nullptr, 0, s, w.spin, zb3(bt, 0, 0)));
    return correction_z(bt, n, nrhs, LU, ldlu, G, B, ldb, strideB, X, ldx, strideX, false, w, 1, nullptr, s, false);
}

rmge_status rmge_refine_uniform_batched(int64_t count, int64_t n, int64_t nrhs, const double* A, int64_t lda,
                                        int64_t strideA, const double* LU, int64_t ldlu, int64_t strideLU,
                                        const double* G, int64_t strideG, const double* B, int64_t ldb,
                                        int64_t strideB, double* X, int64_t ldx, int64_t strideX, rmge_prec prec,
                                        int32_t max_iters, double be_tol, double* berr, int32_t* iters, void* ws,
                                        size_t ws_bytes, rmge_stream_t stream) {
    Bt bt{};
    Ws w{};
    if (!mat_ok(A, n, n, lda, strideA) || !mat_ok(B, n, nrhs, ldb, strideB) || !mat_ok(X, n, nrhs, ldx, strideX) ||
        max_iters < 0 || max_iters > kMaxSweeps || !(be_tol >= 0.0))
        return RMGE_ERR_INVALID_ARG;
    RMGE_TRY(uniform_setup(count, n, nrhs, prec, LU, ldlu, strideLU, G, strideG, ws, ws_bytes, &bt, &w));
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    return refine_loop_z(bt, false, n, nrhs, A, lda, strideA, LU, ldlu, G, B, ldb, strideB, X, ldx, strideX,
                         max_iters, be_tol, berr, iters, w, 1, s);
}

rmge_status rmge_solve_backward_uniform_batched(int64_t count, int64_t n, int64_t nrhs, const double* A, int64_t lda,
                                                int64_t strideA, const double* LU, int64_t ldlu, int64_t strideLU,
                                                const double* G, int64_t strideG, const double* X, int64_t ldx,
                                                int64_t strideX, const double* dX, int64_t lddx, int64_t stridedX,
                                                double* dB, int64_t lddb, int64_t stridedB, double* dA, int64_t ldda,
                                                int64_t stridedA, rmge_prec prec, int32_t max_iters, double be_tol,
                                                double* berr, int32_t* iters, void* ws, size_t ws_bytes,
                                                rmge_stream_t stream) {
    Bt bt{};
    Ws w{};
    if (!mat_ok(dX, n, nrhs, lddx, stridedX) || !mat_ok(dB, n, nrhs, lddb, stridedB) ||
        (dA != nullptr && (!mat_ok(dA, n, n, ldda, stridedA) || !mat_ok(X, n, nrhs, ldx, strideX))) ||
        max_iters < 0 || max_iters > kMaxSweeps || (max_iters > 0 && !mat_ok(A, n, n, lda, strideA)) ||
        !(be_tol >= 0.0))
        return RMGE_ERR_INVALID_ARG;
    RMGE_TRY(uniform_setup(count, n, nrhs, prec, LU, ldlu, strideLU, G, strideG, ws, ws_bytes, &bt, &w));
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    RMGE_TRY(state_init(w.st, w.flags, nflags_for(n, nrhs), w.colred, 0, nullptr, 0, s, w.spin, zb3(bt, 0, 0)));
    // dB = A^{-T} dX ~= L^{-T} U^{-T} G^T dX, refined on A^T dB = dX, then dA = -dB X^T
    RMGE_TRY(correction_z(bt, n, nrhs, LU, ldlu, G, dX, lddx, stridedX, dB, lddb, stridedB, false, w, 1, nullptr, s,
                          true));
    if (max_iters > 0)
        RMGE_TRY(refine_loop_z(bt, true, n, nrhs, A, lda, strideA, LU, ldlu, G, dX, lddx, stridedX, dB, lddb,
                               stridedB, max_iters, be_tol, berr, iters, w, 3, s));
    if (dA != nullptr) return outer_neg(n, nrhs, dB, lddb, X, ldx, dA, ldda, s, zb3(bt, stridedB, strideX, stridedA));
    return RMGE_OK;
}

size_t rmge_batched_workspace_size(int64_t nmax, int32_t ctas) {
    if (nmax < 1 || nmax > 4096 || ctas < 1 || ctas > 65535) return 0;
    return batched_scratch_bytes(nmax, ctas);
}

rmge_status rmge_solve_batched(int64_t count, const int32_t* n, const int64_t* offA, const int64_t* offv,
                               const int32_t* order, const double* A, const double* b, double* x, int32_t* info,
                               double* berr, int32_t* sweeps, uint64_t seed, int32_t max_sweeps, double be_tol,
                               int64_t nmax, int32_t config, int32_t ctas, void* ws, size_t ws_bytes,
                               rmge_stream_t stream) {
    return rmge_solve_batched_ex(count, n, offA, offv, order, A, b, x, info, berr, sweeps, seed, max_sweeps, be_tol,
                                 nmax, config, ctas, nullptr, ws, ws_bytes, stream);
}

rmge_status rmge_solve_batched_ex(int64_t count, const int32_t* n, const int64_t* offA, const int64_t* offv,
                                  const int32_t* order, const double* A, const double* b, double* x, int32_t* info,
                                  double* berr, int32_t* sweeps, uint64_t seed, int32_t max_sweeps, double be_tol,
                                  int64_t nmax, int32_t config, int32_t ctas, const rmge_options* opts, void* ws,
                                  size_t ws_bytes, rmge_stream_t stream) {
    Opts o;
    if (!opts_of(opts, &o) || count < 1 || count > INT32_MAX || n == nullptr || offA == nullptr || offv == nullptr ||
        order == nullptr || A == nullptr || b == nullptr || x == nullptr || info == nullptr || berr == nullptr ||
        sweeps == nullptr || max_sweeps < 0 || max_sweeps > kMaxSweeps || !(be_tol >= 0.0) || config < 0 ||
        config > 2)
        return RMGE_ERR_INVALID_ARG;
    const size_t need = rmge_batched_workspace_size(nmax, ctas);
    if (need == 0) return RMGE_ERR_INVALID_ARG;
    if (ws == nullptr || ((uintptr_t)ws & 255) != 0 || ws_bytes < need) return RMGE_ERR_WORKSPACE;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    if (cudaMemsetAsync(ws, 0, 256, s) != cudaSuccess) {
        (void)cudaGetLastError();
        return RMGE_ERR_CUDA;
    }
    RMGE_TRY(batched_solve(count, n, offA, offv, order, A, b, x, info, berr, sweeps, seed, max_sweeps, be_tol, nmax,
                           config, ctas, o.spin, ws, s));
    if (!o.report()) return RMGE_OK;
    RMGE_TRY(batched_status(count, info, ws, o.status, s));
    if (!o.sync) return RMGE_OK;
    int h = RMGE_OK;
    if (cudaMemcpyAsync(&h, static_cast<char*>(ws) + 32, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) {
        (void)cudaGetLastError();
        return RMGE_ERR_CUDA;
    }
    return (rmge_status)h;
}

}  // extern "C"
