// kernels.cuh -- host-side launchers of the librmge kernels (one translation unit each).
#pragma once

#include "common.cuh"

namespace rmge {

// A uniform batch for the solve-path kernels: `count` systems, blockIdx.z picks one.  m0 .. m3 are the
// element strides between the systems' copies of the launcher's first to fourth array argument (in the
// order of its parameter list, control-block pointers not counted), ws the byte stride between their
// workspace blocks, where every control-block pointer (DevState, skip and halt flags, solve flags,
// reductions) lives.  The default is a single system.
struct Zb {
    int count = 1;
    int64_t m0 = 0, m1 = 0, m2 = 0, m3 = 0;
    int64_t ws = 0;
};

template <typename T>
__device__ __forceinline__ T* zmat(T* p, int64_t stride) {
    return p == nullptr ? p : p + (int64_t)blockIdx.z * stride;
}
template <typename T>
__device__ __forceinline__ T* zws(T* p, int64_t bytes) {
    return p == nullptr ? p
                        : reinterpret_cast<T*>(reinterpret_cast<char*>(const_cast<void*>(static_cast<const void*>(p))) +
                                               (int64_t)blockIdx.z * bytes);
}

// gen.cu: the multiplier draws (Def. 4.1, Ex. 5.1) from Philox4x32-10.
rmge_status launch_gaussian(int64_t count, uint64_t seed, uint64_t subseq, double* out, cudaStream_t s);
rmge_status launch_gaussian(int64_t count, uint64_t seed, uint64_t subseq, float* out, cudaStream_t s);
rmge_status launch_uniform_pm1(int64_t count, uint64_t seed, uint64_t subseq, double* out, cudaStream_t s);
rmge_status launch_unitary_spectrum(int64_t N, uint64_t seed, uint64_t subseq, double2* u, cudaStream_t s);

// gemm.cu: C = alpha * op(A) * B + beta * C on the SIMT FMA pipes (op(A) = A, or A^T when trans_a).
// A is M x K (or K x M when trans_a), B is K x N, C is M x N; all row-major.  beta == 0 never
// reads C.  When halt is non-NULL and *halt != 0 at kernel start the kernel does nothing.
template <typename T>
rmge_status gemm(bool trans_a, int64_t M, int64_t N, int64_t K, T alpha, const T* A, int64_t lda, const T* B,
                 int64_t ldb, T beta, T* C, int64_t ldc, const int* halt, cudaStream_t s, const Zb& zb = Zb{});
// E <- E - L21 U12 (M x N, K <= 64) for GENP, whose CTA on tile (0, 0) then factors the b x b pivot
// block at E's top-left corner (pivot_block_genp); a breakdown at its step s records k + s in *info
// (atomicMin) and raises *halt_w.  halt: as for gemm.
template <typename T>
rmge_status gemm_update_fused(int64_t M, int64_t N, int64_t K, const T* A, int64_t lda, const T* B, int64_t ldb, T* C,
                              int64_t ldc, const int* halt, int b, int64_t k, int* info, int* halt_w, cudaStream_t s);

// C (FP32) = A (FP64, rounded to FP32 on load) * B (FP32): M = A G for the FP32 working matrix.
rmge_status gemm_f64a_f32(int64_t M, int64_t N, int64_t K, const double* A, int64_t lda, const float* B, int64_t ldb,
                          float* C, int64_t ldc, cudaStream_t s);

// tc_gemm.cu: C (FP32) <- beta C + alpha sum_t A_t B_t^T on tcgen05 tensor cores, A_t (M x K) and
// B_t (N x K) BF16 or FP16 K-major with leading dimensions multiples of 8.  terms = 1: A0 B0^T;
// terms = 3: A0 B0^T + A0 B1^T + A1 B0^T (two-term splits).  *err <- RMGE_ERR_TIMEOUT if a bounded
// wait expires.
// mxa/mxb (may be NULL): bits of max|A|, max|B| used by the FP16 power-of-two operand scaling; the
// epilogue divides the scales back out.
rmge_status tc_gemm(int64_t M, int64_t N, int64_t K, int terms, bool bf16, const void* A0, const void* A1, int64_t lda,
                    const void* B0, const void* B1, int64_t ldb, float alpha, float beta, float* C, int64_t ldc,
                    int* err, const int* halt, const unsigned long long* mxa, const unsigned long long* mxb,
                    cudaStream_t s);
// hi (+ lo when non-NULL) = two-term split of scale * 2^e(mx) * src (rows x cols), stored K-major:
// dst[i][j] (trans = false) or dst[j][i] (trans = true), leading dimension ldd.
template <typename S>
rmge_status tc_split(int64_t rows, int64_t cols, const S* src, int64_t lds, bool trans, float scale,
                     const unsigned long long* mx, bool bf16, void* hi, void* lo, int64_t ldd, cudaStream_t s);
uint32_t tc_idesc(bool bf16);

// oz_gemm.cu: C (FP64) <- beta C + alpha A B with the product emulated on BF16 tensor cores from
// s balanced base-256 digit planes of A (rows) and B (columns); s = kOzSlices reproduces FP64.  planesA/planesB: oz_plane_bytes(M, K, s) and
// oz_plane_bytes(N, K, s) bytes; ea[M], eb[N] ints of scratch.  kmaxA/kmaxB (both or neither): the
// per-k maxima max_i |A_ik| and max_j |B_kj| (FP64 bit patterns, K <= 64), which balance column k of A
// against row k of B by an exact power of two.
// *err <- RMGE_ERR_TIMEOUT if a bounded wait expires; nothing happens while *halt != 0 (halt may be NULL).
constexpr int kOzSlices = 7;
size_t oz_plane_bytes(int64_t rows, int64_t k, int s);
// The pivot block of the next GENP step, factored inside the update launch (K <= 64, kOzSlices digits): the
// b x b block at D (b <= 64, leading dimension ldd) must lie in the first 128 x 64 tile of C; a
// breakdown at its step s records k + s in *info (atomicMin) and raises *halt.
struct OzFuse {
    double* D;
    int64_t ldd;
    int b;
    int64_t k;
    int* info;
    int* halt;
};
// A batch of `count` products of one shape (the systems of a uniform batched solve): the element strides
// between the systems' A, B and C, the slots between their per-k maxima (kmaxA and kmaxB move together),
// and the ints between their fused-pivot info / halt words; count = 1 is a single product.  planesA,
// planesB, ea and eb then hold count consecutive per-system blocks of the single sizes (planes of
// Mp x Kp and Np x Kp per digit, Mp and Np exponents).  With count > 1 a set halt word does not skip work.
struct OzBatch {
    int count = 1;
    int64_t sA = 0, sB = 0, sC = 0;
    int64_t sK = 0;
    int64_t sFlag = 0;
};
rmge_status oz_gemm(int64_t M, int64_t N, int64_t K, int s, double alpha, const double* A, int64_t lda,
                    const double* B, int64_t ldb, double beta, double* C, int64_t ldc, void* planesA, void* planesB,
                    int* ea, int* eb, const unsigned long long* kmaxA, const unsigned long long* kmaxB, int* err,
                    const int* halt, cudaStream_t st, const OzFuse* fuse = nullptr, const OzBatch& bt = OzBatch{});
// E -= A B with K = 128 (two pivot blocks of GENP at once; A is M x 128, B is 128 x N), the digit planes
// of A and B from s = 4 .. kOzSlices digits with the per-k balancing maxima kmaxA[0..128), kmaxB[0..128),
// then the persistent 128-deep update kernel.  fuse and bt as for oz_gemm (the tile holding C's top-left
// corner also factors the pivot block there).
rmge_status oz_update128(int64_t M, int64_t N, int s, const double* A, int64_t lda, const double* B, int64_t ldb,
                         double* C, int64_t ldc, void* planesA, void* planesB, int* ea, int* eb,
                         const unsigned long long* kmaxA, const unsigned long long* kmaxB, int* err, const int* halt,
                         cudaStream_t st, const OzFuse* fuse = nullptr, const OzBatch& bt = OzBatch{});
// launch_timing.cu: CUDA event pairs around the emulated Schur-update launches while rmge_launch_timing(1) is
// on.  timing_begin records the first event of launch class `kernel` (rmge_timed_kernel) with its MMA flops
// and returns a token for timing_end; a negative token means nothing was recorded.
int64_t timing_begin(int kernel, cudaStream_t s, double mma_flops);
void timing_end(int64_t token, cudaStream_t s);
// Slots of per-k maxima per system for the emulated factorization: for each pair of pivot steps, the
// 64 + 64 column maxima of L21 and then the 64 + 64 row maxima of U12 (256 slots), so that the 128-deep
// update of a pair finds both operands' maxima contiguous.
inline int64_t oz_kmax_per_system(int64_t n) {
    const int64_t steps = (n + kNb - 1) / kNb;
    return 256 * ((steps + 1) / 2);
}
struct OzUpdate {
    void* planesA;
    void* planesB;
    int* ea;
    int* eb;
    unsigned long long* kmax;  // 128 zeroed slots per pivot-block step: column maxima of L21, row maxima of U12
};

// genp.cu: in-place blocked GENP of an n x n matrix with DevState bookkeeping.
template <typename T>
rmge_status genp_factor(int64_t n, T* M, int64_t ldm, DevState* st, cudaStream_t s);
// Tensor-core trailing updates for the FP32 working matrix: operand buffers of n x ldk 16-bit values
// (hi, lo for A and B), per-step max-abs slots (FP16 scaling), terms 1 or 3.
struct TcUpdate {
    int terms;
    bool bf16;
    bool scale;
    void* a_hi;
    void* a_lo;
    void* b_hi;
    void* b_lo;
    int64_t ldk;
    unsigned long long* mx;  // 2 slots per pivot step, zeroed by the caller
};
rmge_status genp_factor_tc(int64_t n, float* M, int64_t ldm, DevState* st, const TcUpdate& tc,
                           cudaStream_t s);
// FP64 working matrix with the Schur-complement updates as balanced FP64 products emulated on the
// tensor cores (oz_gemm); pivot blocks and panels on the FP64 pipe.
// count > 1: a batch of count equal-size systems, matrices sM elements apart, control blocks st[0..count),
// per-system blocks of digit planes, exponents and per-k maxima in oz (OzBatch); one launch per kernel
// and step covers every system.  digits (4 .. kOzSlices): balanced base-256 digits per operand of the
// emulated updates (digits (digits + 1) / 2 digit-pair products; kOzSlices reproduces FP64 rounding).
rmge_status genp_factor_oz(int64_t n, double* M, int64_t ldm, DevState* st, const OzUpdate& oz, cudaStream_t s,
                           int count = 1, int64_t sM = 0, int digits = kOzSlices);
// growth = max|U| / max|M| and info from the DevState (writes the caller's outputs); count consecutive
// control blocks to count outputs.
rmge_status genp_finish(DevState* st, int32_t* info, double* growth, cudaStream_t s, int count = 1);
template <typename T>
rmge_status maxabs(int64_t rows, int64_t cols, const T* P, int64_t ldp, bool upper_only,
                   unsigned long long* out_bits, cudaStream_t s);

// trsv.cu: in-place triangular solves with the packed factors, nrhs columns, one launch each.
//   kind 0: L y = b (unit lower)      kind 1: U y = b (upper)
//   kind 2: U^T y = b (lower, diag U) kind 3: L^T y = b (unit upper)
// epoch: a value unique within the call (flags are zeroed at call start); the ticket counters in
// st must be zero at launch (state_init, and each solve re-arms them).  skip: as for gemm's halt.
template <typename T>
rmge_status trsv(int kind, int64_t n, int64_t nrhs, const T* LU, int64_t ldlu, T* B, int64_t ldb,
                 DevState* st, int* flags, int epoch, const int* skip, cudaStream_t s, const Zb& zb = Zb{});

// refine.cu
// Resets the control block (with the spin limit of the call's bounded waits), zeroes nflags solve flags and
// ncolred reduction slots, sets berr_out[0..nberr) to -1 (berr_out may be NULL).
rmge_status state_init(DevState* st, int* flags, int64_t nflags, double* colred, int ncolred, double* berr_out,
                       int nberr, cudaStream_t s, long long spin_limit = kSpinLimit, const Zb& zb = Zb{});
// count consecutive control blocks reset (as state_init does for one) and nzero 64-bit words cleared.
rmge_status states_init(DevState* st, int count, unsigned long long* zero, int64_t nzero, cudaStream_t s,
                        long long spin_limit = kSpinLimit);
// st->norm_a = ||A||_inf (transposed: ||A^T||_inf)
rmge_status abs_sums_max(int64_t n, const double* A, int64_t lda, bool transposed, DevState* st, cudaStream_t s,
                         const Zb& zb = Zb{});
// R = B (copy, n x k)
template <typename Tin, typename Tout>
rmge_status copy_matrix(int64_t rows, int64_t cols, const Tin* src, int64_t lds, Tout* dst, int64_t ldd,
                        const int* skip, cudaStream_t s, const Zb& zb = Zb{});
// X += D (FP64 X, D of type T), skipped when *skip != 0
template <typename T>
rmge_status add_update(int64_t rows, int64_t cols, const T* D, int64_t ldd, double* X, int64_t ldx,
                       const int* skip, cudaStream_t s, const Zb& zb = Zb{});
// backward error of (R, X, B) into berr_out[sweep] and the stop test; see rmge_refine.
rmge_status backward_error(int64_t n, int64_t k, const double* R, int64_t ldr, const double* X, int64_t ldx,
                           const double* B, int64_t ldb, DevState* st, double* colred, int sweep,
                           double be_tol, int max_iters, double* berr_out, cudaStream_t s, bool hybrid = false,
                           const Zb& zb = Zb{});
rmge_status refine_finish(DevState* st, int max_iters, double* berr_out, int32_t* iters, cudaStream_t s,
                          const Zb& zb = Zb{});
// st->nonfinite <- 1 if P (rows x cols) holds an Inf or NaN.
template <typename T>
rmge_status nonfinite_scan(int64_t rows, int64_t cols, const T* P, int64_t ldp, DevState* st, cudaStream_t s);
// The call's rmge_status from the control block into st->status and *out (out may be NULL): what is
// kStatusFactor (breakdown, non-finite values, growth above growth_tol > 0), kStatusSolve (non-finite
// result) or kStatusRefine (non-finite result, backward error above be_tol); a timeout comes first.
constexpr int kStatusFactor = 0, kStatusSolve = 1, kStatusRefine = 2;
rmge_status write_status(DevState* st, int what, double growth_tol, double be_tol, int32_t* out, cudaStream_t s);
// dA = -dB X^T
rmge_status outer_neg(int64_t n, int64_t k, const double* dB, int64_t lddb, const double* X, int64_t ldx,
                      double* dA, int64_t ldda, cudaStream_t s, const Zb& zb = Zb{});

// gmres.cu: one FGMRES(m) cycle on op(A) d = R (op(A) = A^T when trans_a) for all k columns, right-preconditioned by P
// (z = P v applied in the factor precision), X += d.  buf: gmres_bytes(n, k, m) bytes.  Uses epochs
// epoch0 .. epoch0 + 2 m - 1 for P's triangular solves.
struct GmresPrecond {
    rmge_status (*apply)(const void* ctx, const double* v, double* z, int epoch, const int* skip, cudaStream_t s);
    const void* ctx;
};
size_t gmres_bytes(int64_t n, int64_t k, int m);
rmge_status gmres_cycle(int64_t n, int64_t k, int m, const double* A, int64_t lda, bool trans_a, const double* R,
                        double* X, int64_t ldx, double* buf, const GmresPrecond& P, int epoch0, const int* skip,
                        cudaStream_t s);

// batched.cu: persistent one-CTA-per-system solves (see rmge_solve_batched).
size_t batched_scratch_bytes(int64_t nmax, int ctas);
rmge_status batched_solve(int64_t count, const int32_t* n, const int64_t* offA, const int64_t* offv,
                          const int32_t* order, const double* A, const double* b, double* x, int32_t* info,
                          double* berr, int32_t* sweeps, uint64_t seed, int max_sweeps, double tol, int64_t nmax,
                          int config, int ctas, long long spin_limit, void* ws, cudaStream_t s);
// RMGE_ERR_TIMEOUT if some info[i] is -1, else RMGE_OK, into the int at byte 32 of ws and *out (may be NULL).
rmge_status batched_status(int64_t count, const int32_t* info, void* ws, int32_t* out, cudaStream_t s);

// fft.cu: circulant multiplier (Theorem 5.1).  G = [c (n doubles) | u = F(c) (n double2)];
// FFT kinds (fft.cu), N the transform length (n for a circulant, 2n for a Toeplitz multiplier, the
// leading n x n block of an N x N circulant); G = [c (N) | u = F(c) (N complex)]; tw: N/2 double2.
rmge_status circulant_spectrum(int64_t N, double* G, double2* tw, cudaStream_t s);
// c = Re F^{-1}(u) from the spectrum in G (the drawn unitary circulant).
rmge_status circulant_from_spectrum(int64_t N, double* G, double2* tw, cudaStream_t s);
// M = A H (rows of A correlated with c), M in FP64 or FP32.
rmge_status circulant_apply_rows(int64_t n, int64_t N, const double* A, int64_t lda, const double* G, double2* tw,
                                 void* M, int64_t ldm, bool out_f32, cudaStream_t s);
// M (rows x nout) = the first nout columns of A C for an n x n circulant C (A: rows x n), FP64.
rmge_status circulant_apply_rows_block(int64_t rows, int64_t n, int64_t nout, const double* A, int64_t lda,
                                       const double* G, double2* tw, double* M, int64_t ldm, cudaStream_t s);
// X (+)= H Y, or H^T Y when transpose, k columns, FP64; nothing when *skip != 0.
rmge_status circulant_apply_cols(int64_t n, int64_t N, int64_t k, const double* G, double2* tw, bool transpose,
                                 const double* Y, int64_t ldy, double* X, int64_t ldx, bool accumulate,
                                 const int* skip, cudaStream_t s);

// lowrank.cu: Algorithm 6.1 (B = A H, Q = Q(B) by CholeskyQR2, Z = Q^T A); kind 0 a dense n x l H, else
// the n x l leading block of an n x n circulant (G storage); ws: lowrank_workspace_bytes.
size_t lowrank_workspace_bytes(int64_t n, int l, bool fft);
rmge_status lowrank_basis(int kind, int64_t m, int64_t n, int l, const double* A, int64_t lda, const double* H,
                          double* Q, int64_t ldq, int32_t* info, void* ws, cudaStream_t s);
rmge_status lowrank_project(int64_t m, int64_t n, int l, const double* Q, int64_t ldq, const double* A, int64_t lda,
                            double* Z, int64_t ldz, cudaStream_t s);

}  // namespace rmge
