// kernels.cuh -- host-side launchers of the librmge kernels (one translation unit each).
#pragma once

#include "common.cuh"

namespace rmge {

// gen.cu: the multiplier draws (Def. 4.1, Ex. 5.1) from Philox4x32-10.
rmge_status launch_gaussian(int64_t count, uint64_t seed, uint64_t subseq, double* out, cudaStream_t s);
rmge_status launch_gaussian(int64_t count, uint64_t seed, uint64_t subseq, float* out, cudaStream_t s);
rmge_status launch_uniform_pm1(int64_t count, uint64_t seed, uint64_t subseq, double* out, cudaStream_t s);

// gemm.cu: C = alpha * op(A) * B + beta * C on the SIMT FMA pipes (op(A) = A, or A^T when trans_a).
// A is M x K (or K x M when trans_a), B is K x N, C is M x N; all row-major.  beta == 0 never
// reads C.  When halt is non-NULL and *halt != 0 at kernel start the kernel does nothing.
template <typename T>
rmge_status gemm(bool trans_a, int64_t M, int64_t N, int64_t K, T alpha, const T* A, int64_t lda, const T* B,
                 int64_t ldb, T beta, T* C, int64_t ldc, const int* halt, cudaStream_t s);

// genp.cu: in-place blocked GENP of an n x n matrix with DevState bookkeeping.
template <typename T>
rmge_status genp_factor(int64_t n, T* M, int64_t ldm, DevState* st, T* inv, cudaStream_t s);
// growth = max|U| / max|M| and info from the DevState (writes the caller's outputs).
rmge_status genp_finish(DevState* st, int32_t* info, double* growth, cudaStream_t s);
template <typename T>
rmge_status maxabs(int64_t rows, int64_t cols, const T* P, int64_t ldp, bool upper_only,
                   unsigned long long* out_bits, cudaStream_t s);

// trsv.cu: in-place triangular solves with the packed factors, nrhs columns, one launch each.
//   kind 0: L y = b (unit lower)      kind 1: U y = b (upper)
//   kind 2: U^T y = b (lower, diag U) kind 3: L^T y = b (unit upper)
// epoch: a value unique within the call and larger than every epoch used earlier in the call;
// ticket: a slot of st->tickets zeroed at call start, used once.  skip: as for gemm's halt.
template <typename T>
rmge_status trsv(int kind, int64_t n, int64_t nrhs, const T* LU, int64_t ldlu, T* B, int64_t ldb,
                 DevState* st, int* flags, int ticket, int epoch, const int* skip, cudaStream_t s);

// refine.cu
// Resets the control block, zeroes nflags solve flags and ncolred reduction slots, sets
// berr_out[0..nberr) to -1 (berr_out may be NULL).
rmge_status state_init(DevState* st, int* flags, int64_t nflags, double* colred, int ncolred, double* berr_out,
                       int nberr, cudaStream_t s);
// st->norm_a = ||A||_inf
rmge_status row_abs_sums(int64_t n, const double* A, int64_t lda, DevState* st, cudaStream_t s);
// R = B (copy, n x k)
template <typename Tin, typename Tout>
rmge_status copy_matrix(int64_t rows, int64_t cols, const Tin* src, int64_t lds, Tout* dst, int64_t ldd,
                        const int* skip, cudaStream_t s);
// X += D (FP64 X, D of type T), skipped when *skip != 0
template <typename T>
rmge_status add_update(int64_t rows, int64_t cols, const T* D, int64_t ldd, double* X, int64_t ldx,
                       const int* skip, cudaStream_t s);
// backward error of (R, X, B) into berr_out[sweep] and the stop test; see rmge_refine.
rmge_status backward_error(int64_t n, int64_t k, const double* R, int64_t ldr, const double* X, int64_t ldx,
                           const double* B, int64_t ldb, DevState* st, double* colred, int sweep,
                           double be_tol, int max_iters, double* berr_out, cudaStream_t s);
rmge_status refine_finish(DevState* st, int max_iters, double* berr_out, int32_t* iters, cudaStream_t s);
// dA = -dB X^T
rmge_status outer_neg(int64_t n, int64_t k, const double* dB, int64_t lddb, const double* X, int64_t ldx,
                      double* dA, int64_t ldda, cudaStream_t s);

// fft.cu: circulant multiplier (Theorem 5.1).  G = [c (n doubles) | u = F(c) (n double2)];
// tw: n/2 double2 of scratch for the twiddle table.
rmge_status circulant_spectrum(int64_t n, double* G, double2* tw, cudaStream_t s);
// M = A C (rows of A correlated with c), M in FP64 or FP32.
rmge_status circulant_apply_rows(int64_t n, const double* A, int64_t lda, const double* G, double2* tw, void* M,
                                 int64_t ldm, bool out_f32, cudaStream_t s);
// X (+)= C Y, or C^T Y when transpose, k columns, FP64; nothing when *skip != 0.
rmge_status circulant_apply_cols(int64_t n, int64_t k, const double* G, double2* tw, bool transpose,
                                 const double* Y, int64_t ldy, double* X, int64_t ldx, bool accumulate,
                                 const int* skip, cudaStream_t s);

}  // namespace rmge
