// fft.cu -- the circulant and Toeplitz multipliers applied by FFT (Sec. 5, Theorem 5.1).
//
// C = (c_{(i-j) mod n}) is diagonalised by the DFT: with F(x)_f = sum_t x_t w^{f t},
// w = exp(2 pi sqrt(-1) / n) (the matrix Omega of Sec. 5) and u = F(c):
//   C y  = F^{-1}( u       .* F(y) )   (circular convolution; recovery X = C Y, Fact 4.1)
//   y^T C -> row of A C, and C^T y = F^{-1}( conj(u) .* F(y) )   (circular cross-correlation)
// for real c.  Both maps send real vectors to real vectors and are C-linear, so two real vectors
// a, b travel together as z = a + sqrt(-1) b and come back as Re / Im of the result.
//
// One CTA per vector pair: the pair is staged in shared memory in bit-reversed order, transformed
// by a radix-2 decimation-in-time FFT (natural-order output), multiplied by the spectrum, and
// transformed back by a radix-2 decimation-in-frequency inverse FFT (bit-reversed output, read
// back through the same permutation).  Twiddles w^m, m < n/2, come from a table built once per
// call by twiddle_kernel.  n = 2^p, 2 <= n <= 8192 (the pair plus the table fit in shared memory).
// FP64 throughout; on GB300 this runs on the DFMA pipe (about 8 n log2 n FP64 operations per pair).
#include "kernels.cuh"

namespace rmge {
namespace {

constexpr int kFftThreads = 512;

__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
    return make_double2(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
}

__global__ void twiddle_kernel(int n, double2* tw) {
    for (int m = blockIdx.x * blockDim.x + threadIdx.x; m < n / 2; m += gridDim.x * blockDim.x) {
        double s, c;
        sincospi(2.0 * (double)m / (double)n, &s, &c);
        tw[m] = make_double2(c, s);
    }
}

// Forward DIT on x (bit-reversed input), sign +1: natural-order output.
__device__ void fft_dit(double2* x, const double2* tw, int n) {
    for (int len = 2; len <= n; len <<= 1) {
        const int half = len >> 1, step = n / len;
        for (int b = threadIdx.x; b < n / 2; b += blockDim.x) {
            const int grp = b / half, j = b % half;
            const int i0 = grp * len + j, i1 = i0 + half;
            const double2 w = tw[j * step];
            const double2 u = x[i0], v = cmul(x[i1], w);
            x[i0] = make_double2(u.x + v.x, u.y + v.y);
            x[i1] = make_double2(u.x - v.x, u.y - v.y);
        }
        __syncthreads();
    }
}

// Inverse DIF (sign -1, unscaled): natural-order input, bit-reversed output.
__device__ void ifft_dif(double2* x, const double2* tw, int n) {
    for (int len = n; len >= 2; len >>= 1) {
        const int half = len >> 1, step = n / len;
        for (int b = threadIdx.x; b < n / 2; b += blockDim.x) {
            const int grp = b / half, j = b % half;
            const int i0 = grp * len + j, i1 = i0 + half;
            const double2 w = tw[j * step];
            const double2 wc = make_double2(w.x, -w.y);
            const double2 u = x[i0], v = x[i1];
            x[i0] = make_double2(u.x + v.x, u.y + v.y);
            x[i1] = cmul(make_double2(u.x - v.x, u.y - v.y), wc);
        }
        __syncthreads();
    }
}

__device__ __forceinline__ int bitrev(int t, int logn) { return (int)(__brev((unsigned)t) >> (32 - logn)); }

// mode 0: spectrum only (G's DFT: out_spec = F(c)), one vector
// mode 1: filter: y -> F^{-1}(s .* F(y)) with s = u (conv) or conj(u) (corr)
// mode 2: inverse of a stored spectrum: dst = Re F^{-1}(spec), one vector (the first column of the
//         circulant whose spectrum was drawn)
// Vectors are rows (src[v*lds + t]) or columns (src[t*lds + v]) of length nin <= n, zero-padded to the
// transform length n; the first nout outputs are written (a Toeplitz multiplier is the leading block of
// a circulant of twice its size).
struct FftArgs {
    int n, logn, count, mode, nin, nout;
    bool cols, conj_spec, out_f32, accumulate;
    const double* src;
    int64_t lds;
    const double2* spec;
    const double2* tw;
    void* dst;
    int64_t ldd;
    double2* out_spec;
    const int* skip;
};

__global__ void __launch_bounds__(kFftThreads) fft_filter_kernel(FftArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    double2* x = reinterpret_cast<double2*>(smem_raw);
    double2* tw = x + a.n;
    if (a.skip != nullptr && *(volatile const int*)a.skip != 0) return;
    const int n = a.n;
    const int v0 = 2 * blockIdx.x;
    const bool has1 = v0 + 1 < a.count;
    for (int m = threadIdx.x; m < n / 2; m += blockDim.x) tw[m] = a.tw[m];
    if (a.mode == 2) {
        for (int t = threadIdx.x; t < n; t += blockDim.x) x[t] = a.spec[t];
        __syncthreads();
        ifft_dif(x, tw, n);
        double* d = static_cast<double*>(a.dst);
        for (int t = threadIdx.x; t < a.nout; t += blockDim.x) d[t] = x[bitrev(t, a.logn)].x / (double)n;
        return;
    }
    for (int t = threadIdx.x; t < n; t += blockDim.x) {
        double re = 0.0, im = 0.0;
        if (t < a.nin) {
            if (a.cols) {
                re = a.src[(int64_t)t * a.lds + v0];
                if (has1) im = a.src[(int64_t)t * a.lds + v0 + 1];
            } else {
                re = a.src[(int64_t)v0 * a.lds + t];
                if (has1) im = a.src[(int64_t)(v0 + 1) * a.lds + t];
            }
        }
        x[bitrev(t, a.logn)] = make_double2(re, im);
    }
    __syncthreads();
    fft_dit(x, tw, n);
    if (a.mode == 0) {
        for (int t = threadIdx.x; t < n; t += blockDim.x) a.out_spec[t] = x[t];
        return;
    }
    for (int t = threadIdx.x; t < n; t += blockDim.x) {
        double2 s = a.spec[t];
        if (a.conj_spec) s.y = -s.y;
        x[t] = cmul(x[t], s);
    }
    __syncthreads();
    ifft_dif(x, tw, n);
    const double scale = 1.0 / (double)n;
    for (int t = threadIdx.x; t < a.nout; t += blockDim.x) {
        const double2 w = x[bitrev(t, a.logn)];
        const double re = w.x * scale, im = w.y * scale;
        if (a.cols) {
            double* d = static_cast<double*>(a.dst);
            double* p0 = d + (int64_t)t * a.ldd + v0;
            *p0 = a.accumulate ? *p0 + re : re;
            if (has1) p0[1] = a.accumulate ? p0[1] + im : im;
        } else if (a.out_f32) {
            float* d = static_cast<float*>(a.dst);
            d[(int64_t)v0 * a.ldd + t] = (float)re;
            if (has1) d[(int64_t)(v0 + 1) * a.ldd + t] = (float)im;
        } else {
            double* d = static_cast<double*>(a.dst);
            d[(int64_t)v0 * a.ldd + t] = re;
            if (has1) d[(int64_t)(v0 + 1) * a.ldd + t] = im;
        }
    }
}

int ilog2(int64_t n) {
    int l = 0;
    while ((1LL << l) < n) ++l;
    return l;
}

rmge_status launch_fft(FftArgs a, int blocks, cudaStream_t s) {
    const size_t smem = (size_t)a.n * sizeof(double2) + (size_t)(a.n / 2) * sizeof(double2);
    if (cudaFuncSetAttribute(fft_filter_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) {
        (void)cudaGetLastError();
        return RMGE_ERR_CUDA;
    }
    fft_filter_kernel<<<blocks, kFftThreads, smem, s>>>(a);
    RMGE_LAUNCH_CHECK();
    return RMGE_OK;
}

}  // namespace

// G layout for the FFT kinds, with N the transform length (n for a circulant, 2n for a Toeplitz
// multiplier): c[0..N), then u = F(c) as N double2 (16-byte aligned because G is 256-byte aligned and N
// is even: offset 8N bytes).  tw: N/2 double2 of scratch.
rmge_status circulant_spectrum(int64_t N, double* G, double2* tw, cudaStream_t s) {
    twiddle_kernel<<<(unsigned)((N / 2 + 255) / 256), 256, 0, s>>>((int)N, tw);
    RMGE_LAUNCH_CHECK();
    FftArgs a{};
    a.n = (int)N;
    a.logn = ilog2(N);
    a.count = 1;
    a.mode = 0;
    a.nin = a.nout = (int)N;
    a.cols = false;
    a.src = G;
    a.lds = N;
    a.tw = tw;
    a.out_spec = reinterpret_cast<double2*>(G + N);
    return launch_fft(a, 1, s);
}

// c = Re F^{-1}(u) into G[0..N) from the spectrum already in G[N..3N) (Theorem 5.1: c = Omega^{-1} u).
// The twiddle table may live in G[0..N): the CTA reads it before writing c.
rmge_status circulant_from_spectrum(int64_t N, double* G, double2* tw, cudaStream_t s) {
    twiddle_kernel<<<(unsigned)((N / 2 + 255) / 256), 256, 0, s>>>((int)N, tw);
    RMGE_LAUNCH_CHECK();
    FftArgs a{};
    a.n = (int)N;
    a.logn = ilog2(N);
    a.count = 1;
    a.mode = 2;
    a.nin = a.nout = (int)N;
    a.spec = reinterpret_cast<const double2*>(G + N);
    a.tw = tw;
    a.dst = G;
    return launch_fft(a, 1, s);
}

rmge_status circulant_apply_rows(int64_t n, int64_t N, const double* A, int64_t lda, const double* G, double2* tw,
                                 void* M, int64_t ldm, bool out_f32, cudaStream_t s) {
    twiddle_kernel<<<(unsigned)((N / 2 + 255) / 256), 256, 0, s>>>((int)N, tw);
    RMGE_LAUNCH_CHECK();
    FftArgs a{};
    a.n = (int)N;
    a.logn = ilog2(N);
    a.count = (int)n;
    a.mode = 1;
    a.nin = a.nout = (int)n;
    a.cols = false;
    a.conj_spec = true;  // row of A C = cross-correlation of the row with c
    a.out_f32 = out_f32;
    a.src = A;
    a.lds = lda;
    a.spec = reinterpret_cast<const double2*>(G + N);
    a.tw = tw;
    a.dst = M;
    a.ldd = ldm;
    return launch_fft(a, (int)((n + 1) / 2), s);
}

rmge_status circulant_apply_rows_block(int64_t rows, int64_t n, int64_t nout, const double* A, int64_t lda,
                                       const double* G, double2* tw, double* M, int64_t ldm, cudaStream_t s) {
    twiddle_kernel<<<(unsigned)((n / 2 + 255) / 256), 256, 0, s>>>((int)n, tw);
    RMGE_LAUNCH_CHECK();
    FftArgs a{};
    a.n = (int)n;
    a.logn = ilog2(n);
    a.count = (int)rows;
    a.mode = 1;
    a.nin = (int)n;
    a.nout = (int)nout;
    a.cols = false;
    a.conj_spec = true;  // row of A C = cross-correlation of the row with c
    a.src = A;
    a.lds = lda;
    a.spec = reinterpret_cast<const double2*>(G + n);
    a.tw = tw;
    a.dst = M;
    a.ldd = ldm;
    return launch_fft(a, (int)((rows + 1) / 2), s);
}

rmge_status circulant_apply_cols(int64_t n, int64_t N, int64_t k, const double* G, double2* tw, bool transpose,
                                 const double* Y, int64_t ldy, double* X, int64_t ldx, bool accumulate, const int* skip,
                                 cudaStream_t s) {
    twiddle_kernel<<<(unsigned)((N / 2 + 255) / 256), 256, 0, s>>>((int)N, tw);
    RMGE_LAUNCH_CHECK();
    FftArgs a{};
    a.n = (int)N;
    a.logn = ilog2(N);
    a.count = (int)k;
    a.mode = 1;
    a.nin = a.nout = (int)n;
    a.cols = true;
    a.conj_spec = transpose;  // C y: convolution; C^T y: correlation
    a.out_f32 = false;
    a.accumulate = accumulate;
    a.src = Y;
    a.lds = ldy;
    a.spec = reinterpret_cast<const double2*>(G + N);
    a.tw = tw;
    a.dst = X;
    a.ldd = ldx;
    a.skip = skip;
    return launch_fft(a, (int)((k + 1) / 2), s);
}

}  // namespace rmge
