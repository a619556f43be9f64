// fft.cu -- the circulant and Toeplitz multipliers applied by FFT (Sec. 5, Theorem 5.1).
//
// C = (c_{(i-j) mod n}) is diagonalised by the DFT: with F(x)_f = sum_t x_t w^{f t},
// w = exp(2 pi sqrt(-1) / n) (the matrix Omega of Sec. 5) and u = F(c):
//   C y  = F^{-1}( u       .* F(y) )   (circular convolution; recovery X = C Y, Fact 4.1)
//   y^T C -> row of A C, and C^T y = F^{-1}( conj(u) .* F(y) )   (circular cross-correlation)
// for real c.  Both maps send real vectors to real vectors, so each spectrum is Hermitian and only its
// bins 0 .. N / 2 are formed.
//
// One CTA per real vector x of length N, transformed as the complex vector z_s = x_{2s} + sqrt(-1) x_{2s+1}
// of half the length h = N / 2 (the standard packing of a real transform): z is staged in shared memory in
// bit-reversed order and transformed by a radix-2 decimation-in-time FFT (natural-order output).  The
// spectrum of x follows from Z by X_f = E_f + w^f O_f with E_f = (Z_f + conj Z_{h-f}) / 2 and
// O_f = (Z_f - conj Z_{h-f}) / (2 sqrt(-1)), one thread per pair (f, h - f).  After the product with the
// filter spectrum, the same pairing packs the Hermitian result back into a length-h complex vector
// (E'_f + sqrt(-1) O'_f with E'_f = Y_f + conj Y_{h-f} and O'_f = (Y_f - conj Y_{h-f}) conj(w^f)),
// which a radix-2 decimation-in-frequency inverse FFT (bit-reversed output) turns into the even and odd
// outputs.  Twiddles come from a quarter table w^m, 0 <= m <= N / 4 (w^{m + N/4} = sqrt(-1) w^m), built
// once per call by twiddle_kernel and staged in shared memory beside z: 12 N + 16 bytes in all, so
// N = 2^p with 4 <= N <= 16384.  FP64 throughout; on GB300 this runs on the DFMA pipe (about
// 5 N log2 N FP64 operations per vector and direction).
#include "kernels.cuh"

namespace rmge {
namespace {

__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
    return make_double2(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
}

__device__ __forceinline__ double2 cconj(double2 a) { return make_double2(a.x, -a.y); }

// w^m = exp(2 pi sqrt(-1) m / N) for 0 <= m <= N / 2 from the quarter table T[0..q], q = N / 4.
__device__ __forceinline__ double2 twid(const double2* T, int m, int q) {
    if (m <= q) return T[m];
    const double2 t = T[m - q];
    return make_double2(-t.y, t.x);
}

__global__ void twiddle_kernel(int N, double2* tw) {
    for (int m = blockIdx.x * blockDim.x + threadIdx.x; m <= N / 4; m += gridDim.x * blockDim.x) {
        double s, c;
        sincospi(2.0 * (double)m / (double)N, &s, &c);
        tw[m] = make_double2(c, s);
    }
}

// Forward DIT of length h (sign +1, w_h^j = w_N^{2j}) on x in bit-reversed order: natural-order output.
__device__ void fft_dit(double2* x, const double2* T, int h, int q) {
    for (int len = 2; len <= h; len <<= 1) {
        const int half = len >> 1, step = h / len;
        for (int b = threadIdx.x; b < h / 2; b += blockDim.x) {
            const int grp = b / half, j = b % half;
            const int i0 = grp * len + j, i1 = i0 + half;
            const double2 w = twid(T, 2 * j * step, q);
            const double2 u = x[i0], v = cmul(x[i1], w);
            x[i0] = make_double2(u.x + v.x, u.y + v.y);
            x[i1] = make_double2(u.x - v.x, u.y - v.y);
        }
        __syncthreads();
    }
}

// Inverse DIF of length h (sign -1, unscaled): natural-order input, bit-reversed output.
__device__ void ifft_dif(double2* x, const double2* T, int h, int q) {
    for (int len = h; len >= 2; len >>= 1) {
        const int half = len >> 1, step = h / len;
        for (int b = threadIdx.x; b < h / 2; b += blockDim.x) {
            const int grp = b / half, j = b % half;
            const int i0 = grp * len + j, i1 = i0 + half;
            const double2 w = cconj(twid(T, 2 * j * step, q));
            const double2 u = x[i0], v = x[i1];
            x[i0] = make_double2(u.x + v.x, u.y + v.y);
            x[i1] = cmul(make_double2(u.x - v.x, u.y - v.y), w);
        }
        __syncthreads();
    }
}

__device__ __forceinline__ int bitrev(int t, int logh) {
    return logh == 0 ? 0 : (int)(__brev((unsigned)t) >> (32 - logh));
}

// X_f of the real vector from Z_f and Z_{h-f} of its half-length packing (w = w^f).
__device__ __forceinline__ double2 unpack_bin(double2 zf, double2 zg, double2 w) {
    const double2 e = make_double2(0.5 * (zf.x + zg.x), 0.5 * (zf.y - zg.y));
    const double2 o = make_double2(0.5 * (zf.y + zg.y), -0.5 * (zf.x - zg.x));
    const double2 wo = cmul(w, o);
    return make_double2(e.x + wo.x, e.y + wo.y);
}

// Twice the half-length packing of bin f of a Hermitian spectrum from Y_f and Y_{h-f} (w = w^f).
__device__ __forceinline__ double2 pack_bin(double2 yf, double2 yg, double2 w) {
    const double2 s = make_double2(yf.x + yg.x, yf.y - yg.y);
    const double2 d = cmul(make_double2(yf.x - yg.x, yf.y + yg.y), cconj(w));
    return make_double2(s.x - d.y, s.y + d.x);
}

// mode 0: spectrum only (G's DFT: out_spec = F(c)), one vector
// mode 1: filter: y -> F^{-1}(s .* F(y)) with s = u (conv) or conj(u) (corr)
// mode 2: inverse of a stored Hermitian spectrum: dst = F^{-1}(spec), one vector (the first column of the
//         circulant whose spectrum was drawn)
// Vectors are rows (src[v*lds + t]) or columns (src[t*lds + v]) of length nin <= N, zero-padded to the
// transform length N; the first nout outputs are written (a Toeplitz multiplier is the leading block of
// a circulant of twice its size).
struct FftArgs {
    int n, logh, count, mode, nin, nout;
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

__global__ void __launch_bounds__(1024) fft_filter_kernel(FftArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int N = a.n, h = N / 2, q = N / 4;
    double2* z = reinterpret_cast<double2*>(smem_raw);
    double2* T = z + h;
    if (a.skip != nullptr && *(volatile const int*)a.skip != 0) return;
    const int v = blockIdx.x;
    for (int m = threadIdx.x; m <= q; m += blockDim.x) T[m] = a.tw[m];
    if (a.mode != 2) {
        for (int s = threadIdx.x; s < h; s += blockDim.x) {
            const int t0 = 2 * s, t1 = 2 * s + 1;
            double re = 0.0, im = 0.0;
            if (a.cols) {
                if (t0 < a.nin) re = a.src[(int64_t)t0 * a.lds + v];
                if (t1 < a.nin) im = a.src[(int64_t)t1 * a.lds + v];
            } else {
                const double* row = a.src + (int64_t)v * a.lds;
                if (t0 < a.nin) re = row[t0];
                if (t1 < a.nin) im = row[t1];
            }
            z[bitrev(s, a.logh)] = make_double2(re, im);
        }
        __syncthreads();
        fft_dit(z, T, h, q);
    } else {
        __syncthreads();  // the table is staged before anything is written (it may share the output's memory)
    }
    // pairs (f, h - f), f = 0 .. h / 2; bin h pairs with bin 0 (Z_h = Z_0) and has no packed slot of its own
    for (int f = threadIdx.x; f <= h / 2; f += blockDim.x) {
        const int g = h - f;
        const double2 wf = twid(T, f, q), wg = twid(T, g, q);
        double2 yf, yg;
        if (a.mode == 2) {
            yf = a.spec[f];
            yg = a.spec[g];
        } else {
            const double2 zf = z[f], zg = z[g == h ? 0 : g];
            const double2 xf = unpack_bin(zf, zg, wf), xg = unpack_bin(zg, zf, wg);
            if (a.mode == 0) {
                a.out_spec[f] = xf;
                a.out_spec[g] = xg;
                if (f > 0) a.out_spec[N - f] = cconj(xf);
                if (g < h && g != f) a.out_spec[N - g] = cconj(xg);
                continue;
            }
            double2 sf = a.spec[f], sg = a.spec[g];
            if (a.conj_spec) {
                sf.y = -sf.y;
                sg.y = -sg.y;
            }
            yf = cmul(xf, sf);
            yg = cmul(xg, sg);
        }
        z[f] = pack_bin(yf, yg, wf);
        if (g < h && g != f) z[g] = pack_bin(yg, yf, wg);
    }
    if (a.mode == 0) return;
    __syncthreads();
    ifft_dif(z, T, h, q);
    const double scale = 1.0 / (double)N;
    for (int s = threadIdx.x; s < h; s += blockDim.x) {
        const int t0 = 2 * s, t1 = 2 * s + 1;
        if (t0 >= a.nout) continue;
        const double2 w = z[bitrev(s, a.logh)];
        const double re = w.x * scale, im = w.y * scale;
        const bool has1 = t1 < a.nout;
        if (a.mode == 2) {
            double* d = static_cast<double*>(a.dst);
            d[t0] = re;
            if (has1) d[t1] = im;
        } else if (a.cols) {
            double* d = static_cast<double*>(a.dst);
            double* p0 = d + (int64_t)t0 * a.ldd + v;
            double* p1 = d + (int64_t)t1 * a.ldd + v;
            *p0 = a.accumulate ? *p0 + re : re;
            if (has1) *p1 = a.accumulate ? *p1 + im : im;
        } else if (a.out_f32) {
            float* d = static_cast<float*>(a.dst) + (int64_t)v * a.ldd;
            d[t0] = (float)re;
            if (has1) d[t1] = (float)im;
        } else {
            double* d = static_cast<double*>(a.dst) + (int64_t)v * a.ldd;
            d[t0] = re;
            if (has1) d[t1] = im;
        }
    }
}

int ilog2(int64_t n) {
    int l = 0;
    while ((1LL << l) < n) ++l;
    return l;
}

// One CTA per vector (a.count of them): 12 N + 16 bytes of shared memory, 1024 threads at N = 16384 (one CTA
// per SM), 512 below.
rmge_status launch_fft(FftArgs a, cudaStream_t s) {
    a.logh = ilog2(a.n) - 1;
    const size_t smem = (size_t)(a.n / 2 + a.n / 4 + 1) * sizeof(double2);
    if (cudaFuncSetAttribute(fft_filter_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) {
        (void)cudaGetLastError();
        return RMGE_ERR_CUDA;
    }
    const int threads = a.n >= 16384 ? 1024 : 512;
    fft_filter_kernel<<<a.count, threads, smem, s>>>(a);
    RMGE_LAUNCH_CHECK();
    return RMGE_OK;
}

rmge_status launch_twiddles(int64_t N, double2* tw, cudaStream_t s) {
    twiddle_kernel<<<(unsigned)((N / 4 + 256) / 256), 256, 0, s>>>((int)N, tw);
    RMGE_LAUNCH_CHECK();
    return RMGE_OK;
}

}  // namespace

// G layout for the FFT kinds, with N the transform length (n for a circulant, 2n for a Toeplitz
// multiplier): c[0..N), then u = F(c) as N double2 (16-byte aligned because G is 256-byte aligned and N
// is even: offset 8N bytes).  tw: N/4 + 1 double2 of scratch (the quarter twiddle table).
rmge_status circulant_spectrum(int64_t N, double* G, double2* tw, cudaStream_t s) {
    RMGE_TRY(launch_twiddles(N, tw, s));
    FftArgs a{};
    a.n = (int)N;
    a.count = 1;
    a.mode = 0;
    a.nin = a.nout = (int)N;
    a.cols = false;
    a.src = G;
    a.lds = N;
    a.tw = tw;
    a.out_spec = reinterpret_cast<double2*>(G + N);
    return launch_fft(a, s);
}

// c = Re F^{-1}(u) into G[0..N) from the spectrum already in G[N..3N) (Theorem 5.1: c = Omega^{-1} u).
// The twiddle table may live in G[0..N): the CTA reads it before writing c.
rmge_status circulant_from_spectrum(int64_t N, double* G, double2* tw, cudaStream_t s) {
    RMGE_TRY(launch_twiddles(N, tw, s));
    FftArgs a{};
    a.n = (int)N;
    a.count = 1;
    a.mode = 2;
    a.nin = a.nout = (int)N;
    a.spec = reinterpret_cast<const double2*>(G + N);
    a.tw = tw;
    a.dst = G;
    return launch_fft(a, s);
}

rmge_status circulant_apply_rows(int64_t n, int64_t N, const double* A, int64_t lda, const double* G, double2* tw,
                                 void* M, int64_t ldm, bool out_f32, cudaStream_t s) {
    RMGE_TRY(launch_twiddles(N, tw, s));
    FftArgs a{};
    a.n = (int)N;
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
    return launch_fft(a, s);
}

rmge_status circulant_apply_rows_block(int64_t rows, int64_t n, int64_t nout, const double* A, int64_t lda,
                                       const double* G, double2* tw, double* M, int64_t ldm, cudaStream_t s) {
    RMGE_TRY(launch_twiddles(n, tw, s));
    FftArgs a{};
    a.n = (int)n;
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
    return launch_fft(a, s);
}

rmge_status circulant_apply_cols(int64_t n, int64_t N, int64_t k, const double* G, double2* tw, bool transpose,
                                 const double* Y, int64_t ldy, double* X, int64_t ldx, bool accumulate, const int* skip,
                                 cudaStream_t s) {
    RMGE_TRY(launch_twiddles(N, tw, s));
    FftArgs a{};
    a.n = (int)N;
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
    return launch_fft(a, s);
}

}  // namespace rmge
