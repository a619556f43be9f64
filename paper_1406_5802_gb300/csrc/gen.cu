// gen.cu -- random multiplier draws (Def. 4.1 Gaussian entries, Ex. 5.1 uniform entries, Ex. 5.2 unit
// spectra of unitary circulants).
//
// Counter-based Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): a 128-bit counter and a
// 64-bit key pass through ten rounds, each two 32x32 multiplies (published multipliers) whose
// high and low halves are permuted and xor-ed with the key; the key advances by the published
// Weyl increments between rounds.  Every output depends only on (counter, key), so each thread
// draws its own entries with no shared state and the stream is identical for any launch shape.
//
// Stream layout: entries e = 2p and 2p+1 come from counter (p_lo, p_hi, sub_lo, sub_hi) and key
// (seed_lo, seed_hi); the four 32-bit outputs x0..x3 form two 53-bit integers
// m1 = x0:x1[31:11], m2 = x2:x3[31:11].
//   Gaussian (Box-Muller): r = sqrt(-2 ln((m1+1) 2^-53)), entries r cos(2 pi m2 2^-53) and
//   r sin(2 pi m2 2^-53).
//   Uniform on [-1, 1): entries 2 m1 2^-53 - 1 and 2 m2 2^-53 - 1 (exact in FP64).
//   FP32 Gaussian (multipliers of the reduced-precision paths): the same Box-Muller pair in FP32
//   arithmetic on 24-bit uniforms: u1 = ((x0 >> 8) + 1) 2^-24, u2 = (x2 >> 8) 2^-24.
#include "kernels.cuh"
#include "box_muller_tables.cuh"

namespace rmge {
namespace {

struct U4 {
    uint32_t x, y, z, w;
};

__device__ __forceinline__ U4 philox10(U4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t a = c.x, b = c.z;
        const uint32_t hi_a = __umulhi(0xD2511F53u, a), lo_a = 0xD2511F53u * a;
        const uint32_t hi_b = __umulhi(0xCD9E8D57u, b), lo_b = 0xCD9E8D57u * b;
        c = U4{hi_b ^ c.y ^ k0, lo_b, hi_a ^ c.w ^ k1, lo_a};
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return c;
}

__device__ __forceinline__ U4 block_for(uint64_t p, uint64_t seed, uint64_t subseq) {
    return philox10(U4{(uint32_t)p, (uint32_t)(p >> 32), (uint32_t)subseq, (uint32_t)(subseq >> 32)},
                    (uint32_t)seed, (uint32_t)(seed >> 32));
}

__device__ __forceinline__ uint64_t join53(uint32_t hi, uint32_t lo) {
    return ((uint64_t)hi << 21) | (uint64_t)(lo >> 11);
}

// ln((m1 + 1) 2^-53) by the table-driven method of Tang (ACM TOMS 16(4), 1990), mostly in integer
// operations: x = m1 + 1 = f 2^p with f in [1, 2); F_j = 1 + j/256 is the table point nearest f (j = 256,
// that is F = 2, moves to the next binade as F = 1, so that u1 near 1 keeps its full relative accuracy);
// g = f - F_j is exact, t = g / F_j, and ln(1 + t) for |t| <= 2^-9 is its Taylor series to t^6 (the first
// term left out is below 2^-63).  (p - 53) ln 2 + ln F_j take the split constants of the table, whose
// high parts add exactly.
__device__ __forceinline__ double ln_uniform53(uint64_t m1, const double (*lt)[3]) {
    const uint64_t x = m1 + 1;  // 1 .. 2^53
    const int lz = __clzll((long long)x);
    const uint64_t mant = ((x << lz) >> 11) & 0xFFFFFFFFFFFFFull;  // exact: x has at most 53 significant bits
    uint64_t j = (mant + (1ull << 43)) >> 44;                       // nearest of the 256ths, 0 .. 256
    const double f = __longlong_as_double((long long)((1023ull << 52) | mant));
    double g = f - __longlong_as_double((long long)((1023ull << 52) + (j << 44)));  // exact (Sterbenz)
    int e = 63 - lz - 53;
    if (j == 256) {
        g *= 0.5;
        j = 0;
        ++e;
    }
    const double t = g * lt[j][0];
    const double q = fma(t, fma(t, fma(t, fma(t, -1.0 / 6, 0.2), -0.25), 1.0 / 3), -0.5);
    const double poly = fma(t, t * q, t);  // t + t^2 (-1/2 + t/3 - t^2/4 + t^3/5 - t^4/6)
    const double ed = (double)e;
    return fma(ed, bm::kLn2Hi, lt[j][1]) + (fma(ed, bm::kLn2Lo, lt[j][2]) + poly);
}

// cos and sin of 2 pi m2 2^-53: k = the nearest 256th of the turn, phi = 2 pi (m2 2^-53 - k/256) with
// |phi| <= pi / 256; cos phi = 1 - c2 and sin phi from their Taylor series (first terms left out below
// 1e-17), then the addition theorems with the tabulated cos, sin of 2 pi k / 256.
__device__ __forceinline__ void sincos_turn53(uint64_t m2, const double (*sc)[2], double* s, double* c) {
    const uint64_t k = (m2 + (1ull << 44)) >> 45;  // 0 .. 256
    const double phi = (double)((long long)m2 - (long long)(k << 45)) * bm::kTwoPi53;
    const double z = phi * phi;
    const double sp = fma(phi * z, fma(z, 1.0 / 120, -1.0 / 6), phi);
    const double c2 = z * fma(z, fma(z, 1.0 / 720, -1.0 / 24), 0.5);
    const double ck = sc[k & 255][0], sk = sc[k & 255][1];
    *c = ck - fma(ck, c2, sk * sp);
    *s = sk + fma(ck, sp, -sk * c2);
}

__global__ void gaussian_kernel(int64_t count, uint64_t seed, uint64_t subseq, double* __restrict__ out) {
    __shared__ double lt[256][3];
    __shared__ double sc[256][2];
    for (int i = threadIdx.x; i < 256; i += blockDim.x) {
        lt[i][0] = bm::kLogTable[i][0];
        lt[i][1] = bm::kLogTable[i][1];
        lt[i][2] = bm::kLogTable[i][2];
        sc[i][0] = bm::kSinCosTable[i][0];
        sc[i][1] = bm::kSinCosTable[i][1];
    }
    __syncthreads();
    const int64_t pairs = (count + 1) / 2;
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < pairs;
         p += (int64_t)gridDim.x * blockDim.x) {
        const U4 x = block_for((uint64_t)p, seed, subseq);
        const double r = sqrt(-2.0 * ln_uniform53(join53(x.x, x.y), lt));
        double sn, cs;
        sincos_turn53(join53(x.z, x.w), sc, &sn, &cs);
        out[2 * p] = r * cs;
        if (2 * p + 1 < count) out[2 * p + 1] = r * sn;
    }
}

__global__ void gaussian_f32_kernel(int64_t count, uint64_t seed, uint64_t subseq, float* __restrict__ out) {
    const int64_t pairs = (count + 1) / 2;
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < pairs;
         p += (int64_t)gridDim.x * blockDim.x) {
        const U4 x = block_for((uint64_t)p, seed, subseq);
        const float u1 = (float)((x.x >> 8) + 1u) * 0x1p-24f;
        const float u2 = (float)(x.z >> 8) * 0x1p-24f;
        const float r = sqrtf(-2.0f * logf(u1));
        float sn, cs;
        sincospif(2.0f * u2, &sn, &cs);
        out[2 * p] = r * cs;
        if (2 * p + 1 < count) out[2 * p + 1] = r * sn;
    }
}

__global__ void uniform_pm1_kernel(int64_t count, uint64_t seed, uint64_t subseq, double* __restrict__ out) {
    const int64_t pairs = (count + 1) / 2;
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < pairs;
         p += (int64_t)gridDim.x * blockDim.x) {
        const U4 x = block_for((uint64_t)p, seed, subseq);
        out[2 * p] = 2.0 * ((double)join53(x.x, x.y) * 0x1p-53) - 1.0;
        if (2 * p + 1 < count) out[2 * p + 1] = 2.0 * ((double)join53(x.z, x.w) * 0x1p-53) - 1.0;
    }
}

// Spectrum of a random unitary circulant of size N (Ex. 5.2): phases phi_j = m_j 2^-53 in [0, 1) are
// entries j = 0 .. N/2 of the same stream (even entries from x0:x1, odd ones from x2:x3 of block j/2);
// u_j = exp(2 pi phi_j sqrt(-1)) and u_{N-j} = conj(u_j) for 0 < j < N/2, while u_0 and u_{N/2} are
// +1 if phi < 1/2 else -1.  The Hermitian symmetry makes the circulant real (and orthogonal).
__global__ void unitary_spectrum_kernel(int64_t N, uint64_t seed, uint64_t subseq, double2* __restrict__ u) {
    const int64_t h = N / 2;
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j <= h; j += (int64_t)gridDim.x * blockDim.x) {
        const U4 x = block_for((uint64_t)(j / 2), seed, subseq);
        const uint64_t m = (j & 1) ? join53(x.z, x.w) : join53(x.x, x.y);
        const double phi = (double)m * 0x1p-53;
        if (j == 0 || j == h) {
            u[j] = make_double2(phi < 0.5 ? 1.0 : -1.0, 0.0);
        } else {
            double sn, cs;
            sincospi(2.0 * phi, &sn, &cs);
            u[j] = make_double2(cs, sn);
            u[N - j] = make_double2(cs, -sn);
        }
    }
}

int grid_for(int64_t pairs, int threads) {
    int64_t g = (pairs + threads - 1) / threads;
    const int64_t cap = 152 * 16;  // grid-stride beyond 16 blocks per SM
    if (g > cap) g = cap;
    return (int)(g < 1 ? 1 : g);
}

}  // namespace

rmge_status launch_gaussian(int64_t count, uint64_t seed, uint64_t subseq, double* out, cudaStream_t s) {
    const int64_t pairs = (count + 1) / 2;
    gaussian_kernel<<<grid_for(pairs, 256), 256, 0, s>>>(count, seed, subseq, out);
    RMGE_LAUNCH_CHECK();
    return RMGE_OK;
}

rmge_status launch_gaussian(int64_t count, uint64_t seed, uint64_t subseq, float* out, cudaStream_t s) {
    const int64_t pairs = (count + 1) / 2;
    gaussian_f32_kernel<<<grid_for(pairs, 256), 256, 0, s>>>(count, seed, subseq, out);
    RMGE_LAUNCH_CHECK();
    return RMGE_OK;
}

rmge_status launch_unitary_spectrum(int64_t N, uint64_t seed, uint64_t subseq, double2* u, cudaStream_t s) {
    unitary_spectrum_kernel<<<grid_for(N / 2 + 1, 256), 256, 0, s>>>(N, seed, subseq, u);
    RMGE_LAUNCH_CHECK();
    return RMGE_OK;
}

rmge_status launch_uniform_pm1(int64_t count, uint64_t seed, uint64_t subseq, double* out, cudaStream_t s) {
    const int64_t pairs = (count + 1) / 2;
    uniform_pm1_kernel<<<grid_for(pairs, 256), 256, 0, s>>>(count, seed, subseq, out);
    RMGE_LAUNCH_CHECK();
    return RMGE_OK;
}

}  // namespace rmge
