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

__global__ void gaussian_kernel(int64_t count, uint64_t seed, uint64_t subseq, double* __restrict__ out) {
    const int64_t pairs = (count + 1) / 2;
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < pairs;
         p += (int64_t)gridDim.x * blockDim.x) {
        const U4 x = block_for((uint64_t)p, seed, subseq);
        const double u1 = (double)(join53(x.x, x.y) + 1) * 0x1p-53;
        const double u2 = (double)join53(x.z, x.w) * 0x1p-53;
        const double r = sqrt(-2.0 * log(u1));
        double sn, cs;
        sincospi(2.0 * u2, &sn, &cs);
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
