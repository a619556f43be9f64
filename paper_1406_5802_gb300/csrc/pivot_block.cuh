// pivot_block.cuh -- unblocked GENP of one pivot block held in shared memory (eq. (3.1) with 1 x 1
// pivots inside the block), shared by the standalone pivot-block kernel (genp.cu) and the Schur-update
// kernel that factors the next pivot block while the other CTAs finish the update (oz_gemm.cu).
//
// GB300 retires 2 FP64 operations per clock per SM, so every lane of every FP64 instruction is kept
// busy: step s scales column s of L by the reciprocal of the pivot (one division per step, formed by the
// thread that finishes the pivot in the previous step), then the (b-s-1)^2 trailing entries are spread
// evenly over the NT threads, the entry index e split into (row, column) by a multiply-shift reciprocal
// of the width, exact for e < 2^20 / w (here e < 63^2).
#pragma once

namespace rmge {

constexpr int kPivotLds = 65;  // padded row of the 64 x 64 pivot block in shared memory

// a: b x b block (b <= 64, row stride LDS, kPivotLds unless the caller's scratch is tighter) in shared
// memory; rp: one shared value; sync(): a barrier over exactly the NT participating threads, tid in
// [0, NT).  Returns 0, or the 1-based step of the first zero or non-finite pivot (Cor. 3.1); a is then
// left as it was before that step.
template <typename T, int NT, typename Sync, int LDS = kPivotLds>
__device__ int pivot_block_genp(T* a, int b, T* rp, int tid, Sync sync) {
    if (tid == 0) *rp = T(1) / a[0];
    sync();
    for (int s = 0; s < b; ++s) {
        const T piv = a[s * LDS + s];
        if (!(piv != T(0) && isfinite(piv))) return s + 1;  // uniform: every thread read the same pivot
        const int w = b - s - 1;
        if (w == 0) break;
        const T r = *rp;
        if (tid < w) a[(s + 1 + tid) * LDS + s] *= r;  // column s of L
        sync();
        const unsigned mw = ((1u << 20) + (unsigned)w - 1u) / (unsigned)w;
        const T* us = a + s * LDS + s + 1;
        for (int e = tid; e < w * w; e += NT) {
            const int ii = (int)(((unsigned)e * mw) >> 20), jj = e - ii * w;
            T* dst = a + (s + 1 + ii) * LDS + s + 1 + jj;
            const T v = fma(-a[(s + 1 + ii) * LDS + s], us[jj], *dst);
            *dst = v;
            if (ii == 0 && jj == 0) *rp = T(1) / v;  // the next pivot is final now
        }
        sync();
    }
    return 0;
}

}  // namespace rmge
