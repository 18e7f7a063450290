// md_corr.cuh -- device side of the blocking scheme for time-correlation
// functions (Sec. 2.5): the tagged-particle mean-square displacement and the
// self intermediate scattering function F_s(q, t) between one origin snapshot
// and up to kCorrMaxJ later snapshots of the same block.
//
// Snapshots hold unwrapped positions in FP64 by original particle index.
// Per particle i of species a and per later snapshot j: d = r_j - r_0 (FP64),
// |d|^2 (FP64) and the average over the n_q wavevectors of cos(q . d) (phase in
// FP64, cosine in FP32).  Sums per block of 256 particles go to a partial array;
// k_corr_reduce adds the partials in block order into the accumulator of the
// block level (deterministic).
#pragma once

#include <cuda_runtime.h>

namespace mdk {

constexpr int kCorrMaxJ = 31;      // at most 32 entries per block level
constexpr int kCorrMaxQ = 64;
constexpr int kCorrBlock = 256;

struct CorrArgs {
    const double *s0;               // origin snapshot [n][3]
    const double *sj[kCorrMaxJ];    // later snapshots
    int nj, n, nq;
    const int *species;             // [n] by original index
    const double *q;                // [nq][3]
    double *part;                   // [nblocks][nj][4]: (msd A, fs A, msd B, fs B)
    double *acc;                    // [nj][4] accumulator of this block level
    int nblocks;
};

__global__ void __launch_bounds__(kCorrBlock) k_corr(CorrArgs c)
{
    __shared__ double sh[kCorrBlock / 32][4];
    __shared__ double sq[kCorrMaxQ * 3];
    for (int t = threadIdx.x; t < 3 * c.nq; t += blockDim.x)
        sq[t] = c.q[t];
    __syncthreads();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const bool valid = i < c.n;
    double x0 = 0.0, y0 = 0.0, z0 = 0.0;
    int sp = 0;
    if (valid) {
        x0 = c.s0[3 * (size_t)i];
        y0 = c.s0[3 * (size_t)i + 1];
        z0 = c.s0[3 * (size_t)i + 2];
        sp = c.species[i];
    }
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int j = 0; j < c.nj; ++j) {
        double v[4] = {0.0, 0.0, 0.0, 0.0};
        if (valid) {
            const double *s = c.sj[j] + 3 * (size_t)i;
            const double dx = s[0] - x0, dy = s[1] - y0, dz = s[2] - z0;
            float cs = 0.0f;
            for (int k = 0; k < c.nq; ++k) {
                const double ph = sq[3 * k] * dx + sq[3 * k + 1] * dy + sq[3 * k + 2] * dz;
                cs += cosf((float)ph);
            }
            const double msd = dx * dx + dy * dy + dz * dz;
            const double fs = (double)cs / (double)c.nq;
            v[2 * sp] = msd;
            v[2 * sp + 1] = fs;
        }
#pragma unroll
        for (int k = 0; k < 4; ++k)
#pragma unroll
            for (int o = 16; o > 0; o >>= 1)
                v[k] += __shfl_xor_sync(0xffffffffu, v[k], o);
        if (lane == 0)
#pragma unroll
            for (int k = 0; k < 4; ++k)
                sh[w][k] = v[k];
        __syncthreads();
        if (threadIdx.x < 4) {
            double t = 0.0;
            for (int u = 0; u < kCorrBlock / 32; ++u)
                t += sh[u][threadIdx.x];
            c.part[((size_t)blockIdx.x * c.nj + j) * 4 + threadIdx.x] = t;
        }
        __syncthreads();
    }
}

__global__ void k_corr_reduce(CorrArgs c)
{
    for (int t = threadIdx.x; t < 4 * c.nj; t += blockDim.x) {
        double s = 0.0;
        for (int b = 0; b < c.nblocks; ++b)
            s += c.part[(size_t)b * c.nj * 4 + t];
        c.acc[t] += s;
    }
}

}  // namespace mdk
