// kernels_esdf.cu -- per-voxel brute-force ESDF of a union of axis-aligned cuboids.
//
// One thread per voxel; the cuboids stream through shared memory in chunks, so
// every box is read from global memory once per block.  For each voxel centre
// p the kernel keeps, over all boxes, the smallest squared outside distance
// |max(|p - c| - h, 0)|^2 and the smallest max_i(|p - c|_i - h_i).  If the
// latter is <= 0 some box contains p and it is the union's signed distance (the
// deepest-penetration reading of min_k sdf_k); otherwise min_k sdf_k is the
// square root of the former.  Both equal min_k sdf_k exactly.
#include <cuda_runtime.h>
#include <math_constants.h>

#include "internal.h"

namespace dseed {

constexpr int kEsdfThreads = 256;
constexpr int kEsdfChunk = 256;

__global__ void __launch_bounds__(kEsdfThreads)
    k_esdf_build(const float *__restrict__ cub, int n, DseedGrid g, long long nvox, float *__restrict__ phi) {
    __shared__ float sb[kEsdfChunk * 6];
    const long long v = (long long)blockIdx.x * kEsdfThreads + threadIdx.x;
    const bool live = v < nvox;
    const long long nxy = (long long)g.nx * g.ny;
    const int k = live ? (int)(v / nxy) : 0;
    const long long r = live ? v - (long long)k * nxy : 0;
    const int j = (int)(r / g.nx), i = (int)(r - (long long)j * g.nx);
    const float px = fmaf((float)i + 0.5f, g.res, g.origin[0]);
    const float py = fmaf((float)j + 0.5f, g.res, g.origin[1]);
    const float pz = fmaf((float)k + 0.5f, g.res, g.origin[2]);
    float out2 = CUDART_INF_F, in = CUDART_INF_F;
    for (int c0 = 0; c0 < n; c0 += kEsdfChunk) {
        const int cnt = min(kEsdfChunk, n - c0);
        __syncthreads();
        for (int t = threadIdx.x; t < cnt * 6; t += kEsdfThreads) sb[t] = cub[(size_t)c0 * 6 + t];
        __syncthreads();
        for (int q = 0; q < cnt; ++q) {
            const float *bx = sb + q * 6;
            const float dx = fabsf(px - bx[0]) - bx[3];
            const float dy = fabsf(py - bx[1]) - bx[4];
            const float dz = fabsf(pz - bx[2]) - bx[5];
            const float ox = fmaxf(dx, 0.f), oy = fmaxf(dy, 0.f), oz = fmaxf(dz, 0.f);
            out2 = fminf(out2, fmaf(ox, ox, fmaf(oy, oy, oz * oz)));
            in = fminf(in, fmaxf(dx, fmaxf(dy, dz)));
        }
    }
    if (live) {
        const float s = in <= 0.f ? in : sqrtf(out2);
        phi[v] = fminf(s, DSEED_ESDF_FAR);
    }
}

int launch_esdf_build(const float *cuboids, int n, const DseedGrid &g, float *esdf, cudaStream_t st) {
    const long long nvox = (long long)g.nx * g.ny * g.nz;
    if (nvox == 0) return cudaSuccess;
    k_esdf_build<<<(unsigned)((nvox + kEsdfThreads - 1) / kEsdfThreads), kEsdfThreads, 0, st>>>(cuboids, n, g, nvox, esdf);
    return (int)cudaGetLastError();
}

}  // namespace dseed
