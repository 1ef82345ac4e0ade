// kernels_esdf.cu -- per-voxel brute-force ESDF of a union of axis-aligned cuboids.
//
// phi(p) = min(FAR, min_k sdf_k(p)) at every voxel centre p.  For each voxel the
// kernel keeps, over the boxes, the smallest squared outside distance
// |max(|p - c| - h, 0)|^2 and the smallest max_i(|p - c|_i - h_i).  If the
// latter is <= 0 some box contains p and it is the union's signed distance (the
// deepest-penetration reading of min_k sdf_k); otherwise min_k sdf_k is the
// square root of the former.  Both equal min_k sdf_k exactly.
//
// One block owns an 8x8x8 tile of voxels (a thread per column of kZPer voxels) of one scene;
// a launch covers up to kMaxJobs scenes (job descriptors travel in the kernel
// parameters, so no device-side table is needed).  Before the per-voxel loop
// the block drops the boxes that cannot be the minimum anywhere in the tile:
// sdf_k is nondecreasing in each |p_i - c_i|, so its maximum over the tile is
// at the corner voxel centre farthest from the box centre along every axis (an
// upper bound U_k from one evaluation), and its minimum over the tile is at least
// the distance from the tile's box of voxel centres to the cuboid (a lower
// bound L_k, or -inf when they overlap).  A box with L_k > min_j U_j + 1e-4 is
// larger than another box's value at every voxel of the tile, so skipping it
// leaves every min, and every output bit, unchanged; the remaining boxes go
// through the same per-voxel arithmetic as without the culling (checked
// bitwise against a build without culling on the benchmark workloads).
//
// A kept box's z terms depend only on its z-slice of the tile, so they are
// formed once per box and slice (dz = |z - c_z| - h_z and max(dz, 0), 8 of each)
// and read from shared memory by the columns; the per-voxel work is one fused
// multiply-add and three min/max, with the same roundings as forming them in place.
#include <cuda_runtime.h>
#include <math_constants.h>

#include "internal.h"

namespace dseed {

constexpr int kTile = 8;
#ifndef DSEED_ESDF_ZPER
#define DSEED_ESDF_ZPER 4
#endif
constexpr int kZPer = DSEED_ESDF_ZPER;                // voxels per thread along z (4 or 8)
static_assert(kZPer == 4 || kZPer == 8, "a thread owns 4 or 8 voxels of a column");
constexpr int kEsdfThreads = kTile * kTile * kTile / kZPer;   // 64 or 128
constexpr int kEsdfChunk = 256;                       // boxes staged per pass

struct EsdfBatch {
    int n_jobs;
    int tiles_z;                                      // max over the jobs
    DseedEsdfJob job[kMaxEsdfJobs];
};

__device__ __forceinline__ float box_sdf(float px, float py, float pz, const float *bx) {
    const float dx = fabsf(px - bx[0]) - bx[3];
    const float dy = fabsf(py - bx[1]) - bx[4];
    const float dz = fabsf(pz - bx[2]) - bx[5];
    const float ox = fmaxf(dx, 0.f), oy = fmaxf(dy, 0.f), oz = fmaxf(dz, 0.f);
    const float in = fmaxf(dx, fmaxf(dy, dz));
    return sqrtf(fmaf(ox, ox, fmaf(oy, oy, oz * oz))) + fminf(in, 0.f);
}

// One block = one 8^3 tile of one scene; a thread owns a column of kZPer voxels
// along z, so each box's x and y terms are formed once for the column.
__global__ void __launch_bounds__(kEsdfThreads) k_esdf_build(const __grid_constant__ EsdfBatch batch) {
    __shared__ float4 s_xy[kEsdfChunk];                // kept boxes: (cx, cy, hx, hy)
    __shared__ float2 s_zc[kEsdfChunk];                // (cz, hz)
    __shared__ float4 s_dz[kEsdfChunk][2];             // dz of the tile's 8 z-slices
    __shared__ float4 s_oz[kEsdfChunk][2];             // max(dz, 0)
    __shared__ float s_red[kEsdfThreads / 32];
    __shared__ int s_count;
    const int jid = blockIdx.z / batch.tiles_z;
    const int tz = blockIdx.z - jid * batch.tiles_z;
    const int tx = blockIdx.x, ty = blockIdx.y;
    const DseedEsdfJob &job = batch.job[jid];
    const DseedGrid &g = job.grid;
    if (tx * kTile >= g.nx || ty * kTile >= g.ny || tz * kTile >= g.nz) return;   // whole block: tile outside this grid
    const float *__restrict__ cub = job.cuboids_dev;
    const int n = job.n;
    const int lx = threadIdx.x & 7, ly = (threadIdx.x >> 3) & 7, lz = threadIdx.x >> 6;
    const int i = tx * kTile + lx, j = ty * kTile + ly, k0 = tz * kTile + lz * kZPer;
    const float px = fmaf((float)i + 0.5f, g.res, g.origin[0]);
    const float py = fmaf((float)j + 0.5f, g.res, g.origin[1]);
    // tile extent in voxel centres (the full 8^3 tile, also past the grid edge)
    float lo[3], hi[3];
    lo[0] = fmaf((float)(tx * kTile) + 0.5f, g.res, g.origin[0]);
    lo[1] = fmaf((float)(ty * kTile) + 0.5f, g.res, g.origin[1]);
    lo[2] = fmaf((float)(tz * kTile) + 0.5f, g.res, g.origin[2]);
    hi[0] = fmaf((float)(tx * kTile + kTile - 1) + 0.5f, g.res, g.origin[0]);
    hi[1] = fmaf((float)(ty * kTile + kTile - 1) + 0.5f, g.res, g.origin[1]);
    hi[2] = fmaf((float)(tz * kTile + kTile - 1) + 0.5f, g.res, g.origin[2]);

    // pass 1: tau = min over boxes of the max of sdf_k over the tile, taken at the
    // corner farthest from the box along each axis (the same value as the largest
    // of the 8 corner evaluations: every rounded step is monotone too)
    float ub = CUDART_INF_F;
    for (int b = threadIdx.x; b < n; b += kEsdfThreads) {
        float bx[6];
        const float *src = cub + (size_t)b * 6;
#pragma unroll
        for (int c = 0; c < 6; ++c) bx[c] = src[c];
        const float fx = fabsf(hi[0] - bx[0]) >= fabsf(lo[0] - bx[0]) ? hi[0] : lo[0];
        const float fy = fabsf(hi[1] - bx[1]) >= fabsf(lo[1] - bx[1]) ? hi[1] : lo[1];
        const float fz = fabsf(hi[2] - bx[2]) >= fabsf(lo[2] - bx[2]) ? hi[2] : lo[2];
        ub = fminf(ub, box_sdf(fx, fy, fz, bx));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) ub = fminf(ub, __shfl_xor_sync(0xffffffffu, ub, o));
    if ((threadIdx.x & 31) == 0) s_red[threadIdx.x >> 5] = ub;
    __syncthreads();
    float tau = s_red[0];
#pragma unroll
    for (int w = 1; w < kEsdfThreads / 32; ++w) tau = fminf(tau, s_red[w]);
    tau += 1e-4f;

    // pass 2: per chunk, keep the boxes whose lower bound over the tile is <= tau
    float out2[kZPer], in[kZPer];
#pragma unroll
    for (int e = 0; e < kZPer; ++e) { out2[e] = CUDART_INF_F; in[e] = CUDART_INF_F; }
    for (int c0 = 0; c0 < n; c0 += kEsdfChunk) {
        const int cnt = min(kEsdfChunk, n - c0);
        __syncthreads();
        if (threadIdx.x == 0) s_count = 0;
        __syncthreads();
        for (int b = threadIdx.x; b < cnt; b += kEsdfThreads) {
            const float *src = cub + (size_t)(c0 + b) * 6;
            float bx[6];
#pragma unroll
            for (int c = 0; c < 6; ++c) bx[c] = src[c];
            float gap2 = 0.f;
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                const float gl = (bx[a] - bx[3 + a]) - hi[a];   // box above the tile
                const float gh = lo[a] - (bx[a] + bx[3 + a]);   // box below the tile
                const float gap = fmaxf(fmaxf(gl, gh), 0.f);
                gap2 = fmaf(gap, gap, gap2);
            }
            // gap2 == 0: the boxes touch or overlap, no useful lower bound
            const float lb = gap2 > 0.f ? sqrtf(gap2) : -CUDART_INF_F;
            if (lb <= tau) {
                const int slot = atomicAdd(&s_count, 1);
                s_xy[slot] = make_float4(bx[0], bx[1], bx[3], bx[4]);
                s_zc[slot] = make_float2(bx[2], bx[5]);
            }
        }
        __syncthreads();
        const int kept = s_count;
        // the z terms of every kept box, once per z-slice of the tile
        for (int w = threadIdx.x; w < kept * kTile; w += kEsdfThreads) {
            const int q = w >> 3, zl = w & 7;
            const float pz = fmaf((float)(tz * kTile + zl) + 0.5f, g.res, g.origin[2]);
            const float2 zc = s_zc[q];
            const float dz = fabsf(pz - zc.x) - zc.y;
            reinterpret_cast<float *>(s_dz[q])[zl] = dz;
            reinterpret_cast<float *>(s_oz[q])[zl] = fmaxf(dz, 0.f);
        }
        __syncthreads();
        for (int q = 0; q < kept; ++q) {
            const float4 b = s_xy[q];
            const float dx = fabsf(px - b.x) - b.z;
            const float dy = fabsf(py - b.y) - b.w;
            const float ox = fmaxf(dx, 0.f), oy = fmaxf(dy, 0.f);
            const float sxy = fmaf(ox, ox, oy * oy);
            const float mxy = fmaxf(dx, dy);
#pragma unroll
            for (int h = 0; h < kZPer / 4; ++h) {
                const float4 o4 = s_oz[q][lz * (kZPer / 4) + h];
                const float oz[4] = {o4.x, o4.y, o4.z, o4.w};
#pragma unroll
                for (int e = 0; e < 4; ++e) out2[4 * h + e] = fminf(out2[4 * h + e], fmaf(oz[e], oz[e], sxy));
            }
            // the inside track can only go <= 0 over the box's x-y footprint (mxy <= 0);
            // elsewhere its value is positive and never read, so a warp with no such
            // column skips it (the output is unchanged)
            if (__any_sync(0xffffffffu, mxy <= 0.f)) {
#pragma unroll
                for (int h = 0; h < kZPer / 4; ++h) {
                    const float4 d4 = s_dz[q][lz * (kZPer / 4) + h];
                    const float dz[4] = {d4.x, d4.y, d4.z, d4.w};
#pragma unroll
                    for (int e = 0; e < 4; ++e) in[4 * h + e] = fminf(in[4 * h + e], fmaxf(mxy, dz[e]));
                }
            }
        }
    }
    if (i < g.nx && j < g.ny) {
#pragma unroll
        for (int e = 0; e < kZPer; ++e) {
            const int k = k0 + e;
            if (k < g.nz) {
                const float s = in[e] <= 0.f ? in[e] : sqrtf(out2[e]);
                job.esdf_dev[((size_t)k * g.ny + j) * g.nx + i] = fminf(s, DSEED_ESDF_FAR);
            }
        }
    }
}

int launch_esdf_build(const DseedEsdfJob *jobs, int n_jobs, cudaStream_t st) {
    for (int j0 = 0; j0 < n_jobs; j0 += kMaxEsdfJobs) {
        EsdfBatch batch;
        batch.n_jobs = n_jobs - j0 < kMaxEsdfJobs ? n_jobs - j0 : kMaxEsdfJobs;
        int tx = 0, ty = 0, tz = 0;
        for (int q = 0; q < batch.n_jobs; ++q) {
            batch.job[q] = jobs[j0 + q];
            const DseedGrid &g = jobs[j0 + q].grid;
            tx = max(tx, (g.nx + kTile - 1) / kTile);
            ty = max(ty, (g.ny + kTile - 1) / kTile);
            tz = max(tz, (g.nz + kTile - 1) / kTile);
        }
        batch.tiles_z = tz;
        const long long gz = (long long)tz * batch.n_jobs;
        if (tx == 0 || ty == 0 || tz == 0) continue;
        if (ty > 65535 || gz > 65535) return (int)cudaErrorInvalidConfiguration;
        k_esdf_build<<<dim3(tx, ty, (unsigned)gz), kEsdfThreads, 0, st>>>(batch);
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return (int)e;
    }
    return cudaSuccess;
}

}  // namespace dseed
