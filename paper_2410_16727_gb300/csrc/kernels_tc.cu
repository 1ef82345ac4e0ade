// kernels_tc.cu -- the denoiser's inference convolutions on the 5th-generation
// tensor cores: an implicit-GEMM 1-D convolution (tcgen05.mma, BF16 operands
// staged by TMA, FP32 accumulators in tensor memory) whose epilogue applies the
// rest of the layer: bias, group norm, Mish, FiLM and the residual add of the
// U-Net's conditional residual blocks (Sec. 4.2), writing BF16 activations.
//
// Geometry.  Activations are channels-last BF16 [samples][L][C].  One CTA owns
// 128 output rows = 128 / L whole samples, and every output channel (N = COUT,
// <= 256, one MMA wide).  The K loop runs over (tap j, 64-channel block): the A
// tile of tap j is the TMA box {64 channels, L rows starting at row j - pad,
// 128 / L samples} of the input; rows outside [0, L) fall out of the tensor and
// arrive as zeros, which is exactly the convolution's zero padding, so no
// im2col buffer exists.  A second source tensor supplies the channels past c0
// (the U-Net's skip concatenations).  A plain GEMM is the case L = 1, one tap.
//
// Roles: thread 0 issues TMA loads into a ring of STAGES stages; thread 32
// issues the MMAs (4 x K=16 per stage) and returns each stage with
// tcgen05.commit; all 8 warps then run the epilogue, warp w reading TMEM lanes
// 32 (w % 4) .. +31 and columns of half w / 4.  Every wait is bounded (2 s);
// one that gives up sets *err and the CTA still releases its tensor memory.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <cstring>
#include <mutex>

#include "internal.h"

namespace dseed {
namespace {

constexpr int kTileM = 128;
constexpr int kBlockK = 64;                  // BF16 channels per K block: one 128-byte swizzle row
constexpr int kTcThreads = 256;
constexpr int kGroups = 8;                   // group-norm groups (the network's)
constexpr unsigned long long kWaitNs = 2000000000ull;

enum { kEpiF32 = 0, kEpiBF16 = 1, kEpiGN = 2 };

struct TcParams {
    CUtensorMap a0, a1, w;
    int M, L, taps, pad, c0_blocks, c_blocks;
    int cout, rows_per_sample;
    float gn_eps;
    const float *bias, *gamma, *beta, *film;
    const int *sample_problem;
    const __nv_bfloat16 *res;
    void *out;
    int out_ld;
    int *err;
};

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Wait for the phase of the given parity to complete; false after kWaitNs.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity) {
    if (mbar_try_wait(bar, parity)) return true;
    const unsigned long long t0 = global_ns();
    while (!mbar_try_wait(bar, parity))
        if (global_ns() - t0 > kWaitNs) return false;
    return true;
}

__device__ __forceinline__ void tma_load_3d(void *dst, const CUtensorMap *map, uint64_t *bar, int x, int y, int z) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
        "[%5];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// Shared-memory matrix descriptor of a K-major operand written by TMA with the
// 128-byte swizzle: rows of 128 bytes, 8-row atoms 1024 bytes apart.
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
    uint64_t d = (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)1 << 16;                 // leading-dimension offset (unused by swizzled K-major)
    d |= (uint64_t)(1024 >> 4) << 32;       // stride-dimension offset: one 8-row atom
    d |= (uint64_t)1 << 46;                 // descriptor version of this architecture
    d |= (uint64_t)2 << 61;                 // 128-byte swizzle
    return d;
}

// Instruction descriptor: D FP32, A and B BF16, both K-major, M x N.
__host__ __device__ constexpr uint32_t bf16_idesc(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void umma_bf16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                          uint32_t accumulate) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(
            tmem_d),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate));
}

__device__ __forceinline__ void umma_commit(uint64_t *bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

// 8 consecutive FP32 columns of this thread's TMEM lane (load and wait in one
// statement, so no use of the values can be scheduled before the wait).
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, float (&v)[8]) {
    uint32_t r[8];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];\n"
        "tcgen05.wait::ld.sync.aligned;\n"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
        : "r"(taddr)
        : "memory");
#pragma unroll
    for (int i = 0; i < 8; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ float mish_f(float x) {
    const float sp = x > 20.f ? x : log1pf(expf(x));
    return x * tanhf(sp);
}

__device__ __forceinline__ void load8(const float *p, float (&v)[8]) {
    const float4 a = *reinterpret_cast<const float4 *>(p), b = *reinterpret_cast<const float4 *>(p + 4);
    v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w; v[4] = b.x; v[5] = b.y; v[6] = b.z; v[7] = b.w;
}

__device__ __forceinline__ void store8_bf16(__nv_bfloat16 *p, const float (&v)[8]) {
    uint4 u;
    __nv_bfloat162 h0 = __floats2bfloat162_rn(v[0], v[1]), h1 = __floats2bfloat162_rn(v[2], v[3]);
    __nv_bfloat162 h2 = __floats2bfloat162_rn(v[4], v[5]), h3 = __floats2bfloat162_rn(v[6], v[7]);
    u.x = *reinterpret_cast<uint32_t *>(&h0);
    u.y = *reinterpret_cast<uint32_t *>(&h1);
    u.z = *reinterpret_cast<uint32_t *>(&h2);
    u.w = *reinterpret_cast<uint32_t *>(&h3);
    *reinterpret_cast<uint4 *>(p) = u;
}

__device__ __forceinline__ void load8_bf16(const __nv_bfloat16 *p, float (&v)[8]) {
    const uint4 u = *reinterpret_cast<const uint4 *>(p);
    const __nv_bfloat162 *h = reinterpret_cast<const __nv_bfloat162 *>(&u);
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const float2 f = __bfloat1622float2(h[i]);
        v[2 * i] = f.x;
        v[2 * i + 1] = f.y;
    }
}

__device__ __forceinline__ void record_failure(int *err, int code) {
    if (err) atomicCAS(err, 0, code);
}

// ---------------------------------------------------------------- epilogues
template <int COUT, int MODE>
__device__ __forceinline__ void epilogue(const TcParams &p, uint32_t tmem, int m0, int warp, int lane) {
    constexpr int HALF = COUT / 2;
    const int q = warp & 3, half = warp >> 2;
    const int gm = m0 + q * 32 + lane;
    const bool valid = gm < p.M;
    const uint32_t trow = tmem + ((uint32_t)(q * 32) << 16);
    const int cb = half * HALF;
    if constexpr (MODE == kEpiGN) {
        constexpr int CG = COUT / kGroups, GH = kGroups / 2;
        static_assert(CG % 8 == 0, "group width must be a multiple of 8 columns");
        const int Lg = p.rows_per_sample;
        float mean[GH], rstd[GH];
        // pass 1: group means over the sample's rows (Lg consecutive lanes)
#pragma unroll
        for (int g = 0; g < GH; ++g) {
            float s = 0.f;
#pragma unroll
            for (int c8 = 0; c8 < CG; c8 += 8) {
                const int c = cb + g * CG + c8;
                float v[8], b[8];
                tmem_ld8(trow + c, v);
                load8(p.bias + c, b);
#pragma unroll
                for (int i = 0; i < 8; ++i) s += v[i] + b[i];
            }
            for (int off = 1; off < Lg; off <<= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
            mean[g] = s / (float)(Lg * CG);
        }
        // pass 2: centred second moments (biased variance)
#pragma unroll
        for (int g = 0; g < GH; ++g) {
            float s = 0.f;
#pragma unroll
            for (int c8 = 0; c8 < CG; c8 += 8) {
                const int c = cb + g * CG + c8;
                float v[8], b[8];
                tmem_ld8(trow + c, v);
                load8(p.bias + c, b);
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    const float d = v[i] + b[i] - mean[g];
                    s += d * d;
                }
            }
            for (int off = 1; off < Lg; off <<= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
            rstd[g] = rsqrtf(s / (float)(Lg * CG) + p.gn_eps);
        }
        // pass 3: normalise, affine, Mish, FiLM, residual; BF16 out
        const float *film = nullptr;
        if (p.film && valid) {
            const int prob = p.sample_problem ? p.sample_problem[gm / Lg] : gm / Lg;
            film = p.film + (size_t)prob * 2 * COUT;
        }
        __nv_bfloat16 *out = reinterpret_cast<__nv_bfloat16 *>(p.out) + (size_t)gm * p.out_ld;
#pragma unroll
        for (int g = 0; g < GH; ++g) {
#pragma unroll
            for (int c8 = 0; c8 < CG; c8 += 8) {
                const int c = cb + g * CG + c8;
                float v[8], b[8], ga[8], be[8];
                tmem_ld8(trow + c, v);
                if (valid) {
                    load8(p.bias + c, b);
                    load8(p.gamma + c, ga);
                    load8(p.beta + c, be);
#pragma unroll
                    for (int i = 0; i < 8; ++i) v[i] = mish_f((v[i] + b[i] - mean[g]) * rstd[g] * ga[i] + be[i]);
                    if (film) {
                        float sc[8], sh[8];
                        load8(film + c, sc);
                        load8(film + COUT + c, sh);
#pragma unroll
                        for (int i = 0; i < 8; ++i) v[i] = v[i] * sc[i] + sh[i];
                    }
                    if (p.res) {
                        float r[8];
                        load8_bf16(p.res + (size_t)gm * COUT + c, r);
#pragma unroll
                        for (int i = 0; i < 8; ++i) v[i] += r[i];
                    }
                    store8_bf16(out + c, v);
                }
            }
        }
    } else {
#pragma unroll
        for (int c8 = 0; c8 < HALF; c8 += 8) {
            const int c = cb + c8;
            float v[8];
            tmem_ld8(trow + c, v);
            if (valid && c < p.cout) {
#pragma unroll
                for (int i = 0; i < 8; ++i) v[i] += (p.bias && c + i < p.cout) ? p.bias[c + i] : 0.f;
                if constexpr (MODE == kEpiBF16) {
                    __nv_bfloat16 *out = reinterpret_cast<__nv_bfloat16 *>(p.out) + (size_t)gm * p.out_ld + c;
                    if (c + 8 <= p.cout) store8_bf16(out, v);
                    else
                        for (int i = 0; i < 8 && c + i < p.cout; ++i) out[i] = __float2bfloat16_rn(v[i]);
                } else {
                    float *out = reinterpret_cast<float *>(p.out) + (size_t)gm * p.out_ld + c;
                    for (int i = 0; i < 8 && c + i < p.cout; ++i) out[i] = v[i];
                }
            }
        }
    }
}

// ---------------------------------------------------------------- kernel
template <int COUT, int STAGES, int MODE>
__global__ void __launch_bounds__(kTcThreads, 1) k_conv_tc(const __grid_constant__ TcParams p) {
    constexpr int A_BYTES = kTileM * kBlockK * 2;
    constexpr int B_BYTES = COUT * kBlockK * 2;
    constexpr int STAGE_BYTES = A_BYTES + B_BYTES;
    constexpr uint32_t TMEM_COLS = COUT < 32 ? 32 : COUT;
    constexpr uint32_t IDESC = bf16_idesc(kTileM, COUT);
    static_assert(COUT % 16 == 0 && COUT >= 16 && COUT <= 256, "MMA N");

    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    __shared__ __align__(8) uint64_t full_bar[STAGES], empty_bar[STAGES], done_bar;
    __shared__ uint32_t tmem_slot;
    __shared__ int s_issued, s_consumed, s_fail;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int m0 = blockIdx.x * kTileM;
    const int nk = p.taps * p.c_blocks;

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(&full_bar[s], 1);
            mbar_init(&empty_bar[s], 1);
        }
        mbar_init(&done_bar, 1);
        s_issued = 0;
        s_consumed = 0;
        s_fail = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                     "r"(TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_slot;

    if (warp == 0 && lane == 0) {
        // producer: one stage = the A box of (tap, channel block) and the matching weight box
        const int sample0 = m0 / p.L;
        int kb = 0;
        for (; kb < nk; ++kb) {
            const int s = kb % STAGES;
            if (kb >= STAGES && !mbar_wait(&empty_bar[s], ((kb / STAGES) - 1) & 1)) {
                record_failure(p.err, 1);
                s_fail = 1;
                break;
            }
            const int tap = kb / p.c_blocks, cblk = kb - tap * p.c_blocks;
            uint8_t *sa = smem + s * STAGE_BYTES;
            mbar_expect_tx(&full_bar[s], STAGE_BYTES);
            if (cblk < p.c0_blocks) tma_load_3d(sa, &p.a0, &full_bar[s], cblk * kBlockK, tap - p.pad, sample0);
            else tma_load_3d(sa, &p.a1, &full_bar[s], (cblk - p.c0_blocks) * kBlockK, tap - p.pad, sample0);
            tma_load_3d(sa + A_BYTES, &p.w, &full_bar[s], cblk * kBlockK, tap, 0);
        }
        s_issued = kb;
    } else if (warp == 1 && lane == 0) {
        // MMA issuer: 4 MMAs of K = 16 per stage, the stage returned by commit
        int kb = 0;
        for (; kb < nk; ++kb) {
            const int s = kb % STAGES;
            if (!mbar_wait(&full_bar[s], (kb / STAGES) & 1)) {
                record_failure(p.err, 2);
                s_fail = 1;
                break;
            }
            tc_fence_after();
            const uint32_t a = smem_u32(smem + s * STAGE_BYTES), b = a + A_BYTES;
#pragma unroll
            for (int k = 0; k < kBlockK / 16; ++k)
                umma_bf16(tmem, sw128_desc(a + 32 * k), sw128_desc(b + 32 * k), IDESC, (kb | k) != 0);
            umma_commit(&empty_bar[s]);
        }
        s_consumed = kb;
        umma_commit(&done_bar);      // arrives once every MMA issued above has completed
    }
    __syncwarp();

    if (!mbar_wait(&done_bar, 0)) record_failure(p.err, 3);
    __syncwarp();                    // the tensor-memory loads below are warp-collective
    tc_fence_after();
    epilogue<COUT, MODE>(p, tmem, m0, warp, lane);
    tc_fence_before();
    __syncthreads();
    if (threadIdx.x == 0 && *(volatile int *)&s_fail) {
        // loads issued but never consumed: let them land before the CTA leaves
        for (int kb = *(volatile int *)&s_consumed; kb < *(volatile int *)&s_issued; ++kb)
            if (!mbar_wait(&full_bar[kb % STAGES], (kb / STAGES) & 1)) break;
    }
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
}

// ---------------------------------------------------------------- host side
typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
    static EncodeTiledFn fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(p);
    });
    return fn;
}

// BF16 3-D tensor {d0 (contiguous), d1, d2}, box {64, b1, b2}, 128-byte swizzle.
bool make_map(CUtensorMap *m, const void *base, uint64_t d0, uint64_t d1, uint64_t d2, uint32_t b1, uint32_t b2) {
    EncodeTiledFn enc = encode_fn();
    if (!enc) return false;
    const cuuint64_t dims[3] = {d0, d1, d2};
    const cuuint64_t strides[2] = {d0 * 2, d0 * d1 * 2};
    const cuuint32_t box[3] = {(cuuint32_t)kBlockK, b1, b2};
    const cuuint32_t estr[3] = {1, 1, 1};
    return enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<void *>(base), dims, strides, box, estr,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <int COUT, int STAGES, int MODE>
int launch_tc(const TcParams &p, cudaStream_t st) {
    constexpr int smem = STAGES * (kTileM + COUT) * kBlockK * 2 + 1024;
    static bool configured = false;       // the attribute is per function; setting it twice is harmless
    if (!configured) {
        const cudaError_t e =
            cudaFuncSetAttribute(k_conv_tc<COUT, STAGES, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e != cudaSuccess) return (int)e;
        configured = true;
    }
    const unsigned grid = (unsigned)((p.M + kTileM - 1) / kTileM);
    k_conv_tc<COUT, STAGES, MODE><<<grid, kTcThreads, smem, st>>>(p);
    return (int)cudaGetLastError();
}

template <int MODE>
int launch_mode(int cout_pad, const TcParams &p, cudaStream_t st) {
    switch (cout_pad) {
        case 16:
            if constexpr (MODE == kEpiGN) return (int)cudaErrorInvalidValue;
            else return launch_tc<16, 4, MODE>(p, st);
        case 64: return launch_tc<64, 4, MODE>(p, st);
        case 128: return launch_tc<128, 3, MODE>(p, st);
        case 256: return launch_tc<256, 4, MODE>(p, st);
        default: return (int)cudaErrorInvalidValue;
    }
}

}  // namespace

bool tc_maps_available() { return encode_fn() != nullptr; }

// Validated by the ABI layer; returns a cudaError_t, or -1 when a tensor map
// cannot be encoded.
int nn_conv_tc(const DseedConvTc &d, cudaStream_t st) {
    TcParams p;
    memset(&p, 0, sizeof(p));
    const int cin = d.c0 + d.c1;
    const int spt = kTileM / d.L;      // samples per tile
    if (!make_map(&p.a0, d.a0_dev, (uint64_t)d.c0, (uint64_t)d.L, (uint64_t)d.n_samples, (uint32_t)d.L,
                  (uint32_t)spt))
        return -1;
    if (d.c1 > 0) {
        if (!make_map(&p.a1, d.a1_dev, (uint64_t)d.c1, (uint64_t)d.L, (uint64_t)d.n_samples, (uint32_t)d.L,
                      (uint32_t)spt))
            return -1;
    } else {
        p.a1 = p.a0;
    }
    if (!make_map(&p.w, d.w_dev, (uint64_t)cin, (uint64_t)d.taps, (uint64_t)d.cout_pad, 1u, (uint32_t)d.cout_pad))
        return -1;
    p.M = d.n_samples * d.L;
    p.L = d.L;
    p.taps = d.taps;
    p.pad = d.pad;
    p.c0_blocks = d.c0 / kBlockK;
    p.c_blocks = cin / kBlockK;
    p.cout = d.cout;
    p.rows_per_sample = d.rows_per_sample;
    p.gn_eps = d.gn_eps;
    p.bias = d.bias_dev;
    p.gamma = d.gamma_dev;
    p.beta = d.beta_dev;
    p.film = d.film_dev;
    p.sample_problem = d.sample_problem_dev;
    p.res = reinterpret_cast<const __nv_bfloat16 *>(d.res_dev);
    p.out = d.out_dev;
    p.out_ld = d.out_ld;
    p.err = d.err_dev;
    if (p.M == 0) return cudaSuccess;
    switch (d.epilogue) {
        case kEpiF32: return launch_mode<kEpiF32>(d.cout_pad, p, st);
        case kEpiBF16: return launch_mode<kEpiBF16>(d.cout_pad, p, st);
        case kEpiGN: return launch_mode<kEpiGN>(d.cout_pad, p, st);
        default: return (int)cudaErrorInvalidValue;
    }
}

}  // namespace dseed
