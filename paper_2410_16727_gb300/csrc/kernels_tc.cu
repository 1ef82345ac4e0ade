// kernels_tc.cu -- the denoiser's inference convolutions on the 5th-generation
// tensor cores: an implicit-GEMM 1-D convolution (tcgen05.mma, BF16 operands
// staged by TMA, FP32 accumulators in tensor memory) whose epilogue applies the
// rest of the layer: bias, group norm, Mish, FiLM and the residual add of the
// U-Net's conditional residual blocks (Sec. 4.2), writing BF16 activations.
//
// Geometry.  Activations are channels-last BF16 [samples][L][C].  A tile is
// 128 output rows = 128 / L whole samples by every output channel (N = COUT,
// <= 256, one MMA wide).  The K loop runs over (tap j, 64-channel block): the A
// tile of tap j is the TMA box {64 channels, L rows starting at row j - pad,
// 128 / L samples} of the input; rows outside [0, L) fall out of the tensor and
// arrive as zeros, which is exactly the convolution's zero padding, so no
// im2col buffer exists.  A second source tensor supplies the channels past c0
// (the U-Net's skip concatenations).  A plain GEMM is the case L = 1, one tap.
//
// Roles (persistent CTAs, one per SM, tiles strided by the grid): one lane of
// warp 0 issues TMA loads into a ring of STAGES stages; one lane of warp 1
// issues the MMAs (4 x K=16 per stage), returns each stage with tcgen05.commit
// and alternates between two TMEM accumulator buffers; the remaining warps
// (8 or 16) run the epilogue of one tile while the next tile accumulates, warp
// w reading TMEM lanes 32 (w % 4) .. +31 and column part (w - 2) / 4.  Every wait is
// bounded (2 s); one that gives up sets *err and the CTA still releases its
// tensor memory.
//
// Wide outputs (128 and 256 channels) run in clusters of two CTAs that share the
// weight tile of every stage: each CTA loads one half of it with a multicast
// TMA copy that lands in both CTAs' shared memory, so the pair reads the weight
// bytes from L2 once (the weights are most of a wide layer's operand bytes).
// Each SM still takes in the whole tile; the multicast halves the pair's L2
// reads (which the optimiser kernels sharing L2 in a serving loop feel) without
// changing the layer's own time.  A stage may then be refilled only
// once both CTAs' MMAs have read it: each MMA commit arrives on the stage's
// empty barrier in both CTAs.  The two CTAs walk the same number of tiles (an
// odd last tile is paired with a tile past the end, whose rows are read as the
// TMA fill value and never stored).
//
// Units of two tiles (MT = 2, 128-output layers with long K): a CTA loads the A
// rows of two adjacent tiles in one TMA box and issues both tiles' MMAs against
// each stage's weight tile, so a weight tile feeds 256 output rows; the two
// accumulators (2 x 128 columns) stay double-buffered.
//
// Resident weights (RESW, 64-output layers of at most 8 K blocks): the layer's
// whole weight matrix is loaded once per CTA and the ring carries only A tiles.
//
// Epilogue memory traffic.  The element-wise chain runs on channel pairs with
// packed FP32x2 arithmetic.  Each epilogue warp owns 32 output rows (one per
// lane), so per-lane global accesses would touch 32 rows per instruction:
// instead the warp writes its rows x one column chunk (BF16) into a swizzled
// shared-memory buffer and stores it with one TMA box, and the residual rows
// of the chunk arrive the same way (a TMA box into the same buffer) before the
// output overwrites it.
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

constexpr int kGroups = 8;                   // group-norm groups (the network's)
constexpr unsigned long long kWaitNs = 2000000000ull;

enum { kEpiF32 = 0, kEpiBF16 = 1, kEpiGN = 2 };

struct TcParams {
    CUtensorMap a0, a1, w, w_half;    // w_half: box of half the output rows (cluster multicast)
    CUtensorMap out_map;              // BF16 output rows, box {CH, 32} (staged TMA stores; out_tma)
    CUtensorMap res_map;              // BF16 residual rows, the same boxes (TMA loads; res_tma)
    int out_tma, res_tma;
    int M, L, taps, pad, c0_blocks, c_blocks;
    int cout, rows_per_sample;
    float gn_eps;
    const float *bias, *gamma, *beta, *film, *film_add;
    const int *sample_problem;
    const __nv_bfloat16 *res;
    void *out;
    int out_ld, film_ld;
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

// The same copy multicast to the CTAs of cta_mask: the data lands at the same
// shared-memory offset in each, and each one's mbarrier at bar's offset counts it.
__device__ __forceinline__ void tma_load_3d_mc(void *dst, const CUtensorMap *map, uint64_t *bar, int x, int y, int z,
                                               uint16_t cta_mask) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes.multicast::cluster [%0], [%1, {%2, "
        "%3, %4}], [%5], %6;" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar)), "h"(cta_mask)
        : "memory");
}

__device__ __forceinline__ uint32_t cluster_rank() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}

__device__ __forceinline__ void cluster_sync_all() {
    asm volatile("barrier.cluster.arrive.release.aligned;\nbarrier.cluster.wait.acquire.aligned;" ::: "memory");
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

// Arrive on the mbarrier at bar's offset in every CTA of cta_mask once this
// thread's prior MMAs have completed.
__device__ __forceinline__ void umma_commit_mc(uint64_t *bar, uint16_t cta_mask) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64 [%0], %1;" ::
                     "r"(smem_u32(bar)),
                 "h"(cta_mask)
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

// Staged output rows: each epilogue warp writes its 32 rows x CH columns (BF16)
// into a shared-memory buffer in the tensor map's swizzled layout (16-byte units
// XORed with address bits 7-8 for 64-byte rows, bit 7 for 32-byte rows), then one
// lane stores the box with TMA (rows and columns outside the tensor are dropped).
__device__ __forceinline__ void tma_store_2d(const CUtensorMap *map, const void *src, int x, int y) {
    asm volatile("cp.async.bulk.tensor.2d.global.shared::cta.bulk_group [%0, {%1, %2}], [%3];" ::"l"(
                     reinterpret_cast<uint64_t>(map)),
                 "r"(x), "r"(y), "r"(smem_u32(src))
                 : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_read_all() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *map, uint64_t *bar, int x, int y) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
            smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(bar))
        : "memory");
}

template <int CH>
__device__ __forceinline__ uint32_t stage_offset(int row, int unit) {
    static_assert(CH == 16 || CH == 32, "32- or 64-byte rows");
    if constexpr (CH == 32) return (uint32_t)(row * 64 + ((unit ^ ((row >> 1) & 3)) << 4));
    else return (uint32_t)(row * 32 + ((unit ^ ((row >> 2) & 1)) << 4));
}

// Write this lane's row of the chunk (8-channel units u as uint4) and store the
// warp's box at (column c0, row r0).
template <int CH>
__device__ __forceinline__ void staged_store(const TcParams &p, uint8_t *stage, int lane, const uint4 (&u)[CH / 8],
                                             int c0, int r0) {
    if (lane == 0) bulk_wait_read_all();      // the previous box has left the buffer
    __syncwarp();
#pragma unroll
    for (int j = 0; j < CH / 8; ++j) *reinterpret_cast<uint4 *>(stage + stage_offset<CH>(lane, j)) = u[j];
    fence_async_smem();
    __syncwarp();
    if (lane == 0) {
        tma_store_2d(&p.out_map, stage, c0, r0);
        bulk_commit();
    }
}

__device__ __forceinline__ void record_failure(int *err, int code) {
    if (err) atomicCAS(err, 0, code);
}

// ---------------------------------------------------------------- epilogues
// Columns are read from tensor memory in chunks of CH (32, or the whole half
// for narrow outputs) in one load; a chunk holds whole normalisation groups,
// so the group statistics come from registers (two passes: mean, then the
// centred second moment) reduced over the sample's Lg lanes by shuffles.
template <int N>
__device__ __forceinline__ void tmem_ld(uint32_t taddr, float (&v)[N]);

template <>
__device__ __forceinline__ void tmem_ld<8>(uint32_t taddr, float (&v)[8]) {
    tmem_ld8(taddr, v);
}

template <>
__device__ __forceinline__ void tmem_ld<16>(uint32_t taddr, float (&v)[16]) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15}, [%16];\n"
        "tcgen05.wait::ld.sync.aligned;\n"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr)
        : "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

template <>
__device__ __forceinline__ void tmem_ld<32>(uint32_t taddr, float (&v)[32]) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];\n"
        "tcgen05.wait::ld.sync.aligned;\n"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr)
        : "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// Mish(x) = x tanh(softplus(x)); with e = exp(x), tanh(log(1 + e)) =
// ((1 + e)^2 - 1) / ((1 + e)^2 + 1) = n / (n + 2), n = e (e + 2).  Here on a
// channel pair, with the adds and multiplies packed (exp and the reciprocal
// stay per element).
__device__ __forceinline__ float2 mish2(float2 x) {
    const float2 e = make_float2(__expf(x.x), __expf(x.y));
    const float2 n = __fmul2_rn(e, __fadd2_rn(e, make_float2(2.f, 2.f)));
    const float2 dn = __fadd2_rn(n, make_float2(2.f, 2.f));
    float2 y = __fmul2_rn(x, make_float2(__fdividef(n.x, dn.x), __fdividef(n.y, dn.y)));
    if (x.x > 15.f) y.x = x.x;                // n / (n + 2) = 1 to FP32 precision
    if (x.y > 15.f) y.y = x.y;
    return y;
}

// Per-layer constants, staged in shared memory once per CTA (16-byte aligned:
// the epilogue reads channel pairs as float2).
struct __align__(16) EpiConst {
    float bias[256], gamma[256], beta[256];
};

// Epilogue warps per CTA: 16 for outputs up to 128 channels (a quarter of
// the columns each, chunks of 16), 8 for wider ones (half the columns, chunks
// of 32), keeping the per-thread registers within the CTA's budget.
template <int COUT>
struct EpiShape {
    static constexpr int EW = COUT <= 128 && COUT >= 64 ? 16 : 8;
    static constexpr int PART = COUT / (EW / 4);            // columns per warp
    static constexpr int CH = EW == 16 ? 16 : (PART < 32 ? PART : 32);
};

// stage: this warp's staging buffer; res_bar / res_phase: its mbarrier for the
// residual box loads and the number of loads it has completed so far.
template <int COUT, int MODE>
__device__ __forceinline__ void epilogue(const TcParams &p, const EpiConst &kc, uint32_t tmem, int m0, int q,
                                         int part, int lane, uint8_t *stage, uint64_t *res_bar, int &res_phase) {
    constexpr int HALF = EpiShape<COUT>::PART;
    constexpr int CH = EpiShape<COUT>::CH;
    const int gm = m0 + q * 32 + lane;
    const bool valid = gm < p.M;
    const uint32_t trow = tmem + ((uint32_t)(q * 32) << 16);
    const int cb = part * HALF;
    if constexpr (MODE == kEpiGN) {
        constexpr int CG = COUT / kGroups;
        static_assert(CH % CG == 0, "a chunk must hold whole groups");
        constexpr int GPC = CH / CG;            // groups per chunk
        const int Lg = p.rows_per_sample;
        const float inv_n = 1.f / (float)(Lg * CG);
        const float *film = nullptr;
        if (p.film && valid) {
            const int prob = p.sample_problem ? p.sample_problem[gm / Lg] : gm / Lg;
            film = p.film + (size_t)prob * p.film_ld;
        }
        const __nv_bfloat16 *res = (p.res && valid) ? p.res + (size_t)gm * COUT : nullptr;
        __nv_bfloat16 *out = reinterpret_cast<__nv_bfloat16 *>(p.out) + (size_t)gm * p.out_ld;
#pragma unroll 1
        for (int c0 = cb; c0 < cb + HALF; c0 += CH) {
            // FiLM rows and the residual do not depend on the accumulator: issue
            // their loads first so their latency hides behind the statistics.
            // The element-wise chain runs on channel pairs (packed FP32x2 adds,
            // multiplies and fused multiply-adds: one instruction per pair).
            float2 fsc[CH / 2], fsh[CH / 2];
            uint4 rr[CH / 8];
            if (film) {
#pragma unroll
                for (int j = 0; j < CH / 4; ++j) {
                    const float4 a = *reinterpret_cast<const float4 *>(film + c0 + 4 * j);
                    const float4 b = *reinterpret_cast<const float4 *>(film + COUT + c0 + 4 * j);
                    fsc[2 * j] = make_float2(a.x, a.y);
                    fsc[2 * j + 1] = make_float2(a.z, a.w);
                    fsh[2 * j] = make_float2(b.x, b.y);
                    fsh[2 * j + 1] = make_float2(b.z, b.w);
                }
                if (p.film_add) {
#pragma unroll
                    for (int j = 0; j < CH / 4; ++j) {
                        const float4 a = *reinterpret_cast<const float4 *>(p.film_add + c0 + 4 * j);
                        const float4 b = *reinterpret_cast<const float4 *>(p.film_add + COUT + c0 + 4 * j);
                        fsc[2 * j] = __fadd2_rn(fsc[2 * j], make_float2(a.x, a.y));
                        fsc[2 * j + 1] = __fadd2_rn(fsc[2 * j + 1], make_float2(a.z, a.w));
                        fsh[2 * j] = __fadd2_rn(fsh[2 * j], make_float2(b.x, b.y));
                        fsh[2 * j + 1] = __fadd2_rn(fsh[2 * j + 1], make_float2(b.z, b.w));
                    }
                }
            }
            const bool res_box = p.res && p.res_tma;
            if (res_box) {
                // the residual box of the warp's 32 rows lands in the staging buffer
                // (once the previous output box has left it) while the statistics run
                if (lane == 0) {
                    bulk_wait_read_all();
                    mbar_expect_tx(res_bar, 32 * CH * 2);
                    tma_load_2d(stage, &p.res_map, res_bar, c0, m0 + q * 32);
                }
            } else if (res) {
#pragma unroll
                for (int j = 0; j < CH / 8; ++j) rr[j] = *reinterpret_cast<const uint4 *>(res + c0 + 8 * j);
            }
            float v[CH];
            tmem_ld<CH>(trow + c0, v);
            float2 w[CH / 2];
#pragma unroll
            for (int i = 0; i < CH / 2; ++i)
                w[i] = __fadd2_rn(make_float2(v[2 * i], v[2 * i + 1]),
                                  *reinterpret_cast<const float2 *>(&kc.bias[c0 + 2 * i]));
            float mean[GPC], rstd[GPC];
#pragma unroll
            for (int g = 0; g < GPC; ++g) {
                float2 s2 = make_float2(0.f, 0.f);
#pragma unroll
                for (int i = 0; i < CG / 2; ++i) s2 = __fadd2_rn(s2, w[g * (CG / 2) + i]);
                float s = s2.x + s2.y;
                for (int off = 1; off < Lg; off <<= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
                mean[g] = s * inv_n;
                const float2 nm = make_float2(-mean[g], -mean[g]);
                float2 t2 = make_float2(0.f, 0.f);
#pragma unroll
                for (int i = 0; i < CG / 2; ++i) {
                    const float2 d = __fadd2_rn(w[g * (CG / 2) + i], nm);
                    t2 = __ffma2_rn(d, d, t2);
                }
                float t = t2.x + t2.y;
                for (int off = 1; off < Lg; off <<= 1) t += __shfl_xor_sync(0xffffffffu, t, off);
                rstd[g] = rsqrtf(t * inv_n + p.gn_eps);
            }
#pragma unroll
            for (int i = 0; i < CH / 2; ++i) {
                const int g = (2 * i) / CG;
                const float2 d = __fadd2_rn(w[i], make_float2(-mean[g], -mean[g]));
                const float2 nrm = __fmul2_rn(d, make_float2(rstd[g], rstd[g]));
                float2 y = mish2(__ffma2_rn(nrm, *reinterpret_cast<const float2 *>(&kc.gamma[c0 + 2 * i]),
                                            *reinterpret_cast<const float2 *>(&kc.beta[c0 + 2 * i])));
                if (film) y = __ffma2_rn(y, fsc[i], fsh[i]);
                w[i] = y;
            }
            if (res_box) {
                if (!mbar_wait(res_bar, res_phase & 1)) record_failure(p.err, 7);
                ++res_phase;
#pragma unroll
                for (int j = 0; j < CH / 8; ++j) rr[j] = *reinterpret_cast<const uint4 *>(stage + stage_offset<CH>(lane, j));
                __syncwarp();                  // every lane has its residual row before the buffer is rewritten
            }
            if (res_box || res) {
#pragma unroll
                for (int j = 0; j < CH / 8; ++j) {
                    const __nv_bfloat162 *h = reinterpret_cast<const __nv_bfloat162 *>(&rr[j]);
#pragma unroll
                    for (int e = 0; e < 4; ++e) w[4 * j + e] = __fadd2_rn(w[4 * j + e], __bfloat1622float2(h[e]));
                }
            }
            uint4 u[CH / 8];
#pragma unroll
            for (int j = 0; j < CH / 8; ++j) {
                __nv_bfloat162 h0 = __float22bfloat162_rn(w[4 * j]), h1 = __float22bfloat162_rn(w[4 * j + 1]);
                __nv_bfloat162 h2 = __float22bfloat162_rn(w[4 * j + 2]), h3 = __float22bfloat162_rn(w[4 * j + 3]);
                u[j].x = *reinterpret_cast<uint32_t *>(&h0);
                u[j].y = *reinterpret_cast<uint32_t *>(&h1);
                u[j].z = *reinterpret_cast<uint32_t *>(&h2);
                u[j].w = *reinterpret_cast<uint32_t *>(&h3);
            }
            if (p.out_tma) {
                staged_store<CH>(p, stage, lane, u, c0, m0 + q * 32);
            } else if (valid) {
#pragma unroll
                for (int j = 0; j < CH / 8; ++j) *reinterpret_cast<uint4 *>(out + c0 + 8 * j) = u[j];
            }
        }
    } else {
#pragma unroll 1
        for (int c0 = cb; c0 < cb + HALF; c0 += CH) {
            float v[CH];
            tmem_ld<CH>(trow + c0, v);
            if constexpr (MODE == kEpiBF16 && (CH == 16 || CH == 32)) {
                if (p.out_tma) {
                    uint4 u[CH / 8];
#pragma unroll
                    for (int j = 0; j < CH / 8; ++j) {
                        float y[8];
#pragma unroll
                        for (int e = 0; e < 8; ++e) y[e] = v[8 * j + e] + kc.bias[c0 + 8 * j + e];
                        __nv_bfloat162 h0 = __floats2bfloat162_rn(y[0], y[1]), h1 = __floats2bfloat162_rn(y[2], y[3]);
                        __nv_bfloat162 h2 = __floats2bfloat162_rn(y[4], y[5]), h3 = __floats2bfloat162_rn(y[6], y[7]);
                        u[j].x = *reinterpret_cast<uint32_t *>(&h0);
                        u[j].y = *reinterpret_cast<uint32_t *>(&h1);
                        u[j].z = *reinterpret_cast<uint32_t *>(&h2);
                        u[j].w = *reinterpret_cast<uint32_t *>(&h3);
                    }
                    staged_store<CH>(p, stage, lane, u, c0, m0 + q * 32);
                    continue;
                }
            }
#pragma unroll
            for (int i = 0; i < CH && valid; i += 8) {
                const int c = c0 + i;
                if (c >= p.cout) break;
                float y[8];
#pragma unroll
                for (int e = 0; e < 8; ++e) y[e] = v[i + e] + kc.bias[c + e];
                if constexpr (MODE == kEpiBF16) {
                    __nv_bfloat16 *out = reinterpret_cast<__nv_bfloat16 *>(p.out) + (size_t)gm * p.out_ld + c;
                    if (c + 8 <= p.cout) store8_bf16(out, y);
                    else
                        for (int e = 0; e < 8 && c + e < p.cout; ++e) out[e] = __float2bfloat16_rn(y[e]);
                } else {
                    float *out = reinterpret_cast<float *>(p.out) + (size_t)gm * p.out_ld + c;
                    for (int e = 0; e < 8 && c + e < p.cout; ++e) out[e] = y[e];
                }
            }
        }
    }
}

// ---------------------------------------------------------------- kernel
// Persistent: one CTA per SM walks the tiles blockIdx.x, +gridDim.x, ...
// Warp 0 (one lane) streams stages through the smem ring, warp 1 (one lane)
// issues the MMAs of tile i into accumulator buffer i % 2, and the epilogue warps run
// the epilogue of tile i while the MMAs of tile i + 1 fill the other buffer.
__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// RESW: the layer's whole weight matrix (at most kMaxResK K blocks) is loaded
// once per CTA and stays resident; the ring then carries only A tiles.
constexpr int kMaxResK = 8;

template <int COUT, int STAGES, int MODE, int CL, int MT, bool RESW = false>
__global__ void __launch_bounds__(32 * (2 + EpiShape<COUT>::EW), 1) k_conv_tc(const __grid_constant__ TcParams p) {
    constexpr int TILE_A_BYTES = kTileM * kBlockK * 2;
    constexpr int A_BYTES = MT * TILE_A_BYTES;                 // MT tiles of one unit, one TMA box
    constexpr int B_BYTES = COUT * kBlockK * 2;
    constexpr int STAGE_BYTES = RESW ? A_BYTES : A_BYTES + B_BYTES;
    static_assert(!RESW || (CL == 1 && MT == 1), "resident weights: single CTAs");
    // a unit's accumulators: MT tiles x COUT columns; two buffers when they fit
    constexpr int UNIT_COLS = MT * COUT;
    constexpr int NBUF = 2 * UNIT_COLS <= 512 ? 2 : 1;
    constexpr uint32_t TMEM_COLS = NBUF * UNIT_COLS < 32 ? 32 : NBUF * UNIT_COLS;
    constexpr uint32_t IDESC = bf16_idesc(kTileM, COUT);
    constexpr int kEpiWarps = EpiShape<COUT>::EW;
    static_assert(COUT % 16 == 0 && COUT >= 16 && COUT <= 256, "MMA N");
    static_assert(CL == 1 || (CL == 2 && COUT >= 128), "clusters of two share wide weight tiles");
    static_assert((MT == 1 || MT == 2) && NBUF * UNIT_COLS <= 512, "tensor memory holds 512 columns");
    constexpr uint16_t kPair = 0x3;

    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    __shared__ __align__(8) uint64_t full_bar[STAGES], empty_bar[STAGES], accf_bar[2], acce_bar[2], wfull_bar;
    __shared__ __align__(8) uint64_t res_bar[kEpiWarps];     // residual box loads, one per epilogue warp
    __shared__ uint32_t tmem_slot;
    __shared__ int s_issued, s_consumed, s_fail, s_wissued;
    __shared__ EpiConst s_const;
    uint8_t *const wres = smem + STAGES * STAGE_BYTES;          // resident weight tiles (RESW)
    // output staging of the epilogue warps (32 rows x CH BF16 each), after the ring
    constexpr int kStageWarpBytes = 32 * EpiShape<COUT>::CH * 2;
    uint8_t *const stage_base = wres + (RESW ? kMaxResK * B_BYTES : 0);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nk = p.taps * p.c_blocks;
    const int n_tiles = (p.M + kTileM - 1) / kTileM;
    // work units of CL x MT adjacent tiles: this CTA takes the MT tiles from
    // (CL u + rank) MT of unit u (past the end for a short last unit)
    const int crank = CL > 1 ? (int)cluster_rank() : 0;
    const int n_units = (n_tiles + CL * MT - 1) / (CL * MT);
    const int unit0 = blockIdx.x / CL, unit_step = gridDim.x / CL;

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(&full_bar[s], 1);
            mbar_init(&empty_bar[s], CL);           // every CTA of the cluster reads the stage
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&accf_bar[b], 1);
            mbar_init(&acce_bar[b], kEpiWarps);
        }
        mbar_init(&wfull_bar, 1);
        for (int w = 0; w < kEpiWarps; ++w) mbar_init(&res_bar[w], 1);
        s_issued = 0;
        s_consumed = 0;
        s_fail = 0;
        s_wissued = 0;
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
    if (CL > 1) cluster_sync_all();               // the partner's barriers exist before any multicast
    tc_fence_after();
    const uint32_t tmem = tmem_slot;
    volatile int *fail = &s_fail;

    if (warp == 0) {
        if (lane == 0) {
            // producer
            if (RESW && nk <= kMaxResK) {
                mbar_expect_tx(&wfull_bar, nk * B_BYTES);
                for (int kb = 0; kb < nk; ++kb) {
                    const int tap = kb / p.c_blocks, cblk = kb - tap * p.c_blocks;
                    tma_load_3d(wres + kb * B_BYTES, &p.w, &wfull_bar, cblk * kBlockK, tap, 0);
                }
                s_wissued = 1;
            }
            int g = 0;
            for (int u = unit0; u < n_units && !*fail; u += unit_step) {
                const int tile = (CL * u + crank) * MT;
                const int sample0 = tile * kTileM / p.L;
                for (int kb = 0; kb < nk; ++kb, ++g) {
                    const int s = g % STAGES;
                    if (g >= STAGES && !mbar_wait(&empty_bar[s], ((g / STAGES) - 1) & 1)) {
                        record_failure(p.err, 1);
                        *fail = 1;
                        break;
                    }
                    const int tap = kb / p.c_blocks, cblk = kb - tap * p.c_blocks;
                    uint8_t *sa = smem + s * STAGE_BYTES;
                    mbar_expect_tx(&full_bar[s], STAGE_BYTES);
                    if (cblk < p.c0_blocks)
                        tma_load_3d(sa, &p.a0, &full_bar[s], cblk * kBlockK, tap - p.pad, sample0);
                    else
                        tma_load_3d(sa, &p.a1, &full_bar[s], (cblk - p.c0_blocks) * kBlockK, tap - p.pad, sample0);
                    if (RESW) {
                    } else if (CL > 1) {
                        tma_load_3d_mc(sa + A_BYTES + crank * (B_BYTES / 2), &p.w_half, &full_bar[s],
                                       cblk * kBlockK, tap, crank * (COUT / 2), kPair);
                    } else {
                        tma_load_3d(sa + A_BYTES, &p.w, &full_bar[s], cblk * kBlockK, tap, 0);
                    }
                }
            }
            s_issued = g;
        }
    } else if (warp == 1) {
        if (lane == 0) {
            // MMA issuer
            if (RESW && (nk > kMaxResK || !mbar_wait(&wfull_bar, 0))) {
                record_failure(p.err, 2);
                *fail = 1;
            }
            int g = 0, it = 0;
            for (int u = unit0; u < n_units && !*fail; u += unit_step, ++it) {
                const int b = NBUF == 2 ? (it & 1) : 0;
                const int use = NBUF == 2 ? (it >> 1) : it;      // earlier units in buffer b
                if (use >= 1 && !mbar_wait(&acce_bar[b], (use - 1) & 1)) {
                    record_failure(p.err, 4);
                    *fail = 1;
                    break;
                }
                tc_fence_after();
                const uint32_t d = tmem + (uint32_t)(b * UNIT_COLS);
                for (int kb = 0; kb < nk; ++kb, ++g) {
                    const int s = g % STAGES;
                    if (!mbar_wait(&full_bar[s], (g / STAGES) & 1)) {
                        record_failure(p.err, 2);
                        *fail = 1;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t a = smem_u32(smem + s * STAGE_BYTES);
                    const uint32_t bb = RESW ? smem_u32(wres + kb * B_BYTES) : a + A_BYTES;
                    // the MT tiles of the unit share the stage's weight tile
#pragma unroll
                    for (int k = 0; k < kBlockK / 16; ++k)
#pragma unroll
                        for (int t = 0; t < MT; ++t)
                            umma_bf16(d + (uint32_t)(t * COUT), sw128_desc(a + t * TILE_A_BYTES + 32 * k),
                                      sw128_desc(bb + 32 * k), IDESC, (kb | k) != 0);
                    if (CL > 1) umma_commit_mc(&empty_bar[s], kPair);
                    else umma_commit(&empty_bar[s]);
                }
                umma_commit(&accf_bar[b]);     // arrives once this tile's MMAs have completed
            }
            s_consumed = g;
        }
    } else {
        // epilogue warps: TMEM lanes of quadrant warp % 4, column part (warp - 2) / 4
        const int q = warp & 3, half = (warp - 2) >> 2;
        for (int c = threadIdx.x - 64; c < COUT; c += 32 * kEpiWarps) {
            s_const.bias[c] = (p.bias && c < p.cout) ? p.bias[c] : 0.f;
            s_const.gamma[c] = p.gamma ? p.gamma[c] : 1.f;
            s_const.beta[c] = p.beta ? p.beta[c] : 0.f;
        }
        asm volatile("bar.sync 1, %0;" ::"n"(32 * kEpiWarps) : "memory");     // epilogue warps only
        int it = 0, res_phase = 0;
        for (int u = unit0; u < n_units; u += unit_step, ++it) {
            const int tile = (CL * u + crank) * MT;
            const int b = NBUF == 2 ? (it & 1) : 0;
            const int use = NBUF == 2 ? (it >> 1) : it;
            if (!mbar_wait(&accf_bar[b], use & 1)) {
                record_failure(p.err, 3);
                *fail = 1;
                break;
            }
            __syncwarp();                      // the tensor-memory loads are warp-collective
            tc_fence_after();
            if (!*fail)
#pragma unroll 1
                for (int t = 0; t < MT; ++t)
                    epilogue<COUT, MODE>(p, s_const, tmem + (uint32_t)(b * UNIT_COLS + t * COUT), (tile + t) * kTileM,
                                         q, half, lane, stage_base + (warp - 2) * kStageWarpBytes, &res_bar[warp - 2],
                                         res_phase);
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&acce_bar[b]);
        }
        if (lane == 0) bulk_wait_all();        // this warp's staged output boxes have been written
    }
    __syncthreads();
    if (threadIdx.x == 0 && *fail) {
        // loads issued but never consumed: let them land before the CTA leaves
        for (int g = *(volatile int *)&s_consumed; g < *(volatile int *)&s_issued; ++g)
            if (!mbar_wait(&full_bar[g % STAGES], (g / STAGES) & 1)) break;
        if (RESW && *(volatile int *)&s_wissued) mbar_wait(&wfull_bar, 0);
    }
    tc_fence_before();
    __syncthreads();
    if (CL > 1) cluster_sync_all();               // neither CTA leaves while the other may still reach it
    tc_fence_after();
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

// BF16 output rows [rows][ld] seen as a 2-D tensor {cols, rows}, box {box_cols, 32},
// swizzled to match the epilogue's staging layout (64- or 32-byte rows).
bool make_out_map(CUtensorMap *m, const void *base, uint64_t cols, uint64_t rows, uint64_t ld, uint32_t box_cols) {
    EncodeTiledFn enc = encode_fn();
    if (!enc || (box_cols != 16 && box_cols != 32)) return false;
    const cuuint64_t dims[2] = {cols, rows};
    const cuuint64_t strides[1] = {ld * 2};
    const cuuint32_t box[2] = {box_cols, 32u};
    const cuuint32_t estr[2] = {1, 1};
    return enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void *>(base), dims, strides, box, estr,
               CU_TENSOR_MAP_INTERLEAVE_NONE, box_cols == 32 ? CU_TENSOR_MAP_SWIZZLE_64B : CU_TENSOR_MAP_SWIZZLE_32B,
               CU_TENSOR_MAP_L2_PROMOTION_NONE, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <int COUT, int STAGES, int MODE, int CL, int MT, bool RESW = false>
int launch_tc(const TcParams &p, cudaStream_t st) {
    constexpr int stage_out = EpiShape<COUT>::EW * 32 * EpiShape<COUT>::CH * 2;      // output staging
    constexpr int smem = (RESW ? STAGES * kTileM * kBlockK * 2 + kMaxResK * COUT * kBlockK * 2
                               : STAGES * (MT * kTileM + COUT) * kBlockK * 2) + stage_out + 1024;
    constexpr int threads = 32 * (2 + EpiShape<COUT>::EW);
    auto kern = k_conv_tc<COUT, STAGES, MODE, CL, MT, RESW>;
    static bool configured = false;       // the attribute is per function; setting it twice is harmless
    static int max_units = 0;             // work units (CTAs, or clusters) resident at once
    if (!configured) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e != cudaSuccess) return (int)e;
        int dev = 0, sms = 0;
        cudaGetDevice(&dev);
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1) sms = 1;
        max_units = sms;
        if (CL > 1) {
            cudaLaunchConfig_t cfg = {};
            cudaLaunchAttribute attr;
            attr.id = cudaLaunchAttributeClusterDimension;
            attr.val.clusterDim.x = CL;
            attr.val.clusterDim.y = 1;
            attr.val.clusterDim.z = 1;
            cfg.gridDim = dim3((unsigned)(CL * (sms / CL)));
            cfg.blockDim = dim3(threads);
            cfg.dynamicSmemBytes = smem;
            cfg.attrs = &attr;
            cfg.numAttrs = 1;
            int clusters = 0;
            e = cudaOccupancyMaxActiveClusters(&clusters, kern, &cfg);
            if (e != cudaSuccess) return (int)e;
            max_units = clusters > 0 ? clusters : 1;
        }
        configured = true;
    }
    const int tiles = (p.M + kTileM - 1) / kTileM;
    const int units = (tiles + CL * MT - 1) / (CL * MT);
    const unsigned grid = (unsigned)(CL * (units < max_units ? units : max_units));
    if (CL == 1) {
        kern<<<grid, threads, smem, st>>>(p);
        return (int)cudaGetLastError();
    }
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr;
    attr.id = cudaLaunchAttributeClusterDimension;
    attr.val.clusterDim.x = CL;
    attr.val.clusterDim.y = 1;
    attr.val.clusterDim.z = 1;
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(threads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cfg.attrs = &attr;
    cfg.numAttrs = 1;
    return (int)cudaLaunchKernelEx(&cfg, kern, p);
}

// mt2: units of two tiles per CTA sharing each weight tile, which halves the
// weight bytes per output row.  Measured at the sampling size (32768
// trajectories): 1.3-1.4x faster for 128 outputs over 1280-2560 input values
// per row (the skip-concatenation layers), neutral at 640, and slower for 256
// outputs, whose two 256-column accumulators fill the tensor memory, so the
// epilogue of one unit can no longer overlap the next unit's MMAs.
template <int MODE>
int launch_mode(int cout_pad, bool mt2, const TcParams &p, cudaStream_t st) {
    switch (cout_pad) {
        case 16:
            if constexpr (MODE == kEpiGN) return (int)cudaErrorInvalidValue;
            else return launch_tc<16, 8, MODE, 1, 1>(p, st);
        case 64:
            // 64-output layers with at most kMaxResK K blocks keep their weights resident
            if (p.taps * p.c_blocks <= kMaxResK) return launch_tc<64, 8, MODE, 1, 1, true>(p, st);
            return launch_tc<64, 8, MODE, 1, 1>(p, st);
        case 128: return mt2 ? launch_tc<128, 4, MODE, 2, 2>(p, st) : launch_tc<128, 6, MODE, 2, 1>(p, st);
        case 256: return launch_tc<256, 4, MODE, 2, 1>(p, st);
        default: return (int)cudaErrorInvalidValue;
    }
}

// Two-tile units: 128 outputs, at least 20 K blocks (1280 input values per
// row), and enough tiles for three rounds of two-tile units over the SMs.
constexpr int kMt2MinKBlocks = 20;
constexpr int kMt2MinTiles = 6 * 152;

}  // namespace

bool tc_maps_available() { return encode_fn() != nullptr; }

// Validated by the ABI layer; returns a cudaError_t, or -1 when a tensor map
// cannot be encoded.
int nn_conv_tc(const DseedConvTc &d, cudaStream_t st) {
    TcParams p;
    memset(&p, 0, sizeof(p));
    const int cin = d.c0 + d.c1;
    const long long n_tiles = ((long long)d.n_samples * d.L + kTileM - 1) / kTileM;
    const bool mt2 = d.cout_pad == 128 && d.taps * (cin / kBlockK) >= kMt2MinKBlocks && n_tiles >= kMt2MinTiles;
    const int spt = (mt2 ? 2 : 1) * kTileM / d.L;      // samples per A box (the tiles of one unit)
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
    if (d.cout_pad >= 128 &&
        !make_map(&p.w_half, d.w_dev, (uint64_t)cin, (uint64_t)d.taps, (uint64_t)d.cout_pad, 1u,
                  (uint32_t)(d.cout_pad / 2)))
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
    p.film_add = d.film_add_dev;
    p.sample_problem = d.sample_problem_dev;
    p.res = reinterpret_cast<const __nv_bfloat16 *>(d.res_dev);
    p.out = d.out_dev;
    p.out_ld = d.out_ld;
    // staged TMA stores of BF16 rows (chunks of 16 or 32 columns: outputs of 64 or more)
    p.out_tma = 0;
    p.res_tma = 0;
    if (d.epilogue >= 1 && d.cout_pad >= 64 && ((uintptr_t)d.out_dev & 15) == 0) {
        const uint32_t ch = d.cout_pad == 256 ? 32u : 16u;
        const uint64_t rows = (uint64_t)d.n_samples * d.L;
        if (make_out_map(&p.out_map, d.out_dev, (uint64_t)d.cout, rows, (uint64_t)d.out_ld, ch)) {
            p.out_tma = 1;
            // the residual [rows][cout_pad] in the same boxes, read through the same staging buffer
            if (d.epilogue == kEpiGN && d.res_dev && ((uintptr_t)d.res_dev & 15) == 0 &&
                make_out_map(&p.res_map, d.res_dev, (uint64_t)d.cout_pad, rows, (uint64_t)d.cout_pad, ch))
                p.res_tma = 1;
        }
    }
    p.film_ld = d.film_ld > 0 ? d.film_ld : 2 * d.cout;
    p.err = d.err_dev;
    if (p.M == 0) return cudaSuccess;
    switch (d.epilogue) {
        case kEpiF32: return launch_mode<kEpiF32>(d.cout_pad, mt2, p, st);
        case kEpiBF16: return launch_mode<kEpiBF16>(d.cout_pad, mt2, p, st);
        case kEpiGN: return launch_mode<kEpiGN>(d.cout_pad, mt2, p, st);
        default: return (int)cudaErrorInvalidValue;
    }
}

}  // namespace dseed
