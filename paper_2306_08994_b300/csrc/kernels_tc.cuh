// Tensor-core Schur update on sm_100-family (B300 = sm_103a): S -= L21 U12
// (Sec. 2.2) with tcgen05.mma kind::tf32, FP32 accumulation in tensor memory.
//
// Accuracy: every operand x is split into x_hi = tf32(x) and x_lo =
// tf32(x - x_hi), and the product is accumulated as A_hi B_hi + A_hi B_lo +
// A_lo B_hi (three MMAs per K slice): products accurate to about 2^-21
// relative, FP32-grade Schur complements, which the FP64 refinement needs.
// Two BF16 modes (kind::f16, BF16 operands, FP32 accumulation) serve the
// MF_TF32_BF16 trial on the largest Schur updates: one BF16 product (x
// rounded to BF16, about 2^-9 relative per product) or three split-BF16
// products (hi = bf16(x), lo = bf16(x - hi): about 2^-17).
//
// Two kernels per class:
//  * k_tc_pack splits L21 and U12 of every tensor-core front once into hi and
//    lo copies, already in the MMA's shared-memory image: K-major, no swizzle,
//    core matrices of 8 rows x 16 bytes, core (row group r, K group g) at byte
//    r*512 + g*128 of a (rows x 16) chunk.  Chunks are contiguous per (row
//    tile, 16-wide K slice) and zero-padded, so the GEMM main loop is nothing
//    but bulk copies (cp.async.bulk, the TMA engine) and MMAs.
//  * k_schur_tc: one CTA per 128 x 256 tile of S; warp 0 lane 0 streams the
//    operand chunks into a 4-stage ring (mbarrier expect_tx / complete_tx),
//    warp 1 lane 0 issues the MMAs and returns each stage with
//    tcgen05.commit; after the last commit all 4 warps read the accumulator
//    (tcgen05.ld, warp w = TMEM lanes 32w..32w+31 = rows) and subtract it from
//    S in place.  Every wait is bounded (globaltimer); on expiry the kernel
//    records a timeout, waits (bounded) for its copies and MMAs in flight,
//    frees its tensor memory and returns.
#pragma once

#include <cuda_bf16.h>

#include <cstdint>

#include "kernels_factor.cuh"

namespace tc {

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint32_t to_tf32(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return r;
}

__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = 0;
    d |= (uint64_t)((addr >> 4) & 0x3FFF);
    d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
    d |= (uint64_t)1 << 46;  // descriptor version for the sm_100 family; bits 61-63 = 0: no swizzle
    return d;
}

// instruction descriptor: D f32, A/B tf32, both K-major, M x N
__host__ __device__ constexpr uint32_t idesc_tf32(int M, int N) {
    return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// instruction descriptor of kind::f16: D f32, A/B bf16, both K-major, M x N
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc)
        : "memory");
}

__device__ __forceinline__ void mma_tf32(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc)
        : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t* mbar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(mbar))
                 : "memory");
}

__device__ __forceinline__ void mbar_init(uint64_t* mbar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(mbar)), "r"(count) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* mbar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(mbar)), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ uint64_t globaltimer_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Bounded wait: gives up after `limit_ns` of wall-clock time and returns false.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* mbar, uint32_t parity, uint64_t limit_ns) {
    const uint64_t t0 = globaltimer_ns();
    while (!mbar_try_wait(mbar, parity))
        if (globaltimer_ns() - t0 > limit_ns) return false;
    return true;
}

__device__ __forceinline__ void fence_before_sync() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after_sync() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=f"(v[0]), "=f"(v[1]), "=f"(v[2]), "=f"(v[3]), "=f"(v[4]), "=f"(v[5]), "=f"(v[6]), "=f"(v[7]), "=f"(v[8]),
          "=f"(v[9]), "=f"(v[10]), "=f"(v[11]), "=f"(v[12]), "=f"(v[13]), "=f"(v[14]), "=f"(v[15]), "=f"(v[16]),
          "=f"(v[17]), "=f"(v[18]), "=f"(v[19]), "=f"(v[20]), "=f"(v[21]), "=f"(v[22]), "=f"(v[23]), "=f"(v[24]),
          "=f"(v[25]), "=f"(v[26]), "=f"(v[27]), "=f"(v[28]), "=f"(v[29]), "=f"(v[30]), "=f"(v[31])
        : "r"(taddr)
        : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* mbar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(mbar)) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* mbar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(mbar)), "r"(bytes) : "memory");
}

// 1D bulk copy global -> shared (TMA engine), completion counted on mbar.
__device__ __forceinline__ void bulk_g2s(void* smem_dst, const void* gmem_src, uint32_t bytes, uint64_t* mbar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(smem_u32(smem_dst)),
        "l"(gmem_src), "r"(bytes), "r"(smem_u32(mbar))
        : "memory");
}

constexpr int kTileM = 128, kTileN = 256, kChunkK = 16, kStages = 4;
constexpr int kChunkA = kTileM * kChunkK;  // floats per A chunk (hi or lo): 8 KB
constexpr int kChunkB = kTileN * kChunkK;  // floats per B chunk: 16 KB
constexpr int kStageBytes = 2 * 4 * (kChunkA + kChunkB);  // bytes: A_hi, A_lo, B_hi, B_lo
constexpr int kSmemBytes = kStages * kStageBytes + 1024;

// Product modes.  A chunk is one 16-wide K slice of a 128-row (A) or 256-row
// (B) operand tile in the MMA's shared-memory image; a stage of the ring holds
// kCps consecutive chunks of A and of B (hi, and lo where the mode has one),
// 48 KB in every mode.  TF32 chunks: core matrix (row group r, K group g) at
// r*512 + g*128 bytes (4 K groups of 4 values); BF16 chunks: at r*256 + g*128
// (2 K groups of 8 values).
enum Mode { kTf32x3 = 0, kBf16 = 1, kBf16x3 = 2 };
template <int MODE>
struct ModeCfg {
    static constexpr bool kBf = MODE != kTf32x3;
    static constexpr bool kLo = MODE != kBf16;
    static constexpr int kCps = MODE == kTf32x3 ? 1 : MODE == kBf16 ? 4 : 2;       // chunks per stage
    static constexpr int kFloatsA = kBf ? kChunkA / 2 : kChunkA;                    // floats per chunk
    static constexpr int kFloatsB = kBf ? kChunkB / 2 : kChunkB;
    static constexpr int kSbo = kBf ? 256 : 512;                                    // row-group stride
    static constexpr int kStage = kCps * 4 * (kFloatsA + kFloatsB) * (kLo ? 2 : 1);  // bytes
    static_assert(kStage == kStageBytes, "every mode fills the same ring");
};
__host__ __device__ constexpr int chunk_floats_a(int mode) { return mode == kTf32x3 ? kChunkA : kChunkA / 2; }
__host__ __device__ constexpr int chunk_floats_b(int mode) { return mode == kTf32x3 ? kChunkB : kChunkB / 2; }
constexpr uint32_t kTmemCols = 256;
constexpr uint64_t kWaitLimit = 1000000000ull;  // 1 s


}  // namespace tc

// One product for the tensor cores (a Schur update S -= L21 U12, a trailing
// update of a super-panel, or a level of the pivot-block inversion), with
// the same operand conventions as the SIMT GEMM: A (M x K) element (i, p) at
// arena a_ar [a_off + i + p lda]; B (K x N) element (p, j) at arena b_ar
// [b_off + p + j ldb]; optional triangular masks; op 0: C -= A B, 1: C = A B,
// 2: C = -A B.  Packed as above: A in row tiles of 128, B^T in row tiles of
// 256; hi chunks at a_hi / b_hi, lo chunks lo_off further.
struct TcPack {
    int64_t a_off, b_off;
    int64_t a_hi, b_hi, lo_off;
    int32_t lda, ldb, M, N, K, nkc;
    int8_t a_ar, b_ar, a_mask, b_mask, pad[4];
};
struct TcTile {
    int64_t a_hi, b_hi, lo_off;  // first chunks (K slice 0) of this tile's A row tile and B row tile
    int64_t c_off;               // offset of the tile's (0, 0) element in arena c_ar
    int32_t ldc, mrows, ncols, nkc;
    int32_t c_ar, op;
};

// Pack kernel: one CTA per (product, operand, row tile, 16-wide K slice),
// 256 threads.  The slice is read coalesced into shared memory (A along its
// contiguous rows, B along its contiguous K), then written out as hi and lo
// chunks: 16-byte unit u of a chunk holds row (u / 32) * 8 + u % 8, K group
// (u / 8) % 4, so consecutive threads write consecutive 16-byte units.
struct TcPackJob {
    int32_t task, which, rt, kc;
};

template <int MODE>
__global__ void __launch_bounds__(256) k_tc_pack(const TcPack* __restrict__ tasks, const TcPackJob* __restrict__ jobs,
                                                 Arenas<float> ar, float* __restrict__ pk) {
    using Cfg = tc::ModeCfg<MODE>;
    __shared__ float tile[tc::kTileN][tc::kChunkK + 1];
    const TcPackJob jb = jobs[blockIdx.x];
    const TcPack t = tasks[jb.task];
    const int rows = jb.which == 0 ? tc::kTileM : tc::kTileN;
    const int nrow = jb.which == 0 ? t.M : t.N;
    const float* src = jb.which == 0 ? ar.a[t.a_ar] + t.a_off : ar.a[t.b_ar] + t.b_off;
    const int r0 = jb.rt * rows, p0 = jb.kc * tc::kChunkK;
    // every load of the thread is issued before the first shared-memory store (8 for an A slice,
    // 16 for a B slice)
    if (jb.which == 0) {  // A: column-major, consecutive threads down a column
        constexpr int NL = tc::kTileM * tc::kChunkK / 256;
        float v[NL];
#pragma unroll
        for (int q = 0; q < NL; q++) {
            const int e = threadIdx.x + 256 * q, r = e % tc::kTileM, kk = e / tc::kTileM;
            const int i = r0 + r, p = p0 + kk;
            v[q] = (i < nrow && p < t.K) ? masked(src[i + (int64_t)p * t.lda], t.a_mask, i, p) : 0.f;
        }
#pragma unroll
        for (int q = 0; q < NL; q++) {
            const int e = threadIdx.x + 256 * q;
            tile[e % tc::kTileM][e / tc::kTileM] = v[q];
        }
    } else {  // B: K-contiguous, consecutive threads along K
        constexpr int NL = tc::kTileN * tc::kChunkK / 256;
        float v[NL];
#pragma unroll
        for (int q = 0; q < NL; q++) {
            const int e = threadIdx.x + 256 * q, kk = e % tc::kChunkK, r = e / tc::kChunkK;
            const int i = r0 + r, p = p0 + kk;
            v[q] = (i < nrow && p < t.K) ? masked(src[p + (int64_t)i * t.ldb], t.b_mask, p, i) : 0.f;
        }
#pragma unroll
        for (int q = 0; q < NL; q++) {
            const int e = threadIdx.x + 256 * q;
            tile[e / tc::kChunkK][e % tc::kChunkK] = v[q];
        }
    }
    __syncthreads();
    if constexpr (Cfg::kBf) {
        // BF16 image: 16-byte unit u = row (u / 16) * 8 + u % 8, K group (u / 8) % 2 (8 values each)
        const int64_t chunk = (jb.which == 0 ? t.a_hi : t.b_hi) + ((int64_t)jb.rt * t.nkc + jb.kc) * rows * 8;
        for (int u = threadIdx.x; u < rows * 2; u += blockDim.x) {
            const int r = (u >> 4) * 8 + (u & 7), kk = ((u >> 3) & 1) * 8;
            uint32_t h[4], l[4];
#pragma unroll
            for (int e = 0; e < 4; e++) {
                const float v0 = tile[r][kk + 2 * e], v1 = tile[r][kk + 2 * e + 1];
                const __nv_bfloat16 h0 = __float2bfloat16_rn(v0), h1 = __float2bfloat16_rn(v1);
                const __nv_bfloat16 l0 = __float2bfloat16_rn(v0 - __bfloat162float(h0));
                const __nv_bfloat16 l1 = __float2bfloat16_rn(v1 - __bfloat162float(h1));
                h[e] = (uint32_t)__bfloat16_as_ushort(h0) | ((uint32_t)__bfloat16_as_ushort(h1) << 16);
                l[e] = (uint32_t)__bfloat16_as_ushort(l0) | ((uint32_t)__bfloat16_as_ushort(l1) << 16);
            }
            *reinterpret_cast<uint4*>(pk + chunk + 4 * u) = make_uint4(h[0], h[1], h[2], h[3]);
            if constexpr (Cfg::kLo)
                *reinterpret_cast<uint4*>(pk + t.lo_off + chunk + 4 * u) = make_uint4(l[0], l[1], l[2], l[3]);
        }
        return;
    }
    const int64_t chunk = (jb.which == 0 ? t.a_hi : t.b_hi) + ((int64_t)jb.rt * t.nkc + jb.kc) * rows * tc::kChunkK;
    for (int u = threadIdx.x; u < rows * 4; u += blockDim.x) {
        const int r = (u >> 5) * 8 + (u & 7), kk = ((u >> 3) & 3) * 4;
        uint32_t h[4], l[4];
#pragma unroll
        for (int e = 0; e < 4; e++) {
            const float v = tile[r][kk + e];
            h[e] = tc::to_tf32(v);
            l[e] = tc::to_tf32(v - __uint_as_float(h[e]));
        }
        *reinterpret_cast<uint4*>(pk + chunk + 4 * u) = make_uint4(h[0], h[1], h[2], h[3]);
        *reinterpret_cast<uint4*>(pk + t.lo_off + chunk + 4 * u) = make_uint4(l[0], l[1], l[2], l[3]);
    }
}

// Persistent product kernel: one CTA per SM walks the tile list (tile
// b, b + gridDim.x, ...).  Warp 0 lane 0 streams operand chunks into the
// 4-stage ring across tile boundaries; warp 1 lane 0 issues the MMAs of tile
// i into TMEM accumulator i & 1 (2 x 256 columns) and commits it to acc_full;
// warps 2-5 (TMEM lane quarters 2, 3, 0, 1) drain the accumulator of tile i
// into C while tile i + 1 is being multiplied, then release it (acc_empty).
constexpr int kTcThreads = 192;

template <int MODE>
__global__ void __launch_bounds__(kTcThreads, 1) k_schur_tc(const TcTile* __restrict__ tiles, int ntiles,
                                                            const float* __restrict__ pk, Arenas<float> ar, DevStatus* st) {
    using Cfg = tc::ModeCfg<MODE>;
    extern __shared__ __align__(128) unsigned char smem_tc[];
    uint64_t* full = reinterpret_cast<uint64_t*>(smem_tc + tc::kStages * tc::kStageBytes);
    uint64_t* empty = full + tc::kStages;
    uint64_t* acc_full = empty + tc::kStages;  // [2]
    uint64_t* acc_empty = acc_full + 2;        // [2]
    uint64_t* drain = acc_empty + 2;
    uint32_t* taddr_slot = reinterpret_cast<uint32_t*>(drain + 1);
    __shared__ int s_fail_raw;
    volatile int& s_fail = s_fail_raw;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    if (threadIdx.x == 0) {
        for (int s = 0; s < tc::kStages; s++) {
            tc::mbar_init(&full[s], 1);
            tc::mbar_init(&empty[s], 1);
        }
        for (int b = 0; b < 2; b++) {
            tc::mbar_init(&acc_full[b], 1);
            tc::mbar_init(&acc_empty[b], 4);  // one arrive per epilogue warp
        }
        tc::mbar_init(drain, 1);
        s_fail = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(tc::smem_u32(taddr_slot)),
                     "r"(2 * tc::kTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = *taddr_slot;

    if (warp == 0) {
        if (lane == 0) {  // producer
            int g = 0;  // stage counter across this CTA's tiles
            bool ok = true;
            // stage layout: A_hi (kCps chunks), A_lo, B_hi, B_lo; a tile's last stage may hold fewer chunks
            constexpr int kA = Cfg::kCps * Cfg::kFloatsA * 4, kB = Cfg::kCps * Cfg::kFloatsB * 4;
            constexpr int kLoA = Cfg::kLo ? kA : 0;
            for (int ti = blockIdx.x; ti < ntiles && ok; ti += gridDim.x) {
                const TcTile t = tiles[ti];
                for (int c = 0; c < t.nkc; c += Cfg::kCps, g++) {
                    const int s = g % tc::kStages;
                    if (g >= tc::kStages) ok = tc::mbar_wait_bounded(&empty[s], ((g / tc::kStages) - 1) & 1, tc::kWaitLimit);
                    if (!ok || s_fail) {
                        ok = false;
                        break;
                    }
                    const int nv = min(Cfg::kCps, t.nkc - c);
                    const uint32_t ba = nv * Cfg::kFloatsA * 4, bb = nv * Cfg::kFloatsB * 4;
                    unsigned char* dst = smem_tc + s * tc::kStageBytes;
                    tc::mbar_expect_tx(&full[s], (ba + bb) * (Cfg::kLo ? 2u : 1u));
                    const float* a = pk + t.a_hi + (int64_t)c * Cfg::kFloatsA;
                    const float* b = pk + t.b_hi + (int64_t)c * Cfg::kFloatsB;
                    tc::bulk_g2s(dst, a, ba, &full[s]);
                    if constexpr (Cfg::kLo) tc::bulk_g2s(dst + kA, a + t.lo_off, ba, &full[s]);
                    tc::bulk_g2s(dst + kA + kLoA, b, bb, &full[s]);
                    if constexpr (Cfg::kLo) tc::bulk_g2s(dst + kA + kLoA + kB, b + t.lo_off, bb, &full[s]);
                }
            }
            if (!ok) {
                s_fail = 1;
                // let the copies already issued land before the CTA can exit
                for (int c = max(0, g - tc::kStages); c < g; c++)
                    tc::mbar_wait_bounded(&full[c % tc::kStages], (c / tc::kStages) & 1, tc::kWaitLimit);
            }
        }
        __syncwarp();
    } else if (warp == 1) {
        if (lane == 0) {  // MMA issuer
            constexpr uint32_t idesc = Cfg::kBf ? tc::idesc_bf16(tc::kTileM, tc::kTileN) : tc::idesc_tf32(tc::kTileM, tc::kTileN);
            constexpr int kA = Cfg::kCps * Cfg::kFloatsA * 4, kB = Cfg::kCps * Cfg::kFloatsB * 4;
            constexpr int kLoA = Cfg::kLo ? kA : 0;
            int g = 0, i = 0;
            bool ok = true;
            for (int ti = blockIdx.x; ti < ntiles && ok; ti += gridDim.x, i++) {
                const TcTile t = tiles[ti];
                const int buf = i & 1;
                const uint32_t acc = tmem + buf * tc::kTmemCols;
                if (i >= 2) ok = tc::mbar_wait_bounded(&acc_empty[buf], ((i >> 1) - 1) & 1, tc::kWaitLimit);
                if (!ok) break;
                tc::fence_after_sync();
                for (int c = 0; c < t.nkc; c += Cfg::kCps, g++) {
                    const int s = g % tc::kStages;
                    ok = tc::mbar_wait_bounded(&full[s], (g / tc::kStages) & 1, tc::kWaitLimit);
                    if (!ok || s_fail) {
                        ok = false;
                        break;
                    }
                    tc::fence_after_sync();
                    const int nv = min(Cfg::kCps, t.nkc - c);
                    const uint32_t sa0 = tc::smem_u32(smem_tc + s * tc::kStageBytes);
                    for (int j = 0; j < nv; j++) {
                        const uint32_t sa = sa0 + j * Cfg::kFloatsA * 4, sal = sa + kA;
                        const uint32_t sb = sa0 + kA + kLoA + j * Cfg::kFloatsB * 4, sbl = sb + kB;
                        if constexpr (Cfg::kBf) {  // one K = 16 MMA per chunk (bf16: two 16-byte K groups)
                            const uint64_t dah = tc::smem_desc(sa, 128, Cfg::kSbo), dbh = tc::smem_desc(sb, 128, Cfg::kSbo);
                            if constexpr (Cfg::kLo) {
                                const uint64_t dal = tc::smem_desc(sal, 128, Cfg::kSbo), dbl = tc::smem_desc(sbl, 128, Cfg::kSbo);
                                tc::mma_bf16(acc, dal, dbh, idesc, (c == 0 && j == 0) ? 0u : 1u);
                                tc::mma_bf16(acc, dah, dbl, idesc, 1u);
                                tc::mma_bf16(acc, dah, dbh, idesc, 1u);
                            } else {
                                tc::mma_bf16(acc, dah, dbh, idesc, (c == 0 && j == 0) ? 0u : 1u);
                            }
                        } else {
#pragma unroll
                            for (int ks = 0; ks < tc::kChunkK / 8; ks++) {  // K = 8 per MMA: two 16-byte K groups
                                const uint32_t ko = ks * 256;
                                const uint64_t dah = tc::smem_desc(sa + ko, 128, 512), dal = tc::smem_desc(sal + ko, 128, 512);
                                const uint64_t dbh = tc::smem_desc(sb + ko, 128, 512), dbl = tc::smem_desc(sbl + ko, 128, 512);
                                tc::mma_tf32(acc, dal, dbh, idesc, (c == 0 && j == 0 && ks == 0) ? 0u : 1u);
                                tc::mma_tf32(acc, dah, dbl, idesc, 1u);
                                tc::mma_tf32(acc, dah, dbh, idesc, 1u);
                            }
                        }
                    }
                    tc::mma_commit(&empty[s]);
                }
                tc::mma_commit(&acc_full[buf]);  // the accumulator is complete when these MMAs are
            }
            if (!ok) {
                s_fail = 1;
                // no MMA may still be writing TMEM when it is freed
                tc::mma_commit(drain);
                tc::mbar_wait_bounded(drain, 0, tc::kWaitLimit);
            }
        }
        __syncwarp();
    } else {  // epilogue warps 2..5: TMEM lanes 32 (warp % 4) ..
        const int q = warp & 3;
        const int row = 32 * q + lane;
        int i = 0;
        for (int ti = blockIdx.x; ti < ntiles; ti += gridDim.x, i++) {
            const TcTile t = tiles[ti];
            const int buf = i & 1;
            bool ok = tc::mbar_wait_bounded(&acc_full[buf], (i >> 1) & 1, tc::kWaitLimit);
            ok = __all_sync(0xffffffffu, ok);
            if (!ok) {
                if (lane == 0) s_fail = 1;
                break;
            }
            tc::fence_after_sync();
            float* crow = ar.a[t.c_ar] + t.c_off + row;
#pragma unroll 1
            for (int cg = 0; cg < tc::kTileN / 32; cg++) {
                if (cg * 32 >= t.ncols) break;
                float v[32], cv[32];
                float* cp = crow + (int64_t)(cg * 32) * t.ldc;
                const int nj = min(32, t.ncols - cg * 32);
                // all loads of the row segment first, then the stores: a load-store-load chain on
                // possibly aliasing addresses would serialise 32 memory round trips
                if (row < t.mrows && t.op == 0) {
#pragma unroll
                    for (int j = 0; j < 32; j++) cv[j] = j < nj ? cp[(int64_t)j * t.ldc] : 0.f;
                }
                tc::tmem_ld32(tmem + buf * tc::kTmemCols + ((uint32_t)(32 * q) << 16) + cg * 32, v);
                if (row < t.mrows) {
#pragma unroll
                    for (int j = 0; j < 32; j++)
                        if (j < nj) cp[(int64_t)j * t.ldc] = t.op == 0 ? cv[j] - v[j] : (t.op == 1 ? v[j] : -v[j]);
                }
            }
            tc::fence_before_sync();
            __syncwarp();
            if (lane == 0) tc::mbar_arrive(&acc_empty[buf]);
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    if (s_fail && threadIdx.x == 0) atomicOr(&st->timeout, 1);
    if (warp == 0) {
        tc::fence_after_sync();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(2 * tc::kTmemCols) : "memory");
    }
}

// ---------------------------------------------------------------------------
// Tensor-core product that splits its FP32 operands itself (no pack pass).
// Same tile (128 x 256), accumulators, epilogue and bounded waits as
// k_schur_tc<kTf32x3>; the producer is two groups of four warps instead of one
// bulk-copy thread.  Group q fills the ring stages g with g % 2 == q: each
// thread loads its share of the stage's 128 x 16 slice of A and 256 x 16
// slice of B^T straight from the arenas (any leading dimension: element
// loads, coalesced across the warp), splits every value into tf32 hi and lo
// and stores them as 16-byte rows of the MMA's core matrices; then a proxy
// fence makes the shared-memory writes visible to the tensor core and one
// lane per warp arrives on the stage's barrier (4 arrivals fill a stage).
struct TcTileD {
    int64_t a_off, b_off, c_off;  // operand origins of the product, the tile's (0, 0) in C
    int32_t lda, ldb, ldc;
    int32_t M, N, K;              // the product's extents
    int32_t i0, j0;               // the tile's first row and column within the product
    int8_t a_ar, b_ar, c_ar, op, a_mask, b_mask, pad[2];
};

constexpr int kTcdProducerWarps = 8;
constexpr int kTcdThreads = (kTcdProducerWarps + 1 + 4) * 32;  // producers, MMA issuer, 4 epilogue warps

__global__ void __launch_bounds__(kTcdThreads, 1) k_tc_direct(const TcTileD* __restrict__ tiles, int ntiles,
                                                              Arenas<float> ar, DevStatus* st) {
    extern __shared__ __align__(128) unsigned char smem_tc[];
    uint64_t* full = reinterpret_cast<uint64_t*>(smem_tc + tc::kStages * tc::kStageBytes);
    uint64_t* empty = full + tc::kStages;
    uint64_t* acc_full = empty + tc::kStages;  // [2]
    uint64_t* acc_empty = acc_full + 2;        // [2]
    uint64_t* drain = acc_empty + 2;
    uint32_t* taddr_slot = reinterpret_cast<uint32_t*>(drain + 1);
    __shared__ int s_fail_raw;
    volatile int& s_fail = s_fail_raw;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    constexpr int kMmaWarp = kTcdProducerWarps;
    constexpr int kA = tc::kChunkA * 4, kB = tc::kChunkB * 4;  // bytes of one hi (or lo) image

    if (threadIdx.x == 0) {
        for (int s = 0; s < tc::kStages; s++) {
            tc::mbar_init(&full[s], 4);
            tc::mbar_init(&empty[s], 1);
        }
        for (int b = 0; b < 2; b++) {
            tc::mbar_init(&acc_full[b], 1);
            tc::mbar_init(&acc_empty[b], 4);
        }
        tc::mbar_init(drain, 1);
        s_fail = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == kMmaWarp) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(tc::smem_u32(taddr_slot)),
                     "r"(2 * tc::kTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = *taddr_slot;

    if (warp < kTcdProducerWarps) {
        const int grp = warp >> 2, t = threadIdx.x & 127;  // producer group, thread within the group
        int g = 0;
        bool ok = true;
        for (int ti = blockIdx.x; ti < ntiles && ok; ti += gridDim.x) {
            const TcTileD tl = tiles[ti];
            const float* A = ar.a[tl.a_ar] + tl.a_off;
            const float* B = ar.a[tl.b_ar] + tl.b_off;
            const int nkc = (tl.K + tc::kChunkK - 1) / tc::kChunkK;
            for (int c = 0; c < nkc; c++, g++) {
                if ((g & 1) != grp) continue;
                const int s = g % tc::kStages;
                if (g >= tc::kStages) ok = tc::mbar_wait_bounded(&empty[s], ((g / tc::kStages) - 1) & 1, tc::kWaitLimit);
                if (!ok || s_fail) {
                    ok = false;
                    break;
                }
                const int p0 = c * tc::kChunkK;
                // A: 512 (row, K group) units, 4 per thread; B^T: 1024 units, 8 per thread.  All loads first.
                float va[4][4], vb[8][4];
#pragma unroll
                for (int q = 0; q < 4; q++) {
                    const int u = t + 128 * q, r = u & 127, kg = u >> 7;
                    const int i = tl.i0 + r;
#pragma unroll
                    for (int e = 0; e < 4; e++) {
                        const int p = p0 + 4 * kg + e;
                        va[q][e] = (i < tl.M && p < tl.K) ? masked(A[i + (int64_t)p * tl.lda], (int)tl.a_mask, i, p) : 0.f;
                    }
                }
#pragma unroll
                for (int q = 0; q < 8; q++) {
                    const int u = t + 128 * q, kg = u & 3, jr = u >> 2;
                    const int j = tl.j0 + jr;
#pragma unroll
                    for (int e = 0; e < 4; e++) {
                        const int p = p0 + 4 * kg + e;
                        vb[q][e] = (j < tl.N && p < tl.K) ? masked(B[p + (int64_t)j * tl.ldb], (int)tl.b_mask, p, j) : 0.f;
                    }
                }
                unsigned char* dst = smem_tc + s * tc::kStageBytes;
#pragma unroll
                for (int q = 0; q < 4; q++) {
                    const int u = t + 128 * q, r = u & 127, kg = u >> 7;
                    uint32_t h[4], l[4];
#pragma unroll
                    for (int e = 0; e < 4; e++) {
                        h[e] = tc::to_tf32(va[q][e]);
                        l[e] = tc::to_tf32(va[q][e] - __uint_as_float(h[e]));
                    }
                    const int off = (r >> 3) * 512 + kg * 128 + (r & 7) * 16;
                    *reinterpret_cast<uint4*>(dst + off) = make_uint4(h[0], h[1], h[2], h[3]);
                    *reinterpret_cast<uint4*>(dst + kA + off) = make_uint4(l[0], l[1], l[2], l[3]);
                }
#pragma unroll
                for (int q = 0; q < 8; q++) {
                    const int u = t + 128 * q, kg = u & 3, jr = u >> 2;
                    uint32_t h[4], l[4];
#pragma unroll
                    for (int e = 0; e < 4; e++) {
                        h[e] = tc::to_tf32(vb[q][e]);
                        l[e] = tc::to_tf32(vb[q][e] - __uint_as_float(h[e]));
                    }
                    const int off = (jr >> 3) * 512 + kg * 128 + (jr & 7) * 16;
                    *reinterpret_cast<uint4*>(dst + 2 * kA + off) = make_uint4(h[0], h[1], h[2], h[3]);
                    *reinterpret_cast<uint4*>(dst + 2 * kA + kB + off) = make_uint4(l[0], l[1], l[2], l[3]);
                }
                tc::fence_proxy_async();  // generic-proxy writes -> visible to the tensor core
                __syncwarp();
                if (lane == 0) tc::mbar_arrive(&full[s]);
            }
        }
        if (!ok) s_fail = 1;
        __syncwarp();
    } else if (warp == kMmaWarp) {
        if (lane == 0) {  // MMA issuer: as k_schur_tc<kTf32x3>
            constexpr uint32_t idesc = tc::idesc_tf32(tc::kTileM, tc::kTileN);
            int g = 0, i = 0;
            bool ok = true;
            for (int ti = blockIdx.x; ti < ntiles && ok; ti += gridDim.x, i++) {
                const TcTileD tl = tiles[ti];
                const int nkc = (tl.K + tc::kChunkK - 1) / tc::kChunkK;
                const int buf = i & 1;
                const uint32_t acc = tmem + buf * tc::kTmemCols;
                if (i >= 2) ok = tc::mbar_wait_bounded(&acc_empty[buf], ((i >> 1) - 1) & 1, tc::kWaitLimit);
                if (!ok) break;
                tc::fence_after_sync();
                for (int c = 0; c < nkc; c++, g++) {
                    const int s = g % tc::kStages;
                    ok = tc::mbar_wait_bounded(&full[s], (g / tc::kStages) & 1, tc::kWaitLimit);
                    if (!ok || s_fail) {
                        ok = false;
                        break;
                    }
                    tc::fence_after_sync();
                    const uint32_t sa = tc::smem_u32(smem_tc + s * tc::kStageBytes);
                    const uint32_t sal = sa + kA, sb = sa + 2 * kA, sbl = sb + kB;
#pragma unroll
                    for (int ks = 0; ks < tc::kChunkK / 8; ks++) {
                        const uint32_t ko = ks * 256;
                        const uint64_t dah = tc::smem_desc(sa + ko, 128, 512), dal = tc::smem_desc(sal + ko, 128, 512);
                        const uint64_t dbh = tc::smem_desc(sb + ko, 128, 512), dbl = tc::smem_desc(sbl + ko, 128, 512);
                        tc::mma_tf32(acc, dal, dbh, idesc, (c == 0 && ks == 0) ? 0u : 1u);
                        tc::mma_tf32(acc, dah, dbl, idesc, 1u);
                        tc::mma_tf32(acc, dah, dbh, idesc, 1u);
                    }
                    tc::mma_commit(&empty[s]);
                }
                tc::mma_commit(&acc_full[buf]);
            }
            if (!ok) {
                s_fail = 1;
                tc::mma_commit(drain);
                tc::mbar_wait_bounded(drain, 0, tc::kWaitLimit);
            }
        }
        __syncwarp();
    } else {  // epilogue warps: TMEM lanes 32 (warp % 4) ..
        const int q = warp & 3;
        const int row = 32 * q + lane;
        int i = 0;
        for (int ti = blockIdx.x; ti < ntiles; ti += gridDim.x, i++) {
            const TcTileD tl = tiles[ti];
            const int buf = i & 1;
            bool ok = tc::mbar_wait_bounded(&acc_full[buf], (i >> 1) & 1, tc::kWaitLimit);
            ok = __all_sync(0xffffffffu, ok);
            if (!ok) {
                if (lane == 0) s_fail = 1;
                break;
            }
            tc::fence_after_sync();
            const int mrows = min(tc::kTileM, tl.M - tl.i0), ncols = min(tc::kTileN, tl.N - tl.j0);
            float* crow = ar.a[tl.c_ar] + tl.c_off + row;
#pragma unroll 1
            for (int cg = 0; cg < tc::kTileN / 32; cg++) {
                if (cg * 32 >= ncols) break;
                float v[32], cv[32];
                float* cp = crow + (int64_t)(cg * 32) * tl.ldc;
                const int nj = min(32, ncols - cg * 32);
                if (row < mrows && tl.op == 0) {
#pragma unroll
                    for (int j = 0; j < 32; j++) cv[j] = j < nj ? cp[(int64_t)j * tl.ldc] : 0.f;
                }
                tc::tmem_ld32(tmem + buf * tc::kTmemCols + ((uint32_t)(32 * q) << 16) + cg * 32, v);
                if (row < mrows) {
#pragma unroll
                    for (int j = 0; j < 32; j++)
                        if (j < nj) cp[(int64_t)j * tl.ldc] = tl.op == 0 ? cv[j] - v[j] : (tl.op == 1 ? v[j] : -v[j]);
                }
            }
            tc::fence_before_sync();
            __syncwarp();
            if (lane == 0) tc::mbar_arrive(&acc_empty[buf]);
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    if (s_fail && threadIdx.x == 0) atomicOr(&st->timeout, 1);
    if (warp == kMmaWarp) {
        tc::fence_after_sync();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(2 * tc::kTmemCols) : "memory");
    }
}
