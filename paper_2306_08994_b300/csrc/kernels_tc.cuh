// Tensor-core Schur update on sm_100-family (B300 = sm_103a): C -= A B with
// tcgen05.mma kind::tf32, FP32 accumulation in tensor memory (TMEM).
//
// Accuracy: every operand x is split into x_hi = tf32(x) and x_lo = x - x_hi
// (exact in FP32), and A B is accumulated as A_hi B_hi + A_hi B_lo + A_lo B_hi
// (three MMAs per K slice): products accurate to about 2^-21 relative, i.e.
// FP32-grade Schur complements, which the FP64 refinement needs.
//
// Tile: 128 x 128 of C per CTA (4 warps), K staged 32 at a time in two
// shared-memory buffers.  Operand tiles are written by the threads in the
// K-major, no-swizzle canonical layout of core matrices (8 rows x 16 bytes):
// core (row group r, K group g) at byte r*1024 + g*128, i.e. leading
// (K-direction) byte offset 128 and stride (row-direction) byte offset 1024.
// One thread issues the MMAs of a stage and commits them to that buffer's
// mbarrier; the threads wait on it (bounded) before refilling the buffer.
// The epilogue reads TMEM with tcgen05.ld (warp w owns lanes 32w..32w+31 =
// rows) and subtracts the product from C in global memory.
#pragma once

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

constexpr int kTileM = 128, kTileN = 128, kTileK = 32;
constexpr int kOpBytes = kTileM * kTileK * 4;       // one operand tile (hi or lo): 16 KB
constexpr int kStageBytes = 4 * kOpBytes;           // A_hi, A_lo, B_hi, B_lo
constexpr int kSmemBytes = 2 * kStageBytes + 1024;  // two stages + barriers / TMEM address
constexpr uint64_t kWaitLimit = 1000000000ull;  // 1 s

}  // namespace tc

// Stage a 128 x 32 slice of a column-major operand into core-matrix layout.
//   rows_contig = true : operand element (row, k) at base[row + k*ld]  (A, M-contiguous)
//   rows_contig = false: operand element (row, k) at base[k + row*ld]  (B stored K x N, K-contiguous)
__device__ __forceinline__ void tc_stage(const float* __restrict__ base, int ld, int nrows, int nk, int k0,
                                         bool rows_contig, unsigned char* hi, unsigned char* lo) {
    const int t = threadIdx.x;  // 128 threads
    for (int it = 0; it < 8; it++) {
        int row, g;
        if (rows_contig) {
            row = t;
            g = it;
        } else {
            row = it * 16 + (t >> 3);
            g = t & 7;
        }
        float v[4];
#pragma unroll
        for (int q = 0; q < 4; q++) {
            const int k = k0 + 4 * g + q;
            v[q] = (row < nrows && k < nk) ? (rows_contig ? base[row + (int64_t)k * ld] : base[k + (int64_t)row * ld]) : 0.f;
        }
        uint32_t h[4], l[4];
#pragma unroll
        for (int q = 0; q < 4; q++) {
            h[q] = tc::to_tf32(v[q]);
            l[q] = tc::to_tf32(v[q] - __uint_as_float(h[q]));
        }
        const int off = (row >> 3) * 1024 + g * 128 + (row & 7) * 16;
        *reinterpret_cast<uint4*>(hi + off) = make_uint4(h[0], h[1], h[2], h[3]);
        *reinterpret_cast<uint4*>(lo + off) = make_uint4(l[0], l[1], l[2], l[3]);
    }
}

__global__ void __launch_bounds__(128) k_gemm_tc(const GemmTile* __restrict__ tiles, Arenas<float> ar, DevStatus* st) {
    extern __shared__ __align__(128) unsigned char smem_tc[];
    unsigned char* stage[2] = {smem_tc, smem_tc + tc::kStageBytes};
    uint64_t* mbar = reinterpret_cast<uint64_t*>(smem_tc + 2 * tc::kStageBytes);
    uint32_t* taddr_slot = reinterpret_cast<uint32_t*>(smem_tc + 2 * tc::kStageBytes + 64);
    const GemmTile t = tiles[blockIdx.x];
    const float* A = ar.a[t.a_ar] + t.a_off + t.i0;                  // rows i0.. of A (M x K, column-major)
    const float* B = ar.a[t.b_ar] + t.b_off + (int64_t)t.j0 * t.ldb;  // columns j0.. of B (K x N, column-major)
    float* C = ar.a[t.c_ar] + t.c_off;
    const int mrows = min(tc::kTileM, t.M - t.i0), ncols = min(tc::kTileN, t.N - t.j0);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    if (threadIdx.x == 0) {
        tc::mbar_init(&mbar[0], 1);
        tc::mbar_init(&mbar[1], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(tc::smem_u32(taddr_slot)),
                     "r"(128u)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = *taddr_slot;
    constexpr uint32_t idesc = tc::idesc_tf32(tc::kTileM, tc::kTileN);
    const int nst = (t.K + tc::kTileK - 1) / tc::kTileK;
    bool ok = true;
    for (int s = 0; s < nst && ok; s++) {
        const int b = s & 1;
        if (s >= 2) ok = tc::mbar_wait_bounded(&mbar[b], ((s >> 1) - 1) & 1, tc::kWaitLimit);
        if (!__syncthreads_and(ok)) {
            ok = false;
            break;
        }
        unsigned char* ahi = stage[b];
        unsigned char* alo = ahi + tc::kOpBytes;
        unsigned char* bhi = alo + tc::kOpBytes;
        unsigned char* blo = bhi + tc::kOpBytes;
        tc_stage(A, t.lda, mrows, t.K, s * tc::kTileK, true, ahi, alo);
        tc_stage(B, t.ldb, ncols, t.K, s * tc::kTileK, false, bhi, blo);
        tc::fence_proxy_async();
        __syncthreads();
        if (threadIdx.x == 0) {
            tc::fence_after_sync();
#pragma unroll
            for (int ks = 0; ks < tc::kTileK / 8; ks++) {  // K = 8 per MMA: two K groups of 16 bytes
                const uint32_t koff = ks * 256;
                const uint64_t dah = tc::smem_desc(tc::smem_u32(ahi) + koff, 128, 1024);
                const uint64_t dal = tc::smem_desc(tc::smem_u32(alo) + koff, 128, 1024);
                const uint64_t dbh = tc::smem_desc(tc::smem_u32(bhi) + koff, 128, 1024);
                const uint64_t dbl = tc::smem_desc(tc::smem_u32(blo) + koff, 128, 1024);
                const uint32_t first = (s == 0 && ks == 0) ? 0u : 1u;
                tc::mma_tf32(tmem, dal, dbh, idesc, first);
                tc::mma_tf32(tmem, dah, dbl, idesc, 1u);
                tc::mma_tf32(tmem, dah, dbh, idesc, 1u);
            }
            tc::mma_commit(&mbar[b]);
        }
    }
    if (ok && nst > 0) ok = tc::mbar_wait_bounded(&mbar[(nst - 1) & 1], ((nst - 1) >> 1) & 1, tc::kWaitLimit);
    ok = __syncthreads_and(ok);
    tc::fence_after_sync();
    if (ok && nst > 0) {
        const int row = 32 * warp + lane;
#pragma unroll 1
        for (int cg = 0; cg < tc::kTileN / 32; cg++) {
            float v[32];
            tc::tmem_ld32(tmem + ((uint32_t)(32 * warp) << 16) + cg * 32, v);
            if (row < mrows) {
                float* crow = C + (t.i0 + row) + (int64_t)(t.j0 + cg * 32) * t.ldc;
#pragma unroll
                for (int j = 0; j < 32; j++)
                    if (cg * 32 + j < ncols) crow[(int64_t)j * t.ldc] -= v[j];
            }
        }
    } else if (!ok && threadIdx.x == 0) {
        atomicOr(&st->timeout, 1);
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(128u) : "memory");
}
