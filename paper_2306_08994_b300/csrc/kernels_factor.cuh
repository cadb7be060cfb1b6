// Factorization kernels: one batched pass per Foata class (Sec. 3.3).
//
// Every kernel is launched over a precomputed task list (a "bag of tasks",
// Sec. 3.3): the fronts of one class, or tiles of them, in any order; the
// launch boundary is the barrier between classes.
#pragma once

#include <cstdint>

#include "mf_internal.h"

struct DevStatus {
    unsigned long long n_perturbed;
    unsigned long long first;  // (front << 32) | pivot of the first small pivot (min)
    int nonfinite;
    int timeout;
};

// Asynchronous global -> shared copies of single elements (cp.async): many
// copies stay in flight per thread, unlike a load-then-store loop whose every
// shared store waits for its own global load.
template <typename T>
__device__ __forceinline__ void cp_async_elem(T* smem_dst, const T* gmem_src) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem_dst);
    if constexpr (sizeof(T) == 8)
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gmem_src) : "memory");
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gmem_src) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

template <typename T>
__device__ __forceinline__ T tiny_pivot() { return sizeof(T) == 8 ? (T)1e-300 : (T)1e-37f; }

// Static pivot check (no pivoting, Table 2 divides unconditionally): a pivot
// below thr in magnitude is replaced by sign(p)*thr.  Returns the pivot to use.
template <typename T>
__device__ __forceinline__ T checked_pivot(T piv, T thr, bool record, int32_t front, int32_t p, DevStatus* st) {
    bool bad = !(fabs(piv) >= thr);
    if (bad) {
        if (record) {
            atomicAdd(&st->n_perturbed, 1ull);
            atomicMin(&st->first, ((unsigned long long)(uint32_t)front << 32) | (uint32_t)p);
            if (!isfinite(piv)) atomicOr(&st->nonfinite, 1);
        }
        piv = (piv < T(0)) ? -thr : thr;
    }
    return piv;
}

template <typename T>
__device__ __forceinline__ T block_max_abs(T v, float* red) {
    // v >= 0 expected; returns the max over the block (all threads)
    for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
    int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) red[w] = (float)v;
    __syncthreads();
    float r = 0.f;
    int nw = blockDim.x >> 5;
    for (int i = 0; i < nw; i++) r = fmaxf(r, red[i]);
    return (T)r;
}

// ---------------------------------------------------------------------------
// Fused small front: one CTA per front, the whole front in shared memory.
// Extend-add (or the element matrix at a leaf), partial LU on the k pivots
// with the division (T1), multiplication (T2) and subtraction (T3) tasks of
// Sec. 3 / Table 2, then P, R and the Schur complement S written out.
// Dynamic shared memory: ldm*maxm T + maxm T + 2*maxm int32 + 32 floats.
template <typename T>
__global__ void __launch_bounds__(256) k_front_fused(const FrontDev* __restrict__ fronts, const int32_t* __restrict__ list,
                                                     const int32_t* __restrict__ maps, const double* __restrict__ values,
                                                     int npe, T* __restrict__ fac, T* __restrict__ cbs, int maxm, int ldm,
                                                     double tol_rel, DevStatus* st) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* F = reinterpret_cast<T*>(smem_raw);
    T* urow = F + (size_t)ldm * maxm;
    int32_t* imap = reinterpret_cast<int32_t*>(urow + maxm);
    float* red = reinterpret_cast<float*>(imap + 2 * maxm);

    const int32_t f = list[blockIdx.x];
    const FrontDev fr = fronts[f];
    const int m = fr.m, k = fr.k, nc = m - k;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;

    const int nmap = fr.nchild > 0 ? fr.nchild * m : m;
    for (int i = threadIdx.x; i < nmap; i += blockDim.x) imap[i] = maps[fr.map_off + i];
    __syncthreads();

    // ---- assembly
    T amax = T(0);
    if (fr.nchild == 0) {
        const double* K = values + (int64_t)fr.elem * npe * npe;
        for (int j = warp; j < m; j += nwarp) {
            const int b = imap[j];
            for (int i = lane; i < m; i += 32) {
                T v = (T)K[imap[i] + b * npe];
                F[i + j * ldm] = v;
                amax = max(amax, (T)fabs(v));
            }
        }
    } else {
        const FrontDev c0 = fronts[fr.child[0]];
        const int n0 = c0.m - c0.k;
        const T* S0 = cbs + c0.S_off;
        const T* S1 = nullptr;
        int n1 = 0;
        if (fr.nchild > 1) {
            const FrontDev c1 = fronts[fr.child[1]];
            n1 = c1.m - c1.k;
            S1 = cbs + c1.S_off;
        }
        for (int j = warp; j < m; j += nwarp) {
            const int j0 = imap[j];
            const int j1 = fr.nchild > 1 ? imap[m + j] : -1;
            for (int i = lane; i < m; i += 32) {
                T v = T(0);
                int i0 = imap[i];
                if (i0 >= 0 && j0 >= 0) v += S0[i0 + (int64_t)j0 * n0];
                if (j1 >= 0) {
                    int i1 = imap[m + i];
                    if (i1 >= 0) v += S1[i1 + (int64_t)j1 * n1];
                }
                F[i + j * ldm] = v;
                amax = max(amax, (T)fabs(v));
            }
        }
    }
    amax = block_max_abs(amax, red);  // includes __syncthreads
    const T thr = (T)tol_rel * amax > T(0) ? (T)tol_rel * amax : tiny_pivot<T>();

    // ---- partial LU on the fully assembled pivots (Table 2 compute_front)
    for (int p = 0; p < k; p++) {
        T piv = checked_pivot(F[p + p * ldm], thr, threadIdx.x == 0, f, p, st);
        // T1: divide the pivot row right of the pivot
        for (int j = p + 1 + threadIdx.x; j < m; j += blockDim.x) {
            T u = F[p + j * ldm] / piv;
            F[p + j * ldm] = u;
            urow[j] = u;
        }
        if (threadIdx.x == 0) F[p + p * ldm] = piv;
        __syncthreads();
        // T2/T3: trailing block update
        for (int j = p + 1 + warp; j < m; j += nwarp) {
            const T u = urow[j];
            for (int i = p + 1 + lane; i < m; i += 32) F[i + j * ldm] -= F[i + p * ldm] * u;
        }
        __syncthreads();
    }

    // ---- write P (m x k), R (k x nc), S (nc x nc)
    T* P = fac + fr.P_off;
    for (int j = warp; j < k; j += nwarp)
        for (int i = lane; i < m; i += 32) P[i + (int64_t)j * m] = F[i + j * ldm];
    T* R = fac + fr.R_off;
    for (int j = k + warp; j < m; j += nwarp)
        for (int i = lane; i < k; i += 32) R[i + (int64_t)(j - k) * k] = F[i + j * ldm];
    T* S = cbs + fr.S_off;
    for (int j = k + warp; j < m; j += nwarp)
        for (int i = k + lane; i < m; i += 32) S[(i - k) + (int64_t)(j - k) * nc] = F[i + j * ldm];
}

// ---------------------------------------------------------------------------
// Large fronts.  Assembly of 64x64 tiles straight into P, R and S; the
// per-front max |entry| (for the static pivot threshold) by atomicMax on the
// float bit pattern (non-negative floats order like their bits).
struct AsmTile {
    int32_t front, i0, j0, pad;
};

template <typename T>
__global__ void __launch_bounds__(256) k_assemble_large(const FrontDev* __restrict__ fronts, const AsmTile* __restrict__ tiles,
                                                        const int32_t* __restrict__ maps, T* __restrict__ fac,
                                                        T* __restrict__ cbs, unsigned int* __restrict__ famax) {
    __shared__ float red[8];
    const AsmTile t = tiles[blockIdx.x];
    const FrontDev fr = fronts[t.front];
    const int m = fr.m, k = fr.k, nc = m - k;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const FrontDev c0 = fronts[fr.child[0]];
    const int n0 = c0.m - c0.k;
    const T* S0 = cbs + c0.S_off;
    const T* S1 = nullptr;
    int n1 = 0;
    const bool two = fr.nchild > 1;
    if (two) {
        const FrontDev c1 = fronts[fr.child[1]];
        n1 = c1.m - c1.k;
        S1 = cbs + c1.S_off;
    }
    const int32_t* map0 = maps + fr.map_off;
    const int32_t* map1 = map0 + m;
    int ri[2], r0[2], r1[2];
    for (int q = 0; q < 2; q++) {
        ri[q] = t.i0 + lane + 32 * q;
        r0[q] = ri[q] < m ? map0[ri[q]] : -1;
        r1[q] = (two && ri[q] < m) ? map1[ri[q]] : -1;
    }
    T amax = T(0);
    for (int jj = warp; jj < 64; jj += 8) {
        const int j = t.j0 + jj;
        if (j >= m) break;
        const int cj0 = map0[j];
        const int cj1 = two ? map1[j] : -1;
        for (int q = 0; q < 2; q++) {
            const int i = ri[q];
            if (i >= m) continue;
            T v = T(0);
            if (r0[q] >= 0 && cj0 >= 0) v += S0[r0[q] + (int64_t)cj0 * n0];
            if (r1[q] >= 0 && cj1 >= 0) v += S1[r1[q] + (int64_t)cj1 * n1];
            amax = max(amax, (T)fabs(v));
            if (j < k) fac[fr.P_off + i + (int64_t)j * m] = v;
            else if (i < k) fac[fr.R_off + i + (int64_t)(j - k) * k] = v;
            else cbs[fr.S_off + (i - k) + (int64_t)(j - k) * nc] = v;
        }
    }
    for (int o = 16; o > 0; o >>= 1) amax = max(amax, __shfl_xor_sync(0xffffffffu, amax, o));
    if (lane == 0) red[warp] = (float)amax;
    __syncthreads();
    if (threadIdx.x == 0) {
        float r = 0.f;
        for (int i = 0; i < 8; i++) r = fmaxf(r, red[i]);
        atomicMax(famax + t.front, __float_as_uint(r));
    }
}

// Panel step of the blocked partial LU (large fronts), pivot block
// [kb, kb+w), w <= 64:
//   k_panel_diag: D = F[kb:kb+w, kb:kb+w] = L_D U_D by the Table 2 tasks
//     (division of the pivot row, then multiplication/subtraction on the
//     trailing block) with the static pivot check, written back to P; and
//     the inverses L_D^-1, U_D^-1 packed into the front's panel slot.
//   then one batched k_gemm launch, in place:
//     L21 = F[kb+w:m, kb:kb+w] U_D^-1,   U12 = L_D^-1 F[kb:kb+w, kb+w:m]
//   (each output tile spans the whole w-wide side, so it reads all of its
//   input before writing), then the trailing update k_gemm.
// One CTA per front.
struct DiagTask {
    int32_t front, kb, w, pad;
    int64_t slot;  // panel-slot offset (64 x 64, column-major, ld 64)
};

// One CTA per pivot block, NB/4 x NB/4 threads, each owning a 4x4 register
// tile (rows 4*tr.., columns 4*tc..).  Per pivot the owners of the pivot
// column and row publish them to double-buffered shared memory, one barrier,
// then every thread applies the rank-1 update to its own tile (masked to
// the trailing block).  The block is padded with the identity beyond w.
// The two inverse sweeps run the same way, interleaved: L_D^-1 top-down
// (row p of the inverse scaled by 1/L_pp, rows below lose L_ip * row p) and
// U_D^-1 bottom-up (rows above lose U_iq * row q).
template <typename T, int NB>
__global__ void __launch_bounds__((NB / 4) * (NB / 4)) k_panel_diag(const FrontDev* __restrict__ fronts,
                                                                    const DiagTask* __restrict__ tasks, T* __restrict__ fac,
                                                                    T* __restrict__ slots, const unsigned int* __restrict__ famax,
                                                                    double tol_rel, DevStatus* st) {
    constexpr int TPD = NB / 4;
    __shared__ T Ds[NB][NB + 1];
    __shared__ T colb[2][NB], rowb[2][NB], colc[2][NB], rowc[2][NB];
    const DiagTask t = tasks[blockIdx.x];
    const FrontDev fr = fronts[t.front];
    const int m = fr.m, kb = t.kb, w = t.w;
    const int tid = threadIdx.x, tr = tid / TPD, tc = tid % TPD;
    T* P = fac + fr.P_off;
    for (int j = tid / 32; j < NB; j += TPD * TPD / 32)
        for (int i = tid % 32; i < NB; i += 32) {
            if (i < w && j < w) cp_async_elem(&Ds[i][j], P + (kb + i) + (int64_t)(kb + j) * m);
            else Ds[i][j] = (i == j) ? T(1) : T(0);
        }
    cp_async_wait_all();
    __syncthreads();
    T a[4][4];
#pragma unroll
    for (int r = 0; r < 4; r++)
#pragma unroll
        for (int c = 0; c < 4; c++) a[r][c] = Ds[4 * tr + r][4 * tc + c];
    const T amax = (T)__uint_as_float(famax[t.front]);
    const T thr = (T)tol_rel * amax > T(0) ? (T)tol_rel * amax : tiny_pivot<T>();
    // ---- LU (Table 2 tasks: divide the pivot row, update the trailing block)
    for (int pb = 0; pb < NB; pb += 4) {
#pragma unroll
        for (int pp = 0; pp < 4; pp++) {
            const int p = pb + pp, par = p & 1;
            if (tc == pb / 4) {
#pragma unroll
                for (int r = 0; r < 4; r++) colb[par][4 * tr + r] = a[r][pp];
            }
            if (tr == pb / 4) {
#pragma unroll
                for (int c = 0; c < 4; c++) rowb[par][4 * tc + c] = a[pp][c];
            }
            __syncthreads();
            T piv = rowb[par][p];
            if (p < w) piv = checked_pivot(piv, thr, tid == 0, t.front, kb + p, st);
            const T rinv = T(1) / piv;
#pragma unroll
            for (int r = 0; r < 4; r++) {
                const int i = 4 * tr + r;
                const T li = colb[par][i];
#pragma unroll
                for (int c = 0; c < 4; c++) {
                    const int j = 4 * tc + c;
                    const T uj = rowb[par][j] * rinv;
                    if (i > p && j > p) a[r][c] -= li * uj;
                    else if (i == p && j > p) a[r][c] = uj;
                    else if (i == p && j == p) a[r][c] = piv;
                }
            }
        }
    }
    // factored block back to P (through shared memory, coalesced)
    __syncthreads();
#pragma unroll
    for (int r = 0; r < 4; r++)
#pragma unroll
        for (int c = 0; c < 4; c++) Ds[4 * tr + r][4 * tc + c] = a[r][c];
    __syncthreads();
    for (int j = tid / 32; j < w; j += TPD * TPD / 32)
        for (int i = tid % 32; i < w; i += 32) P[(kb + i) + (int64_t)(kb + j) * m] = Ds[i][j];
    // ---- inverses: x = L_D^-1 (lower incl. diagonal), y = U_D^-1 (strict upper)
    T x[4][4], y[4][4];
#pragma unroll
    for (int r = 0; r < 4; r++)
#pragma unroll
        for (int c = 0; c < 4; c++) {
            const bool d = (4 * tr + r) == (4 * tc + c);
            x[r][c] = d ? T(1) : T(0);
            y[r][c] = d ? T(1) : T(0);
        }
    for (int sb = 0; sb < NB; sb += 4) {
#pragma unroll
        for (int ss = 0; ss < 4; ss++) {
            const int p = sb + ss, par = p & 1;
            const int q = NB - 1 - p;  // q's tile column/row index: (NB-1-sb-ss)/4 = TPD-1-sb/4, offset 3-ss
            const int qb = TPD - 1 - sb / 4, qq = 3 - ss;
            if (tc == sb / 4) {
#pragma unroll
                for (int r = 0; r < 4; r++) colb[par][4 * tr + r] = a[r][ss];  // L column p
            }
            if (tr == sb / 4) {
#pragma unroll
                for (int c = 0; c < 4; c++) rowb[par][4 * tc + c] = x[ss][c];  // inverse row p (unscaled)
            }
            if (tc == qb) {
#pragma unroll
                for (int r = 0; r < 4; r++) colc[par][4 * tr + r] = a[r][qq];  // U column q
            }
            if (tr == qb) {
#pragma unroll
                for (int c = 0; c < 4; c++) rowc[par][4 * tc + c] = y[qq][c];  // U^-1 row q (final)
            }
            __syncthreads();
            const T rinv = T(1) / colb[par][p];
#pragma unroll
            for (int r = 0; r < 4; r++) {
                const int i = 4 * tr + r;
                const T li = colb[par][i], ui = colc[par][i];
#pragma unroll
                for (int c = 0; c < 4; c++) {
                    const int j = 4 * tc + c;
                    const T xp = rowb[par][j] * rinv;
                    if (j <= p) {
                        if (i > p) x[r][c] -= li * xp;
                        else if (i == p) x[r][c] = xp;
                    }
                    if (i < q && j >= q) y[r][c] -= ui * (j == q ? T(1) : rowc[par][j]);
                }
            }
        }
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < 4; r++)
#pragma unroll
        for (int c = 0; c < 4; c++) {
            const int i = 4 * tr + r, j = 4 * tc + c;
            Ds[i][j] = j <= i ? x[r][c] : y[r][c];
        }
    __syncthreads();
    T* Z = slots + t.slot;
    for (int j = tid / 32; j < w; j += TPD * TPD / 32)
        for (int i = tid % 32; i < w; i += 32) Z[i + j * 64] = Ds[i][j];
}

// ---------------------------------------------------------------------------
// Batched SIMT GEMM over column-major operands with explicit leading
// dimensions, 64x64 tiles, 256 threads, 4x4 outputs per thread.
//   op 0: C -= A B      (trailing updates, Schur update S -= L21 U12, Sec. 2.2)
//   op 1: C  = A B      op 2: C = -A B   (triangular inversion levels)
// Operands live in one of the arenas (factor, CB, inverse, scratch, panel
// slots).  A tile may write the operand it reads (panel step) when it spans
// that operand's whole K extent: all loads precede the epilogue's stores.  A
// triangular operand is read through a mask: 1 = lower (entries above the
// diagonal read as 0), 2 = unit upper (below the diagonal 0, diagonal 1),
// relative to the operand's own origin.
enum { AR_FAC = 0, AR_CB = 1, AR_INV = 2, AR_SCR = 3, AR_PNL = 4 };

struct GemmTile {
    int64_t a_off, b_off, c_off;  // element offsets into the arenas named below
    int32_t lda, ldb, ldc;
    int32_t M, N, K;
    int32_t i0, j0;
    int8_t a_ar, b_ar, c_ar, op;
    int8_t a_mask, b_mask, pad0, pad1;
};

template <typename T>
struct Arenas {
    T* a[5];
};

template <typename T>
__device__ __forceinline__ T masked(T v, int mask, int r, int c) {
    if (mask == 1) return r >= c ? v : T(0);
    if (mask == 2) return r < c ? v : (r == c ? T(1) : T(0));
    return v;
}

template <typename T, int BK>
__global__ void __launch_bounds__(256) k_gemm(const GemmTile* __restrict__ tiles, Arenas<T> ar) {
    __shared__ T As[2][BK][64 + 1];
    __shared__ T Bs[2][BK][64 + 1];
    const GemmTile t = tiles[blockIdx.x];
    const T* A = ar.a[t.a_ar] + t.a_off;
    const T* B = ar.a[t.b_ar] + t.b_off;
    T* C = ar.a[t.c_ar] + t.c_off;
    const int tid = threadIdx.x;
    const int tx = tid & 15, ty = tid >> 4;
    T acc[4][4];
#pragma unroll
    for (int r = 0; r < 4; r++)
#pragma unroll
        for (int c = 0; c < 4; c++) acc[r][c] = T(0);

    constexpr int LOADS = 64 * BK / 256;
    T ra[LOADS], rb[LOADS];
    auto load = [&](int kk0) {
#pragma unroll
        for (int r = 0; r < LOADS; r++) {
            int idx = tid + 256 * r;
            int i = idx & 63, kk = idx >> 6;
            int gi = t.i0 + i, gk = kk0 + kk;
            T va = (gi < t.M && gk < t.K) ? A[gi + (int64_t)gk * t.lda] : T(0);
            ra[r] = (gi < t.M && gk < t.K) ? masked(va, t.a_mask, gi, gk) : T(0);
            int kb = idx % BK, j = idx / BK;
            int gj = t.j0 + j, gk2 = kk0 + kb;
            T vb = (gj < t.N && gk2 < t.K) ? B[gk2 + (int64_t)gj * t.ldb] : T(0);
            rb[r] = (gj < t.N && gk2 < t.K) ? masked(vb, t.b_mask, gk2, gj) : T(0);
        }
    };
    auto store = [&](int buf) {
#pragma unroll
        for (int r = 0; r < LOADS; r++) {
            int idx = tid + 256 * r;
            As[buf][idx >> 6][idx & 63] = ra[r];
            Bs[buf][idx % BK][idx / BK] = rb[r];
        }
    };
    int nk = (t.K + BK - 1) / BK;
    load(0);
    store(0);
    __syncthreads();
    for (int kt = 0; kt < nk; kt++) {
        int buf = kt & 1;
        if (kt + 1 < nk) load((kt + 1) * BK);
#pragma unroll
        for (int kk = 0; kk < BK; kk++) {
            T a[4], b[4];
#pragma unroll
            for (int r = 0; r < 4; r++) a[r] = As[buf][kk][tx + 16 * r];
#pragma unroll
            for (int c = 0; c < 4; c++) b[c] = Bs[buf][kk][ty + 16 * c];
#pragma unroll
            for (int r = 0; r < 4; r++)
#pragma unroll
                for (int c = 0; c < 4; c++) acc[r][c] = fma(a[r], b[c], acc[r][c]);
        }
        if (kt + 1 < nk) store(buf ^ 1);
        __syncthreads();
    }
#pragma unroll
    for (int c = 0; c < 4; c++) {
        int gj = t.j0 + ty + 16 * c;
        if (gj >= t.N) continue;
#pragma unroll
        for (int r = 0; r < 4; r++) {
            int gi = t.i0 + tx + 16 * r;
            if (gi >= t.M) continue;
            T* dst = C + gi + (int64_t)gj * t.ldc;
            if (t.op == 0) *dst -= acc[r][c];
            else if (t.op == 1) *dst = acc[r][c];
            else *dst = -acc[r][c];
        }
    }
}

// ---------------------------------------------------------------------------
// Explicit inverses of the pivot blocks of large fronts, used by the solve
// (the triangular solves become wide products).  The inverse block Q (k x k,
// column-major, in the inverse arena) holds L11^-1 on and below the diagonal
// and the strictly upper part of U11^-1 (unit diagonal implied), packed like
// P's own L11\U11 block.  k_inv_diag inverts the 64x64 diagonal blocks; the
// off-diagonal blocks follow by block doubling,
//   [L1 0; L21 L2]^-1 = [X1 0; -X2 L21 X1  X2],
//   [U1 U12; 0 U2]^-1 = [Y1 -Y1 U12 Y2; 0 Y2],
// with two k_gemm launches per doubling level.
struct InvTask {
    int32_t front, kb, w, pad;
    int64_t q_off;  // inverse-arena offset of the front's Q
};

template <typename T>
__global__ void __launch_bounds__(128) k_inv_diag(const FrontDev* __restrict__ fronts, const InvTask* __restrict__ tasks,
                                                  const T* __restrict__ fac, T* __restrict__ inv) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T(*A)[65] = reinterpret_cast<T(*)[65]>(smem_raw);       // 64 x 65
    T(*X)[65] = reinterpret_cast<T(*)[65]>(smem_raw) + 64;  // 64 x 65
    const InvTask t = tasks[blockIdx.x];
    const FrontDev fr = fronts[t.front];
    const int m = fr.m, k = fr.k, kb = t.kb, w = t.w;
    const T* P = fac + fr.P_off;
    for (int j = threadIdx.x >> 5; j < w; j += 4)
        for (int i = threadIdx.x & 31; i < w; i += 32) cp_async_elem(&A[i][j], P + (kb + i) + (int64_t)(kb + j) * m);
    cp_async_wait_all();
    __syncthreads();
    const int c = threadIdx.x & 63;
    if (c < w) {
        if (threadIdx.x < 64) {
            // column c of L^-1: forward substitution on L x = e_c
            X[c][c] = T(1) / A[c][c];
            for (int i = c + 1; i < w; i++) {
                T sacc = T(0);
                for (int q = c; q < i; q++) sacc += A[i][q] * X[q][c];
                X[i][c] = -sacc / A[i][i];
            }
        } else {
            // column c of U^-1 (unit upper): back substitution on U y = e_c
            for (int i = c - 1; i >= 0; i--) {
                T sacc = A[i][c];
                for (int q = i + 1; q < c; q++) sacc += A[i][q] * X[q][c];
                X[i][c] = -sacc;
            }
        }
    }
    __syncthreads();
    T* Q = inv + t.q_off;
    for (int j = threadIdx.x >> 5; j < w; j += 4)
        for (int i = threadIdx.x & 31; i < w; i += 32) Q[(kb + i) + (int64_t)(kb + j) * k] = X[i][j];
}
