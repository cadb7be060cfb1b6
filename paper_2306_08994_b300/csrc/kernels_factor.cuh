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

// Panel step of the blocked partial LU (large fronts).  With the pivot block
// [kb, kb+w):
//   D = F[kb:kb+w, kb:kb+w] = L11 U11     (unblocked Table 2 tasks, in smem)
//   L21 = F[kb+w:m, kb:kb+w] U11^-1       (role 0: a chunk of rows)
//   U12 = L11^-1 F[kb:kb+w, kb+w:m]       (role 1: a chunk of columns, in P or R)
// Every CTA factors D itself from P (w^3/3 flops) instead of waiting for
// another CTA, so D must stay unfactored in P while the step runs: the
// factored diagonal blocks are written back by role 2 tasks in one launch
// after the class's panel loop (nothing else reads or writes them in
// between: the trailing updates start at row/column kb+w).
struct PanelTask {
    int32_t front, kb, w, role, r0, r1, pad0, pad1;
};

template <typename T, int NB>
__device__ __forceinline__ void factor_diag_block(T (*D)[NB + 1], int w, T thr, bool record, int32_t front, int kb,
                                                  DevStatus* st) {
    for (int p = 0; p < w; p++) {
        const T piv = checked_pivot(D[p][p], thr, record && threadIdx.x == 0, front, kb + p, st);
        __syncthreads();
        const int n = w - p - 1;
        if (threadIdx.x == 0) D[p][p] = piv;
        for (int j = p + 1 + (int)threadIdx.x; j < w; j += blockDim.x) D[p][j] = D[p][j] / piv;
        __syncthreads();
        for (int idx = threadIdx.x; idx < n * n; idx += blockDim.x) {
            const int i = p + 1 + idx % n, j = p + 1 + idx / n;
            D[i][j] -= D[i][p] * D[p][j];
        }
        __syncthreads();
    }
}

template <typename T, int NB>
__global__ void __launch_bounds__(256) k_panel(const FrontDev* __restrict__ fronts, const PanelTask* __restrict__ tasks,
                                               T* __restrict__ fac, const unsigned int* __restrict__ famax, double tol_rel,
                                               DevStatus* st) {
    __shared__ T D[NB][NB + 1];
    const PanelTask t = tasks[blockIdx.x];
    const FrontDev fr = fronts[t.front];
    const int m = fr.m, k = fr.k, kb = t.kb, w = t.w;
    T* P = fac + fr.P_off;
    T* R = fac + fr.R_off;
    for (int idx = threadIdx.x; idx < w * w; idx += blockDim.x) {
        int i = idx % w, j = idx / w;
        D[i][j] = P[(kb + i) + (int64_t)(kb + j) * m];
    }
    __syncthreads();
    const T amax = (T)__uint_as_float(famax[t.front]);
    const T thr = (T)tol_rel * amax > T(0) ? (T)tol_rel * amax : tiny_pivot<T>();
    factor_diag_block<T, NB>(D, w, thr, t.role == 2, t.front, kb, st);
    if (t.role == 2) {
        for (int idx = threadIdx.x; idx < w * w; idx += blockDim.x) {
            int i = idx % w, j = idx / w;
            P[(kb + i) + (int64_t)(kb + j) * m] = D[i][j];
        }
        return;
    }
    if (t.role == 0) {
        const int i = t.r0 + threadIdx.x;
        if (i >= t.r1) return;
        T l[NB];
#pragma unroll
        for (int p = 0; p < NB; p++)
            if (p < w) l[p] = P[i + (int64_t)(kb + p) * m];
#pragma unroll
        for (int p = 0; p < NB; p++) {
            if (p < w) {
                T a = l[p];
#pragma unroll
                for (int q = 0; q < NB; q++)
                    if (q < p) a -= l[q] * D[q][p];
                l[p] = a;
            }
        }
#pragma unroll
        for (int p = 0; p < NB; p++)
            if (p < w) P[i + (int64_t)(kb + p) * m] = l[p];
    } else {
        const int j = t.r0 + threadIdx.x;
        if (j >= t.r1) return;
        T* col = (j < k) ? (P + kb + (int64_t)j * m) : (R + kb + (int64_t)(j - k) * k);
        T u[NB];
#pragma unroll
        for (int p = 0; p < NB; p++)
            if (p < w) u[p] = col[p];
#pragma unroll
        for (int p = 0; p < NB; p++) {
            if (p < w) {
                T a = u[p];
#pragma unroll
                for (int q = 0; q < NB; q++)
                    if (q < p) a -= D[p][q] * u[q];
                u[p] = a / D[p][p];
            }
        }
#pragma unroll
        for (int p = 0; p < NB; p++)
            if (p < w) col[p] = u[p];
    }
}

// ---------------------------------------------------------------------------
// Batched SIMT GEMM C -= A B (column-major, explicit leading dimensions),
// 64x64 tiles, 256 threads, 4x4 outputs per thread.  Used for the trailing
// updates of the panel loop and for the Schur update S -= L21 U12 (Sec. 2.2).
struct GemmTile {
    int64_t a_off, b_off, c_off;  // element offsets: A, B in the factor arena; C in factor or CB arena
    int32_t lda, ldb, ldc;
    int32_t M, N, K;
    int32_t i0, j0;
    int32_t c_in_cb;
    int32_t pad;
};

template <typename T, int BK>
__global__ void __launch_bounds__(256) k_gemm_sub(const GemmTile* __restrict__ tiles, const T* __restrict__ fac,
                                                  T* __restrict__ facw, T* __restrict__ cbs) {
    __shared__ T As[2][BK][64 + 1];
    __shared__ T Bs[2][BK][64 + 1];
    const GemmTile t = tiles[blockIdx.x];
    const T* A = fac + t.a_off;
    const T* B = fac + t.b_off;
    T* C = (t.c_in_cb ? cbs : facw) + t.c_off;
    const int tid = threadIdx.x;
    const int tx = tid & 15, ty = tid >> 4;
    T acc[4][4];
#pragma unroll
    for (int r = 0; r < 4; r++)
#pragma unroll
        for (int c = 0; c < 4; c++) acc[r][c] = T(0);

    constexpr int ALOADS = 64 * BK / 256;  // A tile elements per thread
    T ra[ALOADS], rb[ALOADS];
    auto load = [&](int kk0) {
#pragma unroll
        for (int r = 0; r < ALOADS; r++) {
            int idx = tid + 256 * r;
            int i = idx & 63, kk = idx >> 6;
            int gi = t.i0 + i, gk = kk0 + kk;
            ra[r] = (gi < t.M && gk < t.K) ? A[gi + (int64_t)gk * t.lda] : T(0);
            int kb = idx % BK, j = idx / BK;
            int gj = t.j0 + j, gk2 = kk0 + kb;
            rb[r] = (gj < t.N && gk2 < t.K) ? B[gk2 + (int64_t)gj * t.ldb] : T(0);
        }
    };
    auto store = [&](int buf) {
#pragma unroll
        for (int r = 0; r < ALOADS; r++) {
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
            if (gi < t.M) C[gi + (int64_t)gj * t.ldc] -= acc[r][c];
        }
    }
}
