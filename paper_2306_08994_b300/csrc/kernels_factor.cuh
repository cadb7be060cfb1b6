// Factorization kernels: one batched pass per Foata class (Sec. 3.3).
//
// Every kernel is launched over a precomputed task list (a "bag of tasks",
// Sec. 3.3): the fronts of one class, or tiles of them, in any order; the
// launch boundary is the barrier between classes.
#pragma once

#include <cstdint>

#include "mf_internal.h"

// Programmatic dependent launch (used by the substitution kernels).  A kernel
// launched with programmatic stream serialization may be scheduled while the
// previous kernel of its stream is still running.  It reads only
// launch-invariant data (task records, index maps, factor coefficients) before
// pdl_wait, which returns once the predecessor grid has completed and its
// memory is visible (a no-op for an ordinary launch); every thread that reads
// or writes data of earlier kernels calls it first, so a completed grid implies
// a completed predecessor.  pdl_trigger lets the next kernel's CTAs be
// scheduled once every CTA of this grid has started.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

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

// What the fused and lane-group factor kernels read of a front and of its
// children, stored in launch-list order: one load, no list -> descriptor ->
// child-descriptor chain before the children's blocks can be fetched.
struct FactorRec {
    int64_t P_off, R_off, S_off, map_off;
    int64_t cS[2];     // children's contribution blocks (CB arena offsets)
    int32_t m, k, nchild, elem;
    int32_t cn[2];     // children's contribution-block orders (m - k)
    int32_t front, pad;
};

// ---------------------------------------------------------------------------
// Fused small front: one CTA per front, the whole front in shared memory.
// Extend-add (or the element matrix at a leaf), partial LU on the k pivots
// (Sec. 3 / Table 2 tasks), P and R written out, and the Schur complement
// S = F22 - L21 U12 formed straight into the contribution-block arena.
// BLK (fronts with few pivots, k <= 32 for every front of the launch),
// blocked form:
//   (1) one warp factors the k x k pivot block: per pivot the T4 static
//       check, T1 division of the pivot row, T2/T3 on the rows below;
//   (2) one thread per row of L21 solves x U11 = a (U11 unit upper) and,
//       for unsymmetric fronts, one thread per column of U12 solves
//       L11 y = a; for symmetric fronts U12 = D^-1 L21^T (D = diag L11);
//   (3) S from a 4 x 4 register tile per thread on a grid sized to the
//       contribution block (ceil(nc/4)^2 tiles).
// Three block barriers after the assembly, whatever k is.  !BLK (fronts
// with more pivots): right-looking, one pivot at a time over the whole
// block (two barriers per pivot), S deferred to the same tiled product.
// Dynamic shared memory: ldm*maxm T + maxm T + 2*maxm int32 + 32 floats.
template <typename T, bool BLK>
__global__ void __launch_bounds__(256) k_front_fused(const FactorRec* __restrict__ recs,
                                                     const int32_t* __restrict__ maps, const double* __restrict__ values,
                                                     int npe, T* __restrict__ fac, T* __restrict__ cbs, int maxm, int ldm,
                                                     double tol_rel, int sym, DevStatus* st) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* F = reinterpret_cast<T*>(smem_raw);
    T* urow = F + (size_t)ldm * maxm;  // BLK: reciprocals of the pivots; otherwise the scaled pivot row
    int32_t* imap = reinterpret_cast<int32_t*>(urow + maxm);
    float* red = reinterpret_cast<float*>(imap + 2 * maxm);

    const FactorRec fr = recs[blockIdx.x];
    const int32_t f = fr.front;
    const int m = fr.m, k = fr.k, nc = m - k;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
    const int nthr = blockDim.x;

    const int nmap = fr.nchild > 0 ? fr.nchild * m : m;
    for (int i = threadIdx.x; i < nmap; i += nthr) imap[i] = maps[fr.map_off + i];
    __syncthreads();

    // ---- assembly: entries in column-major order over the whole block, 8 per thread in flight
    //      (all loads of a round before its stores); (i, j) stepped by nthr without divisions
    T amax = T(0);
    {
        const int mm = m * m, di = nthr % m, dj = nthr / m;
        const bool leaf = fr.nchild == 0, two = fr.nchild > 1;
        const double* K = values + (int64_t)fr.elem * npe * npe;
        const T* S0 = leaf ? nullptr : cbs + fr.cS[0];
        const T* S1 = two ? cbs + fr.cS[1] : nullptr;
        const int n0 = leaf ? 0 : fr.cn[0], n1 = two ? fr.cn[1] : 0;
        int i = threadIdx.x % m, j = threadIdx.x / m;
        for (int e0 = threadIdx.x; e0 < mm; e0 += 8 * nthr) {
            T v[8];
            int ii[8], jj[8];
#pragma unroll
            for (int u = 0; u < 8; u++) {
                ii[u] = i;
                jj[u] = j;
                T x = T(0);
                if (e0 + u * nthr < mm) {
                    if (leaf) {
                        x = (T)K[imap[i] + imap[j] * npe];
                    } else {
                        const int i0 = imap[i], j0 = imap[j];
                        if (i0 >= 0 && j0 >= 0) x = S0[i0 + j0 * n0];
                        if (two) {
                            const int i1 = imap[m + i], j1 = imap[m + j];
                            if (i1 >= 0 && j1 >= 0) x += S1[i1 + j1 * n1];
                        }
                    }
                }
                v[u] = x;
                i += di;
                j += dj;
                if (i >= m) {
                    i -= m;
                    j++;
                }
            }
#pragma unroll
            for (int u = 0; u < 8; u++)
                if (e0 + u * nthr < mm) {
                    F[ii[u] + jj[u] * ldm] = v[u];
                    amax = max(amax, (T)fabs(v[u]));
                }
        }
    }
    amax = block_max_abs(amax, red);  // includes __syncthreads
    const T thr = (T)tol_rel * amax > T(0) ? (T)tol_rel * amax : tiny_pivot<T>();

    if constexpr (BLK) {
        T* rd = urow;
        // ---- (1) pivot block, one warp: per pivot the static check (T4), the division of the pivot
        //      row (T1, one lane per entry) and the update of the rows below (T2/T3, one lane per row)
        if (warp == 0) {
            for (int p = 0; p < k; p++) {
                const T piv = checked_pivot(F[p + p * ldm], thr, lane == 0, f, p, st);
                const T rinv = T(1) / piv;
                __syncwarp();
                if (lane == 0) {
                    F[p + p * ldm] = piv;
                    rd[p] = rinv;
                }
                for (int c = p + 1 + lane; c < k; c += 32) F[p + c * ldm] *= rinv;
                __syncwarp();
                for (int r = p + 1 + lane; r < k; r += 32) {
                    const T l = F[r + p * ldm];
                    for (int c = p + 1; c < k; c++) F[r + c * ldm] -= l * F[p + c * ldm];
                }
                __syncwarp();
            }
        }
        __syncthreads();
        // ---- (2) L21 by rows (x U11 = a), U12 by columns (L11 y = a) or from L21 (symmetric);
        //      each solve in place in its own row / column, four partial sums per step
        const int nsolve = sym ? nc : 2 * nc;
        for (int t = threadIdx.x; t < nsolve; t += nthr) {
            if (t < nc) {
                const int i = k + t;
                for (int c = 1; c < k; c++) {
                    T s0 = F[i + c * ldm], s1 = T(0), s2 = T(0), s3 = T(0);
                    int q = 0;
                    for (; q + 4 <= c; q += 4) {
                        s0 -= F[i + q * ldm] * F[q + c * ldm];
                        s1 -= F[i + (q + 1) * ldm] * F[q + 1 + c * ldm];
                        s2 -= F[i + (q + 2) * ldm] * F[q + 2 + c * ldm];
                        s3 -= F[i + (q + 3) * ldm] * F[q + 3 + c * ldm];
                    }
                    for (; q < c; q++) s0 -= F[i + q * ldm] * F[q + c * ldm];
                    F[i + c * ldm] = (s0 + s1) + (s2 + s3);
                }
                if (sym)
                    for (int c = 0; c < k; c++) F[c + i * ldm] = F[i + c * ldm] * rd[c];
            } else {
                const int j = k + (t - nc);
                for (int r = 0; r < k; r++) {
                    T s0 = F[r + j * ldm], s1 = T(0), s2 = T(0), s3 = T(0);
                    int q = 0;
                    for (; q + 4 <= r; q += 4) {
                        s0 -= F[r + q * ldm] * F[q + j * ldm];
                        s1 -= F[r + (q + 1) * ldm] * F[q + 1 + j * ldm];
                        s2 -= F[r + (q + 2) * ldm] * F[q + 2 + j * ldm];
                        s3 -= F[r + (q + 3) * ldm] * F[q + 3 + j * ldm];
                    }
                    for (; q < r; q++) s0 -= F[r + q * ldm] * F[q + j * ldm];
                    F[r + j * ldm] = ((s0 + s1) + (s2 + s3)) * rd[r];
                }
            }
        }
        __syncthreads();
    } else {
        // ---- right-looking partial LU, the Schur block deferred: per pivot the division T1 along
        //      the whole pivot row, T2/T3 only on the pivot columns and on the pivot rows' right part
        for (int p = 0; p < k; p++) {
            T piv = checked_pivot(F[p + p * ldm], thr, threadIdx.x == 0, f, p, st);
            for (int j = p + 1 + threadIdx.x; j < m; j += nthr) {
                T u = F[p + j * ldm] / piv;
                F[p + j * ldm] = u;
                urow[j] = u;
            }
            if (threadIdx.x == 0) F[p + p * ldm] = piv;
            __syncthreads();
            for (int i = p + 1 + threadIdx.x; i < m; i += nthr) {
                const T lip = F[i + p * ldm];
                for (int j = p + 1; j < k; j++) F[i + j * ldm] -= lip * urow[j];
            }
            for (int j = k + warp; j < m; j += nwarp) {
                const T u = urow[j];
                for (int i = p + 1 + lane; i < k; i += 32) F[i + j * ldm] -= F[i + p * ldm] * u;
            }
            __syncthreads();
        }
    }

    // ---- write P (m x k), R (k x nc)
    T* P = fac + fr.P_off;
    for (int j = warp; j < k; j += nwarp)
        for (int i = lane; i < m; i += 32) P[i + (int64_t)j * m] = F[i + j * ldm];
    T* R = fac + fr.R_off;
    for (int j = k + warp; j < m; j += nwarp)
        for (int i = lane; i < k; i += 32) R[i + (int64_t)(j - k) * k] = F[i + j * ldm];
    // ---- S = F22 - L21 U12 straight to the contribution-block arena: g = ceil(nc / 4) row and
    //      column groups; thread tile (ti, tj) holds outputs (ti + g a, tj + g b), a, b < 4, so a
    //      warp's shared reads of L21 run down consecutive rows and those of U12 are broadcasts
    if (nc > 0) {
        T* S = cbs + fr.S_off;
        const int g = (nc + 3) >> 2;
        for (int t = threadIdx.x; t < g * g; t += nthr) {
            const int ti = t % g, tj = t / g;
            T acc[4][4];
#pragma unroll
            for (int a = 0; a < 4; a++)
#pragma unroll
                for (int b = 0; b < 4; b++) acc[a][b] = T(0);
            int ri[4], cj[4];
#pragma unroll
            for (int a = 0; a < 4; a++) {
                ri[a] = min(ti + g * a, nc - 1);
                cj[a] = min(tj + g * a, nc - 1);
            }
            for (int l = 0; l < k; l++) {
                T la[4], ub[4];
#pragma unroll
                for (int a = 0; a < 4; a++) {
                    la[a] = F[(k + ri[a]) + l * ldm];
                    ub[a] = F[l + (k + cj[a]) * ldm];
                }
#pragma unroll
                for (int a = 0; a < 4; a++)
#pragma unroll
                    for (int b = 0; b < 4; b++) acc[a][b] += la[a] * ub[b];
            }
#pragma unroll
            for (int b = 0; b < 4; b++) {
                const int j = tj + g * b;
                if (j >= nc) continue;
#pragma unroll
                for (int a = 0; a < 4; a++) {
                    const int i = ti + g * a;
                    if (i < nc) S[i + (int64_t)j * nc] = F[(k + i) + (k + j) * ldm] - acc[a][b];
                }
            }
        }
    }
}

// ---------------------------------------------------------------------------
// Tiny fronts (m <= MJ <= G, G in {4, 8, 16, 32}): a group of G lanes per front,
// 32/G fronts per warp, no shared memory.  Lane i holds row i of F in
// registers; the pivot row, the pivot and the pivot-column entry travel by
// width-G shuffles.  Same tasks as k_front_fused: assembly (element matrix
// at a leaf, extend-add of the children's blocks otherwise), static pivot
// check, T1 division of the pivot row, T2/T3 update, then P, R, S written.
template <typename T, int G, int MJ = G>
__global__ void __launch_bounds__(256) k_front_grp(const FactorRec* __restrict__ recs, int count, const int32_t* __restrict__ maps,
                                                   const double* __restrict__ values, int npe, T* __restrict__ fac,
                                                   T* __restrict__ cbs, double tol_rel, DevStatus* st) {
    const int lane = threadIdx.x & 31;
    const int fidx = (blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)) * (32 / G) + lane / G;
    const bool active = fidx < count;
    const int i = lane % G;
    FactorRec fr{};
    if (active) fr = recs[fidx];
    const int32_t f = active ? fr.front : -1;
    const int m = active ? fr.m : 0, k = active ? fr.k : 0;
    const bool row = i < m;
    T a[MJ];  // MJ <= G: the widest front of the launch
    // ---- assembly: lane i loads its own row's maps; column j's maps are row j's, taken from
    //      lane j by a shuffle (rows and columns of a front share one index set; every lane of
    //      the warp takes part, so the shuffles stay outside the leaf / internal branches).
    //      Children of a front with m <= G have contribution blocks of order <= G, so 32-bit
    //      offsets suffice.
    T amax = T(0);
    {
        const bool leaf = fr.nchild == 0, two = fr.nchild > 1;
        const int32_t* m0 = maps + fr.map_off;
        const int i0 = row ? m0[i] : -1;  // leaf: element-local node; internal: child-0 CB row
        const int i1 = (row && two) ? m0[m + i] : -1;
        const double* K = values + (int64_t)(leaf ? fr.elem : 0) * npe * npe;
        const T* S0 = cbs + fr.cS[0];
        const T* S1 = cbs + (two ? fr.cS[1] : 0);
        const int n0 = fr.cn[0], n1 = two ? fr.cn[1] : 0;
#pragma unroll
        for (int j = 0; j < MJ; j++) {
            const int j0 = __shfl_sync(0xffffffffu, i0, j, G), j1 = __shfl_sync(0xffffffffu, i1, j, G);
            T v = T(0);
            if (leaf) {
                if (i0 >= 0 && j0 >= 0) v = (T)K[i0 + j0 * npe];
            } else {
                if (i0 >= 0 && j0 >= 0) v = S0[i0 + j0 * n0];
                if (i1 >= 0 && j1 >= 0) v += S1[i1 + j1 * n1];
            }
            a[j] = v;
            amax = max(amax, (T)fabs(v));
        }
    }
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) amax = max(amax, __shfl_xor_sync(0xffffffffu, amax, o, G));
    const T thr = (T)tol_rel * amax > T(0) ? (T)tol_rel * amax : tiny_pivot<T>();
    // ---- partial LU (Table 2): all lanes shuffle, each group applies its own pivots
    const int kmax = (int)__reduce_max_sync(0xffffffffu, (unsigned)k);
#pragma unroll
    for (int p = 0; p < MJ; p++) {
        if (p < kmax) {
            const T pv = __shfl_sync(0xffffffffu, a[p], p, G);
            const bool mine = p < k;
            T piv = pv;
            if (mine) piv = checked_pivot(pv, thr, i == 0, f, p, st);
            const T rinv = T(1) / piv;
            const T lp = a[p];
#pragma unroll
            for (int j = p + 1; j < MJ; j++) {
                const T uj = __shfl_sync(0xffffffffu, a[j], p, G) * rinv;
                if (mine) {
                    if (i > p) a[j] -= lp * uj;
                    else if (i == p) a[j] = uj;
                }
            }
            if (mine && i == p) a[p] = piv;
        }
    }
    // ---- P (m x k), R (k x nc), S (nc x nc)
    if (row) {
        const int nc = m - k;
        T* P = fac + fr.P_off;
        T* R = fac + fr.R_off;
        T* S = cbs + fr.S_off;
#pragma unroll
        for (int j = 0; j < MJ; j++) {
            if (j < k) P[i + j * m] = a[j];
            else if (j < m) {
                if (i < k) R[i + (j - k) * k] = a[j];
                else S[(i - k) + (j - k) * nc] = a[j];
            }
        }
    }
}

// ---------------------------------------------------------------------------
// Large fronts.  Assembly of 64x64 tiles straight into P, R and S; the
// per-front max |entry| (for the static pivot threshold) by atomicMax on the
// float bit pattern (non-negative floats order like their bits).
struct AsmTile {
    int32_t front, i0, j0, pad;
};

// One 64 x 64 tile of a large front's extend-add, with everything the tile
// needs of the front and its children in the record itself, so the only
// dependent loads are record -> row/column maps -> child entries.
struct AsmRec {
    int64_t P_off, R_off, S_off;  // the front's P, R (factor arena) and S (CB arena)
    int64_t cS[2];                // children's contribution blocks (CB arena)
    int64_t map_off;              // the front's child maps (nchild blocks of m int32)
    int32_t m, k, cn[2];          // cn: children's contribution-block orders (0 = no child)
    int32_t i0, j0, front, pad;
};

// SYM (symmetric fronts): the children's contribution blocks are read from their lower
// triangles only (entry (a, b) of a child is taken at (max, min)), so the strictly upper part of
// a child's block is never needed; the plan leaves out the tiles this front's own R and strictly
// upper contribution block (overwritten later by the transposing copy of U12 and never read).
template <typename T, bool SYM = false>
__global__ void __launch_bounds__(256) k_assemble_large(const AsmRec* __restrict__ recs, const int32_t* __restrict__ maps,
                                                        T* __restrict__ fac, T* __restrict__ cbs,
                                                        unsigned int* __restrict__ famax) {
    __shared__ float red[8];
    const AsmRec t = recs[blockIdx.x];
    const int m = t.m, k = t.k, nc = m - k;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int n0 = t.cn[0], n1 = t.cn[1];
    const bool one = n0 > 0, two = n1 > 0;
    const T* S0 = cbs + t.cS[0];
    const T* S1 = cbs + t.cS[1];
    const int32_t* map0 = maps + t.map_off;
    const int32_t* map1 = map0 + m;
    // row maps of the thread's two rows and column maps of the warp's 8 columns, all issued
    // before any child entry, then all 16 child entries before the stores
    int ri[2], r0[2], r1[2], cj0[8], cj1[8];
#pragma unroll
    for (int q = 0; q < 2; q++) {
        ri[q] = t.i0 + lane + 32 * q;
        r0[q] = (one && ri[q] < m) ? map0[ri[q]] : -1;
        r1[q] = (two && ri[q] < m) ? map1[ri[q]] : -1;
    }
#pragma unroll
    for (int u = 0; u < 8; u++) {
        const int j = t.j0 + warp + 8 * u;
        cj0[u] = (one && j < m) ? map0[j] : -1;
        cj1[u] = (two && j < m) ? map1[j] : -1;
    }
    T v[8][2];
#pragma unroll
    for (int u = 0; u < 8; u++)
#pragma unroll
        for (int q = 0; q < 2; q++) {
            T x = T(0);
            if (r0[q] >= 0 && cj0[u] >= 0) {
                const int a0 = SYM ? max(r0[q], cj0[u]) : r0[q], b0 = SYM ? min(r0[q], cj0[u]) : cj0[u];
                x += S0[a0 + (int64_t)b0 * n0];
            }
            if (r1[q] >= 0 && cj1[u] >= 0) {
                const int a1 = SYM ? max(r1[q], cj1[u]) : r1[q], b1 = SYM ? min(r1[q], cj1[u]) : cj1[u];
                x += S1[a1 + (int64_t)b1 * n1];
            }
            v[u][q] = x;
        }
    T amax = T(0);
#pragma unroll
    for (int u = 0; u < 8; u++) {
        const int j = t.j0 + warp + 8 * u;
        if (j >= m) break;
#pragma unroll
        for (int q = 0; q < 2; q++) {
            const int i = ri[q];
            if (i >= m) continue;
            amax = max(amax, (T)fabs(v[u][q]));
            if (j < k) fac[t.P_off + i + (int64_t)j * m] = v[u][q];
            else if (i < k) fac[t.R_off + i + (int64_t)(j - k) * k] = v[u][q];
            else cbs[t.S_off + (i - k) + (int64_t)(j - k) * nc] = v[u][q];
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
// With one-panel lookahead the block first takes the update from the pivots
// factored since the last update that reached it (pre of them, kb-pre..kb: the
// panel before it, or every pivot of its super-panel so far):
//   F[kb:kb+w, kb:kb+w] -= L[kb:kb+w, kb-pre:kb] U[kb-pre:kb, kb:kb+w],
// so it can be factored while the rest of those updates runs.
struct DiagTask {
    int32_t front, kb, w, pre;
    int64_t slot;   // panel-slot offset (64 x 64, column-major, ld 64)
    int64_t q_off;  // >= 0: the inverses also go to the front's Q block in the inverse arena (ld k)
};
// dynamic shared memory of k_panel_diag_blk: the U block of the lookahead update (storage type T),
// and with a wider compute type C also the working block D and the inverse block Z (C each)
template <typename T, int NB, typename C = T>
constexpr size_t panel_diag_dyn_smem() {
    return ((size_t)NB * (NB + 1) * sizeof(T) + 15) / 16 * 16 +
           (sizeof(C) == sizeof(T) ? 0 : 2 * (size_t)NB * (NB + 1) * sizeof(C));
}

// Symmetric fronts (option symmetric): for A = A^T the paper's U (unit upper)
// is D^-1 L^T with D = diag(L), so beyond the pivot block only L is
// factored; the Schur update's B operand U12 = D^-1 L21^T is written into R
// by a transposing copy (one 64 x 64 tile of R per CTA through shared
// memory, each U entry one division T1 of Table 2 by the pivot), and the
// update itself computes only the tiles of S on and below the diagonal,
// mirrored afterwards (k_sym_mirror).  Tile (i0, j0) of R covers pivots
// i0.. and contribution-block columns j0..
template <typename T>
__global__ void __launch_bounds__(256) k_sym_r(const FrontDev* __restrict__ fronts, const AsmTile* __restrict__ tiles,
                                               T* __restrict__ fac) {
    __shared__ T tl[64][65];
    const AsmTile t = tiles[blockIdx.x];
    const FrontDev fr = fronts[t.front];
    const int m = fr.m, k = fr.k, nc = m - k;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    T v[16];
#pragma unroll
    for (int u = 0; u < 16; u++) {
        const int pp = warp + 8 * (u >> 1), jj = lane + 32 * (u & 1);
        const int p = t.i0 + pp, j = t.j0 + jj;
        v[u] = (p < k && j < nc) ? fac[fr.P_off + (k + j) + (int64_t)p * m] : T(0);
    }
#pragma unroll
    for (int u = 0; u < 16; u++) tl[warp + 8 * (u >> 1)][lane + 32 * (u & 1)] = v[u];
    __syncthreads();
    T d[2];
#pragma unroll
    for (int h = 0; h < 2; h++) {
        const int p = t.i0 + lane + 32 * h;
        d[h] = p < k ? fac[fr.P_off + p + (int64_t)p * m] : T(1);
    }
#pragma unroll
    for (int u = 0; u < 16; u++) {
        const int jj = warp + 8 * (u >> 1), pp = lane + 32 * (u & 1);
        const int p = t.i0 + pp, j = t.j0 + jj;
        if (p < k && j < nc) fac[fr.R_off + p + (int64_t)j * k] = tl[pp][jj] / d[u & 1];
    }
}

// S[j, i] = S[i, j]: tile (i0, j0), i0 >= j0 + 64 (strictly below the diagonal), of the
// contribution block is read and written transposed; all 16 loads of a thread are issued before
// any shared-memory store, all 16 shared loads before the global stores
template <typename T>
__global__ void __launch_bounds__(256) k_sym_mirror(const FrontDev* __restrict__ fronts, const AsmTile* __restrict__ tiles,
                                                    T* __restrict__ cbs) {
    __shared__ T tl[64][65];
    const AsmTile t = tiles[blockIdx.x];
    const FrontDev fr = fronts[t.front];
    const int nc = fr.m - fr.k;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    T* S = cbs + fr.S_off;
    T v[16];
#pragma unroll
    for (int u = 0; u < 16; u++) {
        const int ii = lane + 32 * (u & 1), jj = warp + 8 * (u >> 1);
        const int i = t.i0 + ii, j = t.j0 + jj;
        v[u] = (i < nc && j < nc) ? S[i + (int64_t)j * nc] : T(0);
    }
#pragma unroll
    for (int u = 0; u < 16; u++) tl[lane + 32 * (u & 1)][warp + 8 * (u >> 1)] = v[u];
    __syncthreads();
#pragma unroll
    for (int u = 0; u < 16; u++) v[u] = tl[warp + 8 * (u >> 1)][lane + 32 * (u & 1)];
#pragma unroll
    for (int u = 0; u < 16; u++) {
        const int ii = warp + 8 * (u >> 1), jj = lane + 32 * (u & 1);
        const int i = t.i0 + ii, j = t.j0 + jj;
        if (i < nc && j < nc) S[j + (int64_t)i * nc] = v[u];
    }
}

// Owners of row q and of column q of the pivot block publish them (and row q
// of L_D^-1, column q of U_D^-1) for elimination step q (k_panel_diag_blk).
template <typename C, int RPT, bool INV>
__device__ __forceinline__ void pivot_strip_publish(const C (&Ft)[RPT][RPT], const C (&Xt)[INV ? RPT : 1][INV ? RPT : 1],
                                                    const C (&Yt)[INV ? RPT : 1][INV ? RPT : 1], int q, int ti, int tj,
                                                    C* colF, C* rowF, C* rowX, C* colY) {
    // the tile row / column is picked by a chain of selects (an indexed register
    // read would put the tiles in local memory)
    const int i0 = ti * RPT, j0 = tj * RPT, rq = q % RPT;
    if (ti == q / RPT) {
#pragma unroll
        for (int c = 0; c < RPT; c++) {
            C f = Ft[0][c], x = INV ? Xt[0][INV ? c : 0] : C(0);
#pragma unroll
            for (int r = 1; r < RPT; r++) {
                f = r == rq ? Ft[r][c] : f;
                if constexpr (INV) x = r == rq ? Xt[r][c] : x;
            }
            rowF[j0 + c] = f;
            if constexpr (INV) rowX[j0 + c] = x;
        }
    }
    if (tj == q / RPT) {
#pragma unroll
        for (int r = 0; r < RPT; r++) {
            C f = Ft[r][0], y = INV ? Yt[INV ? r : 0][0] : C(0);
#pragma unroll
            for (int c = 1; c < RPT; c++) {
                f = c == rq ? Ft[r][c] : f;
                if constexpr (INV) y = c == rq ? Yt[r][c] : y;
            }
            colF[i0 + r] = f;
            if constexpr (INV) colY[i0 + r] = y;
        }
    }
}

// Pivot block of a large front (NB x NB at pivot kb, padded with the
// identity beyond w): partial LU in place (L with its diagonal, unit U) and
// the explicit inverses L_D^-1 (on and below the diagonal) and U_D^-1 (strict
// upper part) into the front's panel slot, for the panel products
// L21 = A21 U_D^-1 and U12 = L_D^-1 A12 that follow.
// 256 threads, each holding a fixed (NB/16) x (NB/16) tile of the block, of
// L_D^-1 and of U_D^-1 in registers for the whole kernel; one right-looking
// elimination step per pivot with one block barrier, the pivot column and row
// passed through a small double-buffered strip of shared memory.  The
// inverses are updated in the same steps from the same column and row, so
// the block costs w barrier-separated steps of a few shared loads and
// 3 (NB/16)^2 FMAs per thread, in a short rolled loop (the whole kernel stays
// small enough for the instruction cache; the block is latency-bound).
// C is the arithmetic of the block (T by default).  With T = float and
// C = double the block is factored and inverted in FP64 from the FP32 front
// and rounded once on the way out: the FP64 pivot blocks of the root
// separator fronts on the FP32-front path.  SYMB (symmetric fronts): for a
// symmetric block U_D = diag(L_D)^-1 L_D^T, so U_D^-1 = L_D^-T diag(L_D) is
// formed from L_D^-1 at the end instead of being carried through the steps.
template <typename T, int NB, typename C = T, bool INV = true, bool SYMB = false>
__global__ void __launch_bounds__(256, sizeof(C) == sizeof(T) ? 2 : 1) k_panel_diag_blk(const FrontDev* __restrict__ fronts,
                                                        const DiagTask* __restrict__ tasks, T* __restrict__ fac,
                                                        T* __restrict__ slots, T* __restrict__ inv,
                                                        const unsigned int* __restrict__ famax,
                                                        double tol_rel, DevStatus* st) {
    constexpr int NBB = NB / 16;
    static_assert(NB % 16 == 0 && NBB <= 4, "NB must be 16, 32, 48 or 64");
    constexpr bool kWide = sizeof(C) != sizeof(T);  // D and Z in dynamic shared memory
    __shared__ C Dst[kWide ? 1 : NB][NB + 1];
    __shared__ C Zst[kWide ? 1 : NB][NB + 1];
    const DiagTask t = tasks[blockIdx.x];
    const FrontDev fr = fronts[t.front];
    const int m = fr.m, kb = t.kb, w = t.w;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    T* P = fac + fr.P_off;
    extern __shared__ __align__(16) unsigned char pd_dyn[];
    T* Us = reinterpret_cast<T*>(pd_dyn);  // U slice of the lookahead update, NB x (NB + 1)
    C(*D)[NB + 1] = Dst;
    C(*Z)[NB + 1] = Zst;
    if constexpr (kWide) {
        D = reinterpret_cast<C(*)[NB + 1]>(pd_dyn + ((size_t)NB * (NB + 1) * sizeof(T) + 15) / 16 * 16);
        Z = D + NB;
    }
    const int pre = t.pre, p0 = kb - t.pre;
    // L slice (rows kb.., columns p0 + c0..) into Z, U slice (rows p0 + c0.., columns kb..) into Us,
    // zero outside w x cw and cw x w, so the identity padding of D takes no update
    auto stage = [&](int c0) {
        const int cw = min(NB, pre - c0);
        for (int j = warp; j < NB; j += 8)
            for (int i = lane; i < NB; i += 32) {
                if (i < w && j < cw) {
                    if constexpr (kWide) Z[i][j] = (C)P[(kb + i) + (int64_t)(p0 + c0 + j) * m];
                    else cp_async_elem(&Z[i][j], P + (kb + i) + (int64_t)(p0 + c0 + j) * m);
                } else {
                    Z[i][j] = C(0);
                }
                if (i < cw && j < w) cp_async_elem(&Us[i * (NB + 1) + j], P + (p0 + c0 + i) + (int64_t)(kb + j) * m);
                else Us[i * (NB + 1) + j] = T(0);
            }
    };
    for (int j = warp; j < NB; j += 8)
        for (int i = lane; i < NB; i += 32) {
            if (i < w && j < w) {
                if constexpr (kWide) D[i][j] = (C)P[(kb + i) + (int64_t)(kb + j) * m];
                else cp_async_elem(&D[i][j], P + (kb + i) + (int64_t)(kb + j) * m);
            } else {
                D[i][j] = (i == j) ? C(1) : C(0);
            }
        }
    if (pre > 0) stage(0);
    cp_async_wait_all();
    __syncthreads();
    // Thread (ti, tj) owns the RPT x RPT tile at rows i0.., columns j0.. of the block for the rest of
    // the kernel: first the pending lookahead update, then the LU and the inverses, all in registers.
    constexpr int RPT = NB / 16;
    const int ti = tid >> 4, tj = tid & 15, i0 = ti * RPT, j0 = tj * RPT;
    C Ft[RPT][RPT];
    {
        C acc[RPT][RPT];
#pragma unroll
        for (int r = 0; r < RPT; r++)
#pragma unroll
            for (int c = 0; c < RPT; c++) acc[r][c] = C(0);
        // the block's share of the pending update, pre pivots deep, NB at a time
        for (int c0 = 0; c0 < pre; c0 += NB) {
            if (c0 > 0) {
                __syncthreads();  // the previous slice is consumed
                stage(c0);
                cp_async_wait_all();
                __syncthreads();
            }
            const int cw = min(NB, pre - c0);
            for (int q = 0; q < cw; q++) {
                C av[RPT], bv[RPT];
#pragma unroll
                for (int r = 0; r < RPT; r++) {
                    av[r] = Z[i0 + r][q];
                    bv[r] = (C)Us[q * (NB + 1) + j0 + r];
                }
#pragma unroll
                for (int r = 0; r < RPT; r++)
#pragma unroll
                    for (int c = 0; c < RPT; c++) acc[r][c] += av[r] * bv[c];
            }
        }
#pragma unroll
        for (int r = 0; r < RPT; r++)
#pragma unroll
            for (int c = 0; c < RPT; c++) Ft[r][c] = D[i0 + r][j0 + c] - acc[r][c];
    }
    const C amax = (C)__uint_as_float(famax[t.front]);
    const C thr = (C)tol_rel * amax > C(0) ? (C)tol_rel * amax : (C)tiny_pivot<T>();

    // Right-looking elimination in steps of BP = RPT pivots, one block barrier per step (Table 2
    // tasks on the block): every thread factors the BP x BP diagonal block of the step itself
    // (T4 static check, T1 division of the pivot row, T2/T3 inside the block; all threads compute
    // the same values), solves its own rows of L (x U_bb = a) and columns of U (L_bb y = a)
    // against it, and applies the rank-BP update to its tile:  F[i, j] -= L[i, blk] U[blk, j].
    // The inverses ride along, from the same strips:
    //   X = L_D^-1:  rows blk final as L_bb^-1 (rows blk as they stand), X[i, :] -= L[i, blk] X[blk, :]
    //   Y = U_D^-1:  columns blk final as (columns blk as they stand) U_bb^-1, Y[:, j] -= Y[:, blk] U[blk, j]
    // Step s reads the columns and rows p0 = s BP .. p0 + BP - 1 of F (and rows of X, columns of Y)
    // as they stand after step s - 1, published by their owners (the threads whose tile holds them:
    // BP = RPT, so one tile column / row of threads) into a double-buffered strip.
    constexpr int BP = RPT;
    __shared__ __align__(16) C colF[2][BP][NB], rowF[2][BP][NB], rowX[2][BP][NB], colY[2][BP][NB];
    C Xt[INV ? RPT : 1][INV ? RPT : 1], Yt[INV ? RPT : 1][INV ? RPT : 1];
    if constexpr (INV) {
#pragma unroll
        for (int r = 0; r < RPT; r++)
#pragma unroll
            for (int c = 0; c < RPT; c++) Xt[r][c] = Yt[r][c] = (i0 + r == j0 + c) ? C(1) : C(0);
    }
    auto publish = [&](int blk, int buf) {
        if (tj == blk) {
#pragma unroll
            for (int c = 0; c < BP; c++)
#pragma unroll
                for (int r = 0; r < RPT; r++) {
                    colF[buf][c][i0 + r] = Ft[r][c];
                    if constexpr (INV && !SYMB) colY[buf][c][i0 + r] = Yt[r][c];
                }
        }
        if (ti == blk) {
#pragma unroll
            for (int q = 0; q < BP; q++)
#pragma unroll
                for (int c = 0; c < RPT; c++) {
                    rowF[buf][q][j0 + c] = Ft[q][c];
                    if constexpr (INV) rowX[buf][q][j0 + c] = Xt[q][c];
                }
        }
    };
    publish(0, 0);
    __syncthreads();
    const int nsteps = (w + BP - 1) / BP;
#pragma unroll 1
    for (int sb = 0; sb < nsteps; sb++) {
        const int bb = sb & 1, p0 = sb * BP;
        // (a) the diagonal block (identity padding beyond w: its pivots are 1 and not checked)
        C d[BP][BP], rv[BP];
#pragma unroll
        for (int a = 0; a < BP; a++)
#pragma unroll
            for (int c = 0; c < BP; c++) d[a][c] = colF[bb][c][p0 + a];
#pragma unroll
        for (int q = 0; q < BP; q++) {
            if (p0 + q < w) d[q][q] = checked_pivot(d[q][q], thr, tid == 0, t.front, kb + p0 + q, st);
            rv[q] = C(1) / d[q][q];
#pragma unroll
            for (int c = q + 1; c < BP; c++) d[q][c] *= rv[q];
#pragma unroll
            for (int a = q + 1; a < BP; a++)
#pragma unroll
                for (int c = q + 1; c < BP; c++) d[a][c] -= d[a][q] * d[q][c];
        }
        // (b) L of my rows below the block, U of my columns right of it (zero elsewhere)
        const bool rows_below = i0 >= p0 + BP, cols_right = j0 >= p0 + BP;
        C lm[RPT][BP], um[RPT][BP];
#pragma unroll
        for (int r = 0; r < RPT; r++) {
#pragma unroll
            for (int c = 0; c < BP; c++) {
                C x = colF[bb][c][i0 + r];
#pragma unroll
                for (int q = 0; q < c; q++) x -= lm[r][q] * d[q][c];
                lm[r][c] = x;
            }
#pragma unroll
            for (int c = 0; c < BP; c++) lm[r][c] = rows_below ? lm[r][c] : C(0);
        }
#pragma unroll
        for (int c = 0; c < RPT; c++) {
#pragma unroll
            for (int q = 0; q < BP; q++) {
                C y = rowF[bb][q][j0 + c];
#pragma unroll
                for (int t2 = 0; t2 < q; t2++) y -= d[q][t2] * um[c][t2];
                um[c][q] = y * rv[q];
            }
#pragma unroll
            for (int q = 0; q < BP; q++) um[c][q] = cols_right ? um[c][q] : C(0);
        }
        // (c) rank-BP update of my tile, then the final values of the block's rows and columns
#pragma unroll
        for (int r = 0; r < RPT; r++)
#pragma unroll
            for (int c = 0; c < RPT; c++) {
                C v = Ft[r][c];
#pragma unroll
                for (int q = 0; q < BP; q++) v -= lm[r][q] * um[c][q];
                Ft[r][c] = v;
            }
        if (ti == sb) {  // my rows are the block's rows: U right of the block, the block itself
#pragma unroll
            for (int r = 0; r < RPT; r++)
#pragma unroll
                for (int c = 0; c < RPT; c++) {
                    if (cols_right) Ft[r][c] = um[c][r];
                    else if (tj == sb) Ft[r][c] = d[r][c];
                }
        }
        if (tj == sb && rows_below) {  // my columns are the block's columns: L below the block
#pragma unroll
            for (int r = 0; r < RPT; r++)
#pragma unroll
                for (int c = 0; c < RPT; c++) Ft[r][c] = lm[r][c];
        }
        if constexpr (INV) {
            // X: the block's rows through L_bb^-1, then the rows below
#pragma unroll
            for (int c = 0; c < RPT; c++) {
                C xf[BP];
#pragma unroll
                for (int q = 0; q < BP; q++) {
                    C x = rowX[bb][q][j0 + c];
#pragma unroll
                    for (int t2 = 0; t2 < q; t2++) x -= d[q][t2] * xf[t2];
                    xf[q] = x * rv[q];
                }
#pragma unroll
                for (int r = 0; r < RPT; r++) {
                    C v = Xt[r][c];
#pragma unroll
                    for (int q = 0; q < BP; q++) v -= lm[r][q] * xf[q];
                    Xt[r][c] = ti == sb ? xf[r] : v;
                }
            }
            // Y: the block's columns through U_bb^-1, then the columns to the right
#pragma unroll
            for (int r = 0; r < RPT && !SYMB; r++) {
                C yf[BP];
#pragma unroll
                for (int q = 0; q < BP; q++) {
                    C y = colY[bb][q][i0 + r];
#pragma unroll
                    for (int t2 = 0; t2 < q; t2++) y -= yf[t2] * d[t2][q];
                    yf[q] = y;
                }
#pragma unroll
                for (int c = 0; c < RPT; c++) {
                    C v = Yt[r][c];
#pragma unroll
                    for (int q = 0; q < BP; q++) v -= yf[q] * um[c][q];
                    Yt[r][c] = tj == sb ? yf[c] : v;
                }
            }
        }
        if (sb + 1 < nsteps) publish(sb + 1, bb ^ 1);
        __syncthreads();
    }
    // factored block back to P and the inverses to the panel slot, through shared memory (coalesced)
#pragma unroll
    for (int r = 0; r < RPT; r++)
#pragma unroll
        for (int c = 0; c < RPT; c++) {
            D[i0 + r][j0 + c] = Ft[r][c];
            if constexpr (INV) Z[i0 + r][j0 + c] = (i0 + r >= j0 + c) ? Xt[r][c] : (SYMB ? C(0) : Yt[r][c]);
        }
    __syncthreads();
    if constexpr (INV && SYMB) {  // U_D^-1[i, j] = L_D^-1[j, i] L_D[j, j] above the diagonal
        for (int j = warp; j < NB; j += 8)
            for (int i = lane; i < j; i += 32) Z[i][j] = Z[j][i] * D[j][j];
        __syncthreads();
    }
    // one pass writes the block to P and (INV) its inverses to the panel slot and Q (ld k): every
    // element of a thread (column warp + 8u, rows lane + 32v) is read from shared memory first, then
    // the stores follow
    constexpr int UJ = NB / 8, VI = (NB + 31) / 32;
    T pv[UJ][VI], zv[UJ][VI];
#pragma unroll
    for (int u = 0; u < UJ; u++)
#pragma unroll
        for (int v = 0; v < VI; v++) {
            const int j = warp + 8 * u, i = lane + 32 * v;
            pv[u][v] = i < NB ? (T)D[i][j] : T(0);
            if constexpr (INV) zv[u][v] = i < NB ? (T)Z[i][j] : T(0);
        }
    T* Zg = slots + t.slot;
    T* Q = inv + (t.q_off >= 0 ? t.q_off : 0);  // the same block of the solve's pivot-block inverse
#pragma unroll
    for (int u = 0; u < UJ; u++)
#pragma unroll
        for (int v = 0; v < VI; v++) {
            const int j = warp + 8 * u, i = lane + 32 * v;
            if (i >= w || j >= w) continue;
            P[(kb + i) + (int64_t)(kb + j) * m] = pv[u][v];
            if constexpr (INV) {  // INV = false: the panel is finished by triangular solves (k_panel_trsm)
                Zg[i + j * 64] = zv[u][v];
                if (t.q_off >= 0) Q[(kb + i) + (int64_t)(kb + j) * fr.k] = zv[u][v];
            }
        }
}

// ---------------------------------------------------------------------------
// Panel of a pivot block finished by triangular solves against the factored
// block D = L_D U_D (Table 2's tasks carried on past the pivot block):
//   side 0, rows below the block:      x U_D = a   (U_D unit upper)  -> L21
//   side 1, pivot columns right of it: L_D y = a   (L_D with its diagonal) -> U12 in P
//   side 2, contribution-block columns: the same, in R
// 128 threads per CTA, one row (side 0) or column (sides 1, 2) per thread, the
// row or column in registers, D in shared memory; right-looking, so every step
// is NB - j independent FMAs.  Each task covers up to 128 rows or columns.
struct TrsmTask {
    int32_t front, kb, w, side, i0, n;
};

template <typename T, int NB>
__global__ void __launch_bounds__(128) k_panel_trsm(const FrontDev* __restrict__ fronts, const TrsmTask* __restrict__ tasks,
                                                    T* __restrict__ fac) {
    __shared__ T D[NB][NB + 1];
    __shared__ T rdiv[NB];
    const TrsmTask t = tasks[blockIdx.x];
    const FrontDev fr = fronts[t.front];
    const int m = fr.m, k = fr.k, kb = t.kb, w = t.w;
    T* P = fac + fr.P_off;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int j = warp; j < NB; j += 4)
        for (int i = lane; i < NB; i += 32)
            D[i][j] = (i < w && j < w) ? P[(kb + i) + (int64_t)(kb + j) * m] : (i == j ? T(1) : T(0));
    __syncthreads();
    if (threadIdx.x < NB) rdiv[threadIdx.x] = D[threadIdx.x][threadIdx.x];
    __syncthreads();
    const int q = threadIdx.x;
    if (q >= t.n) return;
    T x[NB];
    if (t.side == 0) {
        const int64_t i = kb + w + t.i0 + q;  // row of P
#pragma unroll
        for (int j = 0; j < NB; j++) x[j] = j < w ? P[i + (int64_t)(kb + j) * m] : T(0);
#pragma unroll
        for (int j = 0; j < NB; j++) {
            // keep each step's shared-memory reads inside the step (hoisting them all ahead would
            // need ~NB^2/2 registers)
            asm volatile("" ::: "memory");
#pragma unroll
            for (int j2 = j + 1; j2 < NB; j2++) x[j2] -= x[j] * D[j][j2];
        }
#pragma unroll
        for (int j = 0; j < NB; j++)
            if (j < w) P[i + (int64_t)(kb + j) * m] = x[j];
        return;
    }
    // a column of P right of the block (side 1) or of R (side 2): rows kb .. kb + w
    T* col = t.side == 1 ? P + kb + (int64_t)(kb + w + t.i0 + q) * m : fac + fr.R_off + kb + (int64_t)(t.i0 + q) * k;
    (void)k;
#pragma unroll
    for (int i = 0; i < NB; i++) x[i] = i < w ? col[i] : T(0);
#pragma unroll
    for (int i = 0; i < NB; i++) {
        asm volatile("" ::: "memory");
        x[i] = x[i] / rdiv[i];  // the division task T1 by the pivot
#pragma unroll
        for (int i2 = i + 1; i2 < NB; i2++) x[i2] -= D[i2][i] * x[i];
    }
#pragma unroll
    for (int i = 0; i < NB; i++)
        if (i < w) col[i] = x[i];
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
    // epilogue: for C -= A B all 16 loads are issued before any store (a load-store chain on
    // addresses the compiler cannot prove distinct would serialise 16 memory round trips)
    T cv[4][4];
    if (t.op == 0) {
#pragma unroll
        for (int c = 0; c < 4; c++)
#pragma unroll
            for (int r = 0; r < 4; r++) {
                const int gi = t.i0 + tx + 16 * r, gj = t.j0 + ty + 16 * c;
                cv[r][c] = (gi < t.M && gj < t.N) ? C[gi + (int64_t)gj * t.ldc] : T(0);
            }
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
            if (t.op == 0) *dst = cv[r][c] - acc[r][c];
            else if (t.op == 1) *dst = acc[r][c];
            else *dst = -acc[r][c];
        }
    }
}

// 4-byte global -> shared copy that writes zero when `pred` is false (nothing is read then;
// the source address is still kept inside the operand)
__device__ __forceinline__ void cp_async4_zfill(float* smem_dst, const float* gmem_src, bool pred) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem_dst);
    const int n = pred ? 4 : 0;
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(s), "l"(gmem_src), "r"(n) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait_group() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

// FP32 variant of k_gemm for the same 64 x 64 output tiles and 256 threads,
// written against latency: the operand slices of depth BK stream through a
// ring of STAGES shared buffers by cp.async (zero-filled outside the
// operands, masks applied in place by the copying thread), so up to
// STAGES - 1 slices are in flight while one is multiplied; the C tile of
// C -= A B is read into registers at the start.  Each thread holds a
// contiguous 4 x 4 block (rows 4tx.., columns 4ty..) and reads its operands
// as two float4 shared loads per k.  Same tile semantics as k_gemm: op 0
// C -= A B, op 1 C = A B, op 2 C = -A B, triangular operand masks.
template <int BK, int STAGES>
__global__ void __launch_bounds__(256, 3) k_gemm_cp(const GemmTile* __restrict__ tiles, Arenas<float> ar) {
    constexpr int LD = 64 + 4;  // row pitch (floats): 16-byte aligned rows
    __shared__ __align__(16) float As[STAGES][BK][LD];
    __shared__ __align__(16) float Bs[STAGES][BK][LD];
    const GemmTile t = tiles[blockIdx.x];
    const float* A = ar.a[t.a_ar] + t.a_off;
    const float* B = ar.a[t.b_ar] + t.b_off;
    float* C = ar.a[t.c_ar] + t.c_off;
    const int tid = threadIdx.x;
    const int tx = tid & 15, ty = tid >> 4;
    constexpr int PER = 64 * BK / 256;  // elements of each operand slice per thread
    static_assert(PER * 4 == BK || BK == 16, "slice mapping assumes BK = 16");
    const int nk = (t.K + BK - 1) / BK;
    // thread -> slice elements: A (ai, ak + 4r) (down a column), B (bk, bj + 16r) (down a column of B)
    const int ai = tid & 63, ak = tid >> 6, bk = tid & 15, bj = tid >> 4;
    const bool a_row = t.i0 + ai < t.M;
    const float* pa = a_row ? A + (t.i0 + ai) + (int64_t)ak * t.lda : A;
    const float* pb = B + bk + (int64_t)(t.j0 + bj) * t.ldb;
    auto issue = [&](int kt) {
        const int buf = kt % STAGES, kk0 = kt * BK;
#pragma unroll
        for (int r = 0; r < PER; r++) {
            const bool va = a_row && kk0 + ak + 4 * r < t.K;
            cp_async4_zfill(&As[buf][ak + 4 * r][ai], va ? pa + (int64_t)(kk0 + 4 * r) * t.lda : A, va);
            const bool vb = t.j0 + bj + 16 * r < t.N && kk0 + bk < t.K;
            cp_async4_zfill(&Bs[buf][bk][bj + 16 * r], vb ? pb + kk0 + (int64_t)(16 * r) * t.ldb : B, vb);
        }
    };
    auto fix_masks = [&](int kt) {  // the copying thread's own elements, after its wait
        const int buf = kt % STAGES, kk0 = kt * BK;
#pragma unroll
        for (int r = 0; r < PER; r++) {
            const int gi = t.i0 + ai, gk = kk0 + ak + 4 * r;
            if (t.a_mask && gi < t.M && gk < t.K) As[buf][ak + 4 * r][ai] = masked(As[buf][ak + 4 * r][ai], t.a_mask, gi, gk);
            const int gj = t.j0 + bj + 16 * r, gk2 = kk0 + bk;
            if (t.b_mask && gj < t.N && gk2 < t.K) Bs[buf][bk][bj + 16 * r] = masked(Bs[buf][bk][bj + 16 * r], t.b_mask, gk2, gj);
        }
    };
#pragma unroll
    for (int st = 0; st < STAGES - 1; st++) {
        if (st < nk) issue(st);
        cp_async_commit();
    }
    // C of C -= A B: read now, used after the k loop
    float cv[4][4];
    const int ci = t.i0 + 4 * tx, cj = t.j0 + 4 * ty;
    float* pc = C + ci + (int64_t)cj * t.ldc;
#pragma unroll
    for (int c = 0; c < 4; c++)
#pragma unroll
        for (int r = 0; r < 4; r++)
            cv[r][c] = (t.op == 0 && ci + r < t.M && cj + c < t.N) ? pc[r + (int64_t)c * t.ldc] : 0.f;
    float acc[4][4];
#pragma unroll
    for (int r = 0; r < 4; r++)
#pragma unroll
        for (int c = 0; c < 4; c++) acc[r][c] = 0.f;
    const bool any_mask = t.a_mask || t.b_mask;
    for (int kt = 0; kt < nk; kt++) {
        cp_async_wait_group<STAGES - 2>();  // this thread's copies of slice kt have landed
        if (any_mask) fix_masks(kt);
        __syncthreads();                    // everyone's slice kt is visible; slice kt-1 is consumed
        if (kt + STAGES - 1 < nk) issue(kt + STAGES - 1);
        cp_async_commit();
        const int buf = kt % STAGES;
#pragma unroll
        for (int kk = 0; kk < BK; kk++) {
            const float4 a4 = *reinterpret_cast<const float4*>(&As[buf][kk][4 * tx]);
            const float4 b4 = *reinterpret_cast<const float4*>(&Bs[buf][kk][4 * ty]);
            const float a[4] = {a4.x, a4.y, a4.z, a4.w};
            const float b[4] = {b4.x, b4.y, b4.z, b4.w};
#pragma unroll
            for (int r = 0; r < 4; r++)
#pragma unroll
                for (int c = 0; c < 4; c++) acc[r][c] = fmaf(a[r], b[c], acc[r][c]);
        }
    }
    cp_async_wait_group<0>();
#pragma unroll
    for (int c = 0; c < 4; c++) {
        if (cj + c >= t.N) continue;
#pragma unroll
        for (int r = 0; r < 4; r++) {
            if (ci + r >= t.M) continue;
            pc[r + (int64_t)c * t.ldc] = t.op == 0 ? cv[r][c] - acc[r][c] : (t.op == 1 ? acc[r][c] : -acc[r][c]);
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
