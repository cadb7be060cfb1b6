// Subtree fusion for the bottom of the elimination tree.
//
// The fronts of heights 1..h below a cut are grouped into disjoint subtrees;
// one CTA owns one subtree and walks its levels bottom-up (factor, forward
// sweep) or top-down (backward sweep).  The Foata class barrier between two
// levels of one subtree is the CTA barrier: fronts of a level are independent
// (warps take them as a bag of tasks), and a level starts only after the
// previous one is complete (Sec. 3.3).  Contribution blocks and update
// vectors of fronts inside a subtree never leave shared memory; only leaf
// element matrices come in and factors plus the subtree root's contribution
// block go out.
#pragma once

#include <cstdint>

#include "kernels_factor.cuh"
#include "mf_internal.h"

constexpr int kSubMaxLevels = 8;
constexpr int kSubMaxM = 128;  // largest front inside a fused subtree (4 rows per lane)

struct SubtreeTask {
    int32_t first;                          // first entry in the subtree entry list
    int32_t n_levels;
    int32_t level_ptr[kSubMaxLevels + 1];   // entry ranges per level (relative to first)
    int32_t level_mmax[kSubMaxLevels];      // largest m per level
    int32_t pad;
};

struct SubtreeEntry {
    int32_t front;
    int32_t cb_off;           // pool offset (elements) of this front's CB / update vector, -1 at the subtree root
    int32_t child_off[2];     // pool offsets of the children's CBs / update vectors
};

// Shared-memory layout of one subtree CTA (elements of T unless noted):
//   work: warp slots of level_mmax^2 (fronts being processed)         -- work_size
//   pool: contribution blocks (factor) or update vectors (solve), laid
//         out by the host so that blocks alive at the same level never
//         overlap (a block lives from its front's level to its parent's)  -- buf_size
//   maps: 8 x 2 kSubMaxM int32, then 8 floats for block reductions
struct SubtreeLayout {
    int32_t work_size, buf_size;
};

template <typename T>
__device__ __forceinline__ T warp_max(T v) {
    for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// Partial LU of an m x m front held in shared memory (column-major, ld), on
// its first k pivots, by one warp (Table 2 tasks): T1 divides the pivot row,
// T2/T3 update the rows below.  Lane l owns rows l, l+32, l+64, l+96.
template <typename T>
__device__ __forceinline__ void warp_partial_lu(T* F, int ld, int m, int k, T thr, int32_t front, DevStatus* st) {
    const int lane = threadIdx.x & 31;
    for (int p = 0; p < k; p++) {
        const T piv = checked_pivot(F[p + p * ld], thr, lane == 0, front, p, st);
        __syncwarp();
        if (lane == 0) F[p + p * ld] = piv;
        for (int j = p + 1 + lane; j < m; j += 32) F[p + j * ld] = F[p + j * ld] / piv;
        __syncwarp();
        T l[4];
#pragma unroll
        for (int q = 0; q < 4; q++) {
            const int i = lane + 32 * q;
            l[q] = (i > p && i < m) ? F[i + p * ld] : T(0);
        }
        for (int j = p + 1; j < m; j++) {
            const T u = F[p + j * ld];
#pragma unroll
            for (int q = 0; q < 4; q++) {
                const int i = lane + 32 * q;
                if (i > p && i < m) F[i + j * ld] -= l[q] * u;
            }
        }
        __syncwarp();
    }
}

// One front of a fused subtree: assemble (element matrix or children's
// contribution blocks in shared memory), partial LU, write P and R to the
// factor arena and the CB to shared memory (or, at the subtree root, to the
// CB arena).  CTA = false: the calling warp does everything; CTA = true: all
// threads of the block cooperate (warps over columns, lanes over rows).
template <typename T, bool CTA>
__device__ __forceinline__ void subtree_front(const FrontDev* __restrict__ fronts, const SubtreeEntry& en,
                                              const int32_t* __restrict__ maps, const double* __restrict__ values, int npe,
                                              T* __restrict__ fac, T* __restrict__ cbs, const T* cin, T* cout, T* F, int ld,
                                              int32_t* imap, float* red, double tol_rel, DevStatus* st) {
    const int lane = threadIdx.x & 31;
    const int warp = CTA ? (threadIdx.x >> 5) : 0;
    const int nw = CTA ? (blockDim.x >> 5) : 1;
    const int tid = CTA ? threadIdx.x : lane;
    const int nt = CTA ? blockDim.x : 32;
    auto sync = [&]() {
        if (CTA) __syncthreads();
        else __syncwarp();
    };
    const FrontDev fr = fronts[en.front];
    const int m = fr.m, k = fr.k, nc = m - k;
    const int nmap = fr.nchild > 0 ? fr.nchild * m : m;
    for (int i = tid; i < nmap; i += nt) imap[i] = maps[fr.map_off + i];
    sync();
    T amax = T(0);
    if (fr.nchild == 0) {
        const double* K = values + (int64_t)fr.elem * npe * npe;
        for (int j = warp; j < m; j += nw) {
            const int b = imap[j];
            for (int i = lane; i < m; i += 32) {
                const T v = (T)K[imap[i] + b * npe];
                F[i + j * ld] = v;
                amax = max(amax, (T)fabs(v));
            }
        }
    } else {
        const FrontDev c0 = fronts[fr.child[0]];
        const int n0 = c0.m - c0.k;
        const T* S0 = cin + en.child_off[0];
        int n1 = 0;
        const T* S1 = nullptr;
        if (fr.nchild > 1) {
            const FrontDev c1 = fronts[fr.child[1]];
            n1 = c1.m - c1.k;
            S1 = cin + en.child_off[1];
        }
        for (int j = warp; j < m; j += nw) {
            const int j0 = imap[j];
            const int j1 = fr.nchild > 1 ? imap[m + j] : -1;
            for (int i = lane; i < m; i += 32) {
                T v = T(0);
                const int i0 = imap[i];
                if (i0 >= 0 && j0 >= 0) v += S0[i0 + j0 * n0];
                if (j1 >= 0) {
                    const int i1 = imap[m + i];
                    if (i1 >= 0) v += S1[i1 + j1 * n1];
                }
                F[i + j * ld] = v;
                amax = max(amax, (T)fabs(v));
            }
        }
    }
    if (CTA) amax = block_max_abs(amax, red);
    else amax = warp_max(amax);
    const T thr = (T)tol_rel * amax > T(0) ? (T)tol_rel * amax : tiny_pivot<T>();
    sync();
    if (!CTA) {
        warp_partial_lu(F, ld, m, k, thr, en.front, st);
    } else {
        for (int p = 0; p < k; p++) {
            const T piv = checked_pivot(F[p + p * ld], thr, threadIdx.x == 0, en.front, p, st);
            __syncthreads();
            if (threadIdx.x == 0) F[p + p * ld] = piv;
            for (int j = p + 1 + threadIdx.x; j < m; j += blockDim.x) F[p + j * ld] = F[p + j * ld] / piv;
            __syncthreads();
            for (int j = p + 1 + warp; j < m; j += nw) {
                const T u = F[p + j * ld];
                for (int i = p + 1 + lane; i < m; i += 32) F[i + j * ld] -= F[i + p * ld] * u;
            }
            __syncthreads();
        }
    }
    T* P = fac + fr.P_off;
    for (int j = warp; j < k; j += nw)
        for (int i = lane; i < m; i += 32) P[i + (int64_t)j * m] = F[i + j * ld];
    T* Rg = fac + fr.R_off;
    for (int j = k + warp; j < m; j += nw)
        for (int i = lane; i < k; i += 32) Rg[i + (int64_t)(j - k) * k] = F[i + j * ld];
    T* S = en.cb_off >= 0 ? cout + en.cb_off : cbs + fr.S_off;
    for (int j = k + warp; j < m; j += nw)
        for (int i = k + lane; i < m; i += 32) S[(i - k) + (j - k) * nc] = F[i + j * ld];
    sync();
}

template <typename T>
__global__ void __launch_bounds__(256) k_subtree_factor(const FrontDev* __restrict__ fronts,
                                                        const SubtreeTask* __restrict__ tasks,
                                                        const SubtreeEntry* __restrict__ entries,
                                                        const int32_t* __restrict__ maps, const double* __restrict__ values,
                                                        int npe, T* __restrict__ fac, T* __restrict__ cbs, SubtreeLayout lay,
                                                        double tol_rel, DevStatus* st) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* work = reinterpret_cast<T*>(smem_raw);
    T* pool = work + lay.work_size;
    int32_t* mapsm = reinterpret_cast<int32_t*>(pool + lay.buf_size);
    const SubtreeTask task = tasks[blockIdx.x];
    const int warp = threadIdx.x >> 5;
    int32_t* imap = mapsm + warp * 2 * kSubMaxM;
    for (int L = 0; L < task.n_levels; L++) {
        const int e0 = task.first + task.level_ptr[L], e1 = task.first + task.level_ptr[L + 1];
        const int mL = task.level_mmax[L], ld = mL | 1;
        const T* cin = pool;
        T* cout = pool;
        if (e1 - e0 >= 4) {
            // many fronts: one warp per front
            T* F = work + warp * ld * mL;
            for (int e = e0 + warp; e < e1; e += 8) {
                const SubtreeEntry en = entries[e];
                subtree_front<T, false>(fronts, en, maps, values, npe, fac, cbs, cin, cout, F, ld, imap, nullptr, tol_rel,
                                        st);
            }
        } else {
            // few (large) fronts: the whole CTA on each in turn
            for (int e = e0; e < e1; e++) {
                const SubtreeEntry en = entries[e];
                subtree_front<T, true>(fronts, en, maps, values, npe, fac, cbs, cin, cout, work, ld, mapsm,
                                       reinterpret_cast<float*>(mapsm + 8 * 2 * kSubMaxM), tol_rel, st);
                __syncthreads();
            }
        }
        __syncthreads();
    }
}

// Forward sweep of a fused subtree (levels bottom-up), one warp per front.
template <typename T, bool TRANS>
__global__ void __launch_bounds__(256) k_subtree_fwd(const FrontDev* __restrict__ fronts, const SubtreeTask* __restrict__ tasks,
                                                     const SubtreeEntry* __restrict__ entries, const T* __restrict__ fac,
                                                     const int32_t* __restrict__ dofs, const int32_t* __restrict__ maps,
                                                     T* __restrict__ vecs, int64_t vec_size, SubtreeLayout lay,
                                                     double* __restrict__ x, int64_t n_dof) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* pool = reinterpret_cast<T*>(smem_raw);
    const SubtreeTask task = tasks[blockIdx.x];
    const int r = blockIdx.y;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    double* xr = x + (int64_t)r * n_dof;
    T* vr = vecs + (int64_t)r * vec_size;
    for (int L = 0; L < task.n_levels; L++) {
        const int e0 = task.first + task.level_ptr[L], e1 = task.first + task.level_ptr[L + 1];
        const T* uin = pool;
        T* uout = pool;
        for (int e = e0 + warp; e < e1; e += 8) {
            const SubtreeEntry en = entries[e];
            const FrontDev fr = fronts[en.front];
            const int m = fr.m, k = fr.k;
            const int32_t* fd = dofs + fr.dof_off;
            const T* P = fac + fr.P_off;
            const T* R = fac + fr.R_off;
            T w[4];
#pragma unroll
            for (int q = 0; q < 4; q++) {
                const int i = lane + 32 * q;
                T v = T(0);
                if (i < m) {
                    if (i < k) v = (T)xr[fd[i]];
                    for (int c = 0; c < fr.nchild; c++) {
                        const int ic = maps[fr.map_off + (int64_t)c * m + i];
                        if (ic >= 0) v += uin[en.child_off[c] + ic];
                    }
                }
                w[q] = v;
            }
            for (int p = 0; p < k; p++) {
                const int q0 = p >> 5;
                T wp = w[0];
#pragma unroll
                for (int q = 1; q < 4; q++)
                    if (q == q0) wp = w[q];
                const T yp = __shfl_sync(0xffffffffu, wp, p & 31) / (TRANS ? T(1) : P[p + (int64_t)p * m]);
#pragma unroll
                for (int q = 0; q < 4; q++) {
                    const int i = lane + 32 * q;
                    if (i == p) w[q] = yp;
                    else if (i > p && i < m) w[q] -= (!TRANS ? P[i + (int64_t)p * m]
                                                             : (i < k ? P[p + (int64_t)i * m] : R[p + (int64_t)(i - k) * k])) *
                                                     yp;
                }
            }
#pragma unroll
            for (int q = 0; q < 4; q++) {
                const int i = lane + 32 * q;
                if (i < k) xr[fd[i]] = (double)w[q];
                else if (i < m) {
                    if (en.cb_off >= 0) uout[en.cb_off + (i - k)] = w[q];
                    else vr[fr.vec_off + (i - k)] = w[q];
                }
            }
        }
        __syncthreads();
    }
}

// Backward sweep of a fused subtree (levels top-down), one warp per front;
// unknowns travel through x in global memory (visible inside the CTA after
// the level barrier).
template <typename T, bool TRANS>
__global__ void __launch_bounds__(256) k_subtree_bwd(const FrontDev* __restrict__ fronts, const SubtreeTask* __restrict__ tasks,
                                                     const SubtreeEntry* __restrict__ entries, const T* __restrict__ fac,
                                                     const int32_t* __restrict__ dofs, double* __restrict__ x,
                                                     int64_t n_dof) {
    const SubtreeTask task = tasks[blockIdx.x];
    const int r = blockIdx.y;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    double* xr = x + (int64_t)r * n_dof;
    for (int L = task.n_levels - 1; L >= 0; L--) {
        const int e0 = task.first + task.level_ptr[L], e1 = task.first + task.level_ptr[L + 1];
        for (int e = e0 + warp; e < e1; e += 8) {
            const FrontDev fr = fronts[entries[e].front];
            const int m = fr.m, k = fr.k;
            const int32_t* fd = dofs + fr.dof_off;
            const T* P = fac + fr.P_off;
            const T* R = fac + fr.R_off;
            T v[4];
#pragma unroll
            for (int q = 0; q < 4; q++) {
                const int i = lane + 32 * q;
                v[q] = i < m ? (T)xr[fd[i]] : T(0);
            }
            for (int j = m - 1; j >= 0; j--) {
                const int q0 = j >> 5;
                T vj = v[0];
#pragma unroll
                for (int q = 1; q < 4; q++)
                    if (q == q0) vj = v[q];
                T xj = __shfl_sync(0xffffffffu, vj, j & 31);
                if (j < k && TRANS) xj = xj / P[j + (int64_t)j * m];
#pragma unroll
                for (int q = 0; q < 4; q++) {
                    const int i = lane + 32 * q;
                    if (i == j && j < k) v[q] = xj;
                    else if (i < k && i < j)
                        v[q] -= (!TRANS ? (j < k ? P[i + (int64_t)j * m] : R[i + (int64_t)(j - k) * k])
                                        : P[j + (int64_t)i * m]) *
                                xj;
                }
            }
#pragma unroll
            for (int q = 0; q < 4; q++) {
                const int i = lane + 32 * q;
                if (i < k) xr[fd[i]] = (double)v[q];
            }
        }
        __syncthreads();
    }
}
