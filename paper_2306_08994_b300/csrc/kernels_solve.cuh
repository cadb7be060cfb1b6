// Solve-phase kernels: batched forward/backward substitution down the tree
// (`get_solution`, Table 2), FP64 element-by-element residual for iterative
// refinement, norms, and the adjoint gradient contractions.
#pragma once

#include <cstdint>

#include "kernels_factor.cuh"
#include "mf_internal.h"

// ---------------------------------------------------------------------------
// Substitution down the tree (`get_solution`, Table 2), one class per step.
// Per front, with w the front's right-hand side (b at its pivots plus the
// children's update vectors):
//   forward  !TRANS: L11 y = w1, w2 -= L21 y           (L non-unit)
//             TRANS: U11^T y = w1, w2 -= U12^T y       (unit)
//   backward !TRANS: U11 x1 = y - U12 x_CB             (unit)
//             TRANS: L11^T x1 = y - L21^T x_CB
// y is kept in x at the pivots between the two sweeps; w2 goes to the
// front's update vector, pulled by the parent (no two fronts write the same
// entry, so the result is deterministic).
//
// Coefficient accessors.  Forward: coefficient of pivot p in row i (i > p).
template <typename T, bool TRANS>
__device__ __forceinline__ T fcoef(const T* P, const T* R, int m, int k, int i, int p) {
    if (!TRANS) return P[i + (int64_t)p * m];
    return i < k ? P[p + (int64_t)i * m] : R[p + (int64_t)(i - k) * k];
}
// Backward: coefficient of unknown j in pivot row i (j > i).
template <typename T, bool TRANS>
__device__ __forceinline__ T bcoef(const T* P, const T* R, int m, int k, int i, int j) {
    if (!TRANS) return j < k ? P[i + (int64_t)j * m] : R[i + (int64_t)(j - k) * k];
    return P[j + (int64_t)i * m];
}
template <typename T, bool TRANS>
__device__ __forceinline__ T fdiag(const T* P, int m, int p) {
    return TRANS ? T(1) : P[p + (int64_t)p * m];
}
template <typename T, bool TRANS>
__device__ __forceinline__ T bdiag(const T* P, int m, int p) {
    return TRANS ? P[p + (int64_t)p * m] : T(1);
}

// Where row i of a front's right-hand side comes from: its own dof (pivot
// rows) and the update-vector entries of the children that hold it.  The
// children's entries are precomputed per front row (vsrc[2 (dof_off + i) + c],
// -1 when child c does not hold row i), so no child map or child descriptor
// is read on the way.
struct RhsSrc {
    int64_t xi, v0, v1;  // -1 when absent
};

// What the small- and mid-front substitution kernels read of a front, stored
// in substitution-list order (one load, no list -> descriptor indirection).
struct SolveRec {
    int64_t P_off, R_off, dof_off, vec_off;
    int32_t m, k, nchild, pad;
};

template <typename FR>
__device__ __forceinline__ RhsSrc rhs_src(const FR& fr, const int32_t* __restrict__ fd, const int64_t* __restrict__ vsrc,
                                          int i) {
    RhsSrc q{-1, -1, -1};
    if (i < fr.k) q.xi = fd[i];
    if (fr.nchild > 0) {
        const int64_t* v = vsrc + 2 * (fr.dof_off + i);
        q.v0 = v[0];
        q.v1 = v[1];
    }
    return q;
}
template <typename T>
__device__ __forceinline__ T rhs_val(const RhsSrc& q, const T* __restrict__ vr, const double* __restrict__ xr) {
    T v = q.xi >= 0 ? (T)__ldcg(xr + q.xi) : T(0);
    if (q.v0 >= 0) v += __ldcg(vr + q.v0);
    if (q.v1 >= 0) v += __ldcg(vr + q.v1);
    return v;
}

template <typename T, typename FR>
__device__ __forceinline__ T gather_rhs(const FR& fr, const int32_t* __restrict__ fd, const int64_t* __restrict__ vsrc,
                                        const T* __restrict__ vr, const double* __restrict__ xr, int i) {
    return rhs_val<T>(rhs_src<FR>(fr, fd, vsrc, i), vr, xr);
}

// Right-hand sides are processed in chunks inside one launch, so a front's
// coefficients are loaded once per chunk: NR = 1 (single right-hand side,
// fewest registers) or kRhsChunk.
constexpr int kRhsChunk = 4;

// Substitution kernels use programmatic dependent launch (pdl_wait / pdl_trigger,
// kernels_factor.cuh): each loads what no earlier kernel of the solve writes (factor
// coefficients, dof lists, gather sources) before its pdl_wait, and right-hand sides,
// update vectors and pivot values only after it.

// Symmetric solves scale the forward result by D before the backward sweep
// (z = D y).  With scale set, a forward kernel stores the pivot rows as
// y_p d_p (the pivot read from the factor, the product formed in FP64: the
// same value the separate scaling pass computes), so that pass is skipped.
template <typename T>
__device__ __forceinline__ double pivot_out(T y, const T* P, int m, int row, int scale) {
    return scale ? (double)y * (double)P[row + (int64_t)row * m] : (double)y;
}

// y = w / d for one right-hand side, w * (1/d) for several (one reciprocal
// per pivot shared by the chunk).
template <typename T, int NR>
__device__ __forceinline__ T pivot_scale(T d) {
    return NR == 1 ? d : T(1) / d;
}
template <typename T, int NR>
__device__ __forceinline__ T apply_pivot(T w, T ds) {
    return NR == 1 ? w / ds : w * ds;
}

// Small fronts (m <= 64): one warp per front, rows lane and lane+32.
template <typename T, bool TRANS, int NR>
__device__ __forceinline__ void k_fwd_warp_body(const FrontDev* __restrict__ fronts, const SolveRec* __restrict__ list,
                                                  int count, const T* __restrict__ fac, const int32_t* __restrict__ dofs,
                                                  const int64_t* __restrict__ vsrc, T* __restrict__ vecs, int64_t vec_size,
                                                  double* __restrict__ x, int64_t n_dof, int nrhs, int vb, int scale = 0) {
    const int wid = vb * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (wid >= count) return;
    const SolveRec fr = list[wid];
    const int m = fr.m, k = fr.k;
    const int32_t* fd = dofs + fr.dof_off;
    const T* P = fac + fr.P_off;
    const T* R = fac + fr.R_off;
    const int i0 = lane, i1 = lane + 32;
    const RhsSrc s0 = i0 < m ? rhs_src<SolveRec>(fr, fd, vsrc, i0) : RhsSrc{-1, -1, -1};
    const RhsSrc s1 = i1 < m ? rhs_src<SolveRec>(fr, fd, vsrc, i1) : RhsSrc{-1, -1, -1};
    pdl_wait();
    for (int rb = 0; rb < nrhs; rb += NR) {
        const int nr = min(NR, nrhs - rb);
        T w0[NR], w1[NR];
#pragma unroll
        for (int rr = 0; rr < NR; rr++) {
            w0[rr] = w1[rr] = T(0);
            if (rr < nr) {
                const double* xr = x + (int64_t)(rb + rr) * n_dof;
                const T* vr = vecs + (int64_t)(rb + rr) * vec_size;
                w0[rr] = rhs_val<T>(s0, vr, xr);
                w1[rr] = rhs_val<T>(s1, vr, xr);
            }
        }
        for (int pc = 0; pc < k; pc += 8) {
            T c0[8], c1[8], dg[8];
#pragma unroll
            for (int q = 0; q < 8; q++) {
                const int p = pc + q;
                c0[q] = (p < k && i0 > p && i0 < m) ? fcoef<T, TRANS>(P, R, m, k, i0, p) : T(0);
                c1[q] = (p < k && i1 > p && i1 < m) ? fcoef<T, TRANS>(P, R, m, k, i1, p) : T(0);
                dg[q] = p < k ? fdiag<T, TRANS>(P, m, p) : T(1);
            }
#pragma unroll
            for (int q = 0; q < 8; q++) {
                const int p = pc + q;
                if (p >= k) break;
                const T ds = pivot_scale<T, NR>(dg[q]);
#pragma unroll
                for (int rr = 0; rr < NR; rr++) {
                    if (rr >= nr) break;
                    T wp = (p < 32) ? __shfl_sync(0xffffffffu, w0[rr], p) : __shfl_sync(0xffffffffu, w1[rr], p - 32);
                    const T yp = apply_pivot<T, NR>(wp, ds);
                    if (i0 == p) w0[rr] = yp;
                    if (i1 == p) w1[rr] = yp;
                    w0[rr] -= c0[q] * yp;
                    w1[rr] -= c1[q] * yp;
                }
            }
        }
#pragma unroll
        for (int rr = 0; rr < NR; rr++) {
            if (rr >= nr) break;
            double* xr = x + (int64_t)(rb + rr) * n_dof;
            T* vr = vecs + (int64_t)(rb + rr) * vec_size;
            if (i0 < m) {
                if (i0 < k) xr[fd[i0]] = pivot_out(w0[rr], P, m, i0, scale);
                else vr[fr.vec_off + (i0 - k)] = w0[rr];
            }
            if (i1 < m) {
                if (i1 < k) xr[fd[i1]] = pivot_out(w1[rr], P, m, i1, scale);
                else vr[fr.vec_off + (i1 - k)] = w1[rr];
            }
        }
    }
}
template <typename T, bool TRANS, int NR>
__global__ void __launch_bounds__(256, NR == 1 ? 4 : 2) k_fwd_warp(const FrontDev* __restrict__ fronts, const SolveRec* __restrict__ list,
                                                  int count, const T* __restrict__ fac, const int32_t* __restrict__ dofs,
                                                  const int64_t* __restrict__ vsrc, T* __restrict__ vecs, int64_t vec_size,
                                                  double* __restrict__ x, int64_t n_dof, int nrhs, int scale) {
    pdl_trigger();
    k_fwd_warp_body<T, TRANS, NR>(fronts, list, count, fac, dofs, vsrc, vecs, vec_size, x, n_dof, nrhs, blockIdx.x, scale);
}

template <typename T, bool TRANS, int NR>
__device__ __forceinline__ void k_bwd_warp_body(const FrontDev* __restrict__ fronts, const SolveRec* __restrict__ list,
                                                  int count, const T* __restrict__ fac, const int32_t* __restrict__ dofs,
                                                  double* __restrict__ x, int64_t n_dof, int nrhs, int vb) {
    const int wid = vb * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (wid >= count) return;
    const SolveRec fr = list[wid];
    const int m = fr.m, k = fr.k;
    const int32_t* fd = dofs + fr.dof_off;
    const T* P = fac + fr.P_off;
    const T* R = fac + fr.R_off;
    const int i0 = lane, i1 = lane + 32;
    const int d0 = i0 < m ? fd[i0] : 0, d1 = i1 < m ? fd[i1] : 0;
    pdl_wait();
    for (int rb = 0; rb < nrhs; rb += NR) {
        const int nr = min(NR, nrhs - rb);
        // all unknowns of the front: pivots hold y, CB holds the final x
        T v0[NR], v1[NR];
#pragma unroll
        for (int rr = 0; rr < NR; rr++) {
            const double* xr = x + (int64_t)(rb + rr) * n_dof;
            v0[rr] = (rr < nr && i0 < m) ? (T)__ldcg(xr + d0) : T(0);
            v1[rr] = (rr < nr && i1 < m) ? (T)__ldcg(xr + d1) : T(0);
        }
        // eliminate the CB unknowns from the pivot rows (j >= k), then back-substitute
        for (int jc = m - 1; jc >= 0; jc -= 8) {
            T c0[8], c1[8], dg[8];
#pragma unroll
            for (int q = 0; q < 8; q++) {
                const int j = jc - q;
                c0[q] = (j >= 0 && i0 < k && i0 < j) ? bcoef<T, TRANS>(P, R, m, k, i0, j) : T(0);
                c1[q] = (j >= 0 && i1 < k && i1 < j) ? bcoef<T, TRANS>(P, R, m, k, i1, j) : T(0);
                dg[q] = (j >= 0 && j < k) ? bdiag<T, TRANS>(P, m, j) : T(1);
            }
#pragma unroll
            for (int q = 0; q < 8; q++) {
                const int j = jc - q;
                if (j < 0) break;
                const T ds = pivot_scale<T, NR>(dg[q]);
#pragma unroll
                for (int rr = 0; rr < NR; rr++) {
                    if (rr >= nr) break;
                    T xj = (j < 32) ? __shfl_sync(0xffffffffu, v0[rr], j) : __shfl_sync(0xffffffffu, v1[rr], j - 32);
                    if (j < k) {
                        xj = apply_pivot<T, NR>(xj, ds);
                        if (i0 == j) v0[rr] = xj;
                        if (i1 == j) v1[rr] = xj;
                    }
                    v0[rr] -= c0[q] * xj;
                    v1[rr] -= c1[q] * xj;
                }
            }
        }
#pragma unroll
        for (int rr = 0; rr < NR; rr++) {
            if (rr >= nr) break;
            double* xr = x + (int64_t)(rb + rr) * n_dof;
            if (i0 < k) xr[d0] = (double)v0[rr];
            if (i1 < k) xr[d1] = (double)v1[rr];
        }
    }
}
template <typename T, bool TRANS, int NR>
__global__ void __launch_bounds__(256, NR == 1 ? 4 : 2) k_bwd_warp(const FrontDev* __restrict__ fronts, const SolveRec* __restrict__ list,
                                                  int count, const T* __restrict__ fac, const int32_t* __restrict__ dofs,
                                                  double* __restrict__ x, int64_t n_dof, int nrhs) {
    pdl_trigger();
    k_bwd_warp_body<T, TRANS, NR>(fronts, list, count, fac, dofs, x, n_dof, nrhs, blockIdx.x);
}

// Small fronts with few pivots (m <= G R, k <= KM): G lanes per front, lane i
// holding rows i, i + G, ..., i + G (R - 1).  The coefficient arrays are sized
// by the pivot bound KM rather than by the front, so the kernels stay small
// enough for full occupancy, and every load a front needs is issued right
// after its record: the chain is record -> (coefficients, row sources) ->
// right-hand-side values -> the short pivot loop -> stores.
//
// Forward (L y = b restricted to the front, then the update vector): pivot p
// is broadcast from its owner lane and every row below it subtracts its
// coefficient times it.
template <typename T, bool TRANS, int G, int R, int KM, int NR>
__device__ __forceinline__ void k_fwd_lg_body(const SolveRec* __restrict__ list, int count, const T* __restrict__ fac,
                                              const int32_t* __restrict__ dofs, const int64_t* __restrict__ vsrc,
                                              T* __restrict__ vecs, int64_t vec_size, double* __restrict__ x,
                                              int64_t n_dof, int nrhs, int vb, int scale = 0) {
    static_assert(KM <= G * R, "pivot bound beyond the rows of a group");
    const int lane = threadIdx.x & 31;
    const int fidx = (vb * (blockDim.x >> 5) + (threadIdx.x >> 5)) * (32 / G) + lane / G;
    const bool active = fidx < count;
    const int i = lane % G;
    SolveRec fr{};
    if (active) fr = list[fidx];
    const int m = fr.m, k = fr.k;
    const int32_t* fd = dofs + fr.dof_off;
    const T* P = fac + fr.P_off;
    const T* Rb = fac + fr.R_off;
    T c[R][KM], dg[KM];
    RhsSrc src[R];
#pragma unroll
    for (int q = 0; q < R; q++) {
        const int row = i + G * q;
#pragma unroll
        for (int p = 0; p < KM; p++) c[q][p] = (p < k && row > p && row < m) ? fcoef<T, TRANS>(P, Rb, m, k, row, p) : T(0);
        src[q] = (active && row < m) ? rhs_src<SolveRec>(fr, fd, vsrc, row) : RhsSrc{-1, -1, -1};
    }
#pragma unroll
    for (int p = 0; p < KM; p++) dg[p] = p < k ? fdiag<T, TRANS>(P, m, p) : T(1);
    const int kmax = (int)__reduce_max_sync(0xffffffffu, (unsigned)k);  // warp-uniform pivot count
    pdl_wait();
    for (int rb = 0; rb < nrhs; rb += NR) {
        const int nr = min(NR, nrhs - rb);
        T w[R][NR];
#pragma unroll
        for (int q = 0; q < R; q++)
#pragma unroll
            for (int rr = 0; rr < NR; rr++)
                w[q][rr] = rr < nr ? rhs_val<T>(src[q], vecs + (int64_t)(rb + rr) * vec_size, x + (int64_t)(rb + rr) * n_dof)
                                   : T(0);
#pragma unroll
        for (int p = 0; p < KM; p++) {
            if (p >= kmax) break;
            const T ds = pivot_scale<T, NR>(dg[p]);
#pragma unroll
            for (int rr = 0; rr < NR; rr++) {
                const T yp = apply_pivot<T, NR>(__shfl_sync(0xffffffffu, w[p / G][rr], p % G, G), ds);
                if (p < k) {
#pragma unroll
                    for (int q = 0; q < R; q++) {
                        if (i + G * q == p) w[q][rr] = yp;
                        w[q][rr] -= c[q][p] * yp;
                    }
                }
            }
        }
#pragma unroll
        for (int q = 0; q < R; q++) {
            const int row = i + G * q;
            if (!active || row >= m) continue;
#pragma unroll
            for (int rr = 0; rr < NR; rr++) {
                if (rr >= nr) break;
                if (row < k) x[(int64_t)(rb + rr) * n_dof + src[q].xi] = pivot_out(w[q][rr], P, m, row, scale);
                else vecs[(int64_t)(rb + rr) * vec_size + fr.vec_off + (row - k)] = w[q][rr];
            }
        }
    }
}
template <typename T, bool TRANS, int G, int R, int KM, int NR>
__global__ void __launch_bounds__(256) k_fwd_lg(const SolveRec* __restrict__ list, int count, const T* __restrict__ fac,
                                                const int32_t* __restrict__ dofs, const int64_t* __restrict__ vsrc,
                                                T* __restrict__ vecs, int64_t vec_size, double* __restrict__ x,
                                                int64_t n_dof, int nrhs, int scale) {
    pdl_trigger();
    k_fwd_lg_body<T, TRANS, G, R, KM, NR>(list, count, fac, dofs, vsrc, vecs, vec_size, x, n_dof, nrhs, blockIdx.x, scale);
}

// Backward (U x = y on the front's pivot rows; rows >= k already hold their
// final values): lane i holds the coefficients of its own rows in every pivot
// equation, so pivot p needs only the group sum of (coefficient x value) over
// the rows after it (a butterfly of log2 G shuffles) and no broadcast; pivots
// go from k-1 down, each one final before the equations above it read it.
template <typename T, bool TRANS, int G, int R, int KM, int NR>
__device__ __forceinline__ void k_bwd_lg_body(const SolveRec* __restrict__ list, int count, const T* __restrict__ fac,
                                              const int32_t* __restrict__ dofs, double* __restrict__ x, int64_t n_dof,
                                              int nrhs, int vb) {
    static_assert(KM <= G * R, "pivot bound beyond the rows of a group");
    const int lane = threadIdx.x & 31;
    const int fidx = (vb * (blockDim.x >> 5) + (threadIdx.x >> 5)) * (32 / G) + lane / G;
    const bool active = fidx < count;
    const int i = lane % G;
    SolveRec fr{};
    if (active) fr = list[fidx];
    const int m = fr.m, k = fr.k;
    const int32_t* fd = dofs + fr.dof_off;
    const T* P = fac + fr.P_off;
    const T* Rb = fac + fr.R_off;
    T u[R][KM], dg[KM];
    int di[R];
#pragma unroll
    for (int q = 0; q < R; q++) {
        const int row = i + G * q;
#pragma unroll
        for (int p = 0; p < KM; p++) u[q][p] = (p < k && row > p && row < m) ? bcoef<T, TRANS>(P, Rb, m, k, p, row) : T(0);
        di[q] = (active && row < m) ? fd[row] : 0;
    }
#pragma unroll
    for (int p = 0; p < KM; p++) dg[p] = p < k ? bdiag<T, TRANS>(P, m, p) : T(1);
    const int kmax = (int)__reduce_max_sync(0xffffffffu, (unsigned)k);
    pdl_wait();
    for (int rb = 0; rb < nrhs; rb += NR) {
        const int nr = min(NR, nrhs - rb);
        T v[R][NR];
#pragma unroll
        for (int q = 0; q < R; q++)
#pragma unroll
            for (int rr = 0; rr < NR; rr++)
                v[q][rr] = (rr < nr && active && i + G * q < m) ? (T)__ldcg(x + (int64_t)(rb + rr) * n_dof + di[q]) : T(0);
#pragma unroll
        for (int p = KM - 1; p >= 0; p--) {
            if (p >= kmax) continue;
            const T ds = pivot_scale<T, NR>(dg[p]);
#pragma unroll
            for (int rr = 0; rr < NR; rr++) {
                T sum = T(0);
#pragma unroll
                for (int q = 0; q < R; q++) sum += u[q][p] * v[q][rr];
#pragma unroll
                for (int o = G / 2; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o, G);
                if (p < k) {
#pragma unroll
                    for (int q = 0; q < R; q++)
                        if (i + G * q == p) v[q][rr] = apply_pivot<T, NR>(v[q][rr] - sum, ds);
                }
            }
        }
#pragma unroll
        for (int q = 0; q < R; q++) {
            const int row = i + G * q;
            if (!active || row >= k) continue;
#pragma unroll
            for (int rr = 0; rr < NR; rr++)
                if (rr < nr) x[(int64_t)(rb + rr) * n_dof + di[q]] = (double)v[q][rr];
        }
    }
}
template <typename T, bool TRANS, int G, int R, int KM, int NR>
__global__ void __launch_bounds__(256) k_bwd_lg(const SolveRec* __restrict__ list, int count, const T* __restrict__ fac,
                                                const int32_t* __restrict__ dofs, double* __restrict__ x, int64_t n_dof,
                                                int nrhs) {
    pdl_trigger();
    k_bwd_lg_body<T, TRANS, G, R, KM, NR>(list, count, fac, dofs, x, n_dof, nrhs, blockIdx.x);
}

// Tiny fronts (m <= G, G in {4, 8, 16, 32}): 32/G fronts per warp, one lane
// per row, shuffles of width G; all coefficients are loaded once, before the
// short sequential pivot loop.
template <typename T, bool TRANS, int G, int NR>
__device__ __forceinline__ void k_fwd_grp_body(const FrontDev* __restrict__ fronts, const SolveRec* __restrict__ list,
                                                 int count, const T* __restrict__ fac, const int32_t* __restrict__ dofs,
                                                 const int64_t* __restrict__ vsrc, T* __restrict__ vecs, int64_t vec_size,
                                                 double* __restrict__ x, int64_t n_dof, int nrhs, int vb, int scale = 0) {
    const int lane = threadIdx.x & 31;
    const int fidx = (vb * (blockDim.x >> 5) + (threadIdx.x >> 5)) * (32 / G) + lane / G;
    const bool active = fidx < count;
    const int i = lane % G;
    SolveRec fr{};
    int m = 0, k = 0;
    if (active) {
        fr = list[fidx];
        m = fr.m;
        k = fr.k;
    }
    const int32_t* fd = dofs + fr.dof_off;
    const T* P = fac + fr.P_off;
    const T* R = fac + fr.R_off;
    T c[G], dg[G];
#pragma unroll
    for (int p = 0; p < G; p++) {
        c[p] = (p < k && i > p && i < m) ? fcoef<T, TRANS>(P, R, m, k, i, p) : T(0);
        dg[p] = p < k ? fdiag<T, TRANS>(P, m, p) : T(1);
    }
    const RhsSrc src = (active && i < m) ? rhs_src<SolveRec>(fr, fd, vsrc, i) : RhsSrc{-1, -1, -1};
    const int kmax = (int)__reduce_max_sync(0xffffffffu, (unsigned)k);  // warp-uniform pivot count
    pdl_wait();
    for (int rb = 0; rb < nrhs; rb += NR) {
        const int nr = min(NR, nrhs - rb);
        T w[NR];
#pragma unroll
        for (int rr = 0; rr < NR; rr++)
            w[rr] = rr < nr ? rhs_val<T>(src, vecs + (int64_t)(rb + rr) * vec_size, x + (int64_t)(rb + rr) * n_dof) : T(0);
#pragma unroll
        for (int p = 0; p < G; p++) {
            if (p < kmax) {
                const T ds = pivot_scale<T, NR>(dg[p]);
#pragma unroll
                for (int rr = 0; rr < NR; rr++) {
                    const T yp = apply_pivot<T, NR>(__shfl_sync(0xffffffffu, w[rr], p, G), ds);
                    if (p < k) {
                        if (i == p) w[rr] = yp;
                        w[rr] -= c[p] * yp;
                    }
                }
            }
        }
        if (active && i < m) {
#pragma unroll
            for (int rr = 0; rr < NR; rr++) {
                if (rr >= nr) break;
                if (i < k) x[(int64_t)(rb + rr) * n_dof + src.xi] = pivot_out(w[rr], P, m, i, scale);
                else vecs[(int64_t)(rb + rr) * vec_size + fr.vec_off + (i - k)] = w[rr];
            }
        }
    }
}
template <typename T, bool TRANS, int G, int NR>
__global__ void __launch_bounds__(256) k_fwd_grp(const FrontDev* __restrict__ fronts, const SolveRec* __restrict__ list,
                                                 int count, const T* __restrict__ fac, const int32_t* __restrict__ dofs,
                                                 const int64_t* __restrict__ vsrc, T* __restrict__ vecs, int64_t vec_size,
                                                 double* __restrict__ x, int64_t n_dof, int nrhs, int scale) {
    pdl_trigger();
    k_fwd_grp_body<T, TRANS, G, NR>(fronts, list, count, fac, dofs, vsrc, vecs, vec_size, x, n_dof, nrhs, blockIdx.x, scale);
}

template <typename T, bool TRANS, int G, int NR>
__device__ __forceinline__ void k_bwd_grp_body(const FrontDev* __restrict__ fronts, const SolveRec* __restrict__ list,
                                                 int count, const T* __restrict__ fac, const int32_t* __restrict__ dofs,
                                                 double* __restrict__ x, int64_t n_dof, int nrhs, int vb) {
    const int lane = threadIdx.x & 31;
    const int fidx = (vb * (blockDim.x >> 5) + (threadIdx.x >> 5)) * (32 / G) + lane / G;
    const bool active = fidx < count;
    const int i = lane % G;
    SolveRec fr{};
    int m = 0, k = 0;
    if (active) {
        fr = list[fidx];
        m = fr.m;
        k = fr.k;
    }
    const int32_t* fd = dofs + fr.dof_off;
    const T* P = fac + fr.P_off;
    const T* R = fac + fr.R_off;
    T c[G], dg[G];
#pragma unroll
    for (int j = 0; j < G; j++) {
        c[j] = (j < m && i < k && i < j) ? bcoef<T, TRANS>(P, R, m, k, i, j) : T(0);
        dg[j] = j < k ? bdiag<T, TRANS>(P, m, j) : T(1);
    }
    const int di = (active && i < m) ? fd[i] : 0;
    const int mmax = (int)__reduce_max_sync(0xffffffffu, (unsigned)m);  // warp-uniform front size
    pdl_wait();
    for (int rb = 0; rb < nrhs; rb += NR) {
        const int nr = min(NR, nrhs - rb);
        T v[NR];
#pragma unroll
        for (int rr = 0; rr < NR; rr++) v[rr] = (rr < nr && active && i < m) ? (T)__ldcg(x + (int64_t)(rb + rr) * n_dof + di) : T(0);
#pragma unroll
        for (int j = G - 1; j >= 0; j--) {
            if (j >= mmax) continue;
            const T ds = pivot_scale<T, NR>(dg[j]);
#pragma unroll
            for (int rr = 0; rr < NR; rr++) {
                T xj = __shfl_sync(0xffffffffu, v[rr], j, G);
                if (j < k) {
                    xj = apply_pivot<T, NR>(xj, ds);
                    if (i == j) v[rr] = xj;
                }
                v[rr] -= c[j] * xj;
            }
        }
        if (active && i < k) {
#pragma unroll
            for (int rr = 0; rr < NR; rr++)
                if (rr < nr) x[(int64_t)(rb + rr) * n_dof + di] = (double)v[rr];
        }
    }
}
template <typename T, bool TRANS, int G, int NR>
__global__ void __launch_bounds__(256) k_bwd_grp(const FrontDev* __restrict__ fronts, const SolveRec* __restrict__ list,
                                                 int count, const T* __restrict__ fac, const int32_t* __restrict__ dofs,
                                                 double* __restrict__ x, int64_t n_dof, int nrhs) {
    pdl_trigger();
    k_bwd_grp_body<T, TRANS, G, NR>(fronts, list, count, fac, dofs, x, n_dof, nrhs, blockIdx.x);
}

// Mid-size fronts (m > 64, k < kInvMinK): one CTA per front.  The pivot block
// is processed in 32-wide blocks; each 32x32 diagonal block is staged in
// shared memory by all threads, solved by one warp per right-hand side, then
// applied to the later rows, including the contribution-block rows (update
// vector).  Shared memory: 32 x 33 T + kRhsChunk x ldw T (ldw >= m).
template <typename T, bool TRANS, int NR = kRhsChunk>
__device__ __forceinline__ void k_fwd_cta_body(const FrontDev* __restrict__ fronts, const SolveRec* __restrict__ list,
                                                 int rows_all, const T* __restrict__ fac, const int32_t* __restrict__ dofs,
                                                 const int64_t* __restrict__ vsrc, T* __restrict__ vecs, int64_t vec_size,
                                                 double* __restrict__ x, int64_t n_dof, int nrhs, int ldw, int vb, unsigned char* smem_raw,
                                                 int scale = 0) {
    __syncthreads();  // in a persistent sweep the previous body of this CTA may still be reading shared memory
    T* Dg = reinterpret_cast<T*>(smem_raw);  // 32 x 33
    T* w = Dg + 32 * 33;                     // kRhsChunk x ldw
    const SolveRec fr = list[vb];
    const int m = fr.m, k = fr.k;
    const int mr = rows_all ? m : k;
    const int32_t* fd = dofs + fr.dof_off;
    const T* P = fac + fr.P_off;
    const T* R = fac + fr.R_off;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    pdl_wait();
    for (int rb = 0; rb < nrhs; rb += NR) {
        const int nr = min(NR, nrhs - rb);
        for (int i = threadIdx.x; i < mr; i += blockDim.x) {
            const RhsSrc src = rhs_src<SolveRec>(fr, fd, vsrc, i);
            for (int rr = 0; rr < nr; rr++)
                w[rr * ldw + i] = rhs_val<T>(src, vecs + (int64_t)(rb + rr) * vec_size, x + (int64_t)(rb + rr) * n_dof);
        }
        for (int pb = 0; pb < k; pb += 32) {
            const int wb = min(32, k - pb);
            {
                T v[4];
#pragma unroll
                for (int q = 0; q < 4; q++) {
                    const int idx = threadIdx.x + 256 * q, i = idx & 31, p = idx >> 5;  // row pb+i, pivot pb+p
                    v[q] = T(0);
                    if (i < wb && p < wb) v[q] = (i > p) ? fcoef<T, TRANS>(P, R, m, k, pb + i, pb + p)
                                                         : (i == p ? fdiag<T, TRANS>(P, m, pb + p) : T(0));
                }
#pragma unroll
                for (int q = 0; q < 4; q++) {
                    const int idx = threadIdx.x + 256 * q;
                    Dg[(idx & 31) * 33 + (idx >> 5)] = v[q];
                }
            }
            __syncthreads();
            if (warp < nr) {  // warp rr solves right-hand side rr
                T* wr = w + warp * ldw;
                T val = lane < wb ? wr[pb + lane] : T(0);
                for (int p = 0; p < wb; p++) {
                    T yp = __shfl_sync(0xffffffffu, val, p) / Dg[p * 33 + p];
                    if (lane == p) val = yp;
                    if (lane > p) val -= Dg[lane * 33 + p] * yp;
                }
                if (lane < wb) wr[pb + lane] = val;
            }
            __syncthreads();
            for (int i = pb + wb + threadIdx.x; i < mr; i += blockDim.x) {
                T acc[NR];
#pragma unroll
                for (int rr = 0; rr < NR; rr++) acc[rr] = T(0);
                if constexpr (NR == 1) {
                    // one right-hand side: 16 coefficients of the row loaded before their products
                    // (unconditional loads; columns past the block repeat its last one, weighted 0)
                    for (int p0 = 0; p0 < wb; p0 += 16) {
                        T cf[16];
#pragma unroll
                        for (int p = 0; p < 16; p++) cf[p] = fcoef<T, TRANS>(P, R, m, k, i, pb + min(p0 + p, wb - 1));
#pragma unroll
                        for (int p = 0; p < 16; p++) {
                            const T on = p0 + p < wb ? T(1) : T(0);
                            acc[0] += (on * cf[p]) * w[pb + min(p0 + p, wb - 1)];
                        }
                    }
                } else {
#pragma unroll 4
                    for (int p = 0; p < wb; p++) {
                        const T cf = fcoef<T, TRANS>(P, R, m, k, i, pb + p);
#pragma unroll
                        for (int rr = 0; rr < NR; rr++)
                            if (rr < nr) acc[rr] += cf * w[rr * ldw + pb + p];
                    }
                }
#pragma unroll
                for (int rr = 0; rr < NR; rr++)
                    if (rr < nr) w[rr * ldw + i] -= acc[rr];
            }
            __syncthreads();
        }
        for (int i = threadIdx.x; i < mr; i += blockDim.x)
            for (int rr = 0; rr < nr; rr++) {
                if (i < k) x[(int64_t)(rb + rr) * n_dof + fd[i]] = pivot_out(w[rr * ldw + i], P, m, i, scale);
                else vecs[(int64_t)(rb + rr) * vec_size + fr.vec_off + (i - k)] = w[rr * ldw + i];
            }
        __syncthreads();
    }
}
template <typename T, bool TRANS, int NR>
__global__ void __launch_bounds__(256) k_fwd_cta(const FrontDev* __restrict__ fronts, const SolveRec* __restrict__ list,
                                                 int rows_all, const T* __restrict__ fac, const int32_t* __restrict__ dofs,
                                                 const int64_t* __restrict__ vsrc, T* __restrict__ vecs, int64_t vec_size,
                                                 double* __restrict__ x, int64_t n_dof, int nrhs, int ldw, int scale) {
    extern __shared__ __align__(16) unsigned char smem_dyn[];
    pdl_trigger();
    k_fwd_cta_body<T, TRANS, NR>(fronts, list, rows_all, fac, dofs, vsrc, vecs, vec_size, x, n_dof, nrhs, ldw, blockIdx.x, smem_dyn,
                                 scale);
}

// Backward, one CTA per mid-size front: the CB part of the pivot rows first,
// then the unit (or, transposed, L11^T) triangle in 32-wide blocks.
// Shared memory: 32 x 33 T + 8 x 64 x kRhsChunk T + kRhsChunk x ldw T.
template <typename T, bool TRANS, int NR = kRhsChunk>
__device__ __forceinline__ void k_bwd_cta_body(const FrontDev* __restrict__ fronts, const SolveRec* __restrict__ list,
                                                 int cb_done, const T* __restrict__ fac, const int32_t* __restrict__ dofs,
                                                 double* __restrict__ x, int64_t n_dof, int nrhs, int ldw, int vb, unsigned char* smem_raw) {
    __syncthreads();  // in a persistent sweep the previous body of this CTA may still be reading shared memory
    T* Dg = reinterpret_cast<T*>(smem_raw);
    T* red = Dg + 32 * 33;                // 8 warps x 64 rows x kRhsChunk
    T* v = red + 8 * 64 * kRhsChunk;      // kRhsChunk x ldw
    const SolveRec fr = list[vb];
    const int m = fr.m, k = fr.k;
    const int32_t* fd = dofs + fr.dof_off;
    const T* P = fac + fr.P_off;
    const T* R = fac + fr.R_off;
    const int mv = cb_done ? k : m;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    pdl_wait();
    for (int rb = 0; rb < nrhs; rb += NR) {
        const int nr = min(NR, nrhs - rb);
        for (int i = threadIdx.x; i < mv; i += blockDim.x) {
            const int d = fd[i];
            for (int rr = 0; rr < nr; rr++) v[rr * ldw + i] = (T)__ldcg(x + (int64_t)(rb + rr) * n_dof + d);
        }
        __syncthreads();
        if (!cb_done && TRANS) {
            // L^T: pivot row i is column i of L below the pivot block, contiguous in P: one warp per
            // pivot row, lanes along the column (coalesced), a shuffle tree per row
            for (int i = warp; i < k; i += 8) {
                const T* col = P + (int64_t)i * m;
                T acc[NR];
#pragma unroll
                for (int rr = 0; rr < NR; rr++) acc[rr] = T(0);
                int j = k + lane;
                for (; j + 32 * 11 < m; j += 32 * 12) {  // 12 loads in flight per lane
                    T c[12];
#pragma unroll
                    for (int u = 0; u < 12; u++) c[u] = col[j + 32 * u];
#pragma unroll
                    for (int u = 0; u < 12; u++)
#pragma unroll
                        for (int rr = 0; rr < NR; rr++)
                            if (rr < nr) acc[rr] += c[u] * v[rr * ldw + j + 32 * u];
                }
                {  // the remaining < 12 column chunks, guarded, all loads first
                    T c[12];
#pragma unroll
                    for (int u = 0; u < 12; u++) c[u] = j + 32 * u < m ? col[j + 32 * u] : T(0);
#pragma unroll
                    for (int u = 0; u < 12; u++)
                        if (j + 32 * u < m) {
#pragma unroll
                            for (int rr = 0; rr < NR; rr++)
                                if (rr < nr) acc[rr] += c[u] * v[rr * ldw + j + 32 * u];
                        }
                }
#pragma unroll
                for (int rr = 0; rr < NR; rr++) {
                    T sum = acc[rr];
                    for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
                    if (lane == 0 && rr < nr) v[rr * ldw + i] -= sum;
                }
            }
            __syncthreads();
        } else if (!cb_done) {
            // pivot rows (lane, lane + 32; k < 64) minus their CB part; the 8 warps split the columns
            const int i0 = lane, i1 = lane + 32;
            T a0[NR], a1[NR];
#pragma unroll
            for (int rr = 0; rr < NR; rr++) a0[rr] = a1[rr] = T(0);
#pragma unroll 8
            for (int j = k + warp; j < m; j += 8) {
                const T c0 = i0 < k ? bcoef<T, TRANS>(P, R, m, k, i0, j) : T(0);
                const T c1 = i1 < k ? bcoef<T, TRANS>(P, R, m, k, i1, j) : T(0);
#pragma unroll
                for (int rr = 0; rr < NR; rr++) {
                    if (rr < nr) {
                        const T xj = v[rr * ldw + j];
                        a0[rr] += c0 * xj;
                        a1[rr] += c1 * xj;
                    }
                }
            }
#pragma unroll
            for (int rr = 0; rr < NR; rr++) {
                red[(rr * 8 + warp) * 64 + i0] = a0[rr];
                red[(rr * 8 + warp) * 64 + i1] = a1[rr];
            }
            __syncthreads();
            for (int i = threadIdx.x; i < k; i += blockDim.x)
                for (int rr = 0; rr < nr; rr++) {
                    T acc = T(0);
                    for (int w = 0; w < 8; w++) acc += red[(rr * 8 + w) * 64 + i];
                    v[rr * ldw + i] -= acc;
                }
            __syncthreads();
        }
        for (int pe = k; pe > 0; pe -= 32) {
            const int pb = max(0, pe - 32), wb = pe - pb;
            {
                T t[4];
                // row pb+i, unknown pb+j; the index that runs along memory is the fast one across the
                // lanes (i for U, j for L^T, whose coefficient of j in row i is L[j][i])
#pragma unroll
                for (int q = 0; q < 4; q++) {
                    const int idx = threadIdx.x + 256 * q;
                    const int i = TRANS ? idx >> 5 : idx & 31, j = TRANS ? idx & 31 : idx >> 5;
                    t[q] = T(0);
                    if (i < wb && j < wb) t[q] = (i < j) ? bcoef<T, TRANS>(P, R, m, k, pb + i, pb + j)
                                                         : (i == j ? bdiag<T, TRANS>(P, m, pb + j) : T(0));
                }
#pragma unroll
                for (int q = 0; q < 4; q++) {
                    const int idx = threadIdx.x + 256 * q;
                    const int i = TRANS ? idx >> 5 : idx & 31, j = TRANS ? idx & 31 : idx >> 5;
                    Dg[i * 33 + j] = t[q];
                }
            }
            __syncthreads();
            if (warp < nr) {
                T* vr = v + warp * ldw;
                T val = lane < wb ? vr[pb + lane] : T(0);
                for (int j = wb - 1; j >= 0; j--) {
                    T xj = __shfl_sync(0xffffffffu, val, j) / Dg[j * 33 + j];
                    if (lane == j) val = xj;
                    if (lane < j) val -= Dg[lane * 33 + j] * xj;
                }
                if (lane < wb) vr[pb + lane] = val;
            }
            __syncthreads();
            if (TRANS) {  // rows above the block: warp per row, lane = unknown (contiguous in L's column)
                for (int i = warp; i < pb; i += 8) {
                    const T cf = lane < wb ? bcoef<T, TRANS>(P, R, m, k, i, pb + lane) : T(0);
#pragma unroll
                    for (int rr = 0; rr < NR; rr++) {
                        T sum = rr < nr ? cf * v[rr * ldw + pb + min(lane, wb - 1)] : T(0);
                        for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
                        if (lane == 0 && rr < nr) v[rr * ldw + i] -= sum;
                    }
                }
            }
            for (int i = threadIdx.x; i < pb && !TRANS; i += blockDim.x) {
                T acc[NR];
#pragma unroll
                for (int rr = 0; rr < NR; rr++) acc[rr] = T(0);
#pragma unroll 4
                for (int j = 0; j < wb; j++) {
                    const T cf = bcoef<T, TRANS>(P, R, m, k, i, pb + j);
#pragma unroll
                    for (int rr = 0; rr < NR; rr++)
                        if (rr < nr) acc[rr] += cf * v[rr * ldw + pb + j];
                }
#pragma unroll
                for (int rr = 0; rr < NR; rr++)
                    if (rr < nr) v[rr * ldw + i] -= acc[rr];
            }
            __syncthreads();
        }
        for (int i = threadIdx.x; i < k; i += blockDim.x) {
            const int d = fd[i];
            for (int rr = 0; rr < nr; rr++) x[(int64_t)(rb + rr) * n_dof + d] = (double)v[rr * ldw + i];
        }
        __syncthreads();
    }
}
template <typename T, bool TRANS, int NR>
__global__ void __launch_bounds__(256) k_bwd_cta(const FrontDev* __restrict__ fronts, const SolveRec* __restrict__ list,
                                                 int cb_done, const T* __restrict__ fac, const int32_t* __restrict__ dofs,
                                                 double* __restrict__ x, int64_t n_dof, int nrhs, int ldw) {
    extern __shared__ __align__(16) unsigned char smem_dyn[];
    pdl_trigger();
    k_bwd_cta_body<T, TRANS, NR>(fronts, list, cb_done, fac, dofs, x, n_dof, nrhs, ldw, blockIdx.x, smem_dyn);
}

// ---------------------------------------------------------------------------
// Fronts with explicit pivot-block inverses (k >= kInvMinK): each sweep is
// two wide products per front, 32 rows per CTA.
//   FWD1: y = L11^-1 w1            (TRANS: U11^-T w1)      -> pivot scratch
//   FWD2: rows < k: y -> x at the pivots; rows >= k: u = w2 - L21 y (TRANS: U12^T y)
//   BWD1: z = y - U12 x_CB         (TRANS: L21^T x_CB)     -> pivot scratch
//   BWD2: x1 = U11^-1 z            (TRANS: L11^-T z)       -> x at the pivots
// !TRANS operands are read column by column (lane = row, the 8 warps split the
// columns, partial sums added in warp order); TRANS operands row by row
// (warp = row, lanes split the columns, shuffle tree).  Both orders are fixed,
// so results are deterministic.
enum { PH_FWD1 = 0, PH_FWD2 = 1, PH_BWD1 = 2, PH_BWD2 = 3 };

struct RowBlock {
    int32_t front, r0, r1, pad;
};

template <typename T, bool TRANS, int PH>
__device__ __forceinline__ T inv_coef(const T* __restrict__ P, const T* __restrict__ R, const T* __restrict__ Q, int m,
                                      int k, int i, int j) {
    if (PH == PH_FWD1) return TRANS ? (j == i ? T(1) : Q[j + (int64_t)i * k]) : Q[i + (int64_t)j * k];
    if (PH == PH_FWD2) return TRANS ? R[j + (int64_t)(i - k) * k] : P[i + (int64_t)j * m];
    if (PH == PH_BWD1) return TRANS ? P[(k + j) + (int64_t)i * m] : R[i + (int64_t)j * k];
    return TRANS ? Q[j + (int64_t)i * k] : (j == i ? T(1) : Q[i + (int64_t)j * k]);
}

template <typename T, bool TRANS, int PH, int NW>
__device__ __forceinline__ void k_inv_gemv_body(const FrontDev* __restrict__ fronts, const RowBlock* __restrict__ tasks,
                                                  const T* __restrict__ fac, const T* __restrict__ inv,
                                                  const int32_t* __restrict__ dofs, const int64_t* __restrict__ vsrc,
                                                  T* __restrict__ vecs, int64_t vec_size, T* __restrict__ ys,
                                                  int64_t ys_size, double* __restrict__ x, int64_t n_dof, int vb, unsigned char* smem_raw, int rr,
                                                  int scale = 0) {
    __syncthreads();  // in a persistent sweep the previous body of this CTA may still be reading shared memory
    T* red = reinterpret_cast<T*>(smem_raw);  // NW x 32
    T* vin = red + NW * 32;
    const RowBlock t = tasks[vb];
    const int r = rr;
    const FrontDev fr = fronts[t.front];
    const int m = fr.m, k = fr.k;
    const int32_t* fd = dofs + fr.dof_off;
    double* xr = x + (int64_t)r * n_dof;
    T* vr = vecs + (int64_t)r * vec_size;
    T* yr = ys + (int64_t)r * ys_size + fr.y_off;
    const T* P = fac + fr.P_off;
    const T* R = fac + fr.R_off;
    const T* Q = inv + (fr.q_off >= 0 ? fr.q_off : 0);
    if (PH == PH_FWD2 && t.r0 < k) {
        pdl_wait();
        for (int i = t.r0 + threadIdx.x; i < t.r1; i += blockDim.x) xr[fd[i]] = pivot_out(__ldcg(yr + i), P, m, i, scale);
        return;
    }
    const int nin = (PH == PH_BWD1) ? m - k : k;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    // column range of row i
    auto lo = [&](int i) { return PH == PH_BWD2 ? i : 0; };
    auto hi = [&](int i) { return PH == PH_FWD1 ? i + 1 : nin; };
    // The first chunk of each row's coefficients is loaded before the wait for the previous
    // kernel; the operand of the row's final update (its right-hand-side entry, or the dof it is
    // written to) before the inputs are staged.
    constexpr int RW = TRANS ? (32 + NW - 1) / NW : 1;  // rows per warp (TRANS) / per lane (!TRANS)
    constexpr int PC = 8;  // coefficients per row issued early (before the wait for the previous kernel)
    T pre[RW][PC];
    T rhs[RW];
    int xi[RW];
    // !TRANS: full columns for every row of the block: FWD1 [0, r0); BWD2 [r1, k); else [0, nin)
    const int f0 = PH == PH_BWD2 ? t.r1 : 0;
    const int f1 = PH == PH_FWD1 ? t.r0 : nin;
#pragma unroll
    for (int q = 0; q < RW; q++) {
        const int i = TRANS ? t.r0 + warp + NW * q : t.r0 + lane;
        const bool valid = i < t.r1;
        rhs[q] = T(0);
        xi[q] = 0;
#pragma unroll
        for (int u = 0; u < PC; u++) {
            if (!TRANS) {
                const int j = f0 + warp + NW * u;
                pre[q][u] = (valid && j < f1) ? inv_coef<T, TRANS, PH>(P, R, Q, m, k, i, j) : T(0);
            } else {
                const int j = (valid ? lo(i) : 0) + lane + 32 * u;
                pre[q][u] = (valid && j < hi(i)) ? inv_coef<T, TRANS, PH>(P, R, Q, m, k, i, j) : T(0);
            }
        }
    }
    pdl_wait();
#pragma unroll
    for (int q = 0; q < RW; q++) {
        const int i = TRANS ? t.r0 + warp + NW * q : t.r0 + lane;
        if (i < t.r1 && (TRANS ? lane == 0 : warp == 0)) {
            if (PH == PH_FWD2) rhs[q] = gather_rhs<T, FrontDev>(fr, fd, vsrc, vr, xr, i);
            else if (PH == PH_BWD1) rhs[q] = (T)__ldcg(xr + fd[i]);
            else if (PH == PH_BWD2) xi[q] = fd[i];
        }
    }
    for (int j = threadIdx.x; j < nin; j += blockDim.x) {
        T v;
        if (PH == PH_FWD1) v = gather_rhs<T, FrontDev>(fr, fd, vsrc, vr, xr, j);
        else if (PH == PH_BWD1) v = (T)__ldcg(xr + fd[k + j]);
        else v = __ldcg(yr + j);
        vin[j] = v;
    }
    __syncthreads();
    auto finish = [&](int i, int q, T acc) {
        if (PH == PH_FWD1) yr[i] = acc;
        else if (PH == PH_FWD2) vr[fr.vec_off + (i - k)] = rhs[q] - acc;
        else if (PH == PH_BWD1) yr[i] = rhs[q] - acc;
        else xr[xi[q]] = (double)acc;
    };
    if (!TRANS) {
        // lane = row, the NW warps split the columns; the rectangle part of the
        // column range needs no per-element test, only the triangle edge does
        const int i = t.r0 + lane;
        const bool valid = i < t.r1;
        T acc[8];
#pragma unroll
        for (int u = 0; u < 8; u++) acc[u] = T(0);
        if (valid) {
#pragma unroll
            for (int u = 0; u < PC; u++) {
                const int j = f0 + warp + NW * u;
                if (j < f1) acc[u] += pre[0][u] * vin[j];
            }
            int j = f0 + warp + NW * PC;
            for (; j + 7 * NW < f1; j += 8 * NW) {
#pragma unroll
                for (int u = 0; u < 8; u++) acc[u] += inv_coef<T, TRANS, PH>(P, R, Q, m, k, i, j + NW * u) * vin[j + NW * u];
            }
            for (; j < f1; j += NW) acc[0] += inv_coef<T, TRANS, PH>(P, R, Q, m, k, i, j) * vin[j];
            // triangle edge: columns of the block's own diagonal band
            if (PH == PH_FWD1 || PH == PH_BWD2) {
                for (int jj = t.r0 + warp; jj < t.r1; jj += NW)
                    if (jj >= lo(i) && jj < hi(i)) acc[1] += inv_coef<T, TRANS, PH>(P, R, Q, m, k, i, jj) * vin[jj];
            }
        }
        red[warp * 32 + lane] = ((acc[0] + acc[1]) + (acc[2] + acc[3])) + ((acc[4] + acc[5]) + (acc[6] + acc[7]));
        __syncthreads();
        if (warp == 0 && valid) {
            T sum = T(0);
            for (int w = 0; w < NW; w++) sum += red[w * 32 + lane];
            finish(i, 0, sum);
        }
    } else {
#pragma unroll
        for (int q = 0; q < RW; q++) {  // one row per warp at a time
            const int i = t.r0 + warp + NW * q;
            if (i >= t.r1) break;
            T acc[8];
#pragma unroll
            for (int u = 0; u < 8; u++) acc[u] = T(0);
            const int jl = lo(i), jh = hi(i);
#pragma unroll
            for (int u = 0; u < PC; u++) {
                const int j = jl + lane + 32 * u;
                if (j < jh) acc[u] += pre[q][u] * vin[j];
            }
            int j = jl + lane + 32 * PC;
            for (; j + 224 < jh; j += 256) {
#pragma unroll
                for (int u = 0; u < 8; u++) acc[u] += inv_coef<T, TRANS, PH>(P, R, Q, m, k, i, j + 32 * u) * vin[j + 32 * u];
            }
            for (; j < jh; j += 32) acc[0] += inv_coef<T, TRANS, PH>(P, R, Q, m, k, i, j) * vin[j];
            T sum = ((acc[0] + acc[1]) + (acc[2] + acc[3])) + ((acc[4] + acc[5]) + (acc[6] + acc[7]));
            for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
            if (lane == 0) finish(i, q, sum);
        }
    }
}
template <typename T, bool TRANS, int PH, int NW>
__global__ void __launch_bounds__(NW * 32) k_inv_gemv(const FrontDev* __restrict__ fronts, const RowBlock* __restrict__ tasks,
                                                  const T* __restrict__ fac, const T* __restrict__ inv,
                                                  const int32_t* __restrict__ dofs, const int64_t* __restrict__ vsrc,
                                                  T* __restrict__ vecs, int64_t vec_size, T* __restrict__ ys,
                                                  int64_t ys_size, double* __restrict__ x, int64_t n_dof, int scale) {
    extern __shared__ __align__(16) unsigned char smem_dyn[];
    pdl_trigger();
    k_inv_gemv_body<T, TRANS, PH, NW>(fronts, tasks, fac, inv, dofs, vsrc, vecs, vec_size, ys, ys_size, x, n_dof, blockIdx.x, smem_dyn, blockIdx.y,
                                      scale);
}

// ---------------------------------------------------------------------------
// Persistent substitution sweep: one cooperative launch walks every class of
// the forward (or backward) sweep.  A phase is one kernel type of one class
// over its task list; the CTAs take its virtual blocks as a bag of tasks
// (vb = blockIdx.x, +gridDim.x, ...) and run the same bodies as the per-class
// kernels.  Phases of one class touch disjoint fronts; a grid barrier
// separates dependent phases (class c+1 after class c; the second inverse
// product after the first).  The barrier is bounded: after 1 s of waiting
// a CTA records a timeout and the whole sweep returns.  Data written by
// other CTAs earlier in the sweep (x, update vectors, pivot scratch) is
// read through L2 (__ldcg) by the bodies.
enum { SW_GRP4 = 0, SW_GRP8, SW_GRP16, SW_GRP32, SW_WARP, SW_CTA, SW_INV1, SW_INV2 };

struct SweepPhase {
    int32_t kind;     // SW_*
    int32_t count;    // virtual blocks
    int64_t off;      // offset into the substitution list (fronts) or the row blocks (inverse products)
    int32_t n;        // fronts in the list (lane-group and warp kinds)
    int32_t ldw;      // CTA kind: leading dimension of the per-rhs vectors in shared memory
    int32_t barrier;  // nonzero: grid barrier after this phase
    int32_t pad;
};

template <typename T>
struct SweepArgs {
    const FrontDev* fronts;
    const SolveRec* list;
    const RowBlock* rows;
    const T* fac;
    const T* inv;
    const int32_t* dofs;
    const int64_t* vsrc;
    T* vecs;
    int64_t vec_size;
    T* ys;
    int64_t ys_size;
    double* x;
    int64_t n_dof;
    int nrhs;
    const SweepPhase* phases;
    int n_phases;
    unsigned int* bar;  // [0] arrivals, [1] generation
    DevStatus* st;
};

__device__ __forceinline__ uint64_t sweep_clock_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Grid-wide barrier for a cooperative launch (all CTAs resident), bounded.
__device__ __forceinline__ bool sweep_barrier(unsigned int* bar, unsigned int nblocks, DevStatus* st,
                                              unsigned long long limit_ns = 1000000000ull) {
    __shared__ int ok_s;
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        volatile unsigned int* gen = bar + 1;
        const unsigned int g = *gen;
        __threadfence();
        const unsigned int arrived = atomicAdd(bar, 1u) + 1u;
        if (arrived == nblocks) {
            atomicExch(bar, 0u);
            __threadfence();
            atomicAdd(bar + 1, 1u);
        } else {
            const uint64_t t0 = sweep_clock_ns();
            while (*gen == g) {
                if (sweep_clock_ns() - t0 > limit_ns) {
                    ok = 0;
                    atomicOr(&st->timeout, 1);
                    break;
                }
                __nanosleep(64);
            }
        }
        __threadfence();
        ok_s = ok;
    }
    __syncthreads();
    return ok_s != 0;
}

template <typename T, bool TRANS, bool FWD, int NR>
__global__ void __launch_bounds__(256) k_solve_sweep(SweepArgs<T> a) {
    extern __shared__ __align__(16) unsigned char smem_dyn[];
    for (int ph = 0; ph < a.n_phases; ph++) {
        const SweepPhase P = a.phases[ph];
        const SolveRec* L = a.list + P.off;
        for (int vb = blockIdx.x; vb < P.count; vb += gridDim.x) {
            switch (P.kind) {
#define SWEEP_GRP(K, GS)                                                                                              \
    case K:                                                                                                           \
        if (FWD)                                                                                                      \
            k_fwd_grp_body<T, TRANS, GS, NR>(a.fronts, L, P.n, a.fac, a.dofs, a.vsrc, a.vecs, a.vec_size, a.x, a.n_dof, \
                                             a.nrhs, vb);                                                             \
        else                                                                                                          \
            k_bwd_grp_body<T, TRANS, GS, NR>(a.fronts, L, P.n, a.fac, a.dofs, a.x, a.n_dof, a.nrhs, vb);             \
        break;
                SWEEP_GRP(SW_GRP4, 4)
                SWEEP_GRP(SW_GRP8, 8)
                SWEEP_GRP(SW_GRP16, 16)
                SWEEP_GRP(SW_GRP32, 32)
#undef SWEEP_GRP
                case SW_WARP:
                    if (FWD)
                        k_fwd_warp_body<T, TRANS, NR>(a.fronts, L, P.n, a.fac, a.dofs, a.vsrc, a.vecs, a.vec_size, a.x, a.n_dof,
                                                      a.nrhs, vb);
                    else
                        k_bwd_warp_body<T, TRANS, NR>(a.fronts, L, P.n, a.fac, a.dofs, a.x, a.n_dof, a.nrhs, vb);
                    break;
                case SW_CTA:
                    if (FWD)
                        k_fwd_cta_body<T, TRANS, NR>(a.fronts, L, 1, a.fac, a.dofs, a.vsrc, a.vecs, a.vec_size, a.x, a.n_dof, a.nrhs,
                                                 P.ldw, vb, smem_dyn);
                    else
                        k_bwd_cta_body<T, TRANS, NR>(a.fronts, L, 0, a.fac, a.dofs, a.x, a.n_dof, a.nrhs, P.ldw, vb, smem_dyn);
                    break;
                case SW_INV1:
                    for (int r = 0; r < a.nrhs; r++)
                        k_inv_gemv_body<T, TRANS, FWD ? PH_FWD1 : PH_BWD1, 8>(a.fronts, a.rows + P.off, a.fac, a.inv, a.dofs,
                                                                              a.vsrc, a.vecs, a.vec_size, a.ys, a.ys_size,
                                                                              a.x, a.n_dof, vb, smem_dyn, r);
                    break;
                case SW_INV2:
                    for (int r = 0; r < a.nrhs; r++)
                        k_inv_gemv_body<T, TRANS, FWD ? PH_FWD2 : PH_BWD2, 8>(a.fronts, a.rows + P.off, a.fac, a.inv, a.dofs,
                                                                              a.vsrc, a.vecs, a.vec_size, a.ys, a.ys_size,
                                                                              a.x, a.n_dof, vb, smem_dyn, r);
                    break;
            }
        }
        if (P.barrier && !sweep_barrier(a.bar, gridDim.x, a.st)) return;
    }
}

// ---------------------------------------------------------------------------
// FP64 residual, element by element, deterministic:
//   Y[e*npe + a] = sum_b K_e[a,b] x[node(e,b)]          (k_elem_apply)
//   r[d] = b[d] - sum over the (e,a) touching d of Y    (k_gather_residual)
// absmode: |K_e| and x = 1, giving the element-wise bound of ||A||_inf rows.
// trans: the element matrices enter transposed (K_e^T x_e; absmode: column sums), for A^T x.
__global__ void k_elem_apply(const double* __restrict__ values, const int64_t* __restrict__ en, const double* __restrict__ x,
                             double* __restrict__ Y, int64_t n_elem, int npe, int64_t n_dof, int absmode, int trans) {
    const int64_t nE = n_elem * npe;
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int r = blockIdx.y;
    if (idx >= nE) return;
    const int64_t e = idx / npe;
    const int a = (int)(idx - e * npe);
    const double* K = values + e * npe * npe + (trans ? (int64_t)a * npe : a);
    const int ks = trans ? 1 : npe;  // stride between the entries of the lane's row of K_e (or of K_e^T)
    const int64_t* nd = en + e * npe;
    const double* xr = x + (int64_t)r * n_dof;
    double acc = 0.0;
    if (absmode) {
        for (int b = 0; b < npe; b++) acc += fabs(K[b * ks]);
    } else {
        for (int b = 0; b < npe; b++) acc = fma(K[b * ks], xr[nd[b]], acc);
    }
    Y[idx + (int64_t)r * nE] = acc;
}

// Same product with one lane group of G >= npe lanes per element: each lane
// loads its node's x once and the group shares them by shuffles.
template <int G, bool TR>
__global__ void __launch_bounds__(256) k_elem_apply_grp(const double* __restrict__ values, const int64_t* __restrict__ en,
                                                        const double* __restrict__ x, double* __restrict__ Y, int64_t n_elem,
                                                        int npe, int64_t n_dof) {
    const int lane = threadIdx.x & 31;
    const int64_t e = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / G;
    const int a = lane % G;
    const int r = blockIdx.y;
    const bool act = e < n_elem && a < npe;
    const double* xr = x + (int64_t)r * n_dof;
    const double xa = act ? xr[en[e * npe + a]] : 0.0;
    const double* K = values + (act ? e : 0) * npe * npe + (TR ? a * npe : a);
    // all npe loads of the lane's row of K_e (TR: of K_e^T) issued before the products (npe <= G)
    double kv[G];
#pragma unroll
    for (int b = 0; b < G; b++) kv[b] = (act && b < npe) ? K[TR ? b : b * npe] : 0.0;
    double acc = 0.0;
#pragma unroll
    for (int b = 0; b < G; b++) {
        const double xb = __shfl_sync(0xffffffffu, xa, b, G);
        if (b < npe) acc = fma(kv[b], xb, acc);
    }
    if (act) Y[e * npe + a + (int64_t)r * n_elem * npe] = acc;
}

__global__ void k_gather_residual(const int64_t* __restrict__ node_ptr, const int64_t* __restrict__ node_inc,
                                  const double* __restrict__ Y, const double* __restrict__ b, double* __restrict__ out,
                                  int64_t n_dof, int64_t nE, int mode) {
    const int64_t d = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int r = blockIdx.y;
    if (d >= n_dof) return;
    double acc = 0.0;
    for (int64_t t = node_ptr[d]; t < node_ptr[d + 1]; t++) acc += Y[node_inc[t] + (int64_t)r * nE];
    // mode 0: out = b - A x ; mode 1: out = A x (b unused)
    out[d + (int64_t)r * n_dof] = mode == 0 ? b[d + (int64_t)r * n_dof] - acc : acc;
}

// The maxima of |r|, |x|, |b| and of the row sums are taken on the bit patterns: with the sign
// bit cleared, IEEE doubles order like unsigned integers, and a NaN (exponent all ones, mantissa
// nonzero) lies above every number, so the maximum keeps it (an FP64 max would drop it, and FP64
// compares would run on the GPU's small FP64 pipe).
__device__ __forceinline__ unsigned long long abs_bits(double v) {
    return (unsigned long long)__double_as_longlong(v) & 0x7fffffffffffffffull;
}
__device__ __forceinline__ double bits_double(unsigned long long u) { return __longlong_as_double((long long)u); }

// Per right-hand side norms: out[r*6 + {0..5}] = ||r||_inf, ||x||_inf, ||b||_inf,
// ||r||_2^2, ||b||_2^2, ||Arow||_inf (the last one only for r == 0, from rowabs).
// Two stages for a deterministic sum: block partials, then one block.  Each thread loads all of
// its elements (kNormsPer per array, strided by the grid) before it reduces them.
constexpr int kNormsPer = 8;
__global__ void __launch_bounds__(256) k_norms_partial(const double* __restrict__ rv, const double* __restrict__ xv,
                                                       const double* __restrict__ bv, const double* __restrict__ rowabs,
                                                       int64_t n, double* __restrict__ part) {
    const int r = blockIdx.y;
    const double* rr = rv + (int64_t)r * n;
    const double* xx = xv + (int64_t)r * n;
    const double* bb = bv + (int64_t)r * n;
    unsigned long long m0 = 0, m1 = 0, m2 = 0, m5 = 0;
    double a3 = 0, a4 = 0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; base < n; base += kNormsPer * stride) {
        double rq[kNormsPer], xq[kNormsPer], bq[kNormsPer], aq[kNormsPer];
#pragma unroll
        for (int u = 0; u < kNormsPer; u++) {
            const int64_t i = base + u * stride;
            const bool ok = i < n;
            rq[u] = ok ? rr[i] : 0.0;
            xq[u] = ok ? xx[i] : 0.0;
            bq[u] = ok ? bb[i] : 0.0;
            aq[u] = (ok && rowabs) ? rowabs[i] : 0.0;
        }
#pragma unroll
        for (int u = 0; u < kNormsPer; u++) {
            m0 = max(m0, abs_bits(rq[u]));
            m1 = max(m1, abs_bits(xq[u]));
            m2 = max(m2, abs_bits(bq[u]));
            m5 = max(m5, abs_bits(aq[u]));
            a3 = fma(rq[u], rq[u], a3);
            a4 = fma(bq[u], bq[u], a4);
        }
    }
    __shared__ unsigned long long shm[4][8];
    __shared__ double shs[2][8];
    for (int o = 16; o > 0; o >>= 1) {
        m0 = max(m0, __shfl_xor_sync(0xffffffffu, m0, o));
        m1 = max(m1, __shfl_xor_sync(0xffffffffu, m1, o));
        m2 = max(m2, __shfl_xor_sync(0xffffffffu, m2, o));
        m5 = max(m5, __shfl_xor_sync(0xffffffffu, m5, o));
        a3 += __shfl_xor_sync(0xffffffffu, a3, o);
        a4 += __shfl_xor_sync(0xffffffffu, a4, o);
    }
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) {
        shm[0][w] = m0; shm[1][w] = m1; shm[2][w] = m2; shm[3][w] = m5;
        shs[0][w] = a3; shs[1][w] = a4;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long o0 = 0, o1 = 0, o2 = 0, o5 = 0;
        double o3 = 0, o4 = 0;
        for (int i = 0; i < (int)(blockDim.x >> 5); i++) {
            o0 = max(o0, shm[0][i]); o1 = max(o1, shm[1][i]); o2 = max(o2, shm[2][i]); o5 = max(o5, shm[3][i]);
            o3 += shs[0][i]; o4 += shs[1][i];
        }
        double* q = part + ((int64_t)r * gridDim.x + blockIdx.x) * 6;
        q[0] = bits_double(o0); q[1] = bits_double(o1); q[2] = bits_double(o2);
        q[3] = o3; q[4] = o4; q[5] = bits_double(o5);
    }
}

// one block of 256 threads per right-hand side: every partial of a thread loaded first, then a
// fixed-order reduction (strided per thread, a shuffle tree per warp, the warps in order)
__global__ void __launch_bounds__(256) k_norms_final(const double* __restrict__ part, int nblk, double* __restrict__ out) {
    const int r = blockIdx.x, lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    unsigned long long m0 = 0, m1 = 0, m2 = 0, m5 = 0;
    double o3 = 0, o4 = 0;
    for (int i0 = threadIdx.x; i0 < nblk; i0 += 4 * blockDim.x) {
        double v[4][6];
#pragma unroll
        for (int u = 0; u < 4; u++) {
            const int i = i0 + u * blockDim.x;
#pragma unroll
            for (int c = 0; c < 6; c++) v[u][c] = i < nblk ? part[((int64_t)r * nblk + i) * 6 + c] : 0.0;
        }
#pragma unroll
        for (int u = 0; u < 4; u++) {
            m0 = max(m0, abs_bits(v[u][0])); m1 = max(m1, abs_bits(v[u][1])); m2 = max(m2, abs_bits(v[u][2]));
            m5 = max(m5, abs_bits(v[u][5]));
            o3 += v[u][3]; o4 += v[u][4];
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        m0 = max(m0, __shfl_xor_sync(0xffffffffu, m0, o));
        m1 = max(m1, __shfl_xor_sync(0xffffffffu, m1, o));
        m2 = max(m2, __shfl_xor_sync(0xffffffffu, m2, o));
        m5 = max(m5, __shfl_xor_sync(0xffffffffu, m5, o));
        o3 += __shfl_xor_sync(0xffffffffu, o3, o);
        o4 += __shfl_xor_sync(0xffffffffu, o4, o);
    }
    __shared__ unsigned long long shm[4][8];
    __shared__ double shs[2][8];
    if (lane == 0) {
        shm[0][w] = m0; shm[1][w] = m1; shm[2][w] = m2; shm[3][w] = m5;
        shs[0][w] = o3; shs[1][w] = o4;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long t0 = 0, t1 = 0, t2 = 0, t5 = 0;
        double t3 = 0, t4 = 0;
        for (int i = 0; i < (int)(blockDim.x >> 5); i++) {
            t0 = max(t0, shm[0][i]); t1 = max(t1, shm[1][i]); t2 = max(t2, shm[2][i]); t5 = max(t5, shm[3][i]);
            t3 += shs[0][i]; t4 += shs[1][i];
        }
        double* q = out + r * 6;
        q[0] = bits_double(t0); q[1] = bits_double(t1); q[2] = bits_double(t2);
        q[3] = t3; q[4] = t4; q[5] = bits_double(t5);
    }
}

// Conjugate-gradient refinement (symmetric factors, option refine_cg): the
// FP32 factors give M = L D^-1 L^T, symmetric positive definite for an SPD
// A, so the FP64 correction loop can be the preconditioned conjugate
// gradient method instead of stationary refinement.  Per right-hand side r,
// cg[4r .. 4r+3] = {rho = r^T z, p^T s (s = -A p), rho of the next step, spare}.
// Dot products: per block partial sums in a fixed order, then one warp per
// right-hand side adds them in a fixed order (deterministic).
__global__ void k_dot_partial(const double* __restrict__ a, const double* __restrict__ b, int64_t n, double* __restrict__ part) {
    __shared__ double red[8];
    const int r = blockIdx.y;
    const double* aa = a + (int64_t)r * n;
    const double* bb = b + (int64_t)r * n;
    double acc = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        acc = fma(aa[i], bb[i], acc);
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); w++) t += red[w];
        part[(int64_t)r * gridDim.x + blockIdx.x] = t;
    }
}

// cg[4 r + slot] = sum of the partial sums of right-hand side r (one block, all loads first, fixed
// order).  With it the coefficient the next vector kernel needs, formed once: slot 2 (rho of the
// next step) gives beta = rho_next / rho, slot 1 (p^T s, s = -A p) gives alpha = -rho / p^T s;
// either goes to cg[4 r + 3].
__global__ void __launch_bounds__(256) k_dot_final(const double* __restrict__ part, int nblk, double* __restrict__ cg, int slot) {
    const int r = blockIdx.x, lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    double t = 0.0;
    for (int i0 = threadIdx.x; i0 < nblk; i0 += 4 * blockDim.x) {
        double v[4];
#pragma unroll
        for (int u = 0; u < 4; u++) v[u] = i0 + u * (int)blockDim.x < nblk ? part[(int64_t)r * nblk + i0 + u * blockDim.x] : 0.0;
        t += (v[0] + v[1]) + (v[2] + v[3]);
    }
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    __shared__ double sh[8];
    if (lane == 0) sh[w] = t;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int i = 0; i < (int)(blockDim.x >> 5); i++) s += sh[i];
        double* c = cg + 4 * r;
        c[slot] = s;
        if (slot == 2) c[3] = c[0] != 0.0 ? s / c[0] : 0.0;
        if (slot == 1) c[3] = s != 0.0 ? -c[0] / s : 0.0;
    }
}

// x += alpha p, r += alpha s with s = -A p and alpha = rho / (p^T A p) = -rho / (p^T s) (cg[4 r + 3])
__global__ void k_cg_xr(double* __restrict__ x, double* __restrict__ rv, const double* __restrict__ p,
                        const double* __restrict__ sv, const double* __restrict__ cg, int64_t n) {
    const int r = blockIdx.y;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double alpha = cg[4 * r + 3];
    const int64_t q = (int64_t)r * n + i;
    x[q] = fma(alpha, p[q], x[q]);
    rv[q] = fma(alpha, sv[q], rv[q]);
}

// p = z + beta p with beta = rho_next / rho (cg[4 r + 3]; first: p = z); then rho := rho_next
// (k_cg_commit)
__global__ void k_cg_p(double* __restrict__ p, const double* __restrict__ z, const double* __restrict__ cg, int64_t n,
                       int first) {
    const int r = blockIdx.y;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int64_t q = (int64_t)r * n + i;
    if (first) {
        p[q] = z[q];
        return;
    }
    p[q] = fma(cg[4 * r + 3], p[q], z[q]);
}

// Stop test of the device-side refinement loops, the host's test restated: eta = max over the
// right-hand sides of |r| / (|A| |x| + |b|) from the norms block (a NaN stops the loop); the
// iteration counter grows by inc (the step just taken); continue while eta > tol and fewer than
// the allowed iterations have run (par = {tol, iterations allowed}).
__global__ void k_cg_test(const double* __restrict__ norms, int nrhs, const double* __restrict__ par,
                          int* __restrict__ iter, int inc, cudaGraphConditionalHandle h) {
    if (threadIdx.x != 0) return;
    const double anorm = norms[5];
    double eta = 0.0;
    for (int r = 0; r < nrhs; r++) {
        const double* q = norms + 6 * r;
        const double den = anorm * q[1] + q[2];
        const double e = den > 0 ? q[0] / den : (q[0] > 0 ? INFINITY : 0.0);
        if (isnan(e) || e > eta) eta = e;
    }
    const int it = *iter + inc;
    *iter = it;
    const bool go = eta > par[0] && isfinite(eta) && (double)it < par[1];
    cudaGraphSetConditional(h, go ? 1u : 0u);
}

__global__ void k_cg_params(double* __restrict__ par, double tol, int allowed) {
    par[0] = tol;
    par[1] = (double)allowed;
}

__global__ void k_cg_commit(double* __restrict__ cg, int nrhs) {
    const int r = threadIdx.x;
    if (r < nrhs) cg[4 * r] = cg[4 * r + 2];
}

// Symmetric factors (A = L D^-1 L^T, D = diag(L)): between the forward sweep
// with L and the backward sweep with L^T the pivot values are multiplied by
// their pivots, z = D y.  diag_off[d]: factor-arena offset of dof d's pivot.
// Symmetric solves, z = D y between the two sweeps.  The pivots are gathered
// into dof order once per factorization (k_gather_pivots), so the scaling of
// every solve reads them contiguously.
template <typename T>
__global__ void k_gather_pivots(const int64_t* __restrict__ diag_off, const T* __restrict__ fac, double* __restrict__ pdv,
                                int64_t n) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) pdv[i] = (double)fac[diag_off[i]];
}
__global__ void k_scale_pivots(const double* __restrict__ pdv, double* __restrict__ x, int64_t n, int nrhs) {
    pdl_trigger();
    pdl_wait();
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n * nrhs) return;
    x[i] *= pdv[nrhs == 1 ? i : i % n];
}

__global__ void k_axpy(double* __restrict__ x, const double* __restrict__ d, int64_t n) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) x[i] += d[i];
}

// g_e = -lambda_e^T dK_e x_e: one warp per element.
__global__ void k_element_grad(const double* __restrict__ dK, const int64_t* __restrict__ en, const double* __restrict__ lam,
                               const double* __restrict__ x, double* __restrict__ g, int64_t n_elem, int npe) {
    const int64_t e = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (e >= n_elem) return;
    const double* K = dK + e * npe * npe;
    const int64_t* nd = en + e * npe;
    double acc = 0.0;
    for (int t = lane; t < npe * npe; t += 32) {
        int a = t % npe, b = t / npe;
        acc += lam[nd[a]] * K[t] * x[nd[b]];
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) g[e] = -acc;
}

// G_e[a + b*npe] = -sum_r lambda[node(e,a), r] x[node(e,b), r]
__global__ void k_element_outer(const int64_t* __restrict__ en, const double* __restrict__ lam, const double* __restrict__ x,
                                double* __restrict__ G, int64_t n_elem, int npe, int64_t n_dof, int nrhs) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t nn = (int64_t)npe * npe;
    if (idx >= n_elem * nn) return;
    const int64_t e = idx / nn;
    const int t = (int)(idx - e * nn);
    const int a = t % npe, b = t / npe;
    const int64_t na = en[e * npe + a], nb = en[e * npe + b];
    double acc = 0.0;
    for (int r = 0; r < nrhs; r++) acc += lam[na + (int64_t)r * n_dof] * x[nb + (int64_t)r * n_dof];
    G[idx] = -acc;
}
