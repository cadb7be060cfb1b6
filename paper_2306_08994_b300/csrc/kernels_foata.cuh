// Scalar-task Foata executor for the bottom classes (Sec. 3 task alphabet,
// Sec. 3.3 Foata normal form, Table 2 compute_front).
//
// The paper schedules the factorization as a trace of scalar tasks and runs
// each Foata class as a bag of tasks with a barrier after it; inside a front
// the classes cycle through the four task kinds for each pivot p:
//   T4 assertion  -- the pivot is fully assembled (here: the static pivot
//                    check, |F[p,p]| >= tau, replaced by sign * tau if not),
//   T1 division   -- F[p,j] /= F[p,p] for every j > p,
//   T2 multiply   -- t[i,j] = F[i,p] * F[p,j] for every i, j > p,
//   T3 subtract   -- F[i,j] -= t[i,j].
// This executor runs exactly that schedule for the fronts of one tree level
// (a front-level class): one launch per task kind and pivot step covers the
// step's tasks of every front of the level (the launch boundary is the
// class barrier), after one launch of extend-add tasks (each assembled entry
// pulls its children's contributions in fixed child order) and one that
// takes each front's largest entry for the pivot threshold; a last launch
// writes L, U and the contribution block where the other kernels put them.
// Fronts are dense m x m column-major blocks in a workspace W; the products
// of T2 go to a second workspace X of the same shape.  It is an alternative
// to the fused kernels (one CTA or lane group runs a whole front) for the
// classes at the bottom of the tree.
#pragma once

#include <cstdint>

#include "kernels_factor.cuh"

// Launch geometry: fronts of one class in list order, `bpf` blocks of 256
// threads per front (enough for m^2 entries, or m for the row-wise kinds).
struct FoataArgs {
    const FactorRec* recs;
    const int64_t* woff;  // workspace offset of each listed front
    int nfront, bpf, p;
};

template <typename T>
__global__ void __launch_bounds__(256) k_foata_assemble(FoataArgs A, const int32_t* __restrict__ maps,
                                                        const double* __restrict__ values, int npe,
                                                        const T* __restrict__ cbs, T* __restrict__ W) {
    const int fi = blockIdx.x / A.bpf;
    if (fi >= A.nfront) return;
    const FactorRec r = A.recs[fi];
    const int64_t e = (int64_t)(blockIdx.x % A.bpf) * blockDim.x + threadIdx.x;
    const int m = r.m;
    if (e >= (int64_t)m * m) return;
    const int i = (int)(e % m), j = (int)(e / m);
    T x = T(0);
    if (r.nchild == 0) {
        const int32_t* mp = maps + r.map_off;
        x = (T)values[(int64_t)r.elem * npe * npe + mp[i] + (int64_t)mp[j] * npe];
    } else {
        for (int c = 0; c < r.nchild; c++) {  // child 0, then child 1
            const int32_t* mp = maps + r.map_off + (int64_t)c * m;
            const int ic = mp[i], jc = mp[j];
            if (ic >= 0 && jc >= 0) x += cbs[r.cS[c] + ic + (int64_t)jc * r.cn[c]];
        }
    }
    W[A.woff[fi] + e] = x;
}

// largest |entry| of each assembled front (one block per front): the static pivot threshold's scale
template <typename T>
__global__ void __launch_bounds__(256) k_foata_amax(FoataArgs A, const T* __restrict__ W, unsigned int* __restrict__ famax) {
    __shared__ float red[8];
    const int fi = blockIdx.x;
    const FactorRec r = A.recs[fi];
    const int64_t n = (int64_t)r.m * r.m;
    const T* F = W + A.woff[fi];
    T v = T(0);
    for (int64_t e = threadIdx.x; e < n; e += blockDim.x) v = max(v, (T)fabs(F[e]));
    v = block_max_abs(v, red);
    if (threadIdx.x == 0) famax[r.front] = __float_as_uint((float)v);
}

// T4 at pivot p: one task per front that still has pivot p
template <typename T>
__global__ void __launch_bounds__(256) k_foata_t4(FoataArgs A, T* __restrict__ W, const unsigned int* __restrict__ famax,
                                                  double tol_rel, DevStatus* st) {
    const int fi = blockIdx.x * blockDim.x + threadIdx.x;
    if (fi >= A.nfront) return;
    const FactorRec r = A.recs[fi];
    const int p = A.p, m = r.m;
    if (p >= r.k) return;
    const T amax = (T)__uint_as_float(famax[r.front]);
    const T thr = (T)tol_rel * amax > T(0) ? (T)tol_rel * amax : tiny_pivot<T>();
    T* F = W + A.woff[fi];
    F[p + (int64_t)p * m] = checked_pivot(F[p + (int64_t)p * m], thr, true, r.front, p, st);
}

// T1 at pivot p: F[p, j] /= F[p, p], j > p
template <typename T>
__global__ void __launch_bounds__(256) k_foata_t1(FoataArgs A, T* __restrict__ W) {
    const int fi = blockIdx.x / A.bpf;
    if (fi >= A.nfront) return;
    const FactorRec r = A.recs[fi];
    const int p = A.p, m = r.m;
    if (p >= r.k) return;
    const int j = p + 1 + (blockIdx.x % A.bpf) * blockDim.x + threadIdx.x;
    if (j >= m) return;
    T* F = W + A.woff[fi];
    F[p + (int64_t)j * m] = F[p + (int64_t)j * m] / F[p + (int64_t)p * m];
}

// T2 at pivot p: X[i, j] = F[i, p] F[p, j], i, j > p
template <typename T>
__global__ void __launch_bounds__(256) k_foata_t2(FoataArgs A, const T* __restrict__ W, T* __restrict__ X) {
    const int fi = blockIdx.x / A.bpf;
    if (fi >= A.nfront) return;
    const FactorRec r = A.recs[fi];
    const int p = A.p, m = r.m, n = m - p - 1;
    if (p >= r.k) return;
    const int64_t e = (int64_t)(blockIdx.x % A.bpf) * blockDim.x + threadIdx.x;
    if (e >= (int64_t)n * n) return;
    const int i = p + 1 + (int)(e % n), j = p + 1 + (int)(e / n);
    const T* F = W + A.woff[fi];
    X[A.woff[fi] + i + (int64_t)j * m] = F[i + (int64_t)p * m] * F[p + (int64_t)j * m];
}

// T3 at pivot p: F[i, j] -= X[i, j], i, j > p
template <typename T>
__global__ void __launch_bounds__(256) k_foata_t3(FoataArgs A, T* __restrict__ W, const T* __restrict__ X) {
    const int fi = blockIdx.x / A.bpf;
    if (fi >= A.nfront) return;
    const FactorRec r = A.recs[fi];
    const int p = A.p, m = r.m, n = m - p - 1;
    if (p >= r.k) return;
    const int64_t e = (int64_t)(blockIdx.x % A.bpf) * blockDim.x + threadIdx.x;
    if (e >= (int64_t)n * n) return;
    const int i = p + 1 + (int)(e % n), j = p + 1 + (int)(e / n);
    const int64_t q = A.woff[fi] + i + (int64_t)j * m;
    W[q] -= X[q];
}

// P = F[:, 0:k], R = F[0:k, k:m], S = F[k:m, k:m] to the factor and contribution-block arenas
template <typename T>
__global__ void __launch_bounds__(256) k_foata_write(FoataArgs A, const T* __restrict__ W, T* __restrict__ fac,
                                                     T* __restrict__ cbs) {
    const int fi = blockIdx.x / A.bpf;
    if (fi >= A.nfront) return;
    const FactorRec r = A.recs[fi];
    const int m = r.m, k = r.k, nc = m - k;
    const int64_t e = (int64_t)(blockIdx.x % A.bpf) * blockDim.x + threadIdx.x;
    if (e >= (int64_t)m * m) return;
    const int i = (int)(e % m), j = (int)(e / m);
    const T v = W[A.woff[fi] + e];
    if (j < k) fac[r.P_off + i + (int64_t)j * m] = v;
    else if (i < k) fac[r.R_off + i + (int64_t)(j - k) * k] = v;
    else cbs[r.S_off + (i - k) + (int64_t)(j - k) * nc] = v;
}
