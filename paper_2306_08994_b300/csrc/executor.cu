// Executor: builds the per-class launch plan (the Foata classes of Sec. 3.3
// as a sequence of batched launches, each a bag of independent tasks), owns
// the device arenas, and drives factorization, solves and refinement.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <vector>

#include "kernels_factor.cuh"
#include "kernels_solve.cuh"
#include "mf_internal.h"

namespace {

enum LaunchKind { K_FUSED = 0, K_ASM = 1, K_PANEL = 2, K_GEMM = 3 };

struct Launch {
    int kind;
    int cls;
    int count;
    int maxm;     // fused: bucket bound (shared-memory size)
    int64_t off;  // offset into the list of its kind
};

// Solve plan of one class: fronts split by size (see kernels_solve.cuh).
struct ClassList {
    int n_small, n_cta, n_split, n_frows, n_brows;
    int maxm_cta, maxk_split, maxnc_split, maxk_all;
    int64_t off_small, off_cta, off_split;  // into the solve front list
    int64_t off_frows, off_brows;           // into the row-task list
};
constexpr int kSolveWarpMax = 64;   // m <= this: one warp per front
constexpr int kSolveSplitCB = 256;  // m - k > this: CB rows in a separate row-parallel launch

#define CUDA_TRY(x)                          \
    do {                                     \
        cudaError_t e__ = (x);               \
        if (e__ != cudaSuccess) {            \
            (void)cudaGetLastError();        \
            return MF_ECUDA;                 \
        }                                    \
    } while (0)

template <typename T>
int dev_alloc(T** p, size_t n) {
    *p = nullptr;
    if (n == 0) n = 1;
    cudaError_t e = cudaMalloc((void**)p, n * sizeof(T));
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        *p = nullptr;
        return MF_ENOMEM;
    }
    return MF_OK;
}

template <typename T>
int upload(T** p, const std::vector<T>& v) {
    int rc = dev_alloc(p, v.size());
    if (rc) return rc;
    if (!v.empty()) CUDA_TRY(cudaMemcpy(*p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice));
    return MF_OK;
}

constexpr int kPanelNB64 = 32;  // FP64 panel width
constexpr int kPanelNB32 = 64;  // FP32 panel width

__global__ void k_init_status(DevStatus* st) {
    st->n_perturbed = 0ull;
    st->first = ~0ull;
    st->nonfinite = 0;
    st->timeout = 0;
}

}  // namespace

struct mf_factors {
    const mf_analysis* a = nullptr;
    mf_options opt{};
    int prec = MF_F64;
    size_t tsize = 8;
    double tol_rel = 0;
    int nb = 32;
    int small_max = 96;
    int max_nrhs = 4;
    // device
    FrontDev* d_fronts = nullptr;
    int32_t* d_dofs = nullptr;
    int32_t* d_maps = nullptr;
    int64_t* d_en = nullptr;
    int64_t* d_node_ptr = nullptr;
    int64_t* d_node_inc = nullptr;
    void* d_fac = nullptr;
    void* d_cb = nullptr;
    void* d_vec = nullptr;
    int32_t* d_flist = nullptr;
    int32_t* d_slist = nullptr;
    RowTask* d_rows = nullptr;
    AsmTile* d_asm = nullptr;
    PanelTask* d_panel = nullptr;
    GemmTile* d_gemm = nullptr;
    unsigned int* d_famax = nullptr;
    DevStatus* d_status = nullptr;
    double *d_r = nullptr, *d_d = nullptr, *d_Y = nullptr, *d_rowabs = nullptr, *d_part = nullptr, *d_norms = nullptr;
    int norm_blocks = 296;
    bool rowabs_valid = false;
    const double* rowabs_values = nullptr;
    // plan
    std::vector<Launch> plan;
    std::vector<ClassList> classes;
    bool factored = false;
    // algorithmic work per plan entry / per class and direction (per rhs)
    std::vector<double> plan_bytes, plan_flops;
    std::vector<int> plan_fam;
    std::vector<double> fwd_bytes, bwd_bytes, fwd_flops, bwd_flops;
    double resid_bytes = 0, resid_flops = 0;
    // profiling
    bool prof = false;
    std::vector<cudaEvent_t> ev;  // pairs
    std::vector<int> ev_fam;
    size_t ev_used = 0;
    double acc_bytes[MF_PROFILE_FAMILIES] = {};
    double acc_flops[MF_PROFILE_FAMILIES] = {};
    int64_t acc_launch[MF_PROFILE_FAMILIES] = {};
};

enum Family { FAM_FUSED = 0, FAM_ASM = 1, FAM_PANEL = 2, FAM_TRAIL = 3, FAM_SCHUR = 4, FAM_FWD = 5, FAM_BWD = 6,
              FAM_RESID = 7, FAM_OTHER = 8 };

// Bracket one launch: returns a slot index (or -1 when profiling is off).
static int prof_begin(mf_factors* F, cudaStream_t s, int fam, double bytes, double flops, int kernels = 1) {
    F->acc_launch[fam] += kernels;
    F->acc_bytes[fam] += bytes;
    F->acc_flops[fam] += flops;
    if (!F->prof) return -1;
    if (F->ev_used * 2 + 2 > F->ev.size()) {
        for (int i = 0; i < 256; i++) {
            cudaEvent_t e;
            if (cudaEventCreate(&e) != cudaSuccess) return -1;
            F->ev.push_back(e);
        }
        F->ev_fam.resize(F->ev.size() / 2);
    }
    int slot = (int)F->ev_used++;
    F->ev_fam[slot] = fam;
    cudaEventRecord(F->ev[2 * slot], s);
    return slot;
}

static void prof_end(mf_factors* F, cudaStream_t s, int slot) {
    if (slot >= 0) cudaEventRecord(F->ev[2 * slot + 1], s);
}

static void free_factors(mf_factors* f) {
    if (!f) return;
    for (cudaEvent_t e : f->ev) cudaEventDestroy(e);
    void* ptrs[] = {f->d_fronts, f->d_dofs, f->d_maps, f->d_en, f->d_node_ptr, f->d_node_inc, f->d_fac, f->d_cb,
                    f->d_vec, f->d_flist, f->d_slist, f->d_rows, f->d_asm, f->d_panel, f->d_gemm, f->d_famax, f->d_status,
                    f->d_r, f->d_d, f->d_Y, f->d_rowabs, f->d_part, f->d_norms};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    delete f;
}

template <typename T>
static size_t fused_smem(int maxm) {
    int ldm = maxm | 1;
    return (size_t)ldm * maxm * sizeof(T) + (size_t)maxm * sizeof(T) + 2 * (size_t)maxm * sizeof(int32_t) + 32 * sizeof(float);
}

static int build_plan(mf_factors* F) {
    const mf_analysis* a = F->a;
    std::vector<int32_t> flist, slist;
    std::vector<RowTask> rows;
    std::vector<AsmTile> asmt;
    std::vector<PanelTask> pan;
    std::vector<GemmTile> gem;
    const int bounds64[] = {16, 32, 48, 64, 96, 128, 160};
    const int bounds32[] = {16, 32, 48, 64, 96, 128, 160, 192, 224};
    const int* bounds = F->prec == MF_F64 ? bounds64 : bounds32;
    const int nbounds = F->prec == MF_F64 ? 7 : 9;
    const int nb = F->nb;
    const double T = (double)F->tsize;
    double gb = 0, gf = 0;  // running algorithmic counts of the GEMM launch being built
    auto pflops = [](double m, double k) {
        if (k <= 0) return 0.0;
        double a0 = m - k, b0 = m - 1;
        return (a0 + b0) * (b0 - a0 + 1) / 2.0 + 2.0 * (b0 * (b0 + 1) * (2 * b0 + 1) / 6.0 - (a0 - 1) * a0 * (2 * a0 - 1) / 6.0);
    };
    auto push = [&](Launch L, int fam, double bytes, double flops) {
        F->plan.push_back(L);
        F->plan_fam.push_back(fam);
        F->plan_bytes.push_back(bytes);
        F->plan_flops.push_back(flops);
    };
    auto gemm_tiles = [&](int64_t a_off, int lda, int64_t b_off, int ldb, int64_t c_off, int ldc, int M, int N, int K,
                          int c_in_cb) {
        gf += 2.0 * M * N * K;
        gb += T * ((double)M * K + (double)K * N + 2.0 * M * N);
        for (int j0 = 0; j0 < N; j0 += 64)
            for (int i0 = 0; i0 < M; i0 += 64) {
                GemmTile t{};
                t.a_off = a_off; t.b_off = b_off; t.c_off = c_off;
                t.lda = lda; t.ldb = ldb; t.ldc = ldc;
                t.M = M; t.N = N; t.K = K; t.i0 = i0; t.j0 = j0; t.c_in_cb = c_in_cb;
                gem.push_back(t);
            }
    };
    for (int c = 0; c < a->n_cls; c++) {
        const int32_t f0 = a->cls_ptr[c], f1 = a->cls_ptr[c + 1];
        // solve list: all fronts of the class, largest first
        std::vector<int32_t> all;
        int maxm_all = 1;
        for (int32_t f = f0; f < f1; f++) {
            all.push_back(f);
            maxm_all = std::max(maxm_all, a->fronts[f].m);
        }
        std::stable_sort(all.begin(), all.end(), [&](int32_t x, int32_t y) { return a->fronts[x].m > a->fronts[y].m; });
        {
            ClassList C{};
            std::vector<int32_t> sm, ct, sp;
            for (int32_t f : all) {
                const FrontDev& fr = a->fronts[f];
                if (fr.m <= kSolveWarpMax) sm.push_back(f);
                else if (fr.m - fr.k <= kSolveSplitCB) ct.push_back(f);
                else sp.push_back(f);
                C.maxk_all = std::max(C.maxk_all, fr.k);
            }
            C.n_small = (int)sm.size();
            C.off_small = (int64_t)slist.size();
            slist.insert(slist.end(), sm.begin(), sm.end());
            C.n_cta = (int)ct.size();
            C.off_cta = (int64_t)slist.size();
            slist.insert(slist.end(), ct.begin(), ct.end());
            for (int32_t f : ct) C.maxm_cta = std::max(C.maxm_cta, a->fronts[f].m);
            C.n_split = (int)sp.size();
            C.off_split = (int64_t)slist.size();
            slist.insert(slist.end(), sp.begin(), sp.end());
            C.off_frows = (int64_t)rows.size();
            for (int32_t f : sp) {
                const FrontDev& fr = a->fronts[f];
                C.maxk_split = std::max(C.maxk_split, fr.k);
                C.maxnc_split = std::max(C.maxnc_split, fr.m - fr.k);
                for (int i = fr.k; i < fr.m; i += 128) rows.push_back({f, i, std::min(fr.m, i + 128), 0});
            }
            C.n_frows = (int)(rows.size() - C.off_frows);
            C.off_brows = (int64_t)rows.size();
            for (int32_t f : sp) {
                const FrontDev& fr = a->fronts[f];
                for (int i = 0; i < fr.k; i += 128) rows.push_back({f, i, std::min(fr.k, i + 128), 0});
            }
            C.n_brows = (int)(rows.size() - C.off_brows);
            F->classes.push_back(C);
        }
        {
            double fb = 0, bb = 0, ff = 0, bf = 0;
            for (int32_t f : all) {
                const FrontDev& fr = a->fronts[f];
                double m = fr.m, k = fr.k, nc = m - k;
                double nl = m * k - k * (k - 1) / 2, nu = k * (k - 1) / 2 + k * nc;
                double cin = 0;
                for (int q = 0; q < fr.nchild; q++) {
                    const FrontDev& ch = a->fronts[fr.child[q]];
                    cin += ch.m - ch.k;
                }
                fb += T * nl + 8.0 * k * 2 + T * (cin + nc);
                bb += T * nu + 8.0 * (m + k);
                ff += 2.0 * nl;
                bf += 2.0 * nu;
            }
            F->fwd_bytes.push_back(fb);
            F->bwd_bytes.push_back(bb);
            F->fwd_flops.push_back(ff);
            F->bwd_flops.push_back(bf);
        }
        slist.insert(slist.end(), all.begin(), all.end());

        // fused buckets (largest first inside each launch)
        int lo = 0;
        for (int bi = 0; bi < nbounds && lo < F->small_max; bi++) {
            int hi = std::min(bounds[bi], F->small_max);
            std::vector<int32_t> L;
            for (int32_t f : all)
                if (a->fronts[f].m > lo && a->fronts[f].m <= hi) L.push_back(f);
            if (!L.empty()) {
                double by = 0, fl = 0;
                for (int32_t f : L) {
                    const FrontDev& fr = a->fronts[f];
                    double m = fr.m, k = fr.k, nc = m - k;
                    if (fr.nchild == 0) by += 8.0 * a->npe * a->npe;
                    for (int q = 0; q < fr.nchild; q++) {
                        const FrontDev& ch = a->fronts[fr.child[q]];
                        by += T * (double)(ch.m - ch.k) * (ch.m - ch.k);
                    }
                    by += T * (m * k + k * nc + nc * nc);
                    fl += pflops(m, k);
                }
                push({K_FUSED, c, (int)L.size(), hi, (int64_t)flist.size()}, FAM_FUSED, by, fl);
                flist.insert(flist.end(), L.begin(), L.end());
            }
            lo = hi;
        }
        // large fronts
        std::vector<int32_t> big;
        for (int32_t f : all)
            if (a->fronts[f].m > F->small_max) big.push_back(f);
        if (big.empty()) continue;
        {
            int64_t off = (int64_t)asmt.size();
            double by = 0;
            for (int32_t f : big) {
                const FrontDev& fr = a->fronts[f];
                int m = fr.m;
                for (int j0 = 0; j0 < m; j0 += 64)
                    for (int i0 = 0; i0 < m; i0 += 64) asmt.push_back({f, i0, j0, 0});
                for (int q = 0; q < fr.nchild; q++) {
                    const FrontDev& ch = a->fronts[fr.child[q]];
                    by += T * (double)(ch.m - ch.k) * (ch.m - ch.k);
                }
                by += T * (double)m * m;
            }
            push({K_ASM, c, (int)(asmt.size() - off), 0, off}, FAM_ASM, by, 0.0);
        }
        int maxk = 0;
        for (int32_t f : big) maxk = std::max(maxk, a->fronts[f].k);
        std::vector<PanelTask> diag;
        for (int kb = 0; kb < maxk; kb += nb) {
            int64_t poff = (int64_t)pan.size();
            int64_t goff = (int64_t)gem.size();
            double pb = 0, pf = 0;
            gb = gf = 0;
            for (int32_t f : big) {
                const FrontDev& fr = a->fronts[f];
                if (kb >= fr.k) continue;
                const int m = fr.m, k = fr.k, w = std::min(nb, k - kb), r0 = kb + w;
                pb += 2.0 * T * ((double)w * w + 2.0 * (double)(m - r0) * w);
                pf += 2.0 * w * w * w / 3.0 + 2.0 * (double)(m - r0) * w * w;
                diag.push_back({f, kb, w, 2, 0, 0, 0, 0});
                for (int i = r0; i < m; i += 256) pan.push_back({f, kb, w, 0, i, std::min(m, i + 256), 0, 0});
                for (int j = r0; j < m; j += 256) pan.push_back({f, kb, w, 1, j, std::min(m, j + 256), 0, 0});
                // trailing updates restricted to the pivot rows/columns
                if (m - r0 > 0 && k - r0 > 0)
                    gemm_tiles(fr.P_off + r0 + (int64_t)kb * m, m, fr.P_off + kb + (int64_t)r0 * m, m,
                               fr.P_off + r0 + (int64_t)r0 * m, m, m - r0, k - r0, w, 0);
                if (k - r0 > 0 && m - k > 0)
                    gemm_tiles(fr.P_off + r0 + (int64_t)kb * m, m, fr.R_off + kb, k, fr.R_off + r0, k, k - r0, m - k, w, 0);
            }
            if (pan.size() > (size_t)poff) push({K_PANEL, c, (int)(pan.size() - poff), 0, poff}, FAM_PANEL, pb, pf);
            if (gem.size() > (size_t)goff) push({K_GEMM, c, (int)(gem.size() - goff), 0, goff}, FAM_TRAIL, gb, gf);
        }
        // Schur update S -= L21 U12 (Sec. 2.2)
        int64_t goff = (int64_t)gem.size();
        gb = gf = 0;
        for (int32_t f : big) {
            const FrontDev& fr = a->fronts[f];
            const int m = fr.m, k = fr.k;
            if (m - k > 0 && k > 0) gemm_tiles(fr.P_off + k, m, fr.R_off, k, fr.S_off, m - k, m - k, m - k, k, 1);
        }
        if (gem.size() > (size_t)goff) push({K_GEMM, c, (int)(gem.size() - goff), 0, goff}, FAM_SCHUR, gb, gf);
        if (!diag.empty()) {
            int64_t doff = (int64_t)pan.size();
            double db = 0;
            for (const PanelTask& t : diag) db += 2.0 * T * t.w * t.w;
            pan.insert(pan.end(), diag.begin(), diag.end());
            push({K_PANEL, c, (int)diag.size(), 0, doff}, FAM_PANEL, db, 0.0);
        }
    }
    {
        const double nE = (double)a->n_elem * a->npe;
        F->resid_bytes = 8.0 * (nE * a->npe + nE * 2 + nE * 2 + 2.0 * a->n_dof + 3.0 * a->n_dof);
        F->resid_flops = 2.0 * nE * a->npe;
    }
    int rc;
    if ((rc = upload(&F->d_flist, flist))) return rc;
    if ((rc = upload(&F->d_slist, slist))) return rc;
    if ((rc = upload(&F->d_rows, rows))) return rc;
    if ((rc = upload(&F->d_asm, asmt))) return rc;
    if ((rc = upload(&F->d_panel, pan))) return rc;
    if ((rc = upload(&F->d_gemm, gem))) return rc;
    return MF_OK;
}

template <typename T>
static int set_smem_limits() {
    int dev;
    CUDA_TRY(cudaGetDevice(&dev));
    int maxsm = 0;
    CUDA_TRY(cudaDeviceGetAttribute(&maxsm, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    CUDA_TRY(cudaFuncSetAttribute(k_front_fused<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, maxsm));
    CUDA_TRY(cudaFuncSetAttribute(k_fwd_cta<T, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, maxsm));
    CUDA_TRY(cudaFuncSetAttribute(k_fwd_cta<T, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, maxsm));
    CUDA_TRY(cudaFuncSetAttribute(k_bwd_cta<T, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, maxsm));
    CUDA_TRY(cudaFuncSetAttribute(k_bwd_cta<T, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, maxsm));
    CUDA_TRY(cudaFuncSetAttribute(k_fwd_rows<T, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, maxsm));
    CUDA_TRY(cudaFuncSetAttribute(k_fwd_rows<T, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, maxsm));
    CUDA_TRY(cudaFuncSetAttribute(k_bwd_rows<T, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, maxsm));
    CUDA_TRY(cudaFuncSetAttribute(k_bwd_rows<T, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, maxsm));
    return MF_OK;
}

extern "C" int mf_factors_create(const mf_analysis* a, const mf_options* opt, mf_factors** out) {
    if (!a || !out) return MF_EINVAL;
    *out = nullptr;
    mf_factors* F = new mf_factors();
    F->a = a;
    F->opt = opt ? mf_resolve_options(opt) : a->opt;
    F->prec = F->opt.precision;
    if (F->prec != MF_F64 && F->prec != MF_F32 && F->prec != MF_TF32) {
        delete F;
        return MF_EINVAL;
    }
    F->tsize = F->prec == MF_F64 ? 8 : 4;
    F->tol_rel = F->opt.pivot_tol > 0 ? F->opt.pivot_tol : (F->prec == MF_F64 ? 1.1102230246251565e-16 : 5.9604644775390625e-08);
    F->nb = F->opt.panel_width > 0 ? F->opt.panel_width : (F->prec == MF_F64 ? kPanelNB64 : kPanelNB32);
    if (F->nb != (F->prec == MF_F64 ? kPanelNB64 : kPanelNB32)) {
        delete F;
        return MF_ENOTSUP;
    }
    F->small_max = F->opt.small_front_max > 0 ? F->opt.small_front_max : (F->prec == MF_F64 ? 96 : 128);
    F->small_max = std::min(F->small_max, F->prec == MF_F64 ? 160 : 224);
    F->small_max = std::max(F->small_max, a->npe);
    F->max_nrhs = F->opt.max_nrhs > 0 ? F->opt.max_nrhs : 4;
    int rc = MF_OK;
#define TRY(x)                \
    do {                      \
        rc = (x);             \
        if (rc) {             \
            free_factors(F);  \
            return rc;        \
        }                     \
    } while (0)
    TRY(F->prec == MF_F64 ? set_smem_limits<double>() : set_smem_limits<float>());
    TRY(upload(&F->d_fronts, a->fronts));
    TRY(upload(&F->d_dofs, a->dofs));
    TRY(upload(&F->d_maps, a->maps));
    TRY(upload(&F->d_en, a->elem_nodes));
    TRY(upload(&F->d_node_ptr, a->node_ptr));
    TRY(upload(&F->d_node_inc, a->node_inc));
    TRY(dev_alloc((char**)&F->d_fac, (size_t)a->factor_size * F->tsize));
    TRY(dev_alloc((char**)&F->d_cb, (size_t)a->cb_size * F->tsize));
    TRY(dev_alloc((char**)&F->d_vec, (size_t)a->vec_size * F->max_nrhs * F->tsize));
    TRY(dev_alloc(&F->d_famax, (size_t)a->n_front));
    TRY(dev_alloc(&F->d_status, 1));
    const size_t nv = (size_t)a->n_dof * F->max_nrhs;
    TRY(dev_alloc(&F->d_r, nv));
    TRY(dev_alloc(&F->d_d, nv));
    TRY(dev_alloc(&F->d_Y, (size_t)a->n_elem * a->npe * F->max_nrhs));
    TRY(dev_alloc(&F->d_rowabs, (size_t)a->n_dof));
    TRY(dev_alloc(&F->d_part, (size_t)F->norm_blocks * 6 * F->max_nrhs));
    TRY(dev_alloc(&F->d_norms, (size_t)6 * F->max_nrhs));
    TRY(build_plan(F));
#undef TRY
    *out = F;
    return MF_OK;
}

extern "C" void mf_free_factors(mf_factors* f) { free_factors(f); }

template <typename T>
static int run_factor(mf_factors* F, const double* d_values, cudaStream_t s) {
    const mf_analysis* a = F->a;
    T* fac = (T*)F->d_fac;
    T* cb = (T*)F->d_cb;
    int slot = prof_begin(F, s, FAM_OTHER, 0, 0);
    k_init_status<<<1, 1, 0, s>>>(F->d_status);
    CUDA_TRY(cudaMemsetAsync(F->d_famax, 0, sizeof(unsigned int) * a->n_front, s));
    prof_end(F, s, slot);
    for (size_t li = 0; li < F->plan.size(); li++) {
        const Launch& L = F->plan[li];
        slot = prof_begin(F, s, F->plan_fam[li], F->plan_bytes[li], F->plan_flops[li]);
        switch (L.kind) {
            case K_FUSED: {
                int ldm = L.maxm | 1;
                size_t sm = fused_smem<T>(L.maxm);
                int threads = L.maxm <= 32 ? 64 : (L.maxm <= 64 ? 128 : 256);
                k_front_fused<T><<<L.count, threads, sm, s>>>(F->d_fronts, F->d_flist + L.off, F->d_maps, d_values, a->npe,
                                                              fac, cb, L.maxm, ldm, F->tol_rel, F->d_status);
                break;
            }
            case K_ASM:
                k_assemble_large<T><<<L.count, 256, 0, s>>>(F->d_fronts, F->d_asm + L.off, F->d_maps, fac, cb, F->d_famax);
                break;
            case K_PANEL:
                if constexpr (sizeof(T) == 8)
                    k_panel<T, kPanelNB64><<<L.count, 256, 0, s>>>(F->d_fronts, F->d_panel + L.off, fac, F->d_famax,
                                                                   F->tol_rel, F->d_status);
                else
                    k_panel<T, kPanelNB32><<<L.count, 256, 0, s>>>(F->d_fronts, F->d_panel + L.off, fac, F->d_famax,
                                                                   F->tol_rel, F->d_status);
                break;
            case K_GEMM:
                k_gemm_sub<T, sizeof(T) == 8 ? 8 : 16><<<L.count, 256, 0, s>>>(F->d_gemm + L.off, fac, fac, cb);
                break;
        }
        prof_end(F, s, slot);
        CUDA_TRY(cudaGetLastError());
    }
    return MF_OK;
}

extern "C" int mf_factor(mf_factors* F, const double* d_values, mf_stream_t stream) {
    if (!F || !d_values) return MF_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    int rc = F->prec == MF_F64 ? run_factor<double>(F, d_values, s) : run_factor<float>(F, d_values, s);
    if (rc == MF_OK) {
        F->factored = true;
        F->rowabs_valid = false;
    }
    return rc;
}

template <typename T>
static int run_solve(mf_factors* F, double* d_x, int nrhs, bool trans, cudaStream_t s) {
    const mf_analysis* a = F->a;
    const T* fac = (const T*)F->d_fac;
    T* vec = (T*)F->d_vec;
    const FrontDev* fr = F->d_fronts;
    const int32_t* L = F->d_slist;
    const int64_t n = a->n_dof, vs = a->vec_size;
    const size_t dgs = 32 * 33 * sizeof(T);
    for (int c = 0; c < a->n_cls; c++) {
        const ClassList& C = F->classes[c];
        int nk = (C.n_small > 0) + (C.n_cta > 0) + (C.n_split > 0) + (C.n_frows > 0);
        int slot = prof_begin(F, s, FAM_FWD, F->fwd_bytes[c] * nrhs, F->fwd_flops[c] * nrhs, nk);
        if (C.n_small) {
            dim3 g((C.n_small + 7) / 8, nrhs);
            if (!trans) k_fwd_warp<T, false><<<g, 256, 0, s>>>(fr, L + C.off_small, C.n_small, fac, F->d_dofs, F->d_maps, vec, vs, d_x, n);
            else k_fwd_warp<T, true><<<g, 256, 0, s>>>(fr, L + C.off_small, C.n_small, fac, F->d_dofs, F->d_maps, vec, vs, d_x, n);
        }
        if (C.n_cta) {
            dim3 g(C.n_cta, nrhs);
            size_t sm = dgs + (size_t)C.maxm_cta * sizeof(T);
            if (!trans) k_fwd_cta<T, false><<<g, 256, sm, s>>>(fr, L + C.off_cta, 1, fac, F->d_dofs, F->d_maps, vec, vs, d_x, n);
            else k_fwd_cta<T, true><<<g, 256, sm, s>>>(fr, L + C.off_cta, 1, fac, F->d_dofs, F->d_maps, vec, vs, d_x, n);
        }
        if (C.n_split) {
            dim3 g(C.n_split, nrhs);
            size_t sm = dgs + (size_t)C.maxk_split * sizeof(T);
            if (!trans) k_fwd_cta<T, false><<<g, 256, sm, s>>>(fr, L + C.off_split, 0, fac, F->d_dofs, F->d_maps, vec, vs, d_x, n);
            else k_fwd_cta<T, true><<<g, 256, sm, s>>>(fr, L + C.off_split, 0, fac, F->d_dofs, F->d_maps, vec, vs, d_x, n);
        }
        if (C.n_frows) {
            dim3 g(C.n_frows, nrhs);
            size_t sm = (size_t)C.maxk_split * sizeof(T);
            if (!trans) k_fwd_rows<T, false><<<g, 128, sm, s>>>(fr, F->d_rows + C.off_frows, fac, F->d_dofs, F->d_maps, vec, vs, d_x, n);
            else k_fwd_rows<T, true><<<g, 128, sm, s>>>(fr, F->d_rows + C.off_frows, fac, F->d_dofs, F->d_maps, vec, vs, d_x, n);
        }
        prof_end(F, s, slot);
        CUDA_TRY(cudaGetLastError());
    }
    for (int c = a->n_cls - 1; c >= 0; c--) {
        const ClassList& C = F->classes[c];
        int nk = (C.n_small > 0) + (C.n_cta > 0) + (C.n_split > 0) + (C.n_brows > 0);
        int slot = prof_begin(F, s, FAM_BWD, F->bwd_bytes[c] * nrhs, F->bwd_flops[c] * nrhs, nk);
        if (C.n_brows) {
            dim3 g(C.n_brows, nrhs);
            size_t sm = (size_t)C.maxnc_split * sizeof(T);
            if (!trans) k_bwd_rows<T, false><<<g, 128, sm, s>>>(fr, F->d_rows + C.off_brows, fac, F->d_dofs, d_x, n);
            else k_bwd_rows<T, true><<<g, 128, sm, s>>>(fr, F->d_rows + C.off_brows, fac, F->d_dofs, d_x, n);
        }
        if (C.n_split) {
            dim3 g(C.n_split, nrhs);
            size_t sm = dgs + (size_t)C.maxk_split * sizeof(T);
            if (!trans) k_bwd_cta<T, false><<<g, 256, sm, s>>>(fr, L + C.off_split, 1, fac, F->d_dofs, d_x, n);
            else k_bwd_cta<T, true><<<g, 256, sm, s>>>(fr, L + C.off_split, 1, fac, F->d_dofs, d_x, n);
        }
        if (C.n_cta) {
            dim3 g(C.n_cta, nrhs);
            size_t sm = dgs + (size_t)C.maxm_cta * sizeof(T);
            if (!trans) k_bwd_cta<T, false><<<g, 256, sm, s>>>(fr, L + C.off_cta, 0, fac, F->d_dofs, d_x, n);
            else k_bwd_cta<T, true><<<g, 256, sm, s>>>(fr, L + C.off_cta, 0, fac, F->d_dofs, d_x, n);
        }
        if (C.n_small) {
            dim3 g((C.n_small + 7) / 8, nrhs);
            if (!trans) k_bwd_warp<T, false><<<g, 256, 0, s>>>(fr, L + C.off_small, C.n_small, fac, F->d_dofs, d_x, n);
            else k_bwd_warp<T, true><<<g, 256, 0, s>>>(fr, L + C.off_small, C.n_small, fac, F->d_dofs, d_x, n);
        }
        prof_end(F, s, slot);
        CUDA_TRY(cudaGetLastError());
    }
    return MF_OK;
}

static int solve_common(mf_factors* F, double* d_rhs, int nrhs, bool trans, mf_stream_t stream) {
    if (!F || !d_rhs || nrhs < 1) return MF_EINVAL;
    if (!F->factored) return MF_EINVAL;
    if (nrhs > F->max_nrhs) return MF_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    return F->prec == MF_F64 ? run_solve<double>(F, d_rhs, nrhs, trans, s) : run_solve<float>(F, d_rhs, nrhs, trans, s);
}

extern "C" int mf_solve(mf_factors* F, double* d_rhs, int nrhs, mf_stream_t stream) {
    return solve_common(F, d_rhs, nrhs, false, stream);
}

extern "C" int mf_solve_adjoint(mf_factors* F, double* d_rhs, int nrhs, mf_stream_t stream) {
    return solve_common(F, d_rhs, nrhs, true, stream);
}

static int residual_into(const mf_factors* Fc, const double* d_values, const double* d_x, const double* d_b, double* d_r,
                         int nrhs, cudaStream_t s) {
    mf_factors* F = const_cast<mf_factors*>(Fc);
    const mf_analysis* a = F->a;
    const int64_t nE = a->n_elem * a->npe;
    int slot = prof_begin(F, s, FAM_RESID, F->resid_bytes * nrhs, F->resid_flops * nrhs, 2);
    dim3 g1((unsigned)((nE + 255) / 256), nrhs);
    k_elem_apply<<<g1, 256, 0, s>>>(d_values, F->d_en, d_x, F->d_Y, a->n_elem, a->npe, a->n_dof, 0);
    CUDA_TRY(cudaGetLastError());
    dim3 g2((unsigned)((a->n_dof + 255) / 256), nrhs);
    k_gather_residual<<<g2, 256, 0, s>>>(F->d_node_ptr, F->d_node_inc, F->d_Y, d_b, d_r, a->n_dof, nE, 0);
    prof_end(F, s, slot);
    CUDA_TRY(cudaGetLastError());
    return MF_OK;
}

extern "C" int mf_residual(const mf_factors* F, const double* d_values, const double* d_x, const double* d_b, double* d_r,
                           int nrhs, mf_stream_t stream) {
    if (!F || !d_values || !d_x || !d_b || !d_r || nrhs < 1 || nrhs > F->max_nrhs) return MF_EINVAL;
    return residual_into(F, d_values, d_x, d_b, d_r, nrhs, (cudaStream_t)stream);
}

static int compute_rowabs(mf_factors* F, const double* d_values, cudaStream_t s) {
    const mf_analysis* a = F->a;
    const int64_t nE = a->n_elem * a->npe;
    dim3 g1((unsigned)((nE + 255) / 256), 1);
    k_elem_apply<<<g1, 256, 0, s>>>(d_values, F->d_en, nullptr, F->d_Y, a->n_elem, a->npe, a->n_dof, 1);
    CUDA_TRY(cudaGetLastError());
    dim3 g2((unsigned)((a->n_dof + 255) / 256), 1);
    k_gather_residual<<<g2, 256, 0, s>>>(F->d_node_ptr, F->d_node_inc, F->d_Y, nullptr, F->d_rowabs, a->n_dof, nE, 1);
    CUDA_TRY(cudaGetLastError());
    F->rowabs_valid = true;
    F->rowabs_values = d_values;
    return MF_OK;
}

extern "C" int mf_refine_solve(mf_factors* F, const double* d_values, const double* d_b, double* d_x, int nrhs, double tol,
                               int maxit, mf_refine_info* info, mf_stream_t stream) {
    if (!F || !d_values || !d_b || !d_x || nrhs < 1 || nrhs > F->max_nrhs || maxit < 0) return MF_EINVAL;
    if (!F->factored) return MF_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    const mf_analysis* a = F->a;
    const int64_t n = a->n_dof;
    int rc;
    if (!F->rowabs_valid || F->rowabs_values != d_values)
        if ((rc = compute_rowabs(F, d_values, s))) return rc;
    int slot = prof_begin(F, s, FAM_OTHER, 16.0 * n * nrhs, 0, 0);
    CUDA_TRY(cudaMemcpyAsync(d_x, d_b, sizeof(double) * n * nrhs, cudaMemcpyDeviceToDevice, s));
    prof_end(F, s, slot);
    if ((rc = mf_solve(F, d_x, nrhs, stream))) return rc;
    std::vector<double> h(6 * nrhs);
    int it = 0;
    double eta = 0, rel = 0;
    for (;;) {
        if ((rc = residual_into(F, d_values, d_x, d_b, F->d_r, nrhs, s))) return rc;
        dim3 gp(F->norm_blocks, nrhs);
        int slot = prof_begin(F, s, FAM_RESID, 24.0 * n * nrhs, 5.0 * n * nrhs, 2);
        k_norms_partial<<<gp, 256, 0, s>>>(F->d_r, d_x, d_b, F->d_rowabs, n, F->d_part);
        k_norms_final<<<nrhs, 32, 0, s>>>(F->d_part, F->norm_blocks, F->d_norms);
        prof_end(F, s, slot);
        CUDA_TRY(cudaGetLastError());
        CUDA_TRY(cudaMemcpyAsync(h.data(), F->d_norms, sizeof(double) * 6 * nrhs, cudaMemcpyDeviceToHost, s));
        CUDA_TRY(cudaStreamSynchronize(s));
        const double anorm = h[5];
        eta = 0;
        rel = 0;
        for (int r = 0; r < nrhs; r++) {
            const double* q = &h[6 * r];
            double den = anorm * q[1] + q[2];
            double e = den > 0 ? q[0] / den : (q[0] > 0 ? INFINITY : 0.0);
            eta = std::max(eta, e);
            rel = std::max(rel, q[4] > 0 ? std::sqrt(q[3] / q[4]) : std::sqrt(q[3]));
        }
        if (eta <= tol || it >= maxit || !std::isfinite(eta)) break;
        slot = prof_begin(F, s, FAM_OTHER, 16.0 * n * nrhs, 0, 0);
        CUDA_TRY(cudaMemcpyAsync(F->d_d, F->d_r, sizeof(double) * n * nrhs, cudaMemcpyDeviceToDevice, s));
        prof_end(F, s, slot);
        if ((rc = mf_solve(F, F->d_d, nrhs, stream))) return rc;
        slot = prof_begin(F, s, FAM_OTHER, 24.0 * n * nrhs, 1.0 * n * nrhs);
        k_axpy<<<(unsigned)((n * nrhs + 255) / 256), 256, 0, s>>>(d_x, F->d_d, n * nrhs);
        prof_end(F, s, slot);
        CUDA_TRY(cudaGetLastError());
        it++;
    }
    if (info) {
        info->iterations = it;
        info->backward_error = eta;
        info->rel_residual = rel;
    }
    return eta <= tol ? MF_OK : MF_ENOCONV;
}

extern "C" int mf_element_grad(const mf_factors* F, const double* d_dvalues, const double* d_lambda, const double* d_x,
                               double* d_grad, mf_stream_t stream) {
    if (!F || !d_dvalues || !d_lambda || !d_x || !d_grad) return MF_EINVAL;
    const mf_analysis* a = F->a;
    int64_t threads = a->n_elem * 32;
    k_element_grad<<<(unsigned)((threads + 255) / 256), 256, 0, (cudaStream_t)stream>>>(d_dvalues, F->d_en, d_lambda, d_x,
                                                                                         d_grad, a->n_elem, a->npe);
    CUDA_TRY(cudaGetLastError());
    return MF_OK;
}

extern "C" int mf_element_outer(const mf_factors* F, const double* d_lambda, const double* d_x, int nrhs, double* d_gradK,
                                mf_stream_t stream) {
    if (!F || !d_lambda || !d_x || !d_gradK || nrhs < 1) return MF_EINVAL;
    const mf_analysis* a = F->a;
    int64_t n = a->n_elem * a->npe * a->npe;
    k_element_outer<<<(unsigned)((n + 255) / 256), 256, 0, (cudaStream_t)stream>>>(F->d_en, d_lambda, d_x, d_gradK,
                                                                                    a->n_elem, a->npe, a->n_dof, nrhs);
    CUDA_TRY(cudaGetLastError());
    return MF_OK;
}

extern "C" int mf_status(mf_factors* F, mf_status_info* out) {
    if (!F || !out) return MF_EINVAL;
    CUDA_TRY(cudaDeviceSynchronize());
    DevStatus h{};
    CUDA_TRY(cudaMemcpy(&h, F->d_status, sizeof(h), cudaMemcpyDeviceToHost));
    out->n_perturbed = (int64_t)h.n_perturbed;
    if (h.first == ~0ull) {
        out->first_front = -1;
        out->first_pivot = -1;
    } else {
        out->first_front = (int32_t)(h.first >> 32);
        out->first_pivot = (int32_t)(h.first & 0xffffffffu);
    }
    out->nonfinite = h.nonfinite;
    out->timeout = h.timeout;
    if (h.timeout) return MF_ETIMEOUT;
    if (F->opt.pivot_fail && h.n_perturbed > 0) return MF_EZERO_PIVOT;
    return MF_OK;
}

extern "C" int mf_factors_export_front(const mf_factors* F, int32_t front, double* L, double* U) {
    if (!F || !F->factored || front < 0 || front >= F->a->n_front || !L || !U) return MF_EINVAL;
    const FrontDev& fr = F->a->fronts[front];
    const int64_t m = fr.m, k = fr.k;
    CUDA_TRY(cudaDeviceSynchronize());
    std::vector<double> P(m * k), R(k * (m - k));
    if (F->prec == MF_F64) {
        if (m * k) CUDA_TRY(cudaMemcpy(P.data(), (double*)F->d_fac + fr.P_off, sizeof(double) * m * k, cudaMemcpyDeviceToHost));
        if (k * (m - k))
            CUDA_TRY(cudaMemcpy(R.data(), (double*)F->d_fac + fr.R_off, sizeof(double) * k * (m - k), cudaMemcpyDeviceToHost));
    } else {
        std::vector<float> Pf(m * k), Rf(k * (m - k));
        if (m * k) CUDA_TRY(cudaMemcpy(Pf.data(), (float*)F->d_fac + fr.P_off, sizeof(float) * m * k, cudaMemcpyDeviceToHost));
        if (k * (m - k))
            CUDA_TRY(cudaMemcpy(Rf.data(), (float*)F->d_fac + fr.R_off, sizeof(float) * k * (m - k), cudaMemcpyDeviceToHost));
        std::copy(Pf.begin(), Pf.end(), P.begin());
        std::copy(Rf.begin(), Rf.end(), R.begin());
    }
    for (int64_t j = 0; j < k; j++)
        for (int64_t i = 0; i < m; i++) L[i + j * m] = P[i + j * m];
    for (int64_t j = 0; j < m; j++)
        for (int64_t i = 0; i < k; i++) U[i + j * k] = j < k ? P[i + j * m] : R[i + (j - k) * k];
    return MF_OK;
}

extern "C" int mf_profile_enable(mf_factors* F, int enable) {
    if (!F) return MF_EINVAL;
    F->prof = enable != 0;
    return MF_OK;
}

extern "C" int mf_profile_read(mf_factors* F, double* ms, int64_t* launches, double* bytes, double* flops) {
    if (!F) return MF_EINVAL;
    CUDA_TRY(cudaDeviceSynchronize());
    double t[MF_PROFILE_FAMILIES] = {};
    for (size_t i = 0; i < F->ev_used; i++) {
        float e = 0.f;
        CUDA_TRY(cudaEventElapsedTime(&e, F->ev[2 * i], F->ev[2 * i + 1]));
        t[F->ev_fam[i]] += e;
    }
    for (int q = 0; q < MF_PROFILE_FAMILIES; q++) {
        if (ms) ms[q] = t[q];
        if (launches) launches[q] = F->acc_launch[q];
        if (bytes) bytes[q] = F->acc_bytes[q];
        if (flops) flops[q] = F->acc_flops[q];
        F->acc_launch[q] = 0;
        F->acc_bytes[q] = 0;
        F->acc_flops[q] = 0;
    }
    F->ev_used = 0;
    return MF_OK;
}
