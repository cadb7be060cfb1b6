// Executor: builds the per-class launch plan (the Foata classes of Sec. 3.3
// as a sequence of batched launches, each a bag of independent tasks), owns
// the device arenas, and drives factorization, solves and refinement.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <vector>

#include "kernels_factor.cuh"
#include "kernels_foata.cuh"
#include "kernels_solve.cuh"
#include "kernels_subtree.cuh"
#include "kernels_tc.cuh"
#include "mf_internal.h"

// Host-side fault injection for tests (mf_test_fail_alloc): when >= 0, the
// allocation that brings the countdown from 0 to -1 fails as if the device
// were out of memory.
static std::atomic<long long> g_alloc_countdown{-1};
bool mf_alloc_should_fail() {
    long long c = g_alloc_countdown.load();
    while (c >= 0)
        if (g_alloc_countdown.compare_exchange_weak(c, c - 1)) return c == 0;
    return false;
}

namespace {

enum LaunchKind { K_FUSED = 0, K_ASM = 1, K_PDIAG = 2, K_GEMM = 3, K_INVDIAG = 4, K_SUBTREE = 5, K_GEMMTC = 6, K_GRP = 7,
                  K_TCPACK = 8, K_FOATA = 9, K_FORK = 10, K_JOIN = 11, K_SYMR = 13, K_MIRROR = 14, K_TRSM = 15,
                  K_TCD = 16,
                  K_SYNC = 12 };  // K_SYNC: stream `stream` waits for what stream `bucket` issued so far (event `off`)

struct Launch {
    int kind;
    int cls;
    int count;
    int maxm;     // fused: bucket bound (shared-memory size)
    int64_t off;  // offset into the list of its kind
    int bucket = -1;  // fused: size bucket (index into kFusedBounds)
    int threads = 0;  // fused: threads per CTA
    int stream = 0;   // 0: the caller's stream; 1: the side stream (pivot-block inverses); 2: the lookahead stream
    int wide = 0;     // K_PDIAG of FP32 fronts: factor the pivot blocks in FP64 (root separator classes)
    int kmax = 0;     // fused: largest pivot count of the launch's fronts (picks the blocked form)
};

// Solve plan of one class: fronts split by size (see kernels_solve.cuh).
// Lane-group substitution kernels for small fronts with few pivots: (lanes per front G, rows per
// lane R, pivot bound KM) of each list, chosen by m (G R >= m) and k (k <= KM).
constexpr int kLgLists = 15;
constexpr int kLgG[kLgLists] = {4, 4, 4, 4, 4, 4, 8, 8, 8, 16, 16, 16, 32, 32, 32};
constexpr int kLgR[kLgLists] = {1, 2, 2, 4, 4, 4, 4, 4, 4, 4, 4, 4, 3, 3, 3};
// several right-hand sides per launch (each lane carries R x kRhsChunk values): one row per lane
// up to 32 rows, so the same lists run at full occupancy
constexpr int kLgGm[kLgLists] = {4, 8, 8, 16, 16, 16, 32, 32, 32, 32, 32, 32, 32, 32, 32};
constexpr int kLgRm[kLgLists] = {1, 1, 1, 1, 1, 1, 1, 1, 1, 2, 2, 2, 3, 3, 3};
constexpr int kLgKM[kLgLists] = {4, 4, 8, 4, 8, 16, 4, 8, 16, 4, 8, 16, 4, 8, 16};
static int lg_list_of(int m, int k) {
    const int base = m <= 4 ? 0 : m <= 8 ? 1 : m <= 16 ? 3 : m <= 32 ? 6 : m <= 64 ? 9 : m <= 96 ? 12 : -1;
    if (base < 0) return -1;
    const int n = base == 0 ? 1 : base == 1 ? 2 : 3;  // pivot bounds of this size group
    for (int q = base; q < base + n; q++)
        if (k <= kLgKM[q]) return q;
    return -1;
}
struct ClassList {
    int n_small, n_cta, n_piv, n_all;
    int n_lg[kLgLists];           // small fronts with few pivots, per lane-group list
    int64_t off_lg[kLgLists];
    int n_grp[4];                 // fronts with m <= 4, 8, 16, 32 (lane groups of 4, 8, 16, 32)
    int maxm_cta, maxin_inv, maxk_inv, maxnc_inv;
    int64_t off_small, off_cta;   // into the solve front list
    int64_t off_grp[4];
    int64_t off_piv, off_all;     // into the row-block list (inverse fronts)
};
constexpr int kSolveWarpMax = 64;   // m <= this: one warp per front
constexpr int kSweepMaxFronts = 2048;  // classes with at most this many fronts join the persistent sweep

#define CUDA_TRY(x)                          \
    do {                                     \
        cudaError_t e__ = (x);               \
        if (e__ != cudaSuccess) {            \
            (void)cudaGetLastError();        \
            return MF_ECUDA;                 \
        }                                    \
    } while (0)

// Launch with programmatic stream serialization: the kernel may be scheduled
// while the previous kernel of its stream drains; it reads launch-invariant
// data first and waits (griddepcontrol.wait) for that kernel's results before
// touching anything an earlier kernel writes (pdl_wait in kernels_factor.cuh).
// Only kernels that call pdl_wait are launched this way.
template <typename A>
struct NoDeduce {
    using type = A;
};
template <typename... KArgs>
static cudaError_t launch_dep(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                              typename NoDeduce<KArgs>::type... args) {  // converted to the kernel's parameter types
    void* argv[] = {(void*)&args...};
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelExC(&cfg, (const void*)kern, argv);
}

template <typename T>
int dev_alloc(T** p, size_t n) {
    *p = nullptr;
    if (n == 0) n = 1;
    if (mf_alloc_should_fail()) return MF_ENOMEM;
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

constexpr int kFusedBlockedMaxK = 32;  // fused fronts: blocked partial LU when every front has k <= this
constexpr int kPanelNB64 = 32;  // panel width (pivot block of a step), FP64
constexpr int kPanelNB32 = 64;  // FP32

__global__ void k_init_status(DevStatus* st) {
    st->n_perturbed = 0ull;
    st->first = ~0ull;
    st->nonfinite = 0;
    st->timeout = 0;
}

// Subtree fusion plan: disjoint subtrees covering every front of height <= h.
struct SubtreePlan {
    int h = 0;
    std::vector<SubtreeTask> tasks;
    std::vector<SubtreeEntry> ecb, euv;  // factor (CB pool) and solve (update-vector pool) entries
    SubtreeLayout lay_f{0, 0}, lay_s{0, 0};
    size_t smem_f = 0, smem_s = 0;
    double bytes = 0, flops = 0;
};

// first-fit offset for `size` elements among live [off, off+size) ranges
int32_t first_fit(std::vector<std::pair<int32_t, int32_t>> live, int32_t size) {
    std::sort(live.begin(), live.end());
    int32_t off = 0;
    for (const auto& r : live) {
        if (off + size <= r.first) break;
        off = std::max(off, r.first + r.second);
    }
    return off;
}

bool subtree_try(const mf_analysis* a, int h, size_t tsize, size_t budget, SubtreePlan& SP, bool factor = true) {
    SP = SubtreePlan{};
    SP.h = h;
    const std::vector<FrontDev>& Fr = a->fronts;
    std::vector<int32_t> roots;
    for (int32_t f = 0; f < a->n_front; f++)
        if (Fr[f].cls < h && (a->parent[f] < 0 || Fr[a->parent[f]].cls >= h)) roots.push_back(f);
    std::stable_sort(roots.begin(), roots.end(), [&](int32_t x, int32_t y) { return Fr[x].cls > Fr[y].cls; });
    int32_t work_max = 1, pcb_max = 1, puv_max = 1;
    const double T = (double)tsize;
    std::vector<int32_t> cboff(a->n_front, -1), uvoff(a->n_front, -1);
    for (int32_t root : roots) {
        const int nl = Fr[root].cls + 1;
        if (nl > kSubMaxLevels) return false;
        std::vector<std::vector<int32_t>> lev(nl);
        std::vector<int32_t> stack{root};
        while (!stack.empty()) {
            int32_t f = stack.back();
            stack.pop_back();
            lev[Fr[f].cls].push_back(f);
            for (int c = 0; c < Fr[f].nchild; c++) stack.push_back(Fr[f].child[c]);
        }
        SubtreeTask t{};
        t.first = (int32_t)SP.ecb.size();
        t.n_levels = nl;
        // live allocations: (off, size) with the level at which they are freed
        std::vector<std::pair<int32_t, int32_t>> live_cb, live_uv;
        std::vector<int> free_cb, free_uv;
        for (int L = 0; L < nl; L++) {
            std::sort(lev[L].begin(), lev[L].end());
            for (size_t i = live_cb.size(); i-- > 0;)
                if (free_cb[i] <= L) {
                    live_cb.erase(live_cb.begin() + i);
                    free_cb.erase(free_cb.begin() + i);
                }
            for (size_t i = live_uv.size(); i-- > 0;)
                if (free_uv[i] <= L) {
                    live_uv.erase(live_uv.begin() + i);
                    free_uv.erase(free_uv.begin() + i);
                }
            t.level_ptr[L] = (int32_t)SP.ecb.size() - t.first;
            int mmax = 1;
            for (int32_t f : lev[L]) {
                const FrontDev& fr = Fr[f];
                if (fr.m > kSubMaxM) return false;
                mmax = std::max(mmax, fr.m);
                SubtreeEntry ec{f, -1, {-1, -1}}, eu{f, -1, {-1, -1}};
                for (int c = 0; c < fr.nchild; c++) {
                    ec.child_off[c] = cboff[fr.child[c]];
                    eu.child_off[c] = uvoff[fr.child[c]];
                }
                const int32_t nc = fr.m - fr.k;
                if (f != root) {
                    const int fl = Fr[a->parent[f]].cls + 1;
                    ec.cb_off = first_fit(live_cb, nc * nc);
                    live_cb.push_back({ec.cb_off, nc * nc});
                    free_cb.push_back(fl);
                    pcb_max = std::max(pcb_max, ec.cb_off + nc * nc);
                    eu.cb_off = first_fit(live_uv, nc);
                    live_uv.push_back({eu.cb_off, nc});
                    free_uv.push_back(fl);
                    puv_max = std::max(puv_max, eu.cb_off + nc);
                }
                cboff[f] = ec.cb_off;
                uvoff[f] = eu.cb_off;
                SP.ecb.push_back(ec);
                SP.euv.push_back(eu);
                // algorithmic work: inputs once, outputs once
                if (fr.nchild == 0) SP.bytes += 8.0 * a->npe * a->npe;
                SP.bytes += T * ((double)fr.m * fr.k + (double)fr.k * nc) + (f == root ? T * nc * nc : 0.0);
                double am = fr.m - fr.k, bm = fr.m - 1;
                if (fr.k > 0)
                    SP.flops += (am + bm) * (bm - am + 1) / 2.0 +
                                2.0 * (bm * (bm + 1) * (2 * bm + 1) / 6.0 - (am - 1) * am * (2 * am - 1) / 6.0);
            }
            t.level_mmax[L] = mmax;
            const int nlf = (int)lev[L].size();
            const int slots = nlf >= 4 ? std::min(nlf, 8) : 1;
            work_max = std::max(work_max, slots * (mmax | 1) * mmax);
        }
        t.level_ptr[nl] = (int32_t)SP.ecb.size() - t.first;
        SP.tasks.push_back(t);
    }
    SP.lay_f = {work_max, pcb_max};
    SP.lay_s = {0, puv_max};
    SP.smem_f = (size_t)(work_max + pcb_max) * tsize + 8 * 2 * kSubMaxM * sizeof(int32_t) + 64;
    SP.smem_s = (size_t)puv_max * tsize + 16;
    return (!factor || SP.smem_f <= budget) && SP.smem_s <= budget;
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
    int tc_min = 256;
    int bf16_min = 2048;  // MF_TF32_BF16: smallest contribution block with BF16 Schur products
    int sp = 256;  // super-panel depth (pivots)
    int num_sms = 148;
    int max_nrhs = 4;
    // device
    FrontDev* d_fronts = nullptr;
    int32_t* d_dofs = nullptr;
    int32_t* d_maps = nullptr;
    int64_t* d_vsrc = nullptr;  // per front row and child: the child's update-vector index holding it, or -1
    int64_t* d_en = nullptr;
    int64_t* d_node_ptr = nullptr;
    int64_t* d_node_inc = nullptr;
    void* d_fac = nullptr;
    void* d_cb = nullptr;
    void* d_vec = nullptr;
    int32_t* d_flist = nullptr;
    FactorRec* d_frec = nullptr;  // the fused / lane-group launch lists as compact records
    // scalar-task Foata executor of the bottom classes: fronts' workspace offsets (parallel to the
    // factor list), the dense front workspace W and the products' workspace X
    int foata_cls = 0;
    bool sym = false;                 // symmetric factors and solves (option symmetric)
    int64_t* d_pdiag = nullptr;       // symmetric solves: factor-arena offset of each dof's pivot
    double* d_pdv = nullptr;          // the same pivots gathered per dof at the end of each factorization
    AsmTile* d_symt = nullptr;        // tiles of the symmetric-mode R copies and S mirrors
    TrsmTask* d_trsm = nullptr;       // triangular-solve panel tasks
    TcTileD* d_gtcd = nullptr;        // tensor-core tiles that split their own operands
    bool tcd = false;                 // 3xTF32 products without the pack pass (option tc_direct)
    bool pinv = true;                 // panel products through explicit pivot-block inverses (default)
    int64_t* d_fwoff = nullptr;
    void* d_fws = nullptr;
    void* d_fxs = nullptr;
    int64_t fws_size = 0;
    int32_t* d_slist = nullptr;
    SolveRec* d_srec = nullptr;  // the substitution list as compact records
    RowBlock* d_rows = nullptr;
    InvTask* d_invt = nullptr;
    void* d_inv = nullptr;
    void* d_scr = nullptr;
    void* d_ys = nullptr;
    int64_t scr_size = 1;
    AsmRec* d_asm = nullptr;
    DiagTask* d_panel = nullptr;
    void* d_pnl = nullptr;
    int64_t pnl_size = 64 * 64;
    GemmTile* d_gemm = nullptr;
    TcTile* d_gtc = nullptr;    // tensor-core (128 x 256) Schur tiles
    TcPack* d_tcpack = nullptr;  // per tensor-core front: packed operand offsets
    TcPackJob* d_tcjob = nullptr;
    float* d_pk = nullptr;       // packed hi/lo operands of one class (reused class by class)
    int64_t pk_size = 0;
    float* d_pk2 = nullptr;      // the same for the side stream (pivot-block inverses)
    int64_t pk2_size = 0;
    cudaStream_t s1 = nullptr;   // main factorization stream at the highest priority (with s2 / s3)
    cudaEvent_t s1_in = nullptr, s1_out = nullptr;
    cudaStream_t s2 = nullptr;   // side stream: pivot-block inverses overlap the later classes
    cudaStream_t sfan[3] = {};   // the independent kernels of one substitution class run side by side
    cudaEvent_t fan_in = nullptr, fan_out[3] = {};
    bool fan_off = false;        // set while a conditional-node body is captured (single stream there)
    std::vector<cudaEvent_t> fork_ev;
    cudaEvent_t join_ev = nullptr;
    int n_forks = 0;
    bool la = false;             // one-panel lookahead in the large-front partial LU
    cudaStream_t s3 = nullptr;   // lookahead stream: the next pivot block beside the trailing update
    std::vector<cudaEvent_t> sync_ev;
    int n_sync = 0;
    unsigned int* d_famax = nullptr;
    DevStatus* d_status = nullptr;
    // CSR analyses: destination of each CSR entry in the arrowhead element array, and that array
    int64_t* d_csr_dest = nullptr;
    double* d_elemvals = nullptr;
    double *d_r = nullptr, *d_d = nullptr, *d_Y = nullptr, *d_rowabs = nullptr, *d_part = nullptr, *d_norms = nullptr;
    double* d_colabs = nullptr;  // column sums of |A| (||A^T||_inf of the adjoint refinement)
    // conjugate-gradient refinement: search direction p, s = -A p, a zero right-hand side, scalars
    double *d_cgp = nullptr, *d_cgs = nullptr, *d_zero = nullptr, *d_cg = nullptr;
    // device-side CG loop (a while-conditional graph node): stop-test parameters (tol, iteration
    // limit), the iteration counter, and the stream that captures the loop body
    double* d_cgpar = nullptr;
    int* d_cgit = nullptr;
    cudaStream_t s_body = nullptr;
    cudaStream_t s_aux = nullptr;   // captures the solves that loop bodies take as child-graph nodes
    bool loop_failed = false;  // a loop graph could not be built here: iterate from the host
    int loop_first_inc = 0;    // 1 when the loop graph's first step counts as an iteration (CG)
    bool colabs_valid = false;
    const double* colabs_values = nullptr;
    int norm_blocks = 296;
    bool rowabs_valid = false;
    const double* rowabs_values = nullptr;
    // subtree fusion of the bottom classes
    SubtreePlan sub;   // subtree fusion of the bottom classes' factorization
    SubtreePlan subs;  // ... and of their substitutions
    SubtreeTask* d_sub_tasks = nullptr;
    SubtreeEntry* d_sub_ecb = nullptr;
    SubtreeEntry* d_sub_euv = nullptr;
    SubtreeTask* d_subs_tasks = nullptr;
    SubtreeEntry* d_subs_euv = nullptr;
    // captured CUDA graphs, keyed by the buffers they were captured with
    struct GraphEntry {
        int kind;  // 0 factor, 1 refine start, 2 refine step
        const void* p[3];
        int nrhs;
        cudaGraphExec_t exec;
        int64_t launches[MF_PROFILE_FAMILIES];  // what one replay adds to the accounting
        double bytes[MF_PROFILE_FAMILIES], flops[MF_PROFILE_FAMILIES];
    };
    std::vector<GraphEntry> graphs;
    // plan
    std::vector<Launch> plan;
    std::vector<ClassList> classes_f, classes_b;  // substitution lists per class (forward, backward)
    // persistent substitution sweeps: phase tables, shared-memory size, bytes/flops per sweep
    std::vector<SweepPhase> sweep_f, sweep_b;
    SweepPhase* d_sweep_f = nullptr;
    SweepPhase* d_sweep_b = nullptr;
    size_t sweep_smem_f = 0, sweep_smem_b = 0;
    unsigned int* d_bar = nullptr;
    bool use_sweep = true;
    int sweep_c0 = 0;  // classes >= sweep_c0 run in the persistent sweeps, the ones below per class
    bool factored = false;
    // algorithmic work per plan entry / per class and direction (per rhs)
    std::vector<double> plan_bytes, plan_flops;
    std::vector<int> plan_fam;
    std::vector<double> fwd_bytes, bwd_bytes, fwd_flops, bwd_flops;
    double resid_bytes = 0, resid_flops = 0;
    // profiling
    bool prof = false;
    std::vector<cudaEvent_t> ev;  // pairs
    std::vector<mf_trace_rec> ev_rec;  // per event pair: family, kind, class, tasks (ms filled on read)
    std::vector<int> ev_tag;           // fused launches: size bucket; otherwise -1
    size_t ev_used = 0;
    double acc_bytes[MF_PROFILE_FAMILIES] = {};
    double acc_flops[MF_PROFILE_FAMILIES] = {};
    int64_t acc_launch[MF_PROFILE_FAMILIES] = {};
    // work of one body pass of the device-side CG loop (recorded when its graph is captured), so
    // the accounting can follow the number of passes each replay actually ran
    double body_bytes[MF_PROFILE_FAMILIES] = {};
    double body_flops[MF_PROFILE_FAMILIES] = {};
    int64_t body_launch[MF_PROFILE_FAMILIES] = {};
    // solves of F->d_d captured on their own (class kernels side by side) before a loop graph is
    // captured, entered into the loop body as one child-graph node, with their launch accounting
    struct BodySolve {
        int nrhs;
        bool trans;
        cudaGraph_t graph;
        double bytes[MF_PROFILE_FAMILIES], flops[MF_PROFILE_FAMILIES];
        int64_t launches[MF_PROFILE_FAMILIES];
    };
    std::vector<BodySolve> body_solves;
};

enum Family { FAM_FUSED = 0, FAM_ASM = 1, FAM_PANEL = 2, FAM_TRAIL = 3, FAM_SCHUR = 4, FAM_FWD = 5, FAM_BWD = 6,
              FAM_RESID = 7, FAM_OTHER = 8, FAM_INV = 9 };

// Bracket one launch: returns a slot index (or -1 when profiling is off).
// Symmetric solves with per-class launches only (no subtree or persistent sweep planned) take the
// D scaling inside the forward kernels; the factorization then skips gathering the pivots.
static bool scaling_folded(const mf_factors* F) { return F->sym && !F->use_sweep && F->subs.h < 2; }

static int prof_begin(mf_factors* F, cudaStream_t s, int fam, double bytes, double flops, int kernels = 1,
                      int tag = -1, int kind = MF_TRACE_OTHER, int cls = -1, int tasks = 0) {
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
        F->ev_rec.resize(F->ev.size() / 2);
        F->ev_tag.resize(F->ev.size() / 2);
    }
    int slot = (int)F->ev_used++;
    F->ev_rec[slot] = mf_trace_rec{fam, kind, cls, tasks, 0.0, bytes, flops};
    F->ev_tag[slot] = tag;
    cudaEventRecord(F->ev[2 * slot], s);
    return slot;
}

static void prof_end(mf_factors* F, cudaStream_t s, int slot) {
    if (slot >= 0) cudaEventRecord(F->ev[2 * slot + 1], s);
}

static void free_factors(mf_factors* f) {
    if (!f) return;
    for (cudaEvent_t e : f->fork_ev)
        if (e) cudaEventDestroy(e);
    if (f->join_ev) cudaEventDestroy(f->join_ev);
    if (f->s1) cudaStreamDestroy(f->s1);
    if (f->s_body) cudaStreamDestroy(f->s_body);
    if (f->s_aux) cudaStreamDestroy(f->s_aux);
    if (f->s1_in) cudaEventDestroy(f->s1_in);
    if (f->s1_out) cudaEventDestroy(f->s1_out);
    if (f->s2) cudaStreamDestroy(f->s2);
    for (int j = 0; j < 3; j++) {
        if (f->sfan[j]) cudaStreamDestroy(f->sfan[j]);
        if (f->fan_out[j]) cudaEventDestroy(f->fan_out[j]);
    }
    if (f->fan_in) cudaEventDestroy(f->fan_in);
    if (f->s3) cudaStreamDestroy(f->s3);
    for (cudaEvent_t e : f->sync_ev)
        if (e) cudaEventDestroy(e);
    for (auto& g : f->graphs) cudaGraphExecDestroy(g.exec);
    for (auto& b : f->body_solves) cudaGraphDestroy(b.graph);
    for (cudaEvent_t e : f->ev) cudaEventDestroy(e);
    void* ptrs[] = {f->d_fronts, f->d_dofs, f->d_maps, f->d_vsrc, f->d_en, f->d_node_ptr, f->d_node_inc, f->d_fac, f->d_cb,
                    f->d_vec, f->d_flist, f->d_frec, f->d_fwoff, f->d_fws, f->d_fxs, f->d_pdiag, f->d_pdv, f->d_symt, f->d_trsm, f->d_gtcd, f->d_cgp, f->d_cgs, f->d_zero, f->d_cg, f->d_cgpar, f->d_cgit, f->d_slist, f->d_srec, f->d_rows, f->d_invt, f->d_inv, f->d_scr, f->d_ys, f->d_asm, f->d_panel, f->d_pnl, f->d_gemm, f->d_gtc, f->d_tcpack, f->d_tcjob, f->d_pk, f->d_pk2, f->d_sweep_f, f->d_sweep_b, f->d_bar, f->d_sub_tasks, f->d_sub_ecb, f->d_sub_euv, f->d_subs_tasks, f->d_subs_euv, f->d_famax, f->d_status,
                    f->d_csr_dest, f->d_elemvals, f->d_r, f->d_d, f->d_Y, f->d_rowabs, f->d_part, f->d_norms, f->d_colabs};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    delete f;
}

// Replay the graph captured for (kind, p0, p1, p2, nrhs) on stream s, capturing
// `enqueue` first if there is none.  Graphs need a capturable stream: the
// legacy default stream (NULL) runs `enqueue` directly.
template <typename Fn>
static int run_graph(mf_factors* F, int kind, const void* p0, const void* p1, const void* p2, int nrhs, cudaStream_t s,
                     Fn enqueue) {
    if (!F->opt.use_graph || F->prof || s == nullptr) return enqueue(s);
    for (auto& g : F->graphs)
        if (g.kind == kind && g.p[0] == p0 && g.p[1] == p1 && g.p[2] == p2 && g.nrhs == nrhs) {
            CUDA_TRY(cudaGraphLaunch(g.exec, s));
            for (int q = 0; q < MF_PROFILE_FAMILIES; q++) {
                F->acc_launch[q] += g.launches[q];
                F->acc_bytes[q] += g.bytes[q];
                F->acc_flops[q] += g.flops[q];
            }
            return MF_OK;
        }
    int64_t l0[MF_PROFILE_FAMILIES];
    double b0[MF_PROFILE_FAMILIES], f0[MF_PROFILE_FAMILIES];
    for (int q = 0; q < MF_PROFILE_FAMILIES; q++) {
        l0[q] = F->acc_launch[q];
        b0[q] = F->acc_bytes[q];
        f0[q] = F->acc_flops[q];
    }
    cudaGraph_t graph = nullptr;
    CUDA_TRY(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
    int rc = enqueue(s);
    cudaError_t e = cudaStreamEndCapture(s, &graph);
    if (rc != MF_OK || e != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        (void)cudaGetLastError();
        return rc != MF_OK ? rc : MF_ECUDA;
    }
    cudaGraphExec_t exec = nullptr;
    e = cudaGraphInstantiate(&exec, graph, cudaGraphInstantiateFlagUseNodePriority);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        return MF_ECUDA;
    }
    // keep a handful per kind
    int same = 0;
    for (auto& g : F->graphs) same += g.kind == kind;
    if (same >= 4)
        for (size_t i = 0; i < F->graphs.size(); i++)
            if (F->graphs[i].kind == kind) {
                cudaGraphExecDestroy(F->graphs[i].exec);
                F->graphs.erase(F->graphs.begin() + i);
                break;
            }
    mf_factors::GraphEntry ge{};
    ge.kind = kind;
    ge.p[0] = p0;
    ge.p[1] = p1;
    ge.p[2] = p2;
    ge.nrhs = nrhs;
    ge.exec = exec;
    for (int q = 0; q < MF_PROFILE_FAMILIES; q++) {  // the capture already counted this first run
        ge.launches[q] = F->acc_launch[q] - l0[q];
        ge.bytes[q] = F->acc_bytes[q] - b0[q];
        ge.flops[q] = F->acc_flops[q] - f0[q];
    }
    F->graphs.push_back(ge);
    CUDA_TRY(cudaGraphLaunch(exec, s));
    return MF_OK;
}

template <typename T>
static size_t fused_smem(int maxm) {
    int ldm = maxm | 1;
    return (size_t)ldm * maxm * sizeof(T) + (size_t)maxm * sizeof(T) + 2 * (size_t)maxm * sizeof(int32_t) + 32 * sizeof(float);
}

static int build_plan(mf_factors* F) {
    const mf_analysis* a = F->a;
    std::vector<int32_t> flist, slist;
    std::vector<int64_t> fwoff;  // parallel to flist: Foata workspace offsets (-1 for other kernels' fronts)
    std::vector<AsmTile> symt;   // symmetric mode: R tiles and S mirror tiles
    std::vector<TrsmTask> trs;   // triangular-solve panel tasks
    std::vector<TcTileD> gtcd;   // direct tensor-core tiles
    std::vector<RowBlock> rows;
    std::vector<InvTask> invt;
    std::vector<AsmRec> asmt;
    std::vector<DiagTask> pan;
    // fronts whose 64 x 64 pivot-block inverses the pivot-block kernel also writes into Q
    std::vector<char> q_from_pdiag(a->n_front, 0);
    auto diag_q = [&](int32_t f) -> int64_t {
        const FrontDev& fr = a->fronts[f];
        if (!F->pinv || F->nb != 64 || fr.q_off < 0) return -1;
        q_from_pdiag[f] = 1;
        return fr.q_off;
    };
    std::vector<GemmTile> gem;
    std::vector<TcTile> gtc;
    std::vector<TcPack> tcp;
    std::vector<TcPackJob> tcj;
    const int* bounds = kFusedBounds;
    const int nbounds = F->prec == MF_F64 ? kFusedBuckets64 : MF_FUSED_BUCKETS;
    const int nb = F->nb;
    const double T = (double)F->tsize;
    double gb = 0, gf = 0;  // running algorithmic counts of the GEMM launch being built
    auto pflops = [](double m, double k) {
        if (k <= 0) return 0.0;
        double a0 = m - k, b0 = m - 1;
        return (a0 + b0) * (b0 - a0 + 1) / 2.0 + 2.0 * (b0 * (b0 + 1) * (2 * b0 + 1) / 6.0 - (a0 - 1) * a0 * (2 * a0 - 1) / 6.0);
    };
    int cur_stream = 0;  // stream the launches being planned go to
    // FP32-family fronts in the top root_f64 classes factor their pivot blocks in FP64
    auto wide_pdiag = [&](int c) { return F->prec != MF_F64 && F->opt.root_f64 > 0 && c >= a->n_cls - F->opt.root_f64; };
    // symmetric fronts: the front's parent is assembled by the large-front kernel, which reads the
    // children's contribution blocks from their lower triangles only
    auto cb_read_lower = [&](int32_t f) {
        const int32_t pa = a->parent[f];
        return pa >= 0 && a->fronts[pa].m > F->small_max && a->fronts[pa].cls >= F->sub.h &&
               a->fronts[pa].cls >= F->foata_cls;
    };
    auto push = [&](Launch L, int fam, double bytes, double flops) {
        L.stream = cur_stream;
        F->plan.push_back(L);
        F->plan_fam.push_back(fam);
        F->plan_bytes.push_back(bytes);
        F->plan_flops.push_back(flops);
    };
    auto gemm_tiles = [&](int64_t a_off, int lda, int64_t b_off, int ldb, int64_t c_off, int ldc, int M, int N, int K,
                          int c_in_cb, bool lower = false) {
        // lower: only the tiles on and below the diagonal (the symmetric Schur update)
        gf += lower ? (double)M * (M + 1) * K : 2.0 * M * N * K;
        gb += T * ((double)M * K + (double)K * N + (lower ? (double)M * (M + 1) : 2.0 * M * N));
        for (int j0 = 0; j0 < N; j0 += 64)
            for (int i0 = 0; i0 < M; i0 += 64) {
                if (lower && i0 + 64 <= j0) continue;
                GemmTile t{};
                t.a_off = a_off; t.b_off = b_off; t.c_off = c_off;
                t.lda = lda; t.ldb = ldb; t.ldc = ldc;
                t.M = M; t.N = N; t.K = K; t.i0 = i0; t.j0 = j0;
                t.a_ar = AR_FAC; t.b_ar = AR_FAC; t.c_ar = c_in_cb ? AR_CB : AR_FAC; t.op = 0;
                gem.push_back(t);
            }
    };
    // Tensor-core products (MF_TF32): C -= A B with min(M, N) >= tc_min, collected per phase
    // (a trailing step, a Schur update), then one pack launch and one GEMM launch per phase.
    struct TcC {
        int8_t car, op;
        int64_t coff;
        int ldc;
    };
    std::vector<TcC> tcc;
    int64_t tc_hi = 0;
    size_t tc_p0 = 0;
    // a product of depth K < 128 (the trailing update of one 64-pivot super-panel) streams C once for
    // few MMAs per output: it stays on the SIMT tiles unless the threshold on M, N is set below 128
    auto use_tc = [&](int M, int N, int K) {
        return (F->prec == MF_TF32 || F->prec == MF_TF32_BF16) && std::min(M, N) >= F->tc_min && K >= 16 &&
               K >= std::min(128, F->tc_min);
    };
    // per product mode (tc::Mode): packing bytes, product bytes and flops of the pending products
    double tc_pbm[3] = {0, 0, 0}, tc_gbm[3] = {0, 0, 0}, tc_gfm[3] = {0, 0, 0};
    auto tc_add = [&](int8_t aar, int64_t aoff, int lda, int8_t bar, int64_t boff, int ldb, int8_t car, int64_t coff,
                      int ldc, int M, int N, int K, int8_t op = 0, int8_t am = 0, int8_t bm = 0, int mode = tc::kTf32x3,
                      bool lower = false) {
        TcPack q{};
        q.a_ar = aar; q.a_off = aoff; q.lda = lda; q.a_mask = am;
        q.b_ar = bar; q.b_off = boff; q.ldb = ldb; q.b_mask = bm;
        q.M = M; q.N = N; q.K = K;
        q.pad[0] = (int8_t)mode;
        q.pad[1] = lower ? 1 : 0;  // only the output tiles that reach the diagonal or below it
        q.nkc = (K + tc::kChunkK - 1) / tc::kChunkK;
        const int nra = (M + tc::kTileM - 1) / tc::kTileM, nrb = (N + tc::kTileN - 1) / tc::kTileN;
        const int ca = tc::chunk_floats_a(mode), cbk = tc::chunk_floats_b(mode);
        q.a_hi = tc_hi;
        tc_hi += (int64_t)nra * q.nkc * ca;
        q.b_hi = tc_hi;
        tc_hi += (int64_t)nrb * q.nkc * cbk;
        tcp.push_back(q);
        tcc.push_back({car, op, coff, ldc});
        tc_gfm[mode] += lower ? (double)M * (M + 1) * K : 2.0 * M * N * K;
        tc_gbm[mode] += T * ((double)M * K + (double)K * N + (lower ? (double)M * (M + 1) : 2.0 * M * N));
        tc_pbm[mode] += T * ((double)M * K + (double)K * N) +
                        (mode == tc::kBf16 ? 1.0 : 2.0) * 4.0 * ((double)nra * ca + (double)nrb * cbk) * q.nkc;
    };
    auto tc_end = [&](int c, int fam) {
        if (tcp.size() > tc_p0) {
            for (size_t qi = tc_p0; qi < tcp.size(); qi++) tcp[qi].lo_off = tc_hi;  // lo chunks after all hi chunks
            bool packed = false;
            if (F->tcd) {  // 3xTF32 products: tiles that read and split their operands themselves
                const int64_t doff = (int64_t)gtcd.size();
                for (size_t qi = tc_p0; qi < tcp.size(); qi++) {
                    const TcPack& q = tcp[qi];
                    if (q.pad[0] != tc::kTf32x3) continue;
                    const int nra = (q.M + tc::kTileM - 1) / tc::kTileM, nrb = (q.N + tc::kTileN - 1) / tc::kTileN;
                    for (int rb = 0; rb < nrb; rb++)
                        for (int ra = 0; ra < nra; ra++) {
                            if (q.pad[1] && (ra + 1) * tc::kTileM <= rb * tc::kTileN) continue;  // above the diagonal
                            TcTileD t{};
                            t.a_ar = q.a_ar; t.a_off = q.a_off; t.lda = q.lda; t.a_mask = q.a_mask;
                            t.b_ar = q.b_ar; t.b_off = q.b_off; t.ldb = q.ldb; t.b_mask = q.b_mask;
                            t.M = q.M; t.N = q.N; t.K = q.K;
                            t.i0 = ra * tc::kTileM;
                            t.j0 = rb * tc::kTileN;
                            t.c_ar = tcc[qi].car;
                            t.op = tcc[qi].op;
                            t.c_off = tcc[qi].coff + t.i0 + (int64_t)t.j0 * tcc[qi].ldc;
                            t.ldc = tcc[qi].ldc;
                            gtcd.push_back(t);
                        }
                }
                if (gtcd.size() > (size_t)doff)
                    push({K_TCD, c, (int)(gtcd.size() - doff), 0, doff}, fam, tc_gbm[tc::kTf32x3], tc_gfm[tc::kTf32x3]);
            }
            for (int mode = F->tcd ? 1 : 0; mode < 3; mode++) {  // one pack and one product launch per mode in use
                const int64_t joff = (int64_t)tcj.size(), toff = (int64_t)gtc.size();
                const int ca = tc::chunk_floats_a(mode), cbk = tc::chunk_floats_b(mode);
                for (size_t qi = tc_p0; qi < tcp.size(); qi++) {
                    TcPack& q = tcp[qi];
                    if (q.pad[0] != mode) continue;
                    const int nra = (q.M + tc::kTileM - 1) / tc::kTileM, nrb = (q.N + tc::kTileN - 1) / tc::kTileN;
                    for (int rt = 0; rt < nra; rt++)
                        for (int kc = 0; kc < q.nkc; kc++) tcj.push_back({(int32_t)(qi - tc_p0), 0, rt, kc});
                    for (int rt = 0; rt < nrb; rt++)
                        for (int kc = 0; kc < q.nkc; kc++) tcj.push_back({(int32_t)(qi - tc_p0), 1, rt, kc});
                    for (int rb = 0; rb < nrb; rb++)
                        for (int ra = 0; ra < nra; ra++) {
                            if (q.pad[1] && (ra + 1) * tc::kTileM <= rb * tc::kTileN) continue;  // above the diagonal
                            TcTile t{};
                            t.a_hi = q.a_hi + (int64_t)ra * q.nkc * ca;
                            t.b_hi = q.b_hi + (int64_t)rb * q.nkc * cbk;
                            t.lo_off = q.lo_off;
                            const int i0 = ra * tc::kTileM, j0 = rb * tc::kTileN;
                            t.c_ar = tcc[qi].car;
                            t.op = tcc[qi].op;
                            t.c_off = tcc[qi].coff + i0 + (int64_t)j0 * tcc[qi].ldc;
                            t.ldc = tcc[qi].ldc;
                            t.mrows = std::min(tc::kTileM, q.M - i0);
                            t.ncols = std::min(tc::kTileN, q.N - j0);
                            t.nkc = q.nkc;
                            gtc.push_back(t);
                        }
                }
                if (gtc.size() == (size_t)toff) continue;
                packed = true;
                push({K_TCPACK, c, (int)(tcj.size() - joff), 0, joff, (int)tc_p0}, fam, tc_pbm[mode], 0.0);
                F->plan.back().wide = mode;
                push({K_GEMMTC, c, (int)(gtc.size() - toff), 0, toff}, fam, tc_gbm[mode], tc_gfm[mode]);
                F->plan.back().wide = mode;
            }
            int64_t& pks = cur_stream ? F->pk2_size : F->pk_size;  // one packed arena per stream
            if (packed) pks = std::max(pks, 2 * tc_hi);
        }
        tc_hi = 0;
        tc_p0 = tcp.size();
        for (int mode = 0; mode < 3; mode++) tc_pbm[mode] = tc_gbm[mode] = tc_gfm[mode] = 0;
    };
    // subtree fusion of the bottom classes
    {
        int want = F->foata_cls > 0 ? 0 : F->opt.subtree_levels;  // the Foata executor takes the bottom classes
        int hmax = want <= 0 ? 0 : std::min(a->n_cls, want);
        hmax = std::min(hmax, kSubMaxLevels);
        int dev = 0, optin = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
        const size_t budget = (size_t)std::min(optin > 0 ? optin : 100000, 200 * 1024);
        F->sub = SubtreePlan{};
        for (int h = hmax; h >= 2; h--)
            if (subtree_try(a, h, F->tsize, budget, F->sub)) break;
        if (F->sub.tasks.empty() || F->sub.h < 2) F->sub = SubtreePlan{};
        if (F->sub.h >= 2) push({K_SUBTREE, 0, (int)F->sub.tasks.size(), 0, 0}, FAM_FUSED, F->sub.bytes, F->sub.flops);
        // the substitutions may fuse a different number of bottom classes (their update vectors are
        // small, so deeper subtrees fit shared memory); default: as many as the factorization
        int want_s = F->opt.subtree_solve_levels != 0 ? F->opt.subtree_solve_levels : F->sub.h;
        int hs = want_s <= 0 ? 0 : std::min(std::min(a->n_cls, want_s), kSubMaxLevels);
        F->subs = SubtreePlan{};
        if (hs == F->sub.h) F->subs = F->sub;
        else
            for (int h = hs; h >= 2; h--)
                if (subtree_try(a, h, F->tsize, budget, F->subs, false)) break;
        if (F->subs.tasks.empty() || F->subs.h < 2) F->subs = SubtreePlan{};
    }
    // first class of the persistent sweeps: the narrow top of the tree, where launch latency
    // dominates; the wide bottom classes keep their own launches (full occupancy for their many
    // small fronts) and their lane-group lists
    {
        int c0 = a->n_cls;
        if (F->use_sweep) {
            if (F->opt.sweep_kernel > 0) c0 = std::max(0, a->n_cls - F->opt.sweep_kernel);
            else
                while (c0 > 0 && a->cls_ptr[c0] - a->cls_ptr[c0 - 1] <= kSweepMaxFronts) c0--;
        }
        F->sweep_c0 = std::max(c0, F->subs.h);
    }
    // zero update vectors: no pivots in the front's whole subtree (fronts are class-ordered, so
    // children come first)
    std::vector<char> zvec(a->n_front, 0);
    for (int32_t f = 0; f < a->n_front; f++) {
        const FrontDev& fr = a->fronts[f];
        bool z = fr.k == 0;
        for (int q = 0; q < fr.nchild && z; q++) z = zvec[fr.child[q]] != 0;
        zvec[f] = z ? 1 : 0;
    }
    auto class_body = [&](int c) {
        const int32_t f0 = a->cls_ptr[c], f1 = a->cls_ptr[c + 1];
        const bool fused_by_subtree = c < F->sub.h;
        const bool solved_by_subtree = c < F->subs.h;
        // solve list: all fronts of the class, largest first
        std::vector<int32_t> all;
        int maxm_all = 1;
        for (int32_t f = f0; f < f1; f++) {
            all.push_back(f);
            maxm_all = std::max(maxm_all, a->fronts[f].m);
        }
        std::stable_sort(all.begin(), all.end(), [&](int32_t x, int32_t y) { return a->fronts[x].m > a->fronts[y].m; });
        // Substitution lists.  Forward: a front with no pivots whose children all carry zero update
        // vectors has a zero update vector itself (the right-hand side enters at the pivot rows), so
        // it is skipped and its slot of the (zeroed) update-vector arena stays zero.  Backward: a
        // front with no pivots has nothing to solve.
        auto make_list = [&](bool forward) {
            ClassList C{};
            std::vector<int32_t> sm, ct, iv, gp[4], lg[kLgLists];
            for (int32_t f : all) {
                if (solved_by_subtree) break;
                const FrontDev& fr = a->fronts[f];
                if (forward ? zvec[f] : fr.k == 0) continue;
                const int li = c >= F->sweep_c0 ? -1 : lg_list_of(fr.m, fr.k);  // the sweep has no lane-group phase
                if (li >= 0 && fr.q_off < 0) lg[li].push_back(f);
                else if (fr.q_off >= 0) iv.push_back(f);
                else if (fr.m <= 4) gp[0].push_back(f);
                else if (fr.m <= 8) gp[1].push_back(f);
                else if (fr.m <= 16) gp[2].push_back(f);
                else if (fr.m <= 32) gp[3].push_back(f);
                else if (fr.m <= kSolveWarpMax) sm.push_back(f);
                else ct.push_back(f);
            }
            for (int q = 0; q < kLgLists; q++) {
                C.n_lg[q] = (int)lg[q].size();
                C.off_lg[q] = (int64_t)slist.size();
                slist.insert(slist.end(), lg[q].begin(), lg[q].end());
            }
            for (int q = 0; q < 4; q++) {
                C.n_grp[q] = (int)gp[q].size();
                C.off_grp[q] = (int64_t)slist.size();
                slist.insert(slist.end(), gp[q].begin(), gp[q].end());
            }
            C.n_small = (int)sm.size();
            C.off_small = (int64_t)slist.size();
            slist.insert(slist.end(), sm.begin(), sm.end());
            C.n_cta = (int)ct.size();
            C.off_cta = (int64_t)slist.size();
            slist.insert(slist.end(), ct.begin(), ct.end());
            for (int32_t f : ct) C.maxm_cta = std::max(C.maxm_cta, a->fronts[f].m);
            C.off_piv = (int64_t)rows.size();
            for (int32_t f : iv) {
                const FrontDev& fr = a->fronts[f];
                C.maxin_inv = std::max(C.maxin_inv, std::max(fr.k, fr.m - fr.k));
                C.maxk_inv = std::max(C.maxk_inv, fr.k);
                C.maxnc_inv = std::max(C.maxnc_inv, fr.m - fr.k);
                for (int i = 0; i < fr.k; i += 32) rows.push_back({f, i, std::min(fr.k, i + 32), 0});
            }
            C.n_piv = (int)(rows.size() - C.off_piv);
            C.off_all = (int64_t)rows.size();
            for (int32_t f : iv) {
                const FrontDev& fr = a->fronts[f];
                for (int i = 0; i < fr.k; i += 32) rows.push_back({f, i, std::min(fr.k, i + 32), 0});
                for (int i = fr.k; i < fr.m; i += 32) rows.push_back({f, i, std::min(fr.m, i + 32), 0});
            }
            C.n_all = (int)(rows.size() - C.off_all);
            return C;
        };
        F->classes_f.push_back(make_list(true));
        F->classes_b.push_back(make_list(false));
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
                if (!zvec[f]) {  // fronts the forward sweep skips move nothing
                    fb += T * nl + 8.0 * k * 2 + T * (cin + nc);
                    ff += 2.0 * nl;
                }
                if (fr.k > 0) {
                    bb += T * nu + 8.0 * (m + k);
                    bf += 2.0 * nu;
                }
            }
            F->fwd_bytes.push_back(fb);
            F->bwd_bytes.push_back(bb);
            F->fwd_flops.push_back(ff);
            F->bwd_flops.push_back(bf);
        }
        slist.insert(slist.end(), all.begin(), all.end());

        if (fused_by_subtree) return;
        if (c < F->foata_cls) {
            // the Table 2 tasks of every front of the class as Foata classes of scalar tasks: extend-add,
            // front maxima, then per pivot step T4 (check), T1 (divide), T2 (multiply), T3 (subtract),
            // then the write-out; each launch covers the step's tasks of all fronts
            const int64_t off = (int64_t)flist.size();
            int maxm = 1, maxk = 0;
            int64_t ws = 0;
            double by_asm = 0, by_out = 0;
            for (int32_t f : all) {
                const FrontDev& fr = a->fronts[f];
                flist.push_back(f);
                fwoff.push_back(ws);
                ws += (int64_t)fr.m * fr.m;
                maxm = std::max(maxm, fr.m);
                maxk = std::max(maxk, fr.k);
                if (fr.nchild == 0) by_asm += 8.0 * a->npe * a->npe;
                for (int q = 0; q < fr.nchild; q++) {
                    const FrontDev& ch = a->fronts[fr.child[q]];
                    by_asm += T * (double)(ch.m - ch.k) * (ch.m - ch.k);
                }
                by_asm += T * (double)fr.m * fr.m;
                by_out += 2.0 * T * (double)fr.m * fr.m;
            }
            F->fws_size = std::max(F->fws_size, ws);
            const int nf = (int)all.size();
            auto bpf = [](int64_t n) { return (int)std::max<int64_t>(1, (n + 255) / 256); };
            Launch L{K_FOATA, c, nf, bpf((int64_t)maxm * maxm), off, 0, 0};
            push(L, FAM_FUSED, by_asm, 0.0);  // threads = task kind (0 extend-add)
            L.threads = 1;
            push(L, FAM_FUSED, T * (double)ws, (double)ws);  // front maxima
            for (int p = 0; p < maxk; p++) {
                double n1 = 0, n2 = 0, nk = 0;
                for (int32_t f : all) {
                    const FrontDev& fr = a->fronts[f];
                    if (p >= fr.k) continue;
                    nk += 1;
                    n1 += fr.m - p - 1;
                    n2 += (double)(fr.m - p - 1) * (fr.m - p - 1);
                }
                L.bucket = p;
                L.threads = 2;  // T4
                push(L, FAM_FUSED, 2.0 * T * nk, nk);
                L.threads = 3;  // T1
                L.maxm = bpf(maxm - p - 1);
                push(L, FAM_FUSED, 2.0 * T * n1, n1);
                L.threads = 4;  // T2
                L.maxm = bpf((int64_t)(maxm - p - 1) * (maxm - p - 1));
                push(L, FAM_FUSED, 3.0 * T * n2, n2);
                L.threads = 5;  // T3
                push(L, FAM_FUSED, 3.0 * T * n2, n2);
            }
            L.bucket = 0;
            L.threads = 6;  // write-out
            L.maxm = bpf((int64_t)maxm * maxm);
            push(L, FAM_FUSED, by_out, 0.0);
            return;
        }
        // tiny fronts (m <= 32): lane-group kernel, G lanes per front
        auto small_bytes = [&](const std::vector<int32_t>& L, double& by, double& fl) {
            by = fl = 0;
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
        };
        int lo = 0;
        for (int G : {4, 8, 16, 32}) {
            if (lo >= F->small_max) break;
            const int hi = std::min(G, F->small_max);
            std::vector<int32_t> L;
            int mx = 0;
            for (int32_t f : all)
                if (a->fronts[f].m > lo && a->fronts[f].m <= hi) {
                    L.push_back(f);
                    mx = std::max(mx, a->fronts[f].m);
                }
            if (!L.empty()) {
                double by, fl;
                small_bytes(L, by, fl);
                // the launch's widest front bounds the kernel's column loops: 24 for a 32-lane launch
                // whose fronts all have m <= 24
                const int mj = G == 32 && mx <= 24 ? 24 : G;
                push({K_GRP, c, (int)L.size(), mj, (int64_t)flist.size()}, FAM_FUSED, by, fl);
                flist.insert(flist.end(), L.begin(), L.end());
                fwoff.resize(flist.size(), -1);
            }
            lo = hi;
        }
        // fused buckets (largest first inside each launch)
        for (int bi = 0; bi < nbounds && lo < F->small_max; bi++) {
            if (bounds[bi] <= lo) continue;
            int hi = std::min(bounds[bi], F->small_max);
            std::vector<int32_t> L;
            for (int32_t f : all)
                if (a->fronts[f].m > lo && a->fronts[f].m <= hi) L.push_back(f);
            if (!L.empty()) {
                double by, fl;
                small_bytes(L, by, fl);
                int th = F->opt.fused_threads[bi];
                if (th <= 0) th = hi <= 64 ? 128 : 256;
                push({K_FUSED, c, (int)L.size(), hi, (int64_t)flist.size(), bi, th}, FAM_FUSED, by, fl);
                for (int32_t fi : L) F->plan.back().kmax = std::max(F->plan.back().kmax, a->fronts[fi].k);
                flist.insert(flist.end(), L.begin(), L.end());
                fwoff.resize(flist.size(), -1);
            }
            lo = hi;
        }
        // large fronts
        std::vector<int32_t> big;
        for (int32_t f : all)
            if (a->fronts[f].m > F->small_max) big.push_back(f);
        if (big.empty()) return;
        {
            int64_t off = (int64_t)asmt.size();
            double by = 0;
            for (int32_t f : big) {
                const FrontDev& fr = a->fronts[f];
                int m = fr.m;
                AsmRec r{};
                r.P_off = fr.P_off;
                r.R_off = fr.R_off;
                r.S_off = fr.S_off;
                r.map_off = fr.map_off;
                r.m = m;
                r.k = fr.k;
                r.front = f;
                for (int q = 0; q < fr.nchild; q++) {
                    const FrontDev& ch = a->fronts[fr.child[q]];
                    r.cS[q] = ch.S_off;
                    r.cn[q] = ch.m - ch.k;
                }
                // symmetric fronts: no tile whose entries all lie in R (overwritten by the transposing
                // copy of U12) or, when the parent reads only the lower triangle of this front's
                // contribution block, strictly above its diagonal
                const bool lower_cb = F->sym && cb_read_lower(f);
                for (int j0 = 0; j0 < m; j0 += 64)
                    for (int i0 = 0; i0 < m; i0 += 64) {
                        if (F->sym && j0 >= fr.k && i0 + 63 < j0 && (lower_cb || i0 + 64 <= fr.k)) continue;
                        r.i0 = i0;
                        r.j0 = j0;
                        asmt.push_back(r);
                    }
                for (int q = 0; q < fr.nchild; q++) {
                    const FrontDev& ch = a->fronts[fr.child[q]];
                    const double n = ch.m - ch.k;
                    by += T * (F->sym ? n * (n + 1) / 2 : n * n);
                }
                const double nc = m - fr.k;
                by += T * (F->sym ? (double)m * fr.k + (lower_cb ? nc * (nc + 1) / 2 : nc * nc) : (double)m * m);
            }
            push({K_ASM, c, (int)(asmt.size() - off), 0, off}, FAM_ASM, by, 0.0);
        }
        int maxk = 0;
        for (int32_t f : big) maxk = std::max(maxk, a->fronts[f].k);
        F->pnl_size = std::max<int64_t>(F->pnl_size, (int64_t)big.size() * 64 * 64);
        auto tile_raw = [&](int8_t aar, int64_t ao, int lda, int8_t am, int8_t bar, int64_t bo, int ldb, int8_t bm,
                            int8_t car, int64_t co, int ldc, int M, int N, int K, int8_t op) {
            for (int j0 = 0; j0 < N; j0 += 64)
                for (int i0 = 0; i0 < M; i0 += 64) {
                    GemmTile t{};
                    t.a_off = ao; t.b_off = bo; t.c_off = co;
                    t.lda = lda; t.ldb = ldb; t.ldc = ldc;
                    t.M = M; t.N = N; t.K = K; t.i0 = i0; t.j0 = j0;
                    t.a_ar = aar; t.b_ar = bar; t.c_ar = car; t.op = op; t.a_mask = am; t.b_mask = bm;
                    gem.push_back(t);
                }
            gf += 2.0 * M * N * K;
            gb += T * ((double)M * K + (double)K * N + 2.0 * M * N);
        };
        // Pivot blocks in super-panels of kSuperPanel pivots (Crout-style inside, right-looking
        // across): a panel is brought up to date with the pivots of its super-panel just before
        // it is factored (thin strip products), and the rest of the pivot rows and columns takes
        // the whole super-panel in one product of depth kSuperPanel at its end.
        const int SP = F->sp;
        auto any_gemm = [&](int64_t ao, int lda, int64_t bo, int ldb, int8_t car, int64_t co, int ldc, int M, int N,
                            int K) {
            if (M <= 0 || N <= 0 || K <= 0) return;
            if (use_tc(M, N, K)) tc_add(AR_FAC, ao, lda, AR_FAC, bo, ldb, car, co, ldc, M, N, K);
            else gemm_tiles(ao, lda, bo, ldb, co, ldc, M, N, K, car == AR_CB);
        };
        bool la_pending = false;  // a lookahead pivot block is in flight for this step's panel
        for (int kb = 0; kb < maxk; kb += nb) {
            const int s0 = (kb / SP) * SP;
            // (0) strips: panel kb (its columns from row kb down, its rows right of it) minus the
            //     products of this super-panel's earlier pivots s0..kb-1 (with lookahead the pivot
            //     block itself took its share in (A') of the previous step)
            if (kb > s0) {
                int64_t soff = (int64_t)gem.size();
                gb = gf = 0;
                for (int32_t f : big) {
                    const FrontDev& fr = a->fronts[f];
                    if (kb >= fr.k) continue;
                    const int m = fr.m, k = fr.k, w = std::min(nb, k - kb), K0 = kb - s0;
                    const int64_t Lrow = fr.P_off + kb + (int64_t)s0 * m;  // L[kb.., s0..kb)
                    const int r0 = F->la ? w : 0;  // first row of the column strip
                    gemm_tiles(Lrow + r0, m, fr.P_off + s0 + (int64_t)kb * m, m, fr.P_off + kb + r0 + (int64_t)kb * m, m,
                               m - kb - r0, w, K0, 0);
                    if (k - kb - w > 0)
                        gemm_tiles(Lrow, m, fr.P_off + s0 + (int64_t)(kb + w) * m, m, fr.P_off + kb + (int64_t)(kb + w) * m, m,
                                   w, k - kb - w, K0, 0);
                    if (m - k > 0 && !F->sym) gemm_tiles(Lrow, m, fr.R_off + s0, k, fr.R_off + kb, k, w, m - k, K0, 0);
                }
                if (gem.size() > (size_t)soff) push({K_GEMM, c, (int)(gem.size() - soff), 0, soff}, FAM_TRAIL, gb, gf);
            }
            // (A) diagonal blocks: factor + invert, one CTA per front (with lookahead, the blocks
            //     after the first were issued on the lookahead stream in the previous step)
            if (!F->la || kb == 0) {
                int64_t poff = (int64_t)pan.size();
                double pb = 0, pf = 0;
                for (size_t bi = 0; bi < big.size(); bi++) {
                    const FrontDev& fr = a->fronts[big[bi]];
                    if (kb >= fr.k) continue;
                    const int w = std::min(nb, fr.k - kb);
                    pan.push_back({big[bi], kb, w, 0, (int64_t)bi * 64 * 64, diag_q(big[bi])});
                    pb += 3.0 * T * w * w;
                    pf += 2.0 * w * w * w;
                }
                push({K_PDIAG, c, (int)(pan.size() - poff), 0, poff}, FAM_PANEL, pb, pf);
                F->plan.back().wide = wide_pdiag(c);
            }
            if (la_pending) {  // main waits for the lookahead pivot block before the panel products
                push({K_SYNC, c, 0, 0, F->n_sync++, 2}, FAM_OTHER, 0.0, 0.0);
                la_pending = false;
            }
            // (B) the panel: L21 = A21 U_D^-1, U12 = L_D^-1 A12, as products with the pivot block's
            //     explicit inverses (default) or by triangular solves against the factored block
            if (!F->pinv) {
                const int64_t toff = (int64_t)trs.size();
                double tb = 0, tf = 0;
                for (size_t bi = 0; bi < big.size(); bi++) {
                    const int32_t f = big[bi];
                    const FrontDev& fr = a->fronts[f];
                    if (kb >= fr.k) continue;
                    const int m = fr.m, k = fr.k, w = std::min(nb, k - kb), r0 = kb + w;
                    const int ns[3] = {m - r0, k - r0, F->sym ? 0 : m - k};
                    for (int side = 0; side < 3; side++) {
                        for (int i0 = 0; i0 < ns[side]; i0 += 128)
                            trs.push_back({f, kb, w, side, i0, std::min(128, ns[side] - i0)});
                        tb += T * (2.0 * w * ns[side]);
                        tf += (double)w * w * ns[side];
                    }
                    tb += T * (double)w * w;
                }
                if (trs.size() > (size_t)toff) push({K_TRSM, c, (int)(trs.size() - toff), 0, toff}, FAM_PANEL, tb, tf);
            }
            int64_t goff = (int64_t)gem.size();
            gb = gf = 0;
            for (size_t bi = 0; bi < big.size() && F->pinv; bi++) {
                const FrontDev& fr = a->fronts[big[bi]];
                if (kb >= fr.k) continue;
                const int m = fr.m, k = fr.k, w = std::min(nb, k - kb), r0 = kb + w;
                const int64_t slot = (int64_t)bi * 64 * 64;
                if (m - r0 > 0) {
                    const int64_t ab = fr.P_off + r0 + (int64_t)kb * m;
                    tile_raw(AR_FAC, ab, m, 0, AR_PNL, slot, 64, 2, AR_FAC, ab, m, m - r0, w, w, 1);
                }
                if (k - r0 > 0) {
                    const int64_t bb = fr.P_off + kb + (int64_t)r0 * m;
                    tile_raw(AR_PNL, slot, 64, 1, AR_FAC, bb, m, 0, AR_FAC, bb, m, w, k - r0, w, 1);
                }
                if (m - k > 0 && !F->sym) {  // symmetric fronts take U12 from L21 before the Schur update
                    const int64_t bb = fr.R_off + kb;
                    tile_raw(AR_PNL, slot, 64, 1, AR_FAC, bb, k, 0, AR_FAC, bb, k, w, m - k, w, 1);
                }
            }
            if (gem.size() > (size_t)goff) push({K_GEMM, c, (int)(gem.size() - goff), 0, goff}, FAM_PANEL, gb, gf);
            // (A') lookahead: the next pivot block takes the update of every pivot of this
            //      super-panel so far (s0..kb+nb) and is factored on the lookahead stream while (C)
            //      and the next step's strips run on the main one
            if (F->la) {
                const int pre = kb + nb - s0;
                int64_t poff = (int64_t)pan.size();
                double pb = 0, pf = 0;
                for (size_t bi = 0; bi < big.size(); bi++) {
                    const FrontDev& fr = a->fronts[big[bi]];
                    if (kb + nb >= fr.k) continue;
                    const int w = std::min(nb, fr.k - kb - nb);
                    pan.push_back({big[bi], kb + nb, w, pre, (int64_t)bi * 64 * 64, diag_q(big[bi])});
                    pb += T * (3.0 * w * w + 2.0 * w * pre);
                    pf += 2.0 * w * w * w + 2.0 * w * w * pre;
                }
                if (pan.size() > (size_t)poff) {
                    la_pending = true;
                    push({K_SYNC, c, 0, 0, F->n_sync++, 0}, FAM_OTHER, 0.0, 0.0);
                    F->plan.back().stream = 2;
                    cur_stream = 2;
                    push({K_PDIAG, c, (int)(pan.size() - poff), 0, poff}, FAM_PANEL, pb, pf);
                    F->plan.back().wide = wide_pdiag(c);
                    cur_stream = 0;
                }
            }
            // (C) end of a super-panel: the pivot rows and columns beyond it take all of its pivots
            //     (with lookahead: all but the next pivot block, which took its share in (A'))
            if (kb + nb == s0 + SP || kb + nb >= maxk) {
                goff = (int64_t)gem.size();
                gb = gf = 0;
                for (int32_t f : big) {
                    const FrontDev& fr = a->fronts[f];
                    const int m = fr.m, k = fr.k, e = s0 + SP;
                    if (s0 >= k || e >= k) continue;  // the front's pivots end inside this super-panel
                    const int64_t Lb = fr.P_off + e + (int64_t)s0 * m;  // L[e.., s0..e)
                    if (F->la) {
                        const int w2 = std::min(nb, k - e);
                        // below the next pivot block, then everything right of it
                        any_gemm(Lb + w2, m, fr.P_off + s0 + (int64_t)e * m, m, AR_FAC, fr.P_off + e + w2 + (int64_t)e * m, m,
                                 m - e - w2, w2, SP);
                        any_gemm(Lb, m, fr.P_off + s0 + (int64_t)(e + w2) * m, m, AR_FAC, fr.P_off + e + (int64_t)(e + w2) * m,
                                 m, m - e, k - e - w2, SP);
                    } else {
                        any_gemm(Lb, m, fr.P_off + s0 + (int64_t)e * m, m, AR_FAC, fr.P_off + e + (int64_t)e * m, m, m - e,
                                 k - e, SP);
                    }
                    if (!F->sym) any_gemm(Lb, m, fr.R_off + s0, k, AR_FAC, fr.R_off + e, k, k - e, m - k, SP);
                }
                if (gem.size() > (size_t)goff) push({K_GEMM, c, (int)(gem.size() - goff), 0, goff}, FAM_TRAIL, gb, gf);
                tc_end(c, FAM_TRAIL);
            }

        }
        // symmetric fronts: U12 = D^-1 L21^T into R (the Schur update's B operand)
        if (F->sym) {
            const int64_t off = (int64_t)symt.size();
            double by = 0;
            for (int32_t f : big) {
                const FrontDev& fr = a->fronts[f];
                const int k = fr.k, nc = fr.m - fr.k;
                if (nc <= 0 || k <= 0) continue;
                for (int j0 = 0; j0 < nc; j0 += 64)
                    for (int i0 = 0; i0 < k; i0 += 64) symt.push_back({f, i0, j0, 0});
                by += 2.0 * T * k * nc + T * k;
            }
            if (symt.size() > (size_t)off) push({K_SYMR, c, (int)(symt.size() - off), 0, off}, FAM_SCHUR, by, 0.0);
        }
        // Schur update S -= L21 U12 (Sec. 2.2): tensor cores (MF_TF32) for large blocks, SIMT otherwise;
        // symmetric fronts compute only the tiles on and below the diagonal
        int64_t goff = (int64_t)gem.size();
        gb = gf = 0;
        for (int32_t f : big) {
            const FrontDev& fr = a->fronts[f];
            const int m = fr.m, k = fr.k, nc = m - k;
            if (nc <= 0 || k <= 0) continue;
            if (use_tc(nc, nc, k))
                tc_add(AR_FAC, fr.P_off + k, m, AR_FAC, fr.R_off, k, AR_CB, fr.S_off, nc, nc, nc, k, 0, 0, 0,
                       F->prec == MF_TF32_BF16 && nc >= F->bf16_min ? (F->opt.bf16_passes == 3 ? tc::kBf16x3 : tc::kBf16)
                                                                    : tc::kTf32x3,
                       F->sym);
            else
                gemm_tiles(fr.P_off + k, m, fr.R_off, k, fr.S_off, nc, nc, nc, k, 1, F->sym);
        }
        if (gem.size() > (size_t)goff) push({K_GEMM, c, (int)(gem.size() - goff), 0, goff}, FAM_SCHUR, gb, gf);
        tc_end(c, FAM_SCHUR);
        if (F->sym) {  // S[j, i] = S[i, j] for the 64 x 64 tiles above the diagonal the update skipped
            const int64_t off = (int64_t)symt.size();
            double by = 0;
            for (int32_t f : big) {
                const FrontDev& fr = a->fronts[f];
                const int nc = fr.m - fr.k;
                if (nc <= 1 || fr.k <= 0) continue;
                if (cb_read_lower(f)) continue;  // its parent reads only the lower triangle
                const bool on_tc = use_tc(nc, nc, fr.k);
                for (int j0 = 0; j0 < nc; j0 += 64)
                    for (int i0 = j0 + 64; i0 < nc; i0 += 64) {
                        // target tile: rows j0.., columns i0..; a tensor-core tile (128 x 256) that
                        // reaches the diagonal computed it already
                        if (on_tc && ((j0 / tc::kTileM) + 1) * tc::kTileM > (i0 / tc::kTileN) * tc::kTileN) continue;
                        symt.push_back({f, i0, j0, 0});
                        by += 2.0 * T * std::min(64, nc - i0) * std::min(64, nc - j0);
                    }
            }
            if (symt.size() > (size_t)off) push({K_MIRROR, c, (int)(symt.size() - off), 0, off}, FAM_SCHUR, by, 0.0);
        }
    };
    // Explicit pivot-block inverses (used only by the substitutions): those of class c are computed
    // on the side stream right after class c, overlapping the factorization of the later classes.
    int n_forks = 0;
    auto emit_inverses = [&](int cls) {
        std::vector<int32_t> ivf;
        int maxk = 0;
        for (int32_t f = a->cls_ptr[cls]; f < a->cls_ptr[cls + 1]; f++)
            if (a->fronts[f].q_off >= 0) {
                ivf.push_back(f);
                maxk = std::max(maxk, a->fronts[f].k);
            }
        if (!ivf.empty()) {
            push({K_FORK, cls, 0, 0, n_forks++}, FAM_OTHER, 0.0, 0.0);
            cur_stream = 1;
            int64_t off = (int64_t)invt.size();
            double by = 0, fl = 0;
            for (int32_t f : ivf) {
                const FrontDev& fr = a->fronts[f];
                if (q_from_pdiag[f]) continue;  // written by the pivot-block kernel
                for (int kb = 0; kb < fr.k; kb += 64) {
                    int w = std::min(64, fr.k - kb);
                    invt.push_back({f, kb, w, 0, fr.q_off});
                    by += 2.0 * T * w * w;
                    fl += 2.0 * w * w * w / 3.0;
                }
            }
            if (invt.size() > (size_t)off) push({K_INVDIAG, cls, (int)(invt.size() - off), 0, off}, FAM_INV, by, fl);
            for (int S = 64; S < maxk; S *= 2) {
                int64_t scr = 0;
                int64_t g1 = (int64_t)gem.size();
                gb = gf = 0;
                std::vector<GemmTile> ph2;
                struct TcArgs {
                    int8_t aar;
                    int64_t ao;
                    int lda;
                    int8_t am, bar;
                    int64_t bo;
                    int ldb;
                    int8_t bm, car;
                    int64_t co;
                    int ldc, M, N, K;
                    int8_t op;
                };
                std::vector<TcArgs> tc2;  // tensor-core products of the second phase
                for (int32_t f : ivf) {
                    const FrontDev& fr = a->fronts[f];
                    const int m = fr.m, k = fr.k;
                    for (int a0 = 0; a0 + S < k; a0 += 2 * S) {
                        const int n2 = std::min(a0 + 2 * S, k) - (a0 + S);
                        const int64_t t1 = scr, t2 = scr + (int64_t)n2 * S;
                        scr += 2 * (int64_t)n2 * S;
                        auto tiles = [&](std::vector<GemmTile>& out, int8_t aar, int64_t ao, int lda, int8_t am, int8_t bar,
                                         int64_t bo, int ldb, int8_t bm, int64_t co, int ldc, int M, int N, int K, int8_t op) {
                            const int8_t car = op == 2 ? AR_INV : AR_SCR;
                            if (use_tc(M, N, K)) {
                                if (&out == &gem) tc_add(aar, ao, lda, bar, bo, ldb, car, co, ldc, M, N, K, op, am, bm);
                                else tc2.push_back({aar, ao, lda, am, bar, bo, ldb, bm, car, co, ldc, M, N, K, op});
                                return;
                            }
                            for (int j0 = 0; j0 < N; j0 += 64)
                                for (int i0 = 0; i0 < M; i0 += 64) {
                                    GemmTile t{};
                                    t.a_off = ao; t.b_off = bo; t.c_off = co;
                                    t.lda = lda; t.ldb = ldb; t.ldc = ldc;
                                    t.M = M; t.N = N; t.K = K; t.i0 = i0; t.j0 = j0;
                                    t.a_ar = aar; t.b_ar = bar; t.c_ar = op == 2 ? AR_INV : AR_SCR; t.op = op;
                                    t.a_mask = am; t.b_mask = bm;
                                    out.push_back(t);
                                }
                            gf += 2.0 * M * N * K;
                            gb += T * ((double)M * K + (double)K * N + (double)M * N);
                        };
                        const int64_t q = fr.q_off;
                        // T1 = L21 X1 ; T2 = U12 Y2
                        tiles(gem, AR_FAC, fr.P_off + (a0 + S) + (int64_t)a0 * m, m, 0, AR_INV, q + a0 + (int64_t)a0 * k, k, 1,
                              t1, n2, n2, S, S, 1);
                        tiles(gem, AR_FAC, fr.P_off + a0 + (int64_t)(a0 + S) * m, m, 0, AR_INV,
                              q + (a0 + S) + (int64_t)(a0 + S) * k, k, 2, t2, S, S, n2, n2, 1);
                        // Q21 = -X2 T1 ; Q12 = -Y1 T2
                        tiles(ph2, AR_INV, q + (a0 + S) + (int64_t)(a0 + S) * k, k, 1, AR_SCR, t1, n2, 0,
                              q + (a0 + S) + (int64_t)a0 * k, k, n2, S, n2, 2);
                        tiles(ph2, AR_INV, q + a0 + (int64_t)a0 * k, k, 2, AR_SCR, t2, S, 0, q + a0 + (int64_t)(a0 + S) * k, k,
                              S, n2, S, 2);
                    }
                }
                F->scr_size = std::max(F->scr_size, scr);
                // phase 1 (products into scratch), then phase 2 (negated products into the inverse)
                if (gem.size() > (size_t)g1) push({K_GEMM, cls, (int)(gem.size() - g1), 0, g1}, FAM_INV, gb / 2, gf / 2);
                tc_end(cls, FAM_INV);
                for (const TcArgs& x : tc2)
                    tc_add(x.aar, x.ao, x.lda, x.bar, x.bo, x.ldb, x.car, x.co, x.ldc, x.M, x.N, x.K, x.op, x.am, x.bm);
                if (!ph2.empty()) {
                    int64_t g2 = (int64_t)gem.size();
                    gem.insert(gem.end(), ph2.begin(), ph2.end());
                    push({K_GEMM, cls, (int)(gem.size() - g2), 0, g2}, FAM_INV, gb / 2, gf / 2);
                }
                tc_end(cls, FAM_INV);
            }
            cur_stream = 0;
        }
    };
    for (int c = 0; c < a->n_cls; c++) {
        class_body(c);
        emit_inverses(c);
    }
    if (n_forks > 0) push({K_JOIN, a->n_cls - 1, 0, 0, 0}, FAM_OTHER, 0.0, 0.0);
    F->n_forks = n_forks;
    {
        const double nE = (double)a->n_elem * a->npe;
        F->resid_bytes = 8.0 * (nE * a->npe + nE * 2 + nE * 2 + 2.0 * a->n_dof + 3.0 * a->n_dof);
        F->resid_flops = 2.0 * nE * a->npe;
    }
    // persistent-sweep phase tables (classes above the fused subtrees)
    {
        auto add = [&](std::vector<SweepPhase>& out, int kind, int count, int64_t off, int n, int ldw) {
            if (count > 0) out.push_back({kind, count, off, n, ldw, 0, 0});
        };
        auto end_group = [&](std::vector<SweepPhase>& out, size_t start) {
            if (out.size() > start) out.back().barrier = 1;
        };
        const size_t TS = F->tsize;
        F->sweep_smem_f = F->sweep_smem_b = 16;
        for (int c = F->sweep_c0; c < a->n_cls; c++) {
            const ClassList& C = F->classes_f[c];
            size_t st = F->sweep_f.size();
            add(F->sweep_f, SW_GRP4, (C.n_grp[0] + 63) / 64, C.off_grp[0], C.n_grp[0], 0);
            add(F->sweep_f, SW_GRP8, (C.n_grp[1] + 31) / 32, C.off_grp[1], C.n_grp[1], 0);
            add(F->sweep_f, SW_GRP16, (C.n_grp[2] + 15) / 16, C.off_grp[2], C.n_grp[2], 0);
            add(F->sweep_f, SW_WARP, (C.n_grp[3] + 7) / 8, C.off_grp[3], C.n_grp[3], 0);
            add(F->sweep_f, SW_WARP, (C.n_small + 7) / 8, C.off_small, C.n_small, 0);
            add(F->sweep_f, SW_CTA, C.n_cta, C.off_cta, C.n_cta, C.maxm_cta);
            add(F->sweep_f, SW_INV1, C.n_piv, C.off_piv, 0, 0);
            if (C.n_piv > 0) {
                end_group(F->sweep_f, st);
                st = F->sweep_f.size();
                add(F->sweep_f, SW_INV2, C.n_all, C.off_all, 0, 0);
            }
            end_group(F->sweep_f, st);
            if (C.n_cta) F->sweep_smem_f = std::max(F->sweep_smem_f, (32 * 33 + (size_t)kRhsChunk * C.maxm_cta) * TS);
            if (C.n_piv) F->sweep_smem_f = std::max(F->sweep_smem_f, (8 * 32 + (size_t)C.maxin_inv) * TS);
        }
        for (int c = a->n_cls - 1; c >= F->sweep_c0; c--) {
            const ClassList& C = F->classes_b[c];
            size_t st = F->sweep_b.size();
            add(F->sweep_b, SW_GRP4, (C.n_grp[0] + 63) / 64, C.off_grp[0], C.n_grp[0], 0);
            add(F->sweep_b, SW_GRP8, (C.n_grp[1] + 31) / 32, C.off_grp[1], C.n_grp[1], 0);
            add(F->sweep_b, SW_GRP16, (C.n_grp[2] + 15) / 16, C.off_grp[2], C.n_grp[2], 0);
            add(F->sweep_b, SW_GRP32, (C.n_grp[3] + 7) / 8, C.off_grp[3], C.n_grp[3], 0);
            add(F->sweep_b, SW_WARP, (C.n_small + 7) / 8, C.off_small, C.n_small, 0);
            add(F->sweep_b, SW_CTA, C.n_cta, C.off_cta, C.n_cta, C.maxm_cta);
            add(F->sweep_b, SW_INV1, C.n_piv, C.off_piv, 0, 0);
            if (C.n_piv > 0) {
                end_group(F->sweep_b, st);
                st = F->sweep_b.size();
                add(F->sweep_b, SW_INV2, C.n_piv, C.off_piv, 0, 0);
            }
            end_group(F->sweep_b, st);
            if (C.n_cta)
                F->sweep_smem_b = std::max(F->sweep_smem_b, (32 * 33 + 8 * 64 * kRhsChunk + (size_t)kRhsChunk * C.maxm_cta) * TS);
            if (C.n_piv) F->sweep_smem_b = std::max(F->sweep_smem_b, (8 * 32 + (size_t)C.maxin_inv) * TS);
        }
        if (!F->sweep_f.empty()) F->sweep_f.back().barrier = 0;  // the end of the launch is the last barrier
        if (!F->sweep_b.empty()) F->sweep_b.back().barrier = 0;
    }
    int rc;
    if ((rc = upload(&F->d_sweep_f, F->sweep_f))) return rc;
    if ((rc = upload(&F->d_sweep_b, F->sweep_b))) return rc;
    if (!symt.empty() && (rc = upload(&F->d_symt, symt))) return rc;
    if (!trs.empty() && (rc = upload(&F->d_trsm, trs))) return rc;
    if (!gtcd.empty() && (rc = upload(&F->d_gtcd, gtcd))) return rc;
    if ((rc = upload(&F->d_flist, flist))) return rc;
    fwoff.resize(flist.size(), -1);
    if ((rc = upload(&F->d_fwoff, fwoff))) return rc;
    {
        std::vector<FactorRec> frec(flist.size());
        for (size_t i = 0; i < flist.size(); i++) {
            const FrontDev& fr = a->fronts[flist[i]];
            FactorRec r{};
            r.P_off = fr.P_off; r.R_off = fr.R_off; r.S_off = fr.S_off; r.map_off = fr.map_off;
            r.m = fr.m; r.k = fr.k; r.nchild = fr.nchild; r.elem = fr.elem; r.front = flist[i];
            for (int c = 0; c < fr.nchild; c++) {
                const FrontDev& ch = a->fronts[fr.child[c]];
                r.cS[c] = ch.S_off;
                r.cn[c] = ch.m - ch.k;
            }
            frec[i] = r;
        }
        if ((rc = upload(&F->d_frec, frec))) return rc;
    }
    if ((rc = upload(&F->d_slist, slist))) return rc;
    {
        std::vector<SolveRec> srec(slist.size());
        for (size_t i = 0; i < slist.size(); i++) {
            const FrontDev& fr = a->fronts[slist[i]];
            srec[i] = SolveRec{fr.P_off, fr.R_off, fr.dof_off, fr.vec_off, fr.m, fr.k, fr.nchild, 0};
        }
        if ((rc = upload(&F->d_srec, srec))) return rc;
    }
    if ((rc = upload(&F->d_rows, rows))) return rc;
    if ((rc = upload(&F->d_invt, invt))) return rc;
    if ((rc = upload(&F->d_sub_tasks, F->sub.tasks))) return rc;
    if ((rc = upload(&F->d_sub_ecb, F->sub.ecb))) return rc;
    if ((rc = upload(&F->d_sub_euv, F->sub.euv))) return rc;
    if ((rc = upload(&F->d_subs_tasks, F->subs.tasks))) return rc;
    if ((rc = upload(&F->d_subs_euv, F->subs.euv))) return rc;
    if ((rc = upload(&F->d_asm, asmt))) return rc;
    if ((rc = upload(&F->d_panel, pan))) return rc;
    if ((rc = upload(&F->d_gemm, gem))) return rc;
    if ((rc = upload(&F->d_gtc, gtc))) return rc;
    if ((rc = upload(&F->d_tcpack, tcp))) return rc;
    if ((rc = upload(&F->d_tcjob, tcj))) return rc;
    return MF_OK;
}

template <typename T>
static int set_smem_limits() {
    int dev;
    CUDA_TRY(cudaGetDevice(&dev));
    int maxsm = 0;
    CUDA_TRY(cudaDeviceGetAttribute(&maxsm, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    CUDA_TRY(cudaFuncSetAttribute(k_front_fused<T, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, maxsm));
    CUDA_TRY(cudaFuncSetAttribute(k_front_fused<T, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, maxsm));
    CUDA_TRY(cudaFuncSetAttribute(k_fwd_cta<T, false, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, maxsm));
    CUDA_TRY(cudaFuncSetAttribute(k_fwd_cta<T, true, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, maxsm));
    CUDA_TRY(cudaFuncSetAttribute(k_bwd_cta<T, false, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, maxsm));
    CUDA_TRY(cudaFuncSetAttribute(k_bwd_cta<T, true, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, maxsm));
    CUDA_TRY(cudaFuncSetAttribute(k_fwd_cta<T, false, kRhsChunk>, cudaFuncAttributeMaxDynamicSharedMemorySize, maxsm));
    CUDA_TRY(cudaFuncSetAttribute(k_fwd_cta<T, true, kRhsChunk>, cudaFuncAttributeMaxDynamicSharedMemorySize, maxsm));
    CUDA_TRY(cudaFuncSetAttribute(k_bwd_cta<T, false, kRhsChunk>, cudaFuncAttributeMaxDynamicSharedMemorySize, maxsm));
    CUDA_TRY(cudaFuncSetAttribute(k_bwd_cta<T, true, kRhsChunk>, cudaFuncAttributeMaxDynamicSharedMemorySize, maxsm));
    CUDA_TRY(cudaFuncSetAttribute(k_inv_diag<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, maxsm));
    CUDA_TRY(cudaFuncSetAttribute(k_subtree_factor<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, maxsm));
    CUDA_TRY(cudaFuncSetAttribute(k_schur_tc<tc::kTf32x3>, cudaFuncAttributeMaxDynamicSharedMemorySize, tc::kSmemBytes));
    CUDA_TRY(cudaFuncSetAttribute(k_schur_tc<tc::kBf16>, cudaFuncAttributeMaxDynamicSharedMemorySize, tc::kSmemBytes));
    CUDA_TRY(cudaFuncSetAttribute(k_schur_tc<tc::kBf16x3>, cudaFuncAttributeMaxDynamicSharedMemorySize, tc::kSmemBytes));
    CUDA_TRY(cudaFuncSetAttribute(k_tc_direct, cudaFuncAttributeMaxDynamicSharedMemorySize, tc::kSmemBytes));
    CUDA_TRY(cudaFuncSetAttribute(k_subtree_fwd<T, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, maxsm));
    CUDA_TRY(cudaFuncSetAttribute(k_subtree_fwd<T, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, maxsm));
#define SET_INV(TR, PH)                                                                                            \
    CUDA_TRY(cudaFuncSetAttribute(k_inv_gemv<T, TR, PH, 8>, cudaFuncAttributeMaxDynamicSharedMemorySize, maxsm));    \
    CUDA_TRY(cudaFuncSetAttribute(k_inv_gemv<T, TR, PH, 32>, cudaFuncAttributeMaxDynamicSharedMemorySize, maxsm));
    SET_INV(false, PH_FWD1) SET_INV(false, PH_FWD2) SET_INV(false, PH_BWD1) SET_INV(false, PH_BWD2)
    SET_INV(true, PH_FWD1) SET_INV(true, PH_FWD2) SET_INV(true, PH_BWD1) SET_INV(true, PH_BWD2)
#undef SET_INV
    return MF_OK;
}

extern "C" int mf_factors_create(const mf_analysis* a, const mf_options* opt, mf_factors** out) {
    if (!a || !out) return MF_EINVAL;
    *out = nullptr;
    mf_factors* F = new mf_factors();
    F->a = a;
    F->opt = opt ? mf_resolve_options(opt) : a->opt;
    F->prec = F->opt.precision;
    if (F->prec != MF_F64 && F->prec != MF_F32 && F->prec != MF_TF32 && F->prec != MF_TF32_BF16) {
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
    F->tc_min = F->opt.tc_min_cb > 0 ? F->opt.tc_min_cb : 256;
    F->bf16_min = F->opt.bf16_min_cb > 0 ? F->opt.bf16_min_cb : 2048;
    if (F->opt.bf16_passes != 0 && F->opt.bf16_passes != 1 && F->opt.bf16_passes != 3) {
        delete F;
        return MF_EINVAL;
    }
    F->use_sweep = F->opt.sweep_kernel != 0;
    {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&F->num_sms, cudaDevAttrMultiProcessorCount, dev);
        if (F->num_sms <= 0) F->num_sms = 148;
        F->norm_blocks = 8 * F->num_sms;  // norm reduction: 64 warps per SM
    }
    F->sp = F->opt.super_panel > 0 ? F->opt.super_panel : (F->prec == MF_F64 ? F->nb : 256);
    F->sp = std::max(F->nb, (F->sp + F->nb - 1) / F->nb * F->nb);
    F->la = F->opt.lookahead >= 0;
    F->foata_cls = std::max(0, F->opt.foata_classes);
    F->sym = F->opt.symmetric != 0;
    F->pinv = F->opt.panel_trsm == 0;
    F->tcd = F->opt.tc_direct != 0;
    for (int i = 0; i < MF_FUSED_BUCKETS; i++) {
        const int t = F->opt.fused_threads[i];
        if (t != 0 && t != 32 && t != 64 && t != 128 && t != 256) {
            delete F;
            return MF_EINVAL;
        }
    }
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
    {
        // gather sources of the forward substitution, precomputed per front row
        std::vector<int64_t> vsrc(2 * a->dofs.size(), -1);
        for (int32_t f = 0; f < a->n_front; f++) {
            const FrontDev& fr = a->fronts[f];
            for (int c = 0; c < fr.nchild; c++) {
                const int64_t voff = a->fronts[fr.child[c]].vec_off;
                for (int32_t i = 0; i < fr.m; i++) {
                    const int32_t ic = a->maps[fr.map_off + (int64_t)c * fr.m + i];
                    if (ic >= 0) vsrc[2 * (fr.dof_off + i) + c] = voff + ic;
                }
            }
        }
        TRY(upload(&F->d_vsrc, vsrc));
    }
    TRY(upload(&F->d_en, a->elem_nodes));
    if (F->sym) {  // each dof's pivot (diagonal of L) in the factor arena, for the symmetric solves
        std::vector<int64_t> pd(a->n_dof, 0);
        for (int32_t f = 0; f < a->n_front; f++) {
            const FrontDev& fr = a->fronts[f];
            for (int p = 0; p < fr.k; p++) pd[a->dofs[fr.dof_off + p]] = fr.P_off + p + (int64_t)p * fr.m;
        }
        TRY(upload(&F->d_pdiag, pd));
        TRY(dev_alloc(&F->d_pdv, (size_t)a->n_dof));
    }
    if (a->csr_n > 0) {
        TRY(upload(&F->d_csr_dest, a->csr_dest));
        const size_t ne = (size_t)a->n_elem * a->npe * a->npe;
        TRY(dev_alloc(&F->d_elemvals, ne));
        // positions no CSR entry maps to (the arrowheads' empty parts, the padding) stay zero
        if (cudaMemset(F->d_elemvals, 0, ne * sizeof(double)) != cudaSuccess) {
            free_factors(F);
            return MF_ECUDA;
        }
    }
    TRY(upload(&F->d_node_ptr, a->node_ptr));
    TRY(upload(&F->d_node_inc, a->node_inc));
    TRY(dev_alloc((char**)&F->d_fac, (size_t)a->factor_size * F->tsize));
    TRY(dev_alloc((char**)&F->d_cb, (size_t)a->cb_size * F->tsize));
    TRY(dev_alloc((char**)&F->d_vec, (size_t)a->vec_size * F->max_nrhs * F->tsize));
    // update vectors of fronts the forward sweep skips must read as zero
    if (cudaMemset(F->d_vec, 0, (size_t)a->vec_size * F->max_nrhs * F->tsize) != cudaSuccess) {
        free_factors(F);
        return MF_ECUDA;
    }
    TRY(dev_alloc(&F->d_famax, (size_t)a->n_front));
    TRY(dev_alloc(&F->d_status, 1));
    TRY(dev_alloc(&F->d_bar, 2));
    const size_t nv = (size_t)a->n_dof * F->max_nrhs;
    TRY(dev_alloc(&F->d_r, nv));
    TRY(dev_alloc(&F->d_d, nv));
    TRY(dev_alloc(&F->d_Y, (size_t)a->n_elem * a->npe * F->max_nrhs));
    TRY(dev_alloc(&F->d_rowabs, (size_t)a->n_dof));
    TRY(dev_alloc(&F->d_colabs, (size_t)a->n_dof));
    TRY(dev_alloc(&F->d_part, (size_t)F->norm_blocks * 6 * F->max_nrhs));
    TRY(dev_alloc(&F->d_norms, (size_t)6 * F->max_nrhs));
    TRY(dev_alloc(&F->d_cgpar, (size_t)2));
    TRY(dev_alloc(&F->d_cgit, (size_t)1));
    if (cudaStreamCreateWithFlags(&F->s_body, cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamCreateWithFlags(&F->s_aux, cudaStreamNonBlocking) != cudaSuccess) {
        free_factors(F);
        return MF_ECUDA;
    }
    if (F->sym && F->opt.refine_cg) {
        TRY(dev_alloc(&F->d_cgp, nv));
        TRY(dev_alloc(&F->d_cgs, nv));
        TRY(dev_alloc(&F->d_zero, nv));
        TRY(dev_alloc(&F->d_cg, (size_t)4 * F->max_nrhs));
        if (cudaMemset(F->d_zero, 0, nv * sizeof(double)) != cudaSuccess ||
            cudaMemset(F->d_cg, 0, 4 * F->max_nrhs * sizeof(double)) != cudaSuccess) {
            free_factors(F);
            return MF_ECUDA;
        }
    }
    TRY(build_plan(F));
    {
        // the mid-size solve kernels keep kRhsChunk right-hand sides of a front in shared memory
        int dev = 0, maxsm = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&maxsm, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
        for (const ClassList& C : F->classes_b) {
            const size_t need = (32 * 33 + 8 * 64 * kRhsChunk + (size_t)kRhsChunk * C.maxm_cta) * F->tsize;
            if (C.n_cta > 0 && need > (size_t)maxsm) {
                free_factors(F);
                return MF_ENOTSUP;
            }
        }
    }
    if (F->fws_size > 0) {
        TRY(dev_alloc((char**)&F->d_fws, (size_t)F->fws_size * F->tsize));
        TRY(dev_alloc((char**)&F->d_fxs, (size_t)F->fws_size * F->tsize));
    }
    TRY(dev_alloc((char**)&F->d_inv, (size_t)a->inv_size * F->tsize));
    TRY(dev_alloc((char**)&F->d_scr, (size_t)F->scr_size * F->tsize));
    TRY(dev_alloc((char**)&F->d_pnl, (size_t)F->pnl_size * F->tsize));
    if (F->pk_size > 0) TRY(dev_alloc((char**)&F->d_pk, (size_t)F->pk_size * sizeof(float)));
    if (F->pk2_size > 0) TRY(dev_alloc((char**)&F->d_pk2, (size_t)F->pk2_size * sizeof(float)));
    // Stream priorities: the chain of the main stream (and the lookahead pivot blocks beside it) is
    // the critical path; the side stream's inverses fill the SMs it leaves idle, so their CTAs must
    // not hold SMs that the next pivot block or panel product is waiting for.
    int prio_lo = 0, prio_hi = 0;
    if (cudaDeviceGetStreamPriorityRange(&prio_lo, &prio_hi) != cudaSuccess) {
        free_factors(F);
        return MF_ECUDA;
    }
    if (cudaEventCreateWithFlags(&F->fan_in, cudaEventDisableTiming) != cudaSuccess) {
        free_factors(F);
        return MF_ECUDA;
    }
    for (int j = 0; j < 3; j++)
        if (cudaStreamCreateWithPriority(&F->sfan[j], cudaStreamNonBlocking, prio_hi) != cudaSuccess ||
            cudaEventCreateWithFlags(&F->fan_out[j], cudaEventDisableTiming) != cudaSuccess) {
            free_factors(F);
            return MF_ECUDA;
        }
    if (F->n_forks > 0 || F->n_sync > 0) {
        if (cudaStreamCreateWithPriority(&F->s1, cudaStreamNonBlocking, prio_hi) != cudaSuccess ||
            cudaEventCreateWithFlags(&F->s1_in, cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&F->s1_out, cudaEventDisableTiming) != cudaSuccess) {
            free_factors(F);
            return MF_ECUDA;
        }
    }
    if (F->n_forks > 0) {
        if (cudaStreamCreateWithPriority(&F->s2, cudaStreamNonBlocking, prio_lo) != cudaSuccess) {
            free_factors(F);
            return MF_ECUDA;
        }
        F->fork_ev.assign(F->n_forks, nullptr);
        for (int i = 0; i < F->n_forks; i++)
            if (cudaEventCreateWithFlags(&F->fork_ev[i], cudaEventDisableTiming) != cudaSuccess) {
                free_factors(F);
                return MF_ECUDA;
            }
        if (cudaEventCreateWithFlags(&F->join_ev, cudaEventDisableTiming) != cudaSuccess) {
            free_factors(F);
            return MF_ECUDA;
        }
    }
    if (F->n_sync > 0) {
        if (cudaStreamCreateWithPriority(&F->s3, cudaStreamNonBlocking, prio_hi) != cudaSuccess) {
            free_factors(F);
            return MF_ECUDA;
        }
        F->sync_ev.assign(F->n_sync, nullptr);
        for (int i = 0; i < F->n_sync; i++)
            if (cudaEventCreateWithFlags(&F->sync_ev[i], cudaEventDisableTiming) != cudaSuccess) {
                free_factors(F);
                return MF_ECUDA;
            }
    }
    {
        const int s64 = (int)panel_diag_dyn_smem<double, kPanelNB64>(), s32 = (int)panel_diag_dyn_smem<float, kPanelNB32>();
        const int sw = (int)panel_diag_dyn_smem<float, kPanelNB32, double>();
        constexpr cudaFuncAttribute kA = cudaFuncAttributeMaxDynamicSharedMemorySize;
        cudaError_t e = cudaSuccess, e2 = cudaSuccess;
        if (F->prec == MF_F64) {
            e = cudaFuncSetAttribute(k_panel_diag_blk<double, kPanelNB64, double, true>, kA, s64);
            if (e == cudaSuccess) e = cudaFuncSetAttribute(k_panel_diag_blk<double, kPanelNB64, double, false>, kA, s64);
            if (e == cudaSuccess) e = cudaFuncSetAttribute(k_panel_diag_blk<double, kPanelNB64, double, true, true>, kA, s64);
        } else {
            e = cudaFuncSetAttribute(k_panel_diag_blk<float, kPanelNB32, float, true>, kA, s32);
            if (e == cudaSuccess) e = cudaFuncSetAttribute(k_panel_diag_blk<float, kPanelNB32, float, false>, kA, s32);
            if (e == cudaSuccess) e = cudaFuncSetAttribute(k_panel_diag_blk<float, kPanelNB32, float, true, true>, kA, s32);
            e2 = cudaFuncSetAttribute(k_panel_diag_blk<float, kPanelNB32, double, true>, kA, sw);
            if (e2 == cudaSuccess) e2 = cudaFuncSetAttribute(k_panel_diag_blk<float, kPanelNB32, double, false>, kA, sw);
            if (e2 == cudaSuccess) e2 = cudaFuncSetAttribute(k_panel_diag_blk<float, kPanelNB32, double, true, true>, kA, sw);
        }
        if (e != cudaSuccess || e2 != cudaSuccess) {
            (void)cudaGetLastError();
            free_factors(F);
            return MF_ECUDA;
        }
    }
    TRY(dev_alloc((char**)&F->d_ys, (size_t)a->ys_size * F->max_nrhs * F->tsize));
#undef TRY
    *out = F;
    return MF_OK;
}

extern "C" void mf_free_factors(mf_factors* f) { free_factors(f); }

namespace {
__global__ void k_csr_scatter(const double* __restrict__ v, const int64_t* __restrict__ dest, double* __restrict__ out,
                              int64_t nnz) {
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q < nnz) out[dest[q]] = v[q];
}
}  // namespace

// The element matrices the kernels read: the caller's array for a mesh analysis; for a CSR
// analysis, the caller's CSR values scattered into the arrowhead elements (F->d_elemvals).
static int element_values(mf_factors* F, const double* d_values, cudaStream_t s, const double** out) {
    *out = d_values;
    const mf_analysis* a = F->a;
    if (a->csr_n == 0) return MF_OK;
    const int64_t nnz = a->csr_nnz;
    if (nnz > 0) {
        int slot = prof_begin(F, s, FAM_OTHER, 24.0 * nnz, 0.0);
        k_csr_scatter<<<(unsigned)((nnz + 255) / 256), 256, 0, s>>>(d_values, F->d_csr_dest, F->d_elemvals, nnz);
        prof_end(F, s, slot);
        CUDA_TRY(cudaGetLastError());
    }
    *out = F->d_elemvals;
    return MF_OK;
}

template <typename T>
static int run_factor(mf_factors* F, const double* d_values, cudaStream_t s) {
    const mf_analysis* a = F->a;
    T* fac = (T*)F->d_fac;
    T* cb = (T*)F->d_cb;
    int slot = prof_begin(F, s, FAM_OTHER, 0, 0);
    k_init_status<<<1, 1, 0, s>>>(F->d_status);
    CUDA_TRY(cudaMemsetAsync(F->d_famax, 0, sizeof(unsigned int) * a->n_front, s));
    prof_end(F, s, slot);
    const cudaStream_t s_caller = s;
    if (F->s1) {  // the plan runs on the high-priority stream, joined back at the end
        CUDA_TRY(cudaEventRecord(F->s1_in, s_caller));
        CUDA_TRY(cudaStreamWaitEvent(F->s1, F->s1_in, 0));
    }
    const cudaStream_t s_main = F->s1 ? F->s1 : s_caller;
    for (size_t li = 0; li < F->plan.size(); li++) {
        const Launch& L = F->plan[li];
        if (L.kind == K_FORK) {  // the side stream continues after everything issued so far
            CUDA_TRY(cudaEventRecord(F->fork_ev[L.off], s_main));
            CUDA_TRY(cudaStreamWaitEvent(F->s2, F->fork_ev[L.off], 0));
            continue;
        }
        if (L.kind == K_JOIN) {  // the caller's stream waits for the side stream's work
            CUDA_TRY(cudaEventRecord(F->join_ev, F->s2));
            CUDA_TRY(cudaStreamWaitEvent(s_main, F->join_ev, 0));
            continue;
        }
        if (L.kind == K_SYNC) {  // stream L.stream waits for the work issued so far on stream L.bucket
            const cudaStream_t sig = L.bucket == 0 ? s_main : L.bucket == 1 ? F->s2 : F->s3;
            const cudaStream_t wai = L.stream == 0 ? s_main : L.stream == 1 ? F->s2 : F->s3;
            CUDA_TRY(cudaEventRecord(F->sync_ev[L.off], sig));
            CUDA_TRY(cudaStreamWaitEvent(wai, F->sync_ev[L.off], 0));
            continue;
        }
        s = L.stream == 0 ? s_main : L.stream == 1 ? F->s2 : F->s3;
        float* pk = L.stream == 1 ? F->d_pk2 : F->d_pk;
        slot = prof_begin(F, s, F->plan_fam[li], F->plan_bytes[li], F->plan_flops[li], 1,
                          F->plan[li].kind == K_FUSED ? F->plan[li].bucket : -1, F->plan[li].kind, F->plan[li].cls,
                          F->plan[li].count);
        switch (L.kind) {
            case K_FUSED: {
                int ldm = L.maxm | 1;
                size_t sm = fused_smem<T>(L.maxm);
#define FUSED_LAUNCH(BLK)                                                                                          \
    k_front_fused<T, BLK><<<L.count, L.threads, sm, s>>>(F->d_frec + L.off, F->d_maps, d_values, a->npe, fac, cb, \
                                                         L.maxm, ldm, F->tol_rel, F->sym ? 1 : 0, F->d_status)
                if (L.kmax <= kFusedBlockedMaxK) FUSED_LAUNCH(true);
                else FUSED_LAUNCH(false);
#undef FUSED_LAUNCH
                break;
            }
            case K_GRP: {
                const int G = L.maxm <= 4 ? 4 : L.maxm <= 8 ? 8 : L.maxm <= 16 ? 16 : 32;  // L.maxm: widest front
                const unsigned per = 8 * (32 / G);                                          // fronts per 256-thread CTA
                const unsigned g = (unsigned)((L.count + per - 1) / per);
#define GRP_CASE(GS, MJS)                                                                                        \
    case MJS:                                                                                                    \
        k_front_grp<T, GS, MJS><<<g, 256, 0, s>>>(F->d_frec + L.off, L.count, F->d_maps, d_values, a->npe,          \
                                                  fac, cb, F->tol_rel, F->d_status);                             \
        break;
                switch (L.maxm) {
                    GRP_CASE(4, 4)
                    GRP_CASE(8, 8)
                    GRP_CASE(16, 16)
                    GRP_CASE(32, 24)
                    GRP_CASE(32, 32)
                }
#undef GRP_CASE
                break;
            }
            case K_ASM:
                if (F->sym) k_assemble_large<T, true><<<L.count, 256, 0, s>>>(F->d_asm + L.off, F->d_maps, fac, cb, F->d_famax);
                else k_assemble_large<T><<<L.count, 256, 0, s>>>(F->d_asm + L.off, F->d_maps, fac, cb, F->d_famax);
                break;
            case K_PDIAG: {
                constexpr int NB = sizeof(T) == 8 ? kPanelNB64 : kPanelNB32;
                const DiagTask* dt = F->d_panel + L.off;
                if constexpr (sizeof(T) == 4) {
                    if (L.wide) {
                        if (F->pinv && F->sym)
                            k_panel_diag_blk<T, NB, double, true, true><<<L.count, 256, panel_diag_dyn_smem<T, NB, double>(), s>>>(
                                F->d_fronts, dt, fac, (T*)F->d_pnl, (T*)F->d_inv, F->d_famax, F->tol_rel, F->d_status);
                        else if (F->pinv)
                            k_panel_diag_blk<T, NB, double, true><<<L.count, 256, panel_diag_dyn_smem<T, NB, double>(), s>>>(
                                F->d_fronts, dt, fac, (T*)F->d_pnl, (T*)F->d_inv, F->d_famax, F->tol_rel, F->d_status);
                        else
                            k_panel_diag_blk<T, NB, double, false><<<L.count, 256, panel_diag_dyn_smem<T, NB, double>(), s>>>(
                                F->d_fronts, dt, fac, (T*)F->d_pnl, (T*)F->d_inv, F->d_famax, F->tol_rel, F->d_status);
                        break;
                    }
                }
                if (F->pinv && F->sym)
                    k_panel_diag_blk<T, NB, T, true, true><<<L.count, 256, panel_diag_dyn_smem<T, NB>(), s>>>(
                        F->d_fronts, dt, fac, (T*)F->d_pnl, (T*)F->d_inv, F->d_famax, F->tol_rel, F->d_status);
                else if (F->pinv)
                    k_panel_diag_blk<T, NB, T, true><<<L.count, 256, panel_diag_dyn_smem<T, NB>(), s>>>(
                        F->d_fronts, dt, fac, (T*)F->d_pnl, (T*)F->d_inv, F->d_famax, F->tol_rel, F->d_status);
                else
                    k_panel_diag_blk<T, NB, T, false><<<L.count, 256, panel_diag_dyn_smem<T, NB>(), s>>>(
                        F->d_fronts, dt, fac, (T*)F->d_pnl, (T*)F->d_inv, F->d_famax, F->tol_rel, F->d_status);
                break;
            }
            case K_TCD:
                if constexpr (sizeof(T) == 4) {
                    Arenas<float> ar{{fac, cb, (float*)F->d_inv, (float*)F->d_scr, (float*)F->d_pnl}};
                    k_tc_direct<<<(unsigned)std::min(L.count, F->num_sms), kTcdThreads, tc::kSmemBytes, s>>>(
                        F->d_gtcd + L.off, L.count, ar, F->d_status);
                }
                break;
            case K_TRSM: {
                constexpr int NB = sizeof(T) == 8 ? kPanelNB64 : kPanelNB32;
                k_panel_trsm<T, NB><<<L.count, 128, 0, s>>>(F->d_fronts, F->d_trsm + L.off, fac);
                break;
            }
            case K_GEMM: {
                Arenas<T> ar{{fac, cb, (T*)F->d_inv, (T*)F->d_scr, (T*)F->d_pnl}};
                if constexpr (sizeof(T) == 8) k_gemm<T, 8><<<L.count, 256, 0, s>>>(F->d_gemm + L.off, ar);
                else k_gemm_cp<16, 3><<<L.count, 256, 0, s>>>(F->d_gemm + L.off, ar);
                break;
            }
            case K_SUBTREE:
                k_subtree_factor<T><<<L.count, 256, F->sub.smem_f, s>>>(F->d_fronts, F->d_sub_tasks, F->d_sub_ecb, F->d_maps,
                                                                       d_values, a->npe, fac, cb, F->sub.lay_f, F->tol_rel,
                                                                       F->d_status);
                break;
            case K_TCPACK:
                if constexpr (sizeof(T) == 4) {
                    Arenas<float> ar{{fac, cb, (float*)F->d_inv, (float*)F->d_scr, (float*)F->d_pnl}};
                    const TcPack* tp = F->d_tcpack + L.bucket;
                    const TcPackJob* tj = F->d_tcjob + L.off;
                    if (L.wide == tc::kBf16) k_tc_pack<tc::kBf16><<<L.count, 256, 0, s>>>(tp, tj, ar, pk);
                    else if (L.wide == tc::kBf16x3) k_tc_pack<tc::kBf16x3><<<L.count, 256, 0, s>>>(tp, tj, ar, pk);
                    else k_tc_pack<tc::kTf32x3><<<L.count, 256, 0, s>>>(tp, tj, ar, pk);
                }
                break;
            case K_GEMMTC:
                if constexpr (sizeof(T) == 4) {
                    Arenas<float> ar{{fac, cb, (float*)F->d_inv, (float*)F->d_scr, (float*)F->d_pnl}};
                    const unsigned g = (unsigned)std::min(L.count, F->num_sms);
                    const TcTile* tl = F->d_gtc + L.off;
                    if (L.wide == tc::kBf16)
                        k_schur_tc<tc::kBf16><<<g, kTcThreads, tc::kSmemBytes, s>>>(tl, L.count, pk, ar, F->d_status);
                    else if (L.wide == tc::kBf16x3)
                        k_schur_tc<tc::kBf16x3><<<g, kTcThreads, tc::kSmemBytes, s>>>(tl, L.count, pk, ar, F->d_status);
                    else
                        k_schur_tc<tc::kTf32x3><<<g, kTcThreads, tc::kSmemBytes, s>>>(tl, L.count, pk, ar, F->d_status);
                }
                break;
            case K_INVDIAG:
                k_inv_diag<T><<<L.count, 128, 2 * 64 * 65 * sizeof(T), s>>>(F->d_fronts, F->d_invt + L.off, fac, (T*)F->d_inv);
                break;
            case K_SYMR:
                k_sym_r<T><<<L.count, 256, 0, s>>>(F->d_fronts, F->d_symt + L.off, fac);
                break;
            case K_MIRROR:
                k_sym_mirror<T><<<L.count, 256, 0, s>>>(F->d_fronts, F->d_symt + L.off, cb);
                break;
            case K_FOATA: {
                const FoataArgs A{F->d_frec + L.off, F->d_fwoff + L.off, L.count, L.maxm, L.bucket};
                T* W = (T*)F->d_fws;
                T* X = (T*)F->d_fxs;
                const unsigned g = (unsigned)((int64_t)L.count * L.maxm);
                switch (L.threads) {
                    case 0: k_foata_assemble<T><<<g, 256, 0, s>>>(A, F->d_maps, d_values, a->npe, cb, W); break;
                    case 1: k_foata_amax<T><<<L.count, 256, 0, s>>>(A, W, F->d_famax); break;
                    case 2:
                        k_foata_t4<T><<<(L.count + 255) / 256, 256, 0, s>>>(A, W, F->d_famax, F->tol_rel, F->d_status);
                        break;
                    case 3: k_foata_t1<T><<<g, 256, 0, s>>>(A, W); break;
                    case 4: k_foata_t2<T><<<g, 256, 0, s>>>(A, W, X); break;
                    case 5: k_foata_t3<T><<<g, 256, 0, s>>>(A, W, X); break;
                    default: k_foata_write<T><<<g, 256, 0, s>>>(A, W, fac, cb); break;
                }
                break;
            }
        }
        prof_end(F, s, slot);
        CUDA_TRY(cudaGetLastError());
    }
    if (F->sym && !scaling_folded(F)) {  // the pivots in dof order, read by the separate D scaling pass
        const int64_t n = a->n_dof;
        int slot2 = prof_begin(F, s_main, FAM_OTHER, (8.0 + F->tsize + 8.0) * n, 0.0);
        k_gather_pivots<T><<<(unsigned)((n + 255) / 256), 256, 0, s_main>>>(F->d_pdiag, fac, F->d_pdv, n);
        prof_end(F, s_main, slot2);
        CUDA_TRY(cudaGetLastError());
    }
    if (F->s1) {
        CUDA_TRY(cudaEventRecord(F->s1_out, s_main));
        CUDA_TRY(cudaStreamWaitEvent(s_caller, F->s1_out, 0));
    }
    return MF_OK;
}

extern "C" int mf_factor(mf_factors* F, const double* d_values, mf_stream_t stream) {
    if (!F || !d_values) return MF_EINVAL;
    {
        int rc0 = element_values(F, d_values, (cudaStream_t)stream, &d_values);
        if (rc0) return rc0;
    }
    cudaStream_t s = (cudaStream_t)stream;
    int rc = run_graph(F, 0, d_values, nullptr, nullptr, 0, s, [&](cudaStream_t st) {
        return F->prec == MF_F64 ? run_factor<double>(F, d_values, st) : run_factor<float>(F, d_values, st);
    });
    if (rc == MF_OK) {
        F->factored = true;
        F->rowabs_valid = false;
        F->colabs_valid = false;
    }
    return rc;
}

// One cooperative launch of a persistent substitution sweep (all CTAs resident,
// as many per SM as fit).  Returns MF_ENOTSUP when the sweep cannot be
// resident (the caller then uses per-class launches).
template <typename T, bool TR, bool FWD>
static int launch_sweep(mf_factors* F, const SweepArgs<T>& args, size_t smem, int nrhs, cudaStream_t s) {
    void (*kern)(SweepArgs<T>) = nrhs == 1 ? k_solve_sweep<T, TR, FWD, 1> : k_solve_sweep<T, TR, FWD, kRhsChunk>;
    if (smem > 48 * 1024) CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = 0;
    CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 256, smem));
    if (per_sm < 1) return MF_ENOTSUP;
    CUDA_TRY(cudaMemsetAsync(F->d_bar, 0, 2 * sizeof(unsigned int), s));
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3((unsigned)(per_sm * F->num_sms));
    cfg.blockDim = dim3(256);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    CUDA_TRY(cudaLaunchKernelEx(&cfg, kern, args));
    return MF_OK;
}


// Launch a solve kernel templated on the right-hand-side chunk NR: 1 for a
// single right-hand side, kRhsChunk otherwise.
#define SOLVE_UNPAREN(...) __VA_ARGS__
#define SOLVE_NR(KER, TARGS, CFG, ARGS)                                                                      \
    do {                                                                                                     \
        if (nrhs == 1) CUDA_TRY(launch_dep(KER<SOLVE_UNPAREN TARGS, 1>, SOLVE_UNPAREN CFG, SOLVE_UNPAREN ARGS)); \
        else CUDA_TRY(launch_dep(KER<SOLVE_UNPAREN TARGS, kRhsChunk>, SOLVE_UNPAREN CFG, SOLVE_UNPAREN ARGS));   \
    } while (0)

// The kernels of one substitution class cover disjoint fronts, so they need
// not wait for one another: the first runs on the class's stream, the others
// on side streams that start after everything issued before the class and are
// joined back before the class ends (graph branches under capture).
struct Fan {
    static constexpr int kWays = 3;
    mf_factors* F;
    cudaStream_t s;
    bool on;
    int n = 0;
    bool used[kWays] = {};
    cudaError_t err = cudaSuccess;
    Fan(mf_factors* f, cudaStream_t st, int units) : F(f), s(st), on(units > 1 && !f->fan_off) {
        if (on) err = cudaEventRecord(F->fan_in, s);
        if (err != cudaSuccess) on = false;
    }
    cudaStream_t next() {
        const int i = n++;
        if (!on || i == 0) return s;
        const int j = (i - 1) % kWays;
        if (!used[j]) {
            cudaError_t e = cudaStreamWaitEvent(F->sfan[j], F->fan_in, 0);
            if (e != cudaSuccess) {
                if (err == cudaSuccess) err = e;
                return s;
            }
            used[j] = true;
        }
        return F->sfan[j];
    }
    cudaError_t join() {
        for (int j = 0; j < kWays; j++) {
            if (!used[j]) continue;
            cudaError_t e = cudaEventRecord(F->fan_out[j], F->sfan[j]);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(s, F->fan_out[j], 0);
            if (e != cudaSuccess && err == cudaSuccess) err = e;
        }
        return err;
    }
};

template <typename T>
static int run_solve(mf_factors* F, double* d_x, int nrhs, bool trans, cudaStream_t s, bool trans_b, bool scale_d) {
    // trans: the forward sweep solves with U^T instead of L; trans_b: the backward sweep with L^T
    // instead of U; scale_d: multiply the pivot values by their pivots in between (symmetric factors:
    // x = L^-T D L^-1 b)
    const mf_analysis* a = F->a;
    const T* fac = (const T*)F->d_fac;
    const T* inv = (const T*)F->d_inv;
    T* vec = (T*)F->d_vec;
    T* ys = (T*)F->d_ys;
    const FrontDev* fr = F->d_fronts;
    const SolveRec* L = F->d_srec;
    const int64_t n = a->n_dof, vs = a->vec_size, yss = a->ys_size;
    const size_t dgs = 32 * 33 * sizeof(T);
    if (F->subs.h >= 2) {
        int slot = prof_begin(F, s, FAM_FWD, 0, 0, 1, -1, MF_TRACE_SUBTREE_FWD, 0, (int)F->subs.tasks.size());
        dim3 g((unsigned)F->subs.tasks.size(), nrhs);
        if (!trans)
            k_subtree_fwd<T, false><<<g, 256, F->subs.smem_s, s>>>(fr, F->d_subs_tasks, F->d_subs_euv, fac, F->d_dofs, F->d_maps,
                                                               vec, vs, F->subs.lay_s, d_x, n);
        else
            k_subtree_fwd<T, true><<<g, 256, F->subs.smem_s, s>>>(fr, F->d_subs_tasks, F->d_subs_euv, fac, F->d_dofs, F->d_maps,
                                                              vec, vs, F->subs.lay_s, d_x, n);
        prof_end(F, s, slot);
        CUDA_TRY(cudaGetLastError());
    }
    // classes [c_top, n_cls) run in the persistent sweeps when they are enabled and fit
    const bool sweep = F->use_sweep && !F->sweep_f.empty() && !F->sweep_b.empty();
    int c_top = sweep ? F->sweep_c0 : a->n_cls;
    auto run_sweeps = [&](bool forward) -> int {
        double fb = 0, bb = 0, ff = 0, bf = 0;
        for (int c = F->sweep_c0; c < a->n_cls; c++) {
            fb += F->fwd_bytes[c];
            bb += F->bwd_bytes[c];
            ff += F->fwd_flops[c];
            bf += F->bwd_flops[c];
        }
        SweepArgs<T> args{fr, L, F->d_rows, fac, inv, F->d_dofs, F->d_vsrc, vec, vs, ys, yss, d_x, n, nrhs,
                          forward ? F->d_sweep_f : F->d_sweep_b,
                          (int)(forward ? F->sweep_f.size() : F->sweep_b.size()), F->d_bar, F->d_status};
        int slot = forward ? prof_begin(F, s, FAM_FWD, fb * nrhs, ff * nrhs, 1, -1, MF_TRACE_FWD_SWEEP, -1, args.n_phases)
                           : prof_begin(F, s, FAM_BWD, bb * nrhs, bf * nrhs, 1, -1, MF_TRACE_BWD_SWEEP, -1, args.n_phases);
        int rc;
        if (forward)
            rc = trans ? launch_sweep<T, true, true>(F, args, F->sweep_smem_f, nrhs, s)
                       : launch_sweep<T, false, true>(F, args, F->sweep_smem_f, nrhs, s);
        else
            rc = trans_b ? launch_sweep<T, true, false>(F, args, F->sweep_smem_b, nrhs, s)
                         : launch_sweep<T, false, false>(F, args, F->sweep_smem_b, nrhs, s);
        prof_end(F, s, slot);
        return rc;
    };
    if (sweep) {  // the sweep must be resident before any class relies on it
        int per_sm = 0;
        void (*kf)(SweepArgs<T>) = nrhs == 1 ? (trans ? k_solve_sweep<T, true, true, 1> : k_solve_sweep<T, false, true, 1>)
                                             : (trans ? k_solve_sweep<T, true, true, kRhsChunk>
                                                      : k_solve_sweep<T, false, true, kRhsChunk>);
        void (*kb)(SweepArgs<T>) = nrhs == 1 ? (trans_b ? k_solve_sweep<T, true, false, 1> : k_solve_sweep<T, false, false, 1>)
                                             : (trans_b ? k_solve_sweep<T, true, false, kRhsChunk>
                                                        : k_solve_sweep<T, false, false, kRhsChunk>);
        bool ok = true;
        if (F->sweep_smem_f > 48 * 1024)
            CUDA_TRY(cudaFuncSetAttribute(kf, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)F->sweep_smem_f));
        if (F->sweep_smem_b > 48 * 1024)
            CUDA_TRY(cudaFuncSetAttribute(kb, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)F->sweep_smem_b));
        CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kf, 256, F->sweep_smem_f));
        ok = ok && per_sm >= 1;
        CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kb, 256, F->sweep_smem_b));
        ok = ok && per_sm >= 1;
        if (!ok) c_top = a->n_cls;  // not resident: per-class launches for every class
    }
#define INV_LAUNCH(TR, PH, CNT, OFF)                                                                               \
    if ((PH == PH_BWD1 ? C.maxnc_inv : C.maxk_inv) > 512)                                                          \
        CUDA_TRY(launch_dep(k_inv_gemv<T, TR, PH, 32>, dim3(CNT, nrhs), dim3(1024), (32 * 32 + C.maxin_inv) * sizeof(T), \
                            ls, fr, F->d_rows + (OFF), fac, inv, F->d_dofs, F->d_vsrc, vec, vs, ys, yss, d_x, n,     \
                            PH == PH_FWD2 ? fold : 0));                                                        \
    else                                                                                                           \
        CUDA_TRY(launch_dep(k_inv_gemv<T, TR, PH, 8>, dim3(CNT, nrhs), dim3(256), (8 * 32 + C.maxin_inv) * sizeof(T), \
                            ls, fr, F->d_rows + (OFF), fac, inv, F->d_dofs, F->d_vsrc, vec, vs, ys, yss, d_x, n,     \
                            PH == PH_FWD2 ? fold : 0))
    // the D scaling of symmetric solves goes into the forward kernels' pivot-row stores when every
    // class runs as per-class launches (the subtree and persistent sweeps keep the separate pass)
    const int fold = (scale_d && !trans && F->subs.h < 2 && c_top == a->n_cls) ? 1 : 0;  // always when scaling_folded(F)
    for (int c = 0; c < c_top; c++) {
        const ClassList& C = F->classes_f[c];
        int nk = (C.n_small > 0) + (C.n_cta > 0) + 2 * (C.n_piv > 0) + (C.n_grp[0] > 0) + (C.n_grp[1] > 0) + (C.n_grp[2] > 0) + (C.n_grp[3] > 0);
        for (int q = 0; q < kLgLists; q++) nk += C.n_lg[q] > 0;
        int slot = prof_begin(F, s, FAM_FWD, F->fwd_bytes[c] * nrhs, F->fwd_flops[c] * nrhs, nk, -1, MF_TRACE_FWD_CLASS,
                              c, a->cls_ptr[c + 1] - a->cls_ptr[c]);
        Fan fan(F, s, nk - (C.n_piv > 0));
#define GRP_FWD(Q, GS)                                                                                             \
        if (C.n_grp[Q]) {                                                                                          \
            dim3 g((C.n_grp[Q] + 8 * (32 / GS) - 1) / (8 * (32 / GS)));                                             \
            if (!trans) SOLVE_NR(k_fwd_grp, (T, false, GS), (g, 256, 0, fan.next()), (fr, L + C.off_grp[Q], C.n_grp[Q], fac, F->d_dofs, F->d_vsrc, vec, vs, d_x, n, nrhs, fold)); \
            else SOLVE_NR(k_fwd_grp, (T, true, GS), (g, 256, 0, fan.next()), (fr, L + C.off_grp[Q], C.n_grp[Q], fac, F->d_dofs, F->d_vsrc, vec, vs, d_x, n, nrhs, fold)); \
        }
        GRP_FWD(0, 4)
        GRP_FWD(1, 8)
        GRP_FWD(2, 16)
#undef GRP_FWD
#define LG_FWD(Q)                                                                                           \
        if (C.n_lg[Q]) {                                                                                    \
            const int gq = nrhs == 1 ? kLgG[Q] : kLgGm[Q];                                                  \
            const dim3 g((C.n_lg[Q] + 8 * (32 / gq) - 1) / (8 * (32 / gq)));                               \
            const cudaStream_t ls = fan.next();                                                             \
            if (nrhs == 1) {                                                                                \
                if (!trans) CUDA_TRY(launch_dep(k_fwd_lg<T, false, kLgG[Q], kLgR[Q], kLgKM[Q], 1>, g, dim3(256), 0, ls, L + C.off_lg[Q], C.n_lg[Q], fac, F->d_dofs, F->d_vsrc, vec, vs, d_x, n, nrhs, fold)); \
                else CUDA_TRY(launch_dep(k_fwd_lg<T, true, kLgG[Q], kLgR[Q], kLgKM[Q], 1>, g, dim3(256), 0, ls, L + C.off_lg[Q], C.n_lg[Q], fac, F->d_dofs, F->d_vsrc, vec, vs, d_x, n, nrhs, fold)); \
            } else {                                                                                        \
                if (!trans) CUDA_TRY(launch_dep(k_fwd_lg<T, false, kLgGm[Q], kLgRm[Q], kLgKM[Q], kRhsChunk>, g, dim3(256), 0, ls, L + C.off_lg[Q], C.n_lg[Q], fac, F->d_dofs, F->d_vsrc, vec, vs, d_x, n, nrhs, fold)); \
                else CUDA_TRY(launch_dep(k_fwd_lg<T, true, kLgGm[Q], kLgRm[Q], kLgKM[Q], kRhsChunk>, g, dim3(256), 0, ls, L + C.off_lg[Q], C.n_lg[Q], fac, F->d_dofs, F->d_vsrc, vec, vs, d_x, n, nrhs, fold)); \
            }                                                                                               \
        }
        LG_FWD(0)
        LG_FWD(1)
        LG_FWD(2)
        LG_FWD(3)
        LG_FWD(4)
        LG_FWD(5)
        LG_FWD(6)
        LG_FWD(7)
        LG_FWD(8)
        LG_FWD(9)
        LG_FWD(10)
        LG_FWD(11)
        LG_FWD(12)
        LG_FWD(13)
        LG_FWD(14)
#undef LG_FWD
        if (C.n_grp[3]) {  // 16 < m <= 32: the one-front-per-warp kernel is faster forward
            dim3 g((C.n_grp[3] + 7) / 8);
            if (!trans) SOLVE_NR(k_fwd_warp, (T, false), (g, 256, 0, fan.next()), (fr, L + C.off_grp[3], C.n_grp[3], fac, F->d_dofs, F->d_vsrc, vec, vs, d_x, n, nrhs, fold));
            else SOLVE_NR(k_fwd_warp, (T, true), (g, 256, 0, fan.next()), (fr, L + C.off_grp[3], C.n_grp[3], fac, F->d_dofs, F->d_vsrc, vec, vs, d_x, n, nrhs, fold));
        }
        if (C.n_small) {
            dim3 g((C.n_small + 7) / 8);
            if (!trans) SOLVE_NR(k_fwd_warp, (T, false), (g, 256, 0, fan.next()), (fr, L + C.off_small, C.n_small, fac, F->d_dofs, F->d_vsrc, vec, vs, d_x, n, nrhs, fold));
            else SOLVE_NR(k_fwd_warp, (T, true), (g, 256, 0, fan.next()), (fr, L + C.off_small, C.n_small, fac, F->d_dofs, F->d_vsrc, vec, vs, d_x, n, nrhs, fold));
        }
        if (C.n_cta) {
            dim3 g(C.n_cta);
            const int ldw = C.maxm_cta;
            const cudaStream_t ls = fan.next();
            size_t sm = dgs + (size_t)kRhsChunk * ldw * sizeof(T);
            if (!trans) SOLVE_NR(k_fwd_cta, (T, false), (g, 256, sm, ls), (fr, L + C.off_cta, 1, fac, F->d_dofs, F->d_vsrc, vec, vs, d_x, n, nrhs, ldw, fold));
            else SOLVE_NR(k_fwd_cta, (T, true), (g, 256, sm, ls), (fr, L + C.off_cta, 1, fac, F->d_dofs, F->d_vsrc, vec, vs, d_x, n, nrhs, ldw, fold));
        }
        if (C.n_piv) {
            const cudaStream_t ls = fan.next();
            if (!trans) {
                INV_LAUNCH(false, PH_FWD1, C.n_piv, C.off_piv);
                INV_LAUNCH(false, PH_FWD2, C.n_all, C.off_all);
            } else {
                INV_LAUNCH(true, PH_FWD1, C.n_piv, C.off_piv);
                INV_LAUNCH(true, PH_FWD2, C.n_all, C.off_all);
            }
        }
        CUDA_TRY(fan.join());
        prof_end(F, s, slot);
        CUDA_TRY(cudaGetLastError());
    }
    if (c_top < a->n_cls) {
        int rc = run_sweeps(true);
        if (rc != MF_OK) return rc;
    }
    if (scale_d && !fold) {
        int slot = prof_begin(F, s, FAM_OTHER, (16.0 + 8.0) * n * nrhs, 1.0 * n * nrhs);
        CUDA_TRY(launch_dep(k_scale_pivots, dim3((unsigned)((n * nrhs + 255) / 256)), dim3(256), 0, s, F->d_pdv, d_x, n, nrhs));
        prof_end(F, s, slot);
        CUDA_TRY(cudaGetLastError());
    }
    // the backward sweep: with U (trans_b false) or L^T (trans_b true)
    trans = trans_b;
    if (c_top < a->n_cls) {
        int rc = run_sweeps(false);
        if (rc != MF_OK) return rc;
    }
    for (int c = c_top - 1; c >= 0; c--) {
        const ClassList& C = F->classes_b[c];
        int nk = (C.n_small > 0) + (C.n_cta > 0) + 2 * (C.n_piv > 0) + (C.n_grp[0] > 0) + (C.n_grp[1] > 0) + (C.n_grp[2] > 0) + (C.n_grp[3] > 0);
        for (int q = 0; q < kLgLists; q++) nk += C.n_lg[q] > 0;
        int slot = prof_begin(F, s, FAM_BWD, F->bwd_bytes[c] * nrhs, F->bwd_flops[c] * nrhs, nk, -1, MF_TRACE_BWD_CLASS,
                              c, a->cls_ptr[c + 1] - a->cls_ptr[c]);
        Fan fan(F, s, nk - (C.n_piv > 0));
#define GRP_BWD(Q, GS)                                                                                             \
        if (C.n_grp[Q]) {                                                                                          \
            dim3 g((C.n_grp[Q] + 8 * (32 / GS) - 1) / (8 * (32 / GS)));                                             \
            if (!trans) SOLVE_NR(k_bwd_grp, (T, false, GS), (g, 256, 0, fan.next()), (fr, L + C.off_grp[Q], C.n_grp[Q], fac, F->d_dofs, d_x, n, nrhs)); \
            else SOLVE_NR(k_bwd_grp, (T, true, GS), (g, 256, 0, fan.next()), (fr, L + C.off_grp[Q], C.n_grp[Q], fac, F->d_dofs, d_x, n, nrhs)); \
        }
        GRP_BWD(0, 4)
        GRP_BWD(1, 8)
        GRP_BWD(2, 16)
        GRP_BWD(3, 32)
#undef GRP_BWD
#define LG_BWD(Q)                                                                                           \
        if (C.n_lg[Q]) {                                                                                    \
            const int gq = nrhs == 1 ? kLgG[Q] : kLgGm[Q];                                                  \
            const dim3 g((C.n_lg[Q] + 8 * (32 / gq) - 1) / (8 * (32 / gq)));                               \
            const cudaStream_t ls = fan.next();                                                             \
            if (nrhs == 1) {                                                                                \
                if (!trans) CUDA_TRY(launch_dep(k_bwd_lg<T, false, kLgG[Q], kLgR[Q], kLgKM[Q], 1>, g, dim3(256), 0, ls, L + C.off_lg[Q], C.n_lg[Q], fac, F->d_dofs, d_x, n, nrhs)); \
                else CUDA_TRY(launch_dep(k_bwd_lg<T, true, kLgG[Q], kLgR[Q], kLgKM[Q], 1>, g, dim3(256), 0, ls, L + C.off_lg[Q], C.n_lg[Q], fac, F->d_dofs, d_x, n, nrhs)); \
            } else {                                                                                        \
                if (!trans) CUDA_TRY(launch_dep(k_bwd_lg<T, false, kLgGm[Q], kLgRm[Q], kLgKM[Q], kRhsChunk>, g, dim3(256), 0, ls, L + C.off_lg[Q], C.n_lg[Q], fac, F->d_dofs, d_x, n, nrhs)); \
                else CUDA_TRY(launch_dep(k_bwd_lg<T, true, kLgGm[Q], kLgRm[Q], kLgKM[Q], kRhsChunk>, g, dim3(256), 0, ls, L + C.off_lg[Q], C.n_lg[Q], fac, F->d_dofs, d_x, n, nrhs)); \
            }                                                                                               \
        }
        LG_BWD(0)
        LG_BWD(1)
        LG_BWD(2)
        LG_BWD(3)
        LG_BWD(4)
        LG_BWD(5)
        LG_BWD(6)
        LG_BWD(7)
        LG_BWD(8)
        LG_BWD(9)
        LG_BWD(10)
        LG_BWD(11)
        LG_BWD(12)
        LG_BWD(13)
        LG_BWD(14)
#undef LG_BWD
        if (C.n_piv) {
            const cudaStream_t ls = fan.next();
            if (!trans) {
                INV_LAUNCH(false, PH_BWD1, C.n_piv, C.off_piv);
                INV_LAUNCH(false, PH_BWD2, C.n_piv, C.off_piv);
            } else {
                INV_LAUNCH(true, PH_BWD1, C.n_piv, C.off_piv);
                INV_LAUNCH(true, PH_BWD2, C.n_piv, C.off_piv);
            }
        }
        if (C.n_cta) {
            dim3 g(C.n_cta);
            const int ldw = C.maxm_cta;
            const cudaStream_t ls = fan.next();
            size_t sm = dgs + (size_t)(8 * 64 * kRhsChunk + kRhsChunk * ldw) * sizeof(T);
            if (!trans) SOLVE_NR(k_bwd_cta, (T, false), (g, 256, sm, ls), (fr, L + C.off_cta, 0, fac, F->d_dofs, d_x, n, nrhs, ldw));
            else SOLVE_NR(k_bwd_cta, (T, true), (g, 256, sm, ls), (fr, L + C.off_cta, 0, fac, F->d_dofs, d_x, n, nrhs, ldw));
        }
        if (C.n_small) {
            dim3 g((C.n_small + 7) / 8);
            if (!trans) SOLVE_NR(k_bwd_warp, (T, false), (g, 256, 0, fan.next()), (fr, L + C.off_small, C.n_small, fac, F->d_dofs, d_x, n, nrhs));
            else SOLVE_NR(k_bwd_warp, (T, true), (g, 256, 0, fan.next()), (fr, L + C.off_small, C.n_small, fac, F->d_dofs, d_x, n, nrhs));
        }
        CUDA_TRY(fan.join());
        prof_end(F, s, slot);
        CUDA_TRY(cudaGetLastError());
    }
#undef INV_LAUNCH
    if (F->subs.h >= 2) {
        int slot = prof_begin(F, s, FAM_BWD, 0, 0, 1, -1, MF_TRACE_SUBTREE_BWD, 0, (int)F->subs.tasks.size());
        dim3 g((unsigned)F->subs.tasks.size(), nrhs);
        if (!trans)
            k_subtree_bwd<T, false><<<g, 256, 0, s>>>(fr, F->d_subs_tasks, F->d_subs_euv, fac, F->d_dofs, d_x, n);
        else
            k_subtree_bwd<T, true><<<g, 256, 0, s>>>(fr, F->d_subs_tasks, F->d_subs_euv, fac, F->d_dofs, d_x, n);
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
    if (F->fan_off && d_rhs == F->d_d) {
        // s is capturing the body graph of a conditional node: a solve captured beforehand on its
        // own (prepare_body_solve) enters it as one child-graph node, its class kernels side by side
        for (const auto& b : F->body_solves) {
            if (b.nrhs != nrhs || b.trans != trans) continue;
            cudaStreamCaptureStatus cs;
            cudaGraph_t g = nullptr;
            const cudaGraphNode_t* deps = nullptr;
            size_t nd = 0;
            cudaGraphNode_t node = nullptr;
            CUDA_TRY(cudaStreamGetCaptureInfo(s, &cs, nullptr, &g, &deps, nullptr, &nd));
            if (cs != cudaStreamCaptureStatusActive) return MF_EINVAL;
            CUDA_TRY(cudaGraphAddChildGraphNode(&node, g, deps, nd, b.graph));
            CUDA_TRY(cudaStreamUpdateCaptureDependencies(s, &node, nullptr, 1, cudaStreamSetCaptureDependencies));
            for (int q = 0; q < MF_PROFILE_FAMILIES; q++) {
                F->acc_launch[q] += b.launches[q];
                F->acc_bytes[q] += b.bytes[q];
                F->acc_flops[q] += b.flops[q];
            }
            return MF_OK;
        }
    }
    // symmetric factors: A = A^T = L D^-1 L^T, the same sweeps for the solve and the adjoint solve
    const bool tf = F->sym ? false : trans, tb = F->sym ? true : trans;
    return F->prec == MF_F64 ? run_solve<double>(F, d_rhs, nrhs, tf, s, tb, F->sym)
                             : run_solve<float>(F, d_rhs, nrhs, tf, s, tb, F->sym);
}

// Capture (not run) the solve of F->d_d on the auxiliary stream, for the loop bodies; nothing is
// enqueued and the launch accounting is left as it was.  Without it the bodies solve on one stream.
static void prepare_body_solve(mf_factors* F, int nrhs, bool trans) {
    for (const auto& b : F->body_solves)
        if (b.nrhs == nrhs && b.trans == trans) return;
    mf_factors::BodySolve b{};
    b.nrhs = nrhs;
    b.trans = trans;
    double by[MF_PROFILE_FAMILIES], fl[MF_PROFILE_FAMILIES];
    int64_t ln[MF_PROFILE_FAMILIES];
    for (int q = 0; q < MF_PROFILE_FAMILIES; q++) {
        by[q] = F->acc_bytes[q];
        fl[q] = F->acc_flops[q];
        ln[q] = F->acc_launch[q];
    }
    if (cudaStreamBeginCapture(F->s_aux, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        (void)cudaGetLastError();
        return;
    }
    const int rc = solve_common(F, F->d_d, nrhs, trans, (mf_stream_t)F->s_aux);
    cudaGraph_t g = nullptr;
    const cudaError_t e = cudaStreamEndCapture(F->s_aux, &g);
    for (int q = 0; q < MF_PROFILE_FAMILIES; q++) {
        b.bytes[q] = F->acc_bytes[q] - by[q];
        b.flops[q] = F->acc_flops[q] - fl[q];
        b.launches[q] = F->acc_launch[q] - ln[q];
        F->acc_bytes[q] = by[q];
        F->acc_flops[q] = fl[q];
        F->acc_launch[q] = ln[q];
    }
    if (rc != MF_OK || e != cudaSuccess || !g) {
        if (g) cudaGraphDestroy(g);
        (void)cudaGetLastError();
        return;
    }
    b.graph = g;
    F->body_solves.push_back(b);
}

extern "C" int mf_solve(mf_factors* F, double* d_rhs, int nrhs, mf_stream_t stream) {
    if (!F || !d_rhs || nrhs < 1 || !F->factored || nrhs > F->max_nrhs) return MF_EINVAL;
    return run_graph(F, 3, d_rhs, nullptr, nullptr, nrhs, (cudaStream_t)stream,
                     [&](cudaStream_t st) { return solve_common(F, d_rhs, nrhs, false, (mf_stream_t)st); });
}

extern "C" int mf_solve_adjoint(mf_factors* F, double* d_rhs, int nrhs, mf_stream_t stream) {
    if (!F || !d_rhs || nrhs < 1 || !F->factored || nrhs > F->max_nrhs) return MF_EINVAL;
    return run_graph(F, 4, d_rhs, nullptr, nullptr, nrhs, (cudaStream_t)stream,
                     [&](cudaStream_t st) { return solve_common(F, d_rhs, nrhs, true, (mf_stream_t)st); });
}

static int residual_into(const mf_factors* Fc, const double* d_values, const double* d_x, const double* d_b, double* d_r,
                         int nrhs, cudaStream_t s, bool trans = false) {
    mf_factors* F = const_cast<mf_factors*>(Fc);
    const mf_analysis* a = F->a;
    const int64_t nE = a->n_elem * a->npe;
    int slot = prof_begin(F, s, FAM_RESID, F->resid_bytes * nrhs, F->resid_flops * nrhs, 2);
    const int G = a->npe <= 4 ? 4 : a->npe <= 8 ? 8 : a->npe <= 16 ? 16 : a->npe <= 32 ? 32 : 0;
    if (G) {
        const int64_t nthreads = a->n_elem * G;
        dim3 g1((unsigned)((nthreads + 255) / 256), nrhs);
#define ELEM_APPLY(GS)                                                                                        \
    if (trans) k_elem_apply_grp<GS, true><<<g1, 256, 0, s>>>(d_values, F->d_en, d_x, F->d_Y, a->n_elem, a->npe, a->n_dof); \
    else k_elem_apply_grp<GS, false><<<g1, 256, 0, s>>>(d_values, F->d_en, d_x, F->d_Y, a->n_elem, a->npe, a->n_dof);
        if (G == 4) { ELEM_APPLY(4) }
        else if (G == 8) { ELEM_APPLY(8) }
        else if (G == 16) { ELEM_APPLY(16) }
        else { ELEM_APPLY(32) }
#undef ELEM_APPLY
    } else {
        dim3 g1((unsigned)((nE + 255) / 256), nrhs);
        k_elem_apply<<<g1, 256, 0, s>>>(d_values, F->d_en, d_x, F->d_Y, a->n_elem, a->npe, a->n_dof, 0, trans ? 1 : 0);
    }
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
    int rc = element_values(const_cast<mf_factors*>(F), d_values, (cudaStream_t)stream, &d_values);
    if (rc) return rc;
    return residual_into(F, d_values, d_x, d_b, d_r, nrhs, (cudaStream_t)stream);
}

// row sums of |A| (trans: column sums, the row sums of |A^T|), element by element
static int compute_rowabs(mf_factors* F, const double* d_values, const double* key, cudaStream_t s, bool trans = false) {
    const mf_analysis* a = F->a;
    const int64_t nE = a->n_elem * a->npe;
    dim3 g1((unsigned)((nE + 255) / 256), 1);
    k_elem_apply<<<g1, 256, 0, s>>>(d_values, F->d_en, nullptr, F->d_Y, a->n_elem, a->npe, a->n_dof, 1, trans ? 1 : 0);
    CUDA_TRY(cudaGetLastError());
    dim3 g2((unsigned)((a->n_dof + 255) / 256), 1);
    k_gather_residual<<<g2, 256, 0, s>>>(F->d_node_ptr, F->d_node_inc, F->d_Y, nullptr, trans ? F->d_colabs : F->d_rowabs,
                                         a->n_dof, nE, 1);
    CUDA_TRY(cudaGetLastError());
    if (trans) {
        F->colabs_valid = true;
        F->colabs_values = key;
        return MF_OK;
    }
    F->rowabs_valid = true;
    F->rowabs_values = key;
    return MF_OK;
}

// Refinement of A x = b (trans: A^T x = b with the same factors, the adjoint solve and an
// element-by-element residual with the transposed element matrices).
static int refine_impl(mf_factors* F, const double* d_values, const double* d_b, double* d_x, int nrhs, double tol,
                       int maxit, mf_refine_info* info, mf_stream_t stream, bool trans) {
    if (!F || !d_values || !d_b || !d_x || nrhs < 1 || nrhs > F->max_nrhs || maxit < 0) return MF_EINVAL;
    if (!F->factored) return MF_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    const mf_analysis* a = F->a;
    const int64_t n = a->n_dof;
    int rc;
    const double* key = d_values;  // the caller's array names the cached row sums
    if ((rc = element_values(F, d_values, s, &d_values))) return rc;
    if (!trans && (!F->rowabs_valid || F->rowabs_values != key))
        if ((rc = compute_rowabs(F, d_values, key, s))) return rc;
    if (trans && (!F->colabs_valid || F->colabs_values != key))
        if ((rc = compute_rowabs(F, d_values, key, s, true))) return rc;
    const double* anorm_rows = trans ? F->d_colabs : F->d_rowabs;
    const int kind0 = trans ? 5 : 1;  // graph kinds of the first solve and of one correction
    // the residual and its norms after the current x (device only)
    auto residual_norms = [&](cudaStream_t st) -> int {
        int r2;
        if ((r2 = residual_into(F, d_values, d_x, d_b, F->d_r, nrhs, st, trans))) return r2;
        dim3 gp(F->norm_blocks, nrhs);
        int sl = prof_begin(F, st, FAM_RESID, 24.0 * n * nrhs, 5.0 * n * nrhs, 2);
        k_norms_partial<<<gp, 256, 0, st>>>(F->d_r, d_x, d_b, anorm_rows, n, F->d_part);
        k_norms_final<<<nrhs, 256, 0, st>>>(F->d_part, F->norm_blocks, F->d_norms);
        prof_end(F, st, sl);
        CUDA_TRY(cudaGetLastError());
        return MF_OK;
    };
    // first solve: x = A^-1 b, then residual
    auto start = [&](cudaStream_t st) -> int {
        int sl = prof_begin(F, st, FAM_OTHER, 16.0 * n * nrhs, 0, 0);
        CUDA_TRY(cudaMemcpyAsync(d_x, d_b, sizeof(double) * n * nrhs, cudaMemcpyDeviceToDevice, st));
        prof_end(F, st, sl);
        int r2;
        if ((r2 = solve_common(F, d_x, nrhs, trans, (mf_stream_t)st))) return r2;
        return residual_norms(st);
    };
    // one correction: d = A^-1 r, x += d, then residual
    auto step = [&](cudaStream_t st) -> int {
        int sl = prof_begin(F, st, FAM_OTHER, 16.0 * n * nrhs, 0, 0);
        CUDA_TRY(cudaMemcpyAsync(F->d_d, F->d_r, sizeof(double) * n * nrhs, cudaMemcpyDeviceToDevice, st));
        prof_end(F, st, sl);
        int r2;
        if ((r2 = solve_common(F, F->d_d, nrhs, trans, (mf_stream_t)st))) return r2;
        sl = prof_begin(F, st, FAM_OTHER, 24.0 * n * nrhs, 1.0 * n * nrhs);
        k_axpy<<<(unsigned)((n * nrhs + 255) / 256), 256, 0, st>>>(d_x, F->d_d, n * nrhs);
        prof_end(F, st, sl);
        CUDA_TRY(cudaGetLastError());
        return residual_norms(st);
    };
    std::vector<double> h(6 * nrhs);
    int it = 0;
    double eta = 0, rel = 0;
    auto read_eta = [&]() -> int {
        CUDA_TRY(cudaMemcpyAsync(h.data(), F->d_norms, sizeof(double) * 6 * nrhs, cudaMemcpyDeviceToHost, s));
        CUDA_TRY(cudaStreamSynchronize(s));
        const double anorm = h[5];
        eta = 0;
        rel = 0;
        for (int r = 0; r < nrhs; r++) {
            const double* q = &h[6 * r];
            double den = anorm * q[1] + q[2];
            double e = den > 0 ? q[0] / den : (q[0] > 0 ? INFINITY : 0.0);
            if (std::isnan(e) || e > eta) eta = e;  // a NaN norm is never taken for convergence
            rel = std::max(rel, q[4] > 0 ? std::sqrt(q[3] / q[4]) : std::sqrt(q[3]));
        }
        return MF_OK;
    };
    // Device-side loops (graph replay only): the iterations run inside one graph, as a
    // while-conditional node whose body is one iteration followed by the stop test computed on the
    // device (k_cg_test, the host's test restated); the host reads the norms once per loop.
    // capture_loop records, into the capture under way on st: the iteration counter reset, `first`,
    // the stop test (counting `first` as an iteration when first_inc = 1), then the loop node with
    // `body` + stop test captured into its body graph on the side stream s_body.
    const bool device_loop = F->opt.use_graph && !F->prof && F->sweep_f.empty() && s != nullptr && !F->loop_failed;
    auto capture_loop = [&](cudaStream_t st, auto&& first, auto&& body, int first_inc) -> int {
        int r2;
        CUDA_TRY(cudaMemsetAsync(F->d_cgit, 0, sizeof(int), st));
        if ((r2 = first(st))) return r2;
        cudaStreamCaptureStatus cs;
        cudaGraph_t g = nullptr;
        const cudaGraphNode_t* deps = nullptr;
        size_t nd = 0;
        CUDA_TRY(cudaStreamGetCaptureInfo(st, &cs, nullptr, &g, nullptr, nullptr, nullptr));
        if (cs != cudaStreamCaptureStatusActive) return MF_EINVAL;
        cudaGraphConditionalHandle h;
        CUDA_TRY(cudaGraphConditionalHandleCreate(&h, g, 0, 0));
        prof_begin(F, st, FAM_OTHER, 0.0, 0.0, 1);
        k_cg_test<<<1, 32, 0, st>>>(F->d_norms, nrhs, F->d_cgpar, F->d_cgit, first_inc, h);
        CUDA_TRY(cudaGetLastError());
        CUDA_TRY(cudaStreamGetCaptureInfo(st, &cs, nullptr, &g, &deps, nullptr, &nd));
        cudaGraphNodeParams cp{};
        cp.type = cudaGraphNodeTypeConditional;
        cp.conditional.handle = h;
        cp.conditional.type = cudaGraphCondTypeWhile;
        cp.conditional.size = 1;
        cudaGraphNode_t node;
        CUDA_TRY(cudaGraphAddNode(&node, g, deps, nullptr, nd, &cp));
        CUDA_TRY(cudaStreamUpdateCaptureDependencies(st, &node, nullptr, 1, cudaStreamSetCaptureDependencies));
        CUDA_TRY(cudaStreamBeginCaptureToGraph(F->s_body, cp.conditional.phGraph_out[0], nullptr, nullptr, 0,
                                               cudaStreamCaptureModeThreadLocal));
        for (int q = 0; q < MF_PROFILE_FAMILIES; q++) {
            F->body_launch[q] = F->acc_launch[q];
            F->body_bytes[q] = F->acc_bytes[q];
            F->body_flops[q] = F->acc_flops[q];
        }
        F->fan_off = true;  // the body graph of a conditional node is captured on one stream
        r2 = body(F->s_body);
        F->fan_off = false;
        if (r2 == MF_OK) {
            prof_begin(F, F->s_body, FAM_OTHER, 0.0, 0.0, 1);
            k_cg_test<<<1, 32, 0, F->s_body>>>(F->d_norms, nrhs, F->d_cgpar, F->d_cgit, 1, h);
        }
        for (int q = 0; q < MF_PROFILE_FAMILIES; q++) {
            F->body_launch[q] = F->acc_launch[q] - F->body_launch[q];
            F->body_bytes[q] = F->acc_bytes[q] - F->body_bytes[q];
            F->body_flops[q] = F->acc_flops[q] - F->body_flops[q];
        }
        cudaGraph_t bg = nullptr;
        const cudaError_t e1 = cudaGetLastError(), e2 = cudaStreamEndCapture(F->s_body, &bg);
        if (r2 != MF_OK) return r2;
        if (e1 != cudaSuccess || e2 != cudaSuccess) return MF_ECUDA;
        return MF_OK;
    };
    // runs a loop graph (kind) and adds the iterations it ran to `it`
    auto run_loop_graph = [&](int kind, auto&& enqueue_loop) -> int {
        int cnt = 0;
        k_cg_params<<<1, 1, 0, s>>>(F->d_cgpar, tol, maxit - it);
        CUDA_TRY(cudaGetLastError());
        int r2;
        if ((r2 = run_graph(F, kind, d_values, d_b, d_x, nrhs, s, enqueue_loop))) return r2;
        CUDA_TRY(cudaMemcpyAsync(&cnt, F->d_cgit, sizeof(int), cudaMemcpyDeviceToHost, s));
        if ((r2 = read_eta())) return r2;  // synchronises s
        it += cnt;
        // the graph's accounting holds one body pass; the replay ran max(cnt - first_inc, 0) of them
        const int extra = cnt - F->loop_first_inc - 1;
        for (int q = 0; q < MF_PROFILE_FAMILIES; q++) {
            F->acc_launch[q] += (int64_t)extra * F->body_launch[q];
            F->acc_bytes[q] += extra * F->body_bytes[q];
            F->acc_flops[q] += extra * F->body_flops[q];
        }
        return MF_OK;
    };
    if (device_loop && !(F->sym && F->opt.refine_cg && !trans)) {
        // stationary refinement: the first solve, then corrections until the stop test holds
        F->loop_first_inc = 0;
        prepare_body_solve(F, nrhs, trans);
        auto st_loop = [&](cudaStream_t st) -> int { return capture_loop(st, start, step, 0); };
        if ((rc = run_loop_graph(trans ? 12 : 11, st_loop)) == MF_OK) {
            if (info) {
                info->iterations = it;
                info->backward_error = eta;
                info->rel_residual = rel;
            }
            return eta <= tol ? MF_OK : MF_ENOCONV;
        }
        (void)cudaGetLastError();  // no loop graph was captured (nothing of it ran): host-driven loop
        F->loop_failed = true;
        it = 0;
    }
    if ((rc = run_graph(F, kind0, d_values, d_b, d_x, nrhs, s, start))) return rc;
    if ((rc = read_eta())) return rc;
    if (F->sym && F->opt.refine_cg && !trans && maxit > 0 && eta > tol && std::isfinite(eta)) {
        // Preconditioned conjugate gradients in FP64, M^-1 = L^-T D L^-1 from the FP32 factors:
        //   cg_step(first): z = M^-1 r; rho' = r^T z; p = z (first) or z + (rho'/rho) p; rho = rho';
        //                   s = -A p; x += alpha p, r += alpha s, alpha = -rho / p^T s; norms of r
        // The loop stops on the recursively updated residual, then recomputes the true one (the
        // start graph's residual step) and restarts from the current x if drift left it above tol.
        const unsigned nb = (unsigned)F->norm_blocks;
        const dim3 gv((unsigned)((n + 255) / 256), nrhs);
        auto cg_step = [&](bool first) {
            return [&, first](cudaStream_t st) -> int {
                int sl = prof_begin(F, st, FAM_OTHER, 16.0 * n * nrhs, 0, 0);
                CUDA_TRY(cudaMemcpyAsync(F->d_d, F->d_r, sizeof(double) * n * nrhs, cudaMemcpyDeviceToDevice, st));
                prof_end(F, st, sl);
                int r2;
                if ((r2 = solve_common(F, F->d_d, nrhs, false, (mf_stream_t)st))) return r2;
                sl = prof_begin(F, st, FAM_OTHER, 16.0 * n * nrhs, 2.0 * n * nrhs, 2);
                k_dot_partial<<<dim3(nb, nrhs), 256, 0, st>>>(F->d_r, F->d_d, n, F->d_part);
                k_dot_final<<<nrhs, 256, 0, st>>>(F->d_part, nb, F->d_cg, first ? 0 : 2);
                prof_end(F, st, sl);
                sl = prof_begin(F, st, FAM_OTHER, 24.0 * n * nrhs, 2.0 * n * nrhs, first ? 1 : 2);
                k_cg_p<<<gv, 256, 0, st>>>(F->d_cgp, F->d_d, F->d_cg, n, first ? 1 : 0);
                if (!first) k_cg_commit<<<1, 32, 0, st>>>(F->d_cg, nrhs);
                prof_end(F, st, sl);
                CUDA_TRY(cudaGetLastError());
                if ((r2 = residual_into(F, d_values, F->d_cgp, F->d_zero, F->d_cgs, nrhs, st, false))) return r2;
                sl = prof_begin(F, st, FAM_OTHER, 48.0 * n * nrhs, 6.0 * n * nrhs, 3);
                k_dot_partial<<<dim3(nb, nrhs), 256, 0, st>>>(F->d_cgp, F->d_cgs, n, F->d_part);
                k_dot_final<<<nrhs, 256, 0, st>>>(F->d_part, nb, F->d_cg, 1);
                k_cg_xr<<<gv, 256, 0, st>>>(d_x, F->d_r, F->d_cgp, F->d_cgs, F->d_cg, n);
                prof_end(F, st, sl);
                CUDA_TRY(cudaGetLastError());
                sl = prof_begin(F, st, FAM_RESID, 24.0 * n * nrhs, 5.0 * n * nrhs, 2);
                k_norms_partial<<<dim3(nb, nrhs), 256, 0, st>>>(F->d_r, d_x, d_b, anorm_rows, n, F->d_part);
                k_norms_final<<<nrhs, 256, 0, st>>>(F->d_part, nb, F->d_norms);
                prof_end(F, st, sl);
                CUDA_TRY(cudaGetLastError());
                return MF_OK;
            };
        };
        auto true_residual = [&](cudaStream_t st) -> int { return residual_norms(st); };
        // With graph replay the CG iterations run in one loop graph: the restart step and its stop
        // test, then the loop node whose body is one CG step and the stop test.
        auto cg_loop = [&](cudaStream_t st) -> int { return capture_loop(st, cg_step(true), cg_step(false), 1); };
        auto run_loop = [&]() -> int {
            F->loop_first_inc = 1;
            prepare_body_solve(F, nrhs, false);
            return run_loop_graph(10, cg_loop);
        };
        bool loop_built = device_loop;
        if (device_loop && (rc = run_loop())) {
            // no loop graph was captured (nothing of it ran): keep to the host-driven iteration
            (void)cudaGetLastError();
            F->loop_failed = true;
            loop_built = false;
            it = 0;
        }
        if (loop_built) {
            for (;;) {
                if (!std::isfinite(eta)) break;
                if ((rc = run_graph(F, 9, d_values, d_b, d_x, nrhs, s, true_residual))) return rc;
                if ((rc = read_eta())) return rc;
                if (eta <= tol || it >= maxit || !std::isfinite(eta)) break;
                if ((rc = run_loop())) return rc;  // the true residual drifted above tol: restart
            }
            if (info) {
                info->iterations = it;
                info->backward_error = eta;
                info->rel_residual = rel;
            }
            return eta <= tol ? MF_OK : MF_ENOCONV;
        }
        // graph kinds 7-9: CG restart step, CG step, true residual (forward system only)
        if ((rc = run_graph(F, 7, d_values, d_b, d_x, nrhs, s, cg_step(true)))) return rc;
        it = 1;
        for (;;) {
            if ((rc = read_eta())) return rc;
            if (!std::isfinite(eta)) break;
            if (eta <= tol || it >= maxit) {
                if ((rc = run_graph(F, 9, d_values, d_b, d_x, nrhs, s, true_residual))) return rc;
                if ((rc = read_eta())) return rc;
                if (eta <= tol || it >= maxit || !std::isfinite(eta)) break;
                if ((rc = run_graph(F, 7, d_values, d_b, d_x, nrhs, s, cg_step(true)))) return rc;
                it++;
                continue;
            }
            if ((rc = run_graph(F, 8, d_values, d_b, d_x, nrhs, s, cg_step(false)))) return rc;
            it++;
        }
    } else {
        for (;;) {
            if (eta <= tol || it >= maxit || !std::isfinite(eta)) break;
            if ((rc = run_graph(F, kind0 + 1, d_values, d_b, d_x, nrhs, s, step))) return rc;
            it++;
            if ((rc = read_eta())) return rc;
        }
    }
    if (info) {
        info->iterations = it;
        info->backward_error = eta;
        info->rel_residual = rel;
    }
    return eta <= tol ? MF_OK : MF_ENOCONV;
}

extern "C" int mf_refine_solve(mf_factors* F, const double* d_values, const double* d_b, double* d_x, int nrhs, double tol,
                               int maxit, mf_refine_info* info, mf_stream_t stream) {
    return refine_impl(F, d_values, d_b, d_x, nrhs, tol, maxit, info, stream, false);
}

extern "C" int mf_refine_solve_adjoint(mf_factors* F, const double* d_values, const double* d_b, double* d_x, int nrhs,
                                       double tol, int maxit, mf_refine_info* info, mf_stream_t stream) {
    return refine_impl(F, d_values, d_b, d_x, nrhs, tol, maxit, info, stream, true);
}

extern "C" int mf_element_grad(const mf_factors* F, const double* d_dvalues, const double* d_lambda, const double* d_x,
                               double* d_grad, mf_stream_t stream) {
    if (!F || !d_dvalues || !d_lambda || !d_x || !d_grad) return MF_EINVAL;
    const mf_analysis* a = F->a;
    if (a->csr_n > 0) return MF_ENOTSUP;  // a CSR matrix has no elements to differentiate by
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
    if (a->csr_n > 0) return MF_ENOTSUP;
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

int mf_profile_read_buckets(mf_factors* F, double* ms) {
    if (!F || !ms) return MF_EINVAL;
    CUDA_TRY(cudaDeviceSynchronize());
    for (int b = 0; b < MF_FUSED_BUCKETS; b++) ms[b] = 0;
    for (size_t i = 0; i < F->ev_used; i++) {
        const int b = F->ev_tag[i];
        if (b < 0 || b >= MF_FUSED_BUCKETS) continue;
        float e = 0.f;
        CUDA_TRY(cudaEventElapsedTime(&e, F->ev[2 * i], F->ev[2 * i + 1]));
        ms[b] += e;
    }
    return MF_OK;
}

extern "C" int mf_profile_trace(mf_factors* F, mf_trace_rec* out, int cap, int* n) {
    if (!F || !n || cap < 0 || (cap > 0 && !out)) return MF_EINVAL;
    CUDA_TRY(cudaDeviceSynchronize());
    *n = (int)F->ev_used;
    for (size_t i = 0; i < F->ev_used && (int)i < cap; i++) {
        float e = 0.f;
        CUDA_TRY(cudaEventElapsedTime(&e, F->ev[2 * i], F->ev[2 * i + 1]));
        out[i] = F->ev_rec[i];
        out[i].ms = e;
    }
    return MF_OK;
}

extern "C" int mf_profile_read(mf_factors* F, double* ms, int64_t* launches, double* bytes, double* flops) {
    if (!F) return MF_EINVAL;
    CUDA_TRY(cudaDeviceSynchronize());
    double t[MF_PROFILE_FAMILIES] = {};
    for (size_t i = 0; i < F->ev_used; i++) {
        float e = 0.f;
        CUDA_TRY(cudaEventElapsedTime(&e, F->ev[2 * i], F->ev[2 * i + 1]));
        t[F->ev_rec[i].family] += e;
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

// ------------------------------------------------------------- testing hooks
extern "C" void mf_test_fail_alloc(int64_t n) { g_alloc_countdown.store(n < 0 ? -1 : (long long)n); }

namespace {
// One CTA arrives at the substitution sweep's grid barrier expecting a second
// CTA that is never launched: the bounded wait must give up and record a
// timeout.  No asynchronous copies are in flight in this kernel.
__global__ void k_test_bounded_wait(unsigned int* bar, DevStatus* st, unsigned long long limit_ns) {
    (void)sweep_barrier(bar, 2u, st, limit_ns);
}
}  // namespace

extern "C" int mf_test_bounded_wait(mf_factors* F, double limit_ms, mf_stream_t stream) {
    if (!F || !(limit_ms > 0.0) || limit_ms > 10000.0) return MF_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    CUDA_TRY(cudaMemsetAsync(F->d_bar, 0, 2 * sizeof(unsigned int), s));
    k_test_bounded_wait<<<1, 32, 0, s>>>(F->d_bar, F->d_status, (unsigned long long)(limit_ms * 1e6));
    CUDA_TRY(cudaGetLastError());
    // leave the barrier as a sweep launch expects it (every sweep launch clears it again anyway)
    CUDA_TRY(cudaMemsetAsync(F->d_bar, 0, 2 * sizeof(unsigned int), s));
    return MF_OK;
}
