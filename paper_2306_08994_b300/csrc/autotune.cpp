// Plan autotuner (mf_autotune): times the launch plan's free choices on the
// caller's problem and keeps the fastest.  The class order of the fronts is
// fixed by Sec. 3.3; only how one class is cut into launches is tuned.
// Results persist in a JSON Lines cache keyed by the device and the shape of
// the analysis.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <fstream>
#include <string>
#include <vector>

#include "mf_internal.h"

namespace {

struct Timer {
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    Timer() {
        cudaEventCreate(&e0);
        cudaEventCreate(&e1);
    }
    ~Timer() {
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
    }
};

// Version of the launch-plan builder: bumped whenever its kernels or its
// decomposition change enough that plans tuned before are stale.
constexpr int kPlanVersion = 7;
constexpr double kTuneTol = 1e-12;  // refinement target of the timed candidates

int family_of(int precision) { return precision == MF_F64 ? 0 : 1; }

std::string cache_key(const mf_analysis* a, int precision, int symmetric, int refine_cg) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceProp p{};
    cudaGetDeviceProperties(&p, dev);
    std::string name = p.name;
    for (char& c : name)
        if (c == '"' || c == '\\' || c == ':') c = '_';
    char buf[512];
    std::snprintf(buf, sizeof buf, "plan%d:%s:sm%d:%s:dim%d:npe%d:meshes%d:n%lld:fronts%d:classes%d:maxm%d:maxk%d:flops%.6e",
                  kPlanVersion, name.c_str(), p.multiProcessorCount, family_of(precision) == 0 ? "f64" : "f32", a->dim, a->npe,
                  a->n_meshes, (long long)a->n_dof, a->n_front, a->n_cls, a->info.max_m, a->info.max_k,
                  a->info.factor_flops);
    std::string key = buf;
    // symmetric factors and CG refinement are timed as such: their plans are cached apart (the general
    // LU with stationary refinement keeps the key it always had)
    if (symmetric) key += refine_cg ? ":sym:cg" : ":sym";
    return key;
}

// Value after `"field":` in a one-line JSON object, or nullptr.
const char* field(const std::string& line, const char* name) {
    std::string pat = std::string("\"") + name + "\":";
    size_t at = line.find(pat);
    return at == std::string::npos ? nullptr : line.c_str() + at + pat.size();
}

bool cache_lookup(const char* path, const std::string& key, mf_options* o, double* ms) {
    std::ifstream in(path);
    if (!in) return false;
    std::string line, hit;
    const std::string want = "\"key\":\"" + key + "\"";
    while (std::getline(in, line))
        if (line.find(want) != std::string::npos) hit = line;  // the last entry wins
    if (hit.empty()) return false;
    const char* v;
    mf_options t = *o;
    if (!(v = field(hit, "precision"))) return false;
    t.precision = std::atoi(v);
    if (!(v = field(hit, "small_front_max"))) return false;
    t.small_front_max = std::atoi(v);
    if (!(v = field(hit, "subtree_levels"))) return false;
    t.subtree_levels = std::atoi(v);
    if (!(v = field(hit, "tc_min_cb"))) return false;
    t.tc_min_cb = std::atoi(v);
    if (!(v = field(hit, "super_panel"))) return false;
    t.super_panel = std::atoi(v);
    if (!(v = field(hit, "subtree_solve_levels"))) return false;
    t.subtree_solve_levels = std::atoi(v);
    if (!(v = field(hit, "lookahead"))) return false;
    t.lookahead = std::atoi(v);
    if (!(v = field(hit, "fused_threads")) || *v != '[') return false;
    v++;
    for (int b = 0; b < MF_FUSED_BUCKETS; b++) {
        char* end = nullptr;
        long x = std::strtol(v, &end, 10);
        if (end == v) return false;
        t.fused_threads[b] = (int)x;
        v = end;
        while (*v == ',' || *v == ' ') v++;
    }
    if (family_of(t.precision) != family_of(o->precision)) return false;
    *o = t;
    if (ms && (v = field(hit, "ms_best"))) *ms = std::atof(v);
    return true;
}

void cache_append(const char* path, const std::string& key, const mf_options& o, double ms_best, double ms_default,
                  int candidates) {
    FILE* fp = std::fopen(path, "a");
    if (!fp) return;
    std::fprintf(fp, "{\"key\":\"%s\",\"precision\":%d,\"small_front_max\":%d,\"subtree_levels\":%d,\"tc_min_cb\":%d,"
                     "\"super_panel\":%d,\"subtree_solve_levels\":%d,\"lookahead\":%d,\"fused_threads\":[",
                 key.c_str(), o.precision, o.small_front_max, o.subtree_levels, o.tc_min_cb, o.super_panel,
                 o.subtree_solve_levels, o.lookahead);
    for (int b = 0; b < MF_FUSED_BUCKETS; b++) std::fprintf(fp, "%s%d", b ? "," : "", o.fused_threads[b]);
    std::fprintf(fp, "],\"ms_best\":%.4f,\"ms_default\":%.4f,\"candidates\":%d}\n", ms_best, ms_default, candidates);
    std::fclose(fp);
}

struct Ctx {
    const mf_analysis* a;
    const double* d_values;
    const double* d_b;
    double* d_x;
    int reps;
    cudaStream_t s;
    int timed = 0;
};

// Median time (ms) of factor + refined solve (FP64 refinement to a normwise
// backward error of kTuneTol) under options o: the refinement's number of
// corrections depends on the plan (front precision, where the SIMT / tensor-
// core and fused / blocked crossovers fall), so it is part of the objective.
// Returns an error code for plans that cannot be built, fail or do not reach
// the tolerance.
int time_plan(Ctx& c, const mf_options& o, double* ms) {
    mf_factors* F = nullptr;
    int rc = mf_factors_create(c.a, &o, &F);
    if (rc) return rc;
    Timer t;
    std::vector<float> v;
    const size_t bytes = sizeof(double) * (size_t)c.a->n_dof;
    for (int r = 0; r <= c.reps && rc == MF_OK; r++) {
        if (cudaMemcpyAsync(c.d_x, c.d_b, bytes, cudaMemcpyDeviceToDevice, c.s) != cudaSuccess) rc = MF_ECUDA;
        if (!rc && cudaEventRecord(t.e0, c.s) != cudaSuccess) rc = MF_ECUDA;
        if (!rc) rc = mf_factor(F, c.d_values, c.s);
        mf_refine_info ri{};
        if (!rc) rc = mf_refine_solve(F, c.d_values, c.d_b, c.d_x, 1, kTuneTol, 30, &ri, c.s);
        if (!rc && cudaEventRecord(t.e1, c.s) != cudaSuccess) rc = MF_ECUDA;
        if (!rc && cudaEventSynchronize(t.e1) != cudaSuccess) rc = MF_ECUDA;
        float e = 0.f;
        if (!rc && r > 0) {  // the first run builds and captures the graphs
            cudaEventElapsedTime(&e, t.e0, t.e1);
            v.push_back(e);
        }
    }
    if (!rc) {
        mf_status_info st{};
        rc = mf_status(F, &st);
    }
    mf_free_factors(F);
    if (rc) return rc;
    std::sort(v.begin(), v.end());
    *ms = v[v.size() / 2];
    c.timed++;
    return MF_OK;
}

// Per-bucket times of the fused kernel with every bucket at `threads`.
int time_buckets(Ctx& c, const mf_options& base, int threads, double* ms) {
    mf_options o = base;
    o.use_graph = 0;
    o.subtree_levels = 0;
    o.small_front_max = kFusedBounds[(family_of(o.precision) == 0 ? kFusedBuckets64 : MF_FUSED_BUCKETS) - 1];
    for (int b = 0; b < MF_FUSED_BUCKETS; b++) o.fused_threads[b] = threads;
    mf_factors* F = nullptr;
    int rc = mf_factors_create(c.a, &o, &F);
    if (rc) return rc;
    rc = mf_factor(F, c.d_values, c.s);  // untimed first run
    if (!rc) rc = mf_profile_enable(F, 1);
    for (int r = 0; r < c.reps && !rc; r++) rc = mf_factor(F, c.d_values, c.s);
    if (!rc) rc = mf_profile_read_buckets(F, ms);
    if (!rc) rc = mf_profile_read(F, nullptr, nullptr, nullptr, nullptr);
    if (!rc) {
        mf_status_info st{};
        rc = mf_status(F, &st);
    }
    mf_free_factors(F);
    c.timed++;
    return rc;
}

}  // namespace

extern "C" int mf_autotune(const mf_analysis* a, const double* d_values, const double* d_b, const mf_options* base,
                           int reps, const char* cache_path, mf_options* best, mf_tune_info* info, mf_stream_t stream) {
    if (!a || !d_values || !d_b || !best || reps < 1) return MF_EINVAL;
    mf_options o = base ? mf_resolve_options(base) : a->opt;
    if (o.precision != MF_F64 && o.precision != MF_F32 && o.precision != MF_TF32 && o.precision != MF_TF32_BF16)
        return MF_EINVAL;
    const int user_graph = o.use_graph;
    const std::string key = cache_key(a, o.precision, o.symmetric, o.refine_cg);
    if (info) *info = mf_tune_info{};
    if (cache_path) {
        mf_options t = o;
        double ms = 0;
        if (cache_lookup(cache_path, key, &t, &ms)) {
            t.use_graph = user_graph;
            *best = t;
            if (info) {
                info->ms_best = ms;
                info->from_cache = 1;
            }
            return MF_OK;
        }
    }
    cudaStream_t s = (cudaStream_t)stream;
    double* d_x = nullptr;
    if (mf_alloc_should_fail() || cudaMalloc(&d_x, sizeof(double) * (size_t)a->n_dof) != cudaSuccess) return MF_ENOMEM;
    Ctx c{a, d_values, d_b, d_x, reps, s};
    int rc = MF_OK;
    o.use_graph = 1;
    double ms_default = 0, ms_best = 0;
    rc = time_plan(c, o, &ms_default);
    ms_best = ms_default;
    mf_options cur = o;

    // (1) threads per fused size bucket: one profiled sweep per thread count
    if (!rc) {
        const int cand[] = {32, 64, 128, 256};
        double best_b[MF_FUSED_BUCKETS];
        int pick[MF_FUSED_BUCKETS] = {};
        for (int b = 0; b < MF_FUSED_BUCKETS; b++) best_b[b] = 1e300;
        for (int t : cand) {
            double ms[MF_FUSED_BUCKETS];
            int r = time_buckets(c, cur, t, ms);
            if (r) {
                rc = r;
                break;
            }
            for (int b = 0; b < MF_FUSED_BUCKETS; b++)
                if (ms[b] > 0 && ms[b] < best_b[b]) {
                    best_b[b] = ms[b];
                    pick[b] = t;
                }
        }
        if (!rc) {
            mf_options t = cur;
            for (int b = 0; b < MF_FUSED_BUCKETS; b++) t.fused_threads[b] = pick[b];
            double ms = 0;
            rc = time_plan(c, t, &ms);
            if (!rc && ms < ms_best) {
                ms_best = ms;
                cur = t;
            }
        }
    }
    // (2) fused / blocked crossover, (3) subtree fusion depth, (4) Schur GEMM engine
    auto try_one = [&](const mf_options& t) {
        double ms = 0;
        int r = time_plan(c, t, &ms);
        if (r == MF_ENOMEM || r == MF_ECUDA) rc = r;  // anything else: the candidate is skipped
        if (!r && ms < ms_best) {
            ms_best = ms;
            cur = t;
        }
    };
    if (!rc) {
        const mf_options start = cur;
        const int n = family_of(o.precision) == 0 ? kFusedBuckets64 : MF_FUSED_BUCKETS;
        for (int b = 3; b < n && !rc; b++) {
            mf_options t = start;
            t.small_front_max = kFusedBounds[b];
            if (t.small_front_max != start.small_front_max) try_one(t);
        }
    }
    if (!rc) {
        const mf_options start = cur;
        for (int lv : {0, 3, 4, 5}) {
            if (rc) break;
            mf_options t = start;
            t.subtree_levels = lv;
            if (lv != start.subtree_levels) try_one(t);
        }
    }
    if (!rc) {
        const mf_options start = cur;
        for (int lv : {-1, 4, 6, 8}) {
            if (rc) break;
            mf_options t = start;
            t.subtree_solve_levels = lv;
            if (lv != start.subtree_solve_levels) try_one(t);
        }
    }
    if (!rc) {
        const mf_options start = cur;
        for (int sp : {64, 128, 256, 512}) {
            if (rc) break;
            mf_options t = start;
            t.super_panel = sp;
            if (sp != start.super_panel) try_one(t);
        }
    }
    if (!rc) {  // one-panel lookahead on / off
        mf_options t = cur;
        t.lookahead = cur.lookahead >= 0 ? -1 : 0;
        try_one(t);
    }
    if (!rc && family_of(o.precision) == 1) {
        const mf_options start = cur;
        mf_options t = start;
        t.precision = start.precision == MF_F32 ? MF_TF32 : MF_F32;
        if (t.precision == MF_TF32) t.tc_min_cb = 128;
        try_one(t);
        for (int tmin : {256, 512, 1024}) {
            if (rc) break;
            mf_options u = start;
            u.precision = MF_TF32;
            u.tc_min_cb = tmin;
            try_one(u);
        }
    }
    if (!rc && family_of(o.precision) == 1) {
        // the super-panel depth and the tensor-core crossover interact (the deep trailing products
        // of a super-panel are tensor-core candidates): a joint pass over both
        const mf_options start = cur;
        for (int sp : {64, 128, 256, 512})
            for (int tmin : {0, 128, 256, 512}) {  // 0: SIMT products only (MF_F32)
                if (rc) break;
                mf_options t = start;
                t.super_panel = sp;
                t.precision = tmin ? MF_TF32 : MF_F32;
                t.tc_min_cb = tmin;
                if (sp != start.super_panel || t.precision != start.precision || tmin != start.tc_min_cb) try_one(t);
            }
        if (!rc) {
            mf_options t = cur;
            t.lookahead = cur.lookahead >= 0 ? -1 : 0;
            try_one(t);
        }
    }
    cudaFree(d_x);
    if (rc) return rc;
    if (cache_path) cache_append(cache_path, key, cur, ms_best, ms_default, c.timed);
    cur.use_graph = user_graph;
    *best = cur;
    if (info) {
        info->ms_default = ms_default;
        info->ms_best = ms_best;
        info->candidates = c.timed;
        info->from_cache = 0;
    }
    return MF_OK;
}
