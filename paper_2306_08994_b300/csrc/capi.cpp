// C ABI: options, error strings and the analysis entry points.  The factor,
// solve and refinement entry points live in executor.cu.
#include <cstring>
#include <new>

#include "mf_internal.h"

extern "C" void mf_default_options(mf_options* o) {
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    o->precision = MF_F64;
    o->pivot_tol = 0.0;
    o->pivot_fail = 0;
    o->small_front_max = 0;
    o->panel_width = 0;
    o->use_graph = 0;
    o->max_nrhs = 4;
    o->subtree_levels = 0;
}

extern "C" const char* mf_strerror(int code) {
    switch (code) {
        case MF_OK: return "ok";
        case MF_EINVAL: return "invalid argument or handle";
        case MF_ENOMEM: return "out of memory";
        case MF_ECUDA: return "CUDA runtime error";
        case MF_EZERO_PIVOT: return "pivot below the static threshold";
        case MF_ENOCONV: return "refinement did not converge";
        case MF_ETIMEOUT: return "bounded device wait timed out";
        case MF_ENOTSUP: return "not supported";
        case MF_ETOOLARGE: return "larger than the static scratch of mf_residual_noalloc";
        default: return "unknown error";
    }
}

extern "C" int mf_analyze_batch(const mf_mesh_desc* meshes, int count, const mf_options* opt, mf_analysis** out) {
    if (!out) return MF_EINVAL;
    *out = nullptr;
    mf_analysis* a = new (std::nothrow) mf_analysis();
    if (!a) return MF_ENOMEM;
    int rc;
    try {
        rc = mf_symbolic(meshes, count, opt, a);
    } catch (const std::bad_alloc&) {
        rc = MF_ENOMEM;
    } catch (...) {
        rc = MF_EINVAL;
    }
    if (rc) {
        delete a;
        return rc;
    }
    *out = a;
    return MF_OK;
}

extern "C" int mf_analyze_mesh(const mf_mesh_desc* mesh, const mf_options* opt, mf_analysis** out) {
    return mf_analyze_batch(mesh, 1, opt, out);
}

extern "C" int mf_analysis_info(const mf_analysis* a, mf_info* out) {
    if (!a || !out) return MF_EINVAL;
    *out = a->info;
    return MF_OK;
}

extern "C" int mf_analysis_export(const mf_analysis* a, int32_t* parent, int32_t* cls, int32_t* m, int32_t* k,
                                  int64_t* dof_ptr, int32_t* dofs) {
    if (!a) return MF_EINVAL;
    for (int32_t f = 0; f < a->n_front; f++) {
        const FrontDev& F = a->fronts[f];
        if (parent) parent[f] = a->parent[f];
        if (cls) cls[f] = F.cls;
        if (m) m[f] = F.m;
        if (k) k[f] = F.k;
        if (dof_ptr) dof_ptr[f] = F.dof_off;
    }
    if (dof_ptr) dof_ptr[a->n_front] = (int64_t)a->dofs.size();
    if (dofs) std::memcpy(dofs, a->dofs.data(), a->dofs.size() * sizeof(int32_t));
    return MF_OK;
}

extern "C" void mf_free_analysis(mf_analysis* a) { delete a; }
