// Internal data structures shared by the analysis (host), the executor and
// the kernels of libmfsolve.
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include "mfsolve.h"

// One front as the kernels see it.  Fronts are numbered class by class
// (class = height in the elimination tree, Sec. 3.3 Foata classes at front
// granularity), so the fronts of one class are contiguous.
//
// The front F (m x m) is never stored whole.  After assembly its three parts
// live where they end up:
//   P = F[:, 0:k]    m x k,     column-major, ld m,   in the factor arena
//   R = F[0:k, k:m]  k x (m-k), column-major, ld k,   in the factor arena
//   S = F[k:m, k:m]  (m-k)^2,   column-major, ld m-k, in the contribution-block arena
// The partial LU turns P into [L11\U11; L21] and R into U12, and the Schur
// update turns S into the contribution block the parent pulls in.
struct FrontDev {
    int32_t m, k;
    int32_t nchild;   // 0 for a leaf
    int32_t elem;     // leaf: element id; internal: -1
    int32_t child[2]; // children (class-order ids) or -1
    int32_t cls;      // 0-based class
    int32_t pad;
    int64_t P_off;    // factor arena offset of P
    int64_t R_off;    // factor arena offset of R
    int64_t S_off;    // CB arena offset of S
    int64_t vec_off;  // update-vector arena offset ((m-k) per right-hand side)
    int64_t map_off;  // into maps: internal: nchild blocks of m int32 (child CB index of each
                      // front row, -1 if the row is not in that child's CB); leaf: m int32
                      // (element-local node of each front row)
    int64_t dof_off;  // into dofs: m global dof ids (pivots ascending, then CB ascending)
    int64_t q_off;    // fronts with k >= kInvMinK: inverse-arena offset of Q (k x k: L11^-1 on and
                      // below the diagonal, strict upper part of U11^-1); otherwise -1
    int64_t y_off;    // same fronts: offset of their k pivot values in the solve's pivot scratch
};

// Fronts with at least this many pivots get explicit pivot-block inverses,
// so their triangular solves run as wide products.
constexpr int kInvMinK = 64;

struct mf_analysis {
    mf_options opt;
    int dim = 0, npe = 0, n_meshes = 0;
    int64_t n_dof = 0, n_elem = 0;
    int32_t n_front = 0, n_cls = 0;
    std::vector<FrontDev> fronts;     // class-ordered
    std::vector<int32_t> parent;      // class-order parent id, -1 at roots
    std::vector<int32_t> cls_ptr;     // n_cls + 1
    std::vector<int32_t> dofs;
    std::vector<int32_t> maps;
    std::vector<int64_t> elem_nodes;  // n_elem * npe (batch: global dof ids)
    std::vector<int64_t> node_ptr;    // n_dof + 1: incidence CSR (dof -> e*npe + a)
    std::vector<int64_t> node_inc;
    int64_t factor_size = 0, cb_size = 0, vec_size = 0, inv_size = 0, ys_size = 0;
    mf_info info{};
    // CSR input (mf_analyze_csr): the matrix is split into one arrowhead element per vertex; the
    // numeric entry points take the caller's CSR values and scatter entry q to element-array
    // position csr_dest[q] (n_elem * npe * npe doubles, zero elsewhere)
    int64_t csr_n = 0, csr_nnz = 0;  // csr_n = 0: a mesh analysis
    std::vector<int64_t> csr_dest;
};

// Upper bounds on m of the fused small-front kernel's size buckets (FP64
// fronts use the first kFusedBuckets64: a 160 x 160 FP64 front fills the
// shared memory of one CTA).
constexpr int kFusedBounds[MF_FUSED_BUCKETS] = {16, 32, 48, 64, 96, 128, 160, 192, 224};
constexpr int kFusedBuckets64 = 7;

struct mf_factors;
// Fused-kernel time per size bucket (ms) over the launches profiled since the
// last mf_profile_read; synchronises.  Used by the plan autotuner.
int mf_profile_read_buckets(mf_factors* f, double* ms);

// Bisection trees.  Nodes in postorder; child[2v], child[2v+1]; leaf_elem -1
// for internal nodes.
struct HostTree {
    std::vector<int32_t> parent, child, leaf_elem;
};

int mf_build_tree(const mf_mesh_desc* mesh, HostTree& t);
// pretree (count == 1 only): use this element tree instead of cutting one from the mesh geometry
int mf_symbolic(const mf_mesh_desc* meshes, int count, const mf_options* opt, mf_analysis* a,
                const HostTree* pretree = nullptr);

// Options with defaults filled in.
mf_options mf_resolve_options(const mf_options* opt);

// Test hook (mf_test_fail_alloc): true when this device allocation is the one
// chosen to fail.  Every device allocation of the library asks first.
bool mf_alloc_should_fail();
