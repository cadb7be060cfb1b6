// Symbolic analysis (host): elimination tree, pivot sets, front dof lists,
// child-to-parent maps, Foata classes and arena offsets.
//
// Paper anchors (arXiv 2306.08994):
//  * Sec. 2.4 steps 1-5 and Table 3: the tree is built bottom-up from element
//    fronts by joining neighbouring fronts pairwise.  Here the pairing is
//    produced top-down by recursive bisection of the element set (longest
//    axis, floor split, ties x < y < z); on 2^L grids this is the same tree
//    as joining Morton-sorted element fronts pairwise.
//  * Table 2 `compute_front`: a pivot may be eliminated in a front once it
//    belongs to that front only ("front_membership_count == 1").  A dof's
//    pivot front is therefore the lowest common ancestor of the leaves of the
//    elements touching it.
//  * Sec. 3.2: each front is reordered with its pivots first, then the dofs
//    shared with other fronts (its contribution block).
//  * Sec. 3.3: fronts of equal height form one Foata class (no front of a
//    class depends on another; each class needs only the previous ones).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>
#include <stdexcept>

#include "mf_internal.h"

namespace {

// ---------------------------------------------------------------- trees
struct Box {
    int32_t lo[3], hi[3];
};

void bisect_box(const int32_t nel[3], HostTree& t) {
    int64_t ne = (int64_t)nel[0] * nel[1] * nel[2];
    t.parent.assign(2 * ne - 1, -1);
    t.child.assign(2 * (2 * ne - 1), -1);
    t.leaf_elem.assign(2 * ne - 1, -1);
    int32_t next = 0;
    // recursive bisection producing postorder ids
    struct Rec {
        const int32_t* nel;
        HostTree& t;
        int32_t& next;
        int32_t operator()(const Box& b) {
            int32_t n[3] = {b.hi[0] - b.lo[0], b.hi[1] - b.lo[1], b.hi[2] - b.lo[2]};
            if ((int64_t)n[0] * n[1] * n[2] == 1) {
                int32_t id = next++;
                t.leaf_elem[id] = b.lo[0] + nel[0] * (b.lo[1] + nel[1] * b.lo[2]);
                return id;
            }
            int ax = 0;
            if (n[1] > n[ax]) ax = 1;
            if (n[2] > n[ax]) ax = 2;
            Box l = b, r = b;
            l.hi[ax] = b.lo[ax] + n[ax] / 2;
            r.lo[ax] = l.hi[ax];
            int32_t a = (*this)(l);
            int32_t c = (*this)(r);
            int32_t id = next++;
            t.child[2 * id] = a;
            t.child[2 * id + 1] = c;
            t.parent[a] = id;
            t.parent[c] = id;
            return id;
        }
    } rec{nel, t, next};
    Box root{{0, 0, 0}, {nel[0], nel[1], nel[2]}};
    rec(root);
}

void bisect_coords(int64_t ne, int dim, const double* cen, HostTree& t) {
    t.parent.assign(2 * ne - 1, -1);
    t.child.assign(2 * (2 * ne - 1), -1);
    t.leaf_elem.assign(2 * ne - 1, -1);
    std::vector<int32_t> ids(ne);
    std::iota(ids.begin(), ids.end(), 0);
    int32_t next = 0;
    struct Rec {
        int dim;
        const double* cen;
        HostTree& t;
        int32_t& next;
        int32_t operator()(int32_t* b, int64_t n) {
            if (n == 1) {
                int32_t id = next++;
                t.leaf_elem[id] = b[0];
                return id;
            }
            double mn[3] = {1e300, 1e300, 1e300}, mx[3] = {-1e300, -1e300, -1e300};
            for (int64_t i = 0; i < n; i++)
                for (int d = 0; d < dim; d++) {
                    double c = cen[(int64_t)b[i] * dim + d];
                    mn[d] = std::min(mn[d], c);
                    mx[d] = std::max(mx[d], c);
                }
            int ax = 0;
            for (int d = 1; d < dim; d++)
                if (mx[d] - mn[d] > mx[ax] - mn[ax]) ax = d;
            std::sort(b, b + n, [&](int32_t p, int32_t q) {
                double cp = cen[(int64_t)p * dim + ax], cq = cen[(int64_t)q * dim + ax];
                return cp < cq || (cp == cq && p < q);
            });
            int64_t h = n / 2;
            int32_t a = (*this)(b, h);
            int32_t c = (*this)(b + h, n - h);
            int32_t id = next++;
            t.child[2 * id] = a;
            t.child[2 * id + 1] = c;
            t.parent[a] = id;
            t.parent[c] = id;
            return id;
        }
    } rec{dim, cen, t, next};
    rec(ids.data(), ne);
}

inline double pivot_flops(int64_t m, int64_t k) {
    // sum over pivots p < k of (m-p-1) divisions + 2 (m-p-1)^2 mult/sub; t = m-p-1 in [m-k, m-1]
    double a = (double)(m - k), b = (double)(m - 1);
    if (k <= 0) return 0.0;
    double s1 = (a + b) * (b - a + 1) / 2.0;
    double s2 = b * (b + 1) * (2 * b + 1) / 6.0 - (a - 1) * a * (2 * a - 1) / 6.0;
    return s1 + 2.0 * s2;
}

inline int64_t align_up(int64_t x, int64_t a) { return (x + a - 1) / a * a; }

}  // namespace

int mf_build_tree(const mf_mesh_desc* mesh, HostTree& t) {
    if (mesh->n_elem < 1) return MF_EINVAL;
    if (mesh->grid_dims) {
        const int32_t* g = mesh->grid_dims;
        if (g[0] < 1 || g[1] < 1 || g[2] < 1) return MF_EINVAL;
        if ((int64_t)g[0] * g[1] * g[2] != mesh->n_elem) return MF_EINVAL;
        bisect_box(g, t);
        return MF_OK;
    }
    if (!mesh->elem_centroid) return MF_EINVAL;
    bisect_coords(mesh->n_elem, mesh->dim, mesh->elem_centroid, t);
    return MF_OK;
}

mf_options mf_resolve_options(const mf_options* opt) {
    mf_options o;
    mf_default_options(&o);
    if (opt) o = *opt;
    if (o.max_nrhs <= 0) o.max_nrhs = 4;
    return o;
}

// Symbolic analysis of a batch of meshes (a forest).  Each mesh keeps its own
// tree; classes are aligned from the leaves.
int mf_symbolic(const mf_mesh_desc* meshes, int count, const mf_options* opt, mf_analysis* a,
                const HostTree* pretree) {
    if (pretree && count != 1) return MF_EINVAL;
    if (count < 1 || !meshes) return MF_EINVAL;
    a->opt = mf_resolve_options(opt);
    a->npe = meshes[0].nodes_per_elem;
    a->dim = meshes[0].dim;
    a->n_meshes = count;
    if (a->npe < 1 || a->npe > 64) return MF_EINVAL;
    int64_t n_dof = 0, n_elem = 0;
    for (int i = 0; i < count; i++) {
        const mf_mesh_desc& m = meshes[i];
        if (m.nodes_per_elem != a->npe || m.n_nodes < 1 || m.n_elem < 1 || !m.elem_nodes) return MF_EINVAL;
        if (m.dim != 2 && m.dim != 3) return MF_EINVAL;
        n_dof += m.n_nodes;
        n_elem += m.n_elem;
    }
    if (n_dof >= INT32_MAX || 2 * n_elem >= INT32_MAX) return MF_ENOTSUP;
    a->n_dof = n_dof;
    a->n_elem = n_elem;
    const int npe = a->npe;

    // forest in "tree order": mesh by mesh, each tree in postorder
    std::vector<int32_t> tparent, tchild, tleaf;   // tree-order arrays (global element ids)
    std::vector<int32_t> height;
    a->elem_nodes.resize(n_elem * npe);
    {
        int64_t dof0 = 0, el0 = 0;
        for (int i = 0; i < count; i++) {
            const mf_mesh_desc& m = meshes[i];
            HostTree t;
            if (pretree) {
                t = *pretree;
            } else {
                int rc = mf_build_tree(&m, t);
                if (rc) return rc;
            }
            int32_t base = (int32_t)tparent.size();
            for (size_t v = 0; v < t.parent.size(); v++) {
                tparent.push_back(t.parent[v] < 0 ? -1 : t.parent[v] + base);
                tchild.push_back(t.child[2 * v] < 0 ? -1 : t.child[2 * v] + base);
                tchild.push_back(t.child[2 * v + 1] < 0 ? -1 : t.child[2 * v + 1] + base);
                tleaf.push_back(t.leaf_elem[v] < 0 ? -1 : (int32_t)(t.leaf_elem[v] + el0));
            }
            for (int64_t j = 0; j < m.n_elem * npe; j++) {
                int64_t d = m.elem_nodes[j];
                if (d < 0 || d >= m.n_nodes) return MF_EINVAL;
                a->elem_nodes[el0 * npe + j] = d + dof0;
            }
            dof0 += m.n_nodes;
            el0 += m.n_elem;
        }
    }
    const int32_t nt = (int32_t)tparent.size();
    height.assign(nt, 1);
    std::vector<int32_t> depth(nt, 0);
    for (int32_t v = 0; v < nt; v++)  // postorder: children first
        for (int c = 0; c < 2; c++) {
            int32_t ch = tchild[2 * v + c];
            if (ch >= 0) height[v] = std::max(height[v], height[ch] + 1);
        }
    for (int32_t v = nt - 1; v >= 0; v--)  // parents have larger ids
        if (tparent[v] >= 0) depth[v] = depth[tparent[v]] + 1;

    // leaf of each element
    std::vector<int32_t> leaf_of(n_elem, -1);
    for (int32_t v = 0; v < nt; v++)
        if (tleaf[v] >= 0) leaf_of[tleaf[v]] = v;

    // pivot front of every dof: LCA (by depth) of the leaves of its elements
    std::vector<int32_t> elim(n_dof, -1);
    auto lca = [&](int32_t x, int32_t y) {
        while (depth[x] > depth[y]) x = tparent[x];
        while (depth[y] > depth[x]) y = tparent[y];
        while (x != y) {
            x = tparent[x];
            y = tparent[y];
        }
        return x;
    };
    for (int64_t e = 0; e < n_elem; e++) {
        int32_t lv = leaf_of[e];
        for (int j = 0; j < npe; j++) {
            int64_t d = a->elem_nodes[e * npe + j];
            elim[d] = elim[d] < 0 ? lv : lca(elim[d], lv);
        }
    }
    for (int64_t d = 0; d < n_dof; d++)
        if (elim[d] < 0) return MF_EINVAL;  // a dof no element touches: singular

    // pivot lists (ascending dof) via counting sort
    std::vector<int64_t> kptr(nt + 1, 0);
    for (int64_t d = 0; d < n_dof; d++) kptr[elim[d] + 1]++;
    for (int32_t v = 0; v < nt; v++) kptr[v + 1] += kptr[v];
    std::vector<int32_t> piv(n_dof);
    {
        std::vector<int64_t> fill(kptr.begin(), kptr.end() - 1);
        for (int64_t d = 0; d < n_dof; d++) piv[fill[elim[d]]++] = (int32_t)d;
    }

    // contribution-block sets bottom-up: merge the children's sorted sets
    // (leaf: the sorted element dofs) and drop this front's pivots
    std::vector<std::vector<int32_t>> cb(nt);
    std::vector<int32_t> tm(nt), tk(nt);
    std::vector<std::vector<int32_t>> fdofs(nt);
    std::vector<int32_t> buf;
    for (int32_t v = 0; v < nt; v++) {
        buf.clear();
        if (tleaf[v] >= 0) {
            int64_t e = tleaf[v];
            for (int j = 0; j < npe; j++) buf.push_back((int32_t)a->elem_nodes[e * npe + j]);
            std::sort(buf.begin(), buf.end());
            buf.erase(std::unique(buf.begin(), buf.end()), buf.end());
        } else {
            int32_t c0 = tchild[2 * v], c1 = tchild[2 * v + 1];
            if (c1 < 0) {
                buf = cb[c0];
            } else {
                buf.resize(cb[c0].size() + cb[c1].size());
                auto it = std::set_union(cb[c0].begin(), cb[c0].end(), cb[c1].begin(), cb[c1].end(), buf.begin());
                buf.resize(it - buf.begin());
            }
        }
        std::vector<int32_t>& out = cb[v];
        out.clear();
        for (int32_t d : buf)
            if (elim[d] != v) out.push_back(d);
        tk[v] = (int32_t)(kptr[v + 1] - kptr[v]);
        tm[v] = tk[v] + (int32_t)out.size();
        std::vector<int32_t>& fd = fdofs[v];
        fd.assign(piv.begin() + kptr[v], piv.begin() + kptr[v + 1]);
        fd.insert(fd.end(), out.begin(), out.end());
        // children's CB sets are still needed for the maps; freed below
    }

    // class-major renumbering
    int32_t H = *std::max_element(height.begin(), height.end());
    a->n_cls = H;
    a->n_front = nt;
    a->cls_ptr.assign(H + 1, 0);
    for (int32_t v = 0; v < nt; v++) a->cls_ptr[height[v]]++;
    for (int32_t c = 0; c < H; c++) a->cls_ptr[c + 1] += a->cls_ptr[c];
    std::vector<int32_t> newid(nt);
    {
        std::vector<int32_t> fill(a->cls_ptr.begin(), a->cls_ptr.end() - 1);
        for (int32_t v = 0; v < nt; v++) newid[v] = fill[height[v] - 1]++;
    }
    std::vector<int32_t> oldid(nt);
    for (int32_t v = 0; v < nt; v++) oldid[newid[v]] = v;

    a->fronts.assign(nt, FrontDev{});
    a->parent.assign(nt, -1);
    a->dofs.clear();
    a->maps.clear();
    int64_t fac = 0, cbo = 0, vec = 0, inv = 0, ysz = 0;
    std::vector<int32_t> where(n_dof, -1), stamp(n_dof, -1);
    double flops = 0;
    int64_t nnz = 0, scb = 0;
    int32_t maxm = 0, maxk = 0, rootm = 0;
    for (int32_t f = 0; f < nt; f++) {
        int32_t v = oldid[f];
        FrontDev& F = a->fronts[f];
        F.m = tm[v];
        F.k = tk[v];
        F.cls = height[v] - 1;
        F.elem = tleaf[v];
        F.nchild = 0;
        F.child[0] = F.child[1] = -1;
        for (int c = 0; c < 2; c++)
            if (tchild[2 * v + c] >= 0) F.child[F.nchild++] = newid[tchild[2 * v + c]];
        a->parent[f] = tparent[v] >= 0 ? newid[tparent[v]] : -1;
        const int64_t m = F.m, k = F.k;
        int64_t al = (m * k >= 1024) ? 32 : 4;
        fac = align_up(fac, al);
        F.P_off = fac;
        fac += m * k;
        fac = align_up(fac, al);
        F.R_off = fac;
        fac += k * (m - k);
        int64_t alc = ((m - k) * (m - k) >= 1024) ? 32 : 4;
        cbo = align_up(cbo, alc);
        F.S_off = cbo;
        cbo += (m - k) * (m - k);
        F.vec_off = vec;
        vec += m - k;
        if (k >= kInvMinK) {
            inv = align_up(inv, 32);
            F.q_off = inv;
            inv += k * k;
            F.y_off = ysz;
            ysz += k;
        } else {
            F.q_off = -1;
            F.y_off = -1;
        }
        F.dof_off = (int64_t)a->dofs.size();
        const std::vector<int32_t>& fd = fdofs[v];
        a->dofs.insert(a->dofs.end(), fd.begin(), fd.end());
        F.map_off = (int64_t)a->maps.size();
        for (int32_t i = 0; i < (int32_t)m; i++) where[fd[i]] = i;
        if (F.elem >= 0) {
            // front row i holds element-local node map[i]
            std::vector<int32_t> mp(m, -1);
            for (int j = 0; j < npe; j++) {  // first occurrence: a repeated node's later copies carry zeros
                int32_t d = (int32_t)a->elem_nodes[(int64_t)F.elem * npe + j];
                if (mp[where[d]] < 0) mp[where[d]] = j;
            }
            a->maps.insert(a->maps.end(), mp.begin(), mp.end());
        } else {
            for (int c = 0; c < 2; c++) {
                int32_t ch = tchild[2 * v + c];
                if (ch < 0) continue;
                std::vector<int32_t> mp(m, -1);
                const std::vector<int32_t>& ccb = cb[ch];
                for (int32_t t = 0; t < (int32_t)ccb.size(); t++) mp[where[ccb[t]]] = t;
                a->maps.insert(a->maps.end(), mp.begin(), mp.end());
            }
        }
        flops += pivot_flops(m, k);
        nnz += m * k + k * (m - k);
        scb += (m - k) * (m - k);
        maxm = std::max<int32_t>(maxm, F.m);
        maxk = std::max<int32_t>(maxk, F.k);
        if (a->parent[f] < 0) rootm = std::max<int32_t>(rootm, F.m);
    }
    (void)stamp;
    a->factor_size = align_up(fac, 32);
    a->cb_size = align_up(std::max<int64_t>(cbo, 1), 32);
    a->vec_size = std::max<int64_t>(vec, 1);
    a->inv_size = std::max<int64_t>(align_up(inv, 32), 32);
    a->ys_size = std::max<int64_t>(ysz, 1);

    // dof -> (element, local) incidence for the element-by-element residual
    a->node_ptr.assign(n_dof + 1, 0);
    for (int64_t j = 0; j < n_elem * npe; j++) a->node_ptr[a->elem_nodes[j] + 1]++;
    for (int64_t d = 0; d < n_dof; d++) a->node_ptr[d + 1] += a->node_ptr[d];
    a->node_inc.resize(n_elem * npe);
    {
        std::vector<int64_t> fill(a->node_ptr.begin(), a->node_ptr.end() - 1);
        for (int64_t j = 0; j < n_elem * npe; j++) a->node_inc[fill[a->elem_nodes[j]]++] = j;
    }

    mf_info& I = a->info;
    I.n_dof = n_dof;
    I.n_elem = n_elem;
    I.n_front = nt;
    I.n_meshes = count;
    I.n_classes = H;
    I.max_m = maxm;
    I.max_k = maxk;
    I.root_m = rootm;
    int64_t sk = 0;
    for (int32_t f = 0; f < nt; f++) sk += a->fronts[f].k;
    I.sum_k = sk;
    I.nnz_lu = nnz;
    I.sum_cb = scb;
    I.factor_flops = flops;
    I.solve_flops = 2.0 * (double)nnz;
    return MF_OK;
}
