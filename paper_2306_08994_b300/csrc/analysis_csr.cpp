// Symbolic analysis of a general sparse matrix given in CSR form.
//
// The paper applies its method to finite-element systems whose matrix is
// symmetric and invertible (Sec. 2.1), and builds the elimination tree
// bottom-up from element fronts (Sec. 2.4, Table 3).  A CSR matrix carries
// no elements and no coordinates, so both are made here:
//
//  * Tree.  The vertex set of the matrix graph (pattern of A + A^T) is cut in
//    two recursively until single vertices remain.  Each cut orders the
//    part's vertices by breadth-first distance from a pseudo-peripheral
//    vertex of the part (George and Liu's level structure) and finds the
//    level d holding the median vertex.  A level is a vertex separator, but
//    on graphs of higher-order elements one level spans several rows of
//    nodes, so the cut is narrowed: a minimum vertex separator between the
//    levels below d and the levels above d + 1 is found inside the band of
//    levels d and d + 1 by maximum flow (unit vertex capacities, Dinic's
//    algorithm); the band vertices reachable from the lower side join it, the
//    rest go to the upper side.  The result is a binary tree whose leaves are
//    the vertices, numbered in postorder, like the element trees of the mesh
//    analysis.
//  * Elements.  Vertex w's element holds the diagonal entry a_ww and, for
//    every off-diagonal pair {u, w} assigned to w, the entries a_wu and a_uw
//    (an "arrowhead": rows and columns {w, u_1, u_2, ...}, zero elsewhere).
//    Summing the elements gives A exactly.  The pair {u, v} goes to the
//    endpoint whose leaf comes first in postorder, i.e. the one on the left
//    side of the cut that separates them; then a vertex on the left side of a
//    cut is touched only by left-side elements and is eliminated below the
//    cut, while its right-side neighbours across the cut are touched from the
//    left and are eliminated at the cut: the right-side boundary of each cut
//    is its vertex separator.
//  * Elements have different sizes; they are padded to the largest (at most
//    64 nodes) by repeating the element's own vertex with zero rows and
//    columns, so the rest of the library sees a mesh with a fixed number of
//    nodes per element.  The analysis keeps, for every CSR entry, its place
//    in that element array; the numeric entry points scatter the caller's CSR
//    values there before they run.
//
// After that the mesh analysis (pivot sets by the lowest-common-ancestor rule,
// pivots-first fronts, child maps, Foata classes) runs unchanged.
#include <algorithm>
#include <cstring>
#include <new>
#include <numeric>

#include "mf_internal.h"

namespace {

struct Graph {
    int64_t n;
    std::vector<int64_t> ptr;
    std::vector<int32_t> adj;
};

// Pattern of A + A^T without the diagonal, sorted and without duplicates.
int build_graph(int64_t n, const int64_t* rowptr, const int32_t* col, Graph& g) {
    std::vector<int64_t> deg(n + 1, 0);
    for (int64_t i = 0; i < n; i++)
        for (int64_t q = rowptr[i]; q < rowptr[i + 1]; q++) {
            const int64_t j = col[q];
            if (j == i) continue;
            deg[i + 1]++;
            deg[j + 1]++;
        }
    for (int64_t i = 0; i < n; i++) deg[i + 1] += deg[i];
    std::vector<int32_t> adj(deg[n]);
    std::vector<int64_t> fill(deg.begin(), deg.end() - 1);
    for (int64_t i = 0; i < n; i++)
        for (int64_t q = rowptr[i]; q < rowptr[i + 1]; q++) {
            const int64_t j = col[q];
            if (j == i) continue;
            adj[fill[i]++] = (int32_t)j;
            adj[fill[j]++] = (int32_t)i;
        }
    g.n = n;
    g.ptr.assign(n + 1, 0);
    g.adj.clear();
    g.adj.reserve(adj.size());
    for (int64_t i = 0; i < n; i++) {
        auto b = adj.begin() + deg[i], e = adj.begin() + deg[i + 1];
        std::sort(b, e);
        e = std::unique(b, e);
        g.adj.insert(g.adj.end(), b, e);
        g.ptr[i + 1] = (int64_t)g.adj.size();
    }
    return MF_OK;
}

// Maximum flow by Dinic's algorithm (level graph by BFS, blocking flow by an
// iterative depth-first search), then the set reachable from the source in
// the residual graph.
struct MaxFlow {
    struct Edge {
        int32_t to, next;
        int32_t cap;
    };
    std::vector<int32_t> head, level, it;
    std::vector<Edge> e;
    explicit MaxFlow(int32_t n) : head(n, -1), level(n), it(n) {}
    void add(int32_t u, int32_t v, int32_t c) {  // edge 2q and its reverse 2q + 1
        e.push_back({v, head[u], c});
        head[u] = (int32_t)e.size() - 1;
        e.push_back({u, head[v], 0});
        head[v] = (int32_t)e.size() - 1;
    }
    bool bfs(int32_t s, int32_t t) {
        std::fill(level.begin(), level.end(), -1);
        std::vector<int32_t> q{s};
        level[s] = 0;
        for (size_t i = 0; i < q.size(); i++)
            for (int32_t x = head[q[i]]; x >= 0; x = e[x].next)
                if (e[x].cap > 0 && level[e[x].to] < 0) {
                    level[e[x].to] = level[q[i]] + 1;
                    q.push_back(e[x].to);
                }
        return level[t] >= 0;
    }
    int64_t run(int32_t s, int32_t t) {
        int64_t flow = 0;
        std::vector<int32_t> path;  // edge ids from s
        while (bfs(s, t)) {
            it = head;
            path.clear();
            int32_t u = s;
            for (;;) {
                if (u == t) {
                    int32_t b = INT32_MAX;
                    for (int32_t x : path) b = std::min(b, e[x].cap);
                    for (int32_t x : path) {
                        e[x].cap -= b;
                        e[x ^ 1].cap += b;
                    }
                    flow += b;
                    path.clear();
                    u = s;
                    continue;
                }
                int32_t& x = it[u];
                while (x >= 0 && !(e[x].cap > 0 && level[e[x].to] == level[u] + 1)) x = e[x].next;
                if (x >= 0) {
                    path.push_back(x);
                    u = e[x].to;
                    continue;
                }
                if (u == s) break;  // blocking flow found
                level[u] = -1;      // dead end: prune it and step back
                const int32_t back = path.back();
                path.pop_back();
                u = e[back ^ 1].to;
                it[u] = e[it[u]].next;
            }
        }
        return flow;
    }
    void reachable(int32_t s, std::vector<char>& seen) const {
        seen.assign(head.size(), 0);
        std::vector<int32_t> q{s};
        seen[s] = 1;
        for (size_t i = 0; i < q.size(); i++)
            for (int32_t x = head[q[i]]; x >= 0; x = e[x].next)
                if (e[x].cap > 0 && !seen[e[x].to]) {
                    seen[e[x].to] = 1;
                    q.push_back(e[x].to);
                }
    }
};

// Recursive level-structure bisection of the vertex set into a binary tree
// with one leaf per vertex (postorder ids; leaf_elem = vertex).
struct Bisector {
    const Graph& g;
    HostTree& t;
    std::vector<int32_t> part;   // current part id of each vertex (only vertices of the part are followed)
    std::vector<int32_t> dist;   // BFS distance scratch (-1 = unvisited)
    int32_t next = 0;
    int32_t next_part = 1;

    Bisector(const Graph& gr, HostTree& tr) : g(gr), t(tr), part(gr.n, 0), dist(gr.n, -1) {}

    // BFS over the part's vertices from `root`, then from the part's remaining
    // vertices in list order; writes the visiting order into `order`.  Returns
    // the depth of root's own component and leaves its last level's
    // minimum-degree vertex in *far.
    int32_t bfs(const std::vector<int32_t>& verts, int32_t root, int32_t pid, std::vector<int32_t>& order,
                int32_t* far, std::vector<int32_t>* lvl = nullptr, size_t* comp = nullptr) {
        order.clear();
        int32_t depth = 0, far_v = root;
        int64_t far_deg = INT64_MAX;
        size_t start = 0;
        auto run = [&](int32_t r, bool first) {
            dist[r] = 0;
            order.push_back(r);
            while (start < order.size()) {
                const int32_t v = order[start++];
                if (first) {
                    const int64_t dv = g.ptr[v + 1] - g.ptr[v];
                    if (dist[v] > depth || (dist[v] == depth && dv < far_deg)) {
                        depth = dist[v];
                        far_v = v;
                        far_deg = dv;
                    }
                }
                for (int64_t q = g.ptr[v]; q < g.ptr[v + 1]; q++) {
                    const int32_t u = g.adj[q];
                    if (part[u] != pid || dist[u] >= 0) continue;
                    dist[u] = dist[v] + 1;
                    order.push_back(u);
                }
            }
        };
        run(root, true);
        if (comp) *comp = order.size();
        for (int32_t v : verts)
            if (dist[v] < 0) run(v, false);
        if (lvl) {
            lvl->resize(order.size());
            for (size_t i = 0; i < order.size(); i++) (*lvl)[i] = dist[order[i]];
        }
        for (int32_t v : order) dist[v] = -1;
        if (far) *far = far_v;
        return depth;
    }

    // The minimum vertex separator inside the band of levels d and d + 1 (d = the median vertex's
    // level) between the levels below and above it; left = the lower levels and the band vertices
    // reachable from them in the residual graph.  False if the band does not separate anything.
    bool narrow_cut(const std::vector<int32_t>& order, const std::vector<int32_t>& lvl, int64_t h, int32_t pid,
                    std::vector<int32_t>& left, std::vector<int32_t>& right) {
        const int32_t d = lvl[h];
        if (d == 0) return false;
        int32_t nb = 0;
        for (size_t i = 0; i < order.size(); i++)
            if (lvl[i] == d || lvl[i] == d + 1) dist[order[i]] = nb++;  // dist doubles as the band index
        bool above = false;
        for (size_t i = 0; i < order.size(); i++) above |= lvl[i] > d + 1;
        if (!above) {
            for (size_t i = 0; i < order.size(); i++)
                if (lvl[i] == d || lvl[i] == d + 1) dist[order[i]] = -1;
            return false;
        }
        // levels by vertex: the band's own, and below/above from the BFS order
        const int32_t S = 2 * nb, T = 2 * nb + 1;
        MaxFlow fl(2 * nb + 2);
        constexpr int32_t kInf = 1 << 28;
        std::vector<int32_t> bandv(nb);
        for (size_t i = 0; i < order.size(); i++)
            if (lvl[i] == d || lvl[i] == d + 1) bandv[dist[order[i]]] = order[i];
        std::vector<int32_t> lev_of(nb);
        for (size_t i = 0; i < order.size(); i++)
            if (lvl[i] == d || lvl[i] == d + 1) lev_of[dist[order[i]]] = lvl[i];
        for (int32_t b = 0; b < nb; b++) {
            const int32_t v = bandv[b];
            fl.add(2 * b, 2 * b + 1, 1);
            bool lo = false, hi = false;
            for (int64_t q = g.ptr[v]; q < g.ptr[v + 1]; q++) {
                const int32_t u = g.adj[q];
                if (part[u] != pid) continue;
                const int32_t bu = dist[u];
                if (bu >= 0) {
                    fl.add(2 * b + 1, 2 * bu, kInf);
                } else {
                    // a part vertex outside the band: below if v is on level d, above if on level d + 1
                    // (BFS levels of neighbours differ by at most one)
                    if (lev_of[b] == d) lo = true;
                    else hi = true;
                }
            }
            if (lo) fl.add(S, 2 * b, kInf);
            if (hi) fl.add(2 * b + 1, T, kInf);
        }
        fl.run(S, T);
        std::vector<char> seen;
        fl.reachable(S, seen);
        for (size_t i = 0; i < order.size(); i++) {
            const int32_t v = order[i];
            if (lvl[i] < d) left.push_back(v);
            else if (lvl[i] > d + 1) right.push_back(v);
            else if (seen[2 * dist[v] + 1]) left.push_back(v);
            else right.push_back(v);
        }
        for (int32_t b = 0; b < nb; b++) dist[bandv[b]] = -1;
        return true;
    }

    int32_t operator()(std::vector<int32_t>& verts, int32_t pid) {
        const int64_t n = (int64_t)verts.size();
        if (n == 1) {
            const int32_t id = next++;
            t.leaf_elem[id] = verts[0];
            return id;
        }
        // pseudo-peripheral vertex: repeat BFS from the farthest minimum-degree vertex while the
        // depth grows (at most two more sweeps)
        int32_t root = *std::min_element(verts.begin(), verts.end());
        std::vector<int32_t> order;
        int32_t far = root;
        int32_t depth = bfs(verts, root, pid, order, &far);
        for (int it = 0; it < 2 && far != root; it++) {
            int32_t far2 = far;
            const int32_t d2 = bfs(verts, far, pid, order, &far2);
            if (d2 <= depth) break;
            root = far;
            depth = d2;
            far = far2;
        }
        std::vector<int32_t> lvl;
        size_t comp = 0;
        bfs(verts, root, pid, order, nullptr, &lvl, &comp);
        const int64_t h = n / 2;
        std::vector<int32_t> left, right;
        if (comp == order.size() && !narrow_cut(order, lvl, h, pid, left, right)) {
            left.clear();
            right.clear();
        }
        if (left.empty() || right.empty()) {  // disconnected part or no band: split the order in half
            left.assign(order.begin(), order.begin() + h);
            right.assign(order.begin() + h, order.end());
        }
        std::vector<int32_t>().swap(order);
        std::vector<int32_t>().swap(lvl);
        std::vector<int32_t>().swap(verts);
        const int32_t pl = next_part++, pr = next_part++;
        for (int32_t v : left) part[v] = pl;
        for (int32_t v : right) part[v] = pr;
        const int32_t a = (*this)(left, pl);
        const int32_t c = (*this)(right, pr);
        const int32_t id = next++;
        t.child[2 * id] = a;
        t.child[2 * id + 1] = c;
        t.parent[a] = id;
        t.parent[c] = id;
        return id;
    }
};

}  // namespace

int mf_symbolic_csr(int64_t n, const int64_t* rowptr, const int32_t* col, const mf_options* opt, mf_analysis* a) {
    if (n < 1 || !rowptr || !col) return MF_EINVAL;
    if (n >= INT32_MAX / 2) return MF_ENOTSUP;
    if (rowptr[0] != 0) return MF_EINVAL;
    for (int64_t i = 0; i < n; i++) {
        if (rowptr[i + 1] < rowptr[i]) return MF_EINVAL;
        for (int64_t q = rowptr[i]; q < rowptr[i + 1]; q++) {
            if (col[q] < 0 || col[q] >= n) return MF_EINVAL;
            if (q > rowptr[i] && col[q] <= col[q - 1]) return MF_EINVAL;  // strictly increasing columns
        }
    }
    const int64_t nnz = rowptr[n];
    Graph g;
    int rc = build_graph(n, rowptr, col, g);
    if (rc) return rc;

    // vertex tree
    HostTree t;
    t.parent.assign(2 * n - 1, -1);
    t.child.assign(2 * (2 * n - 1), -1);
    t.leaf_elem.assign(2 * n - 1, -1);
    {
        Bisector bis(g, t);
        std::vector<int32_t> all(n);
        std::iota(all.begin(), all.end(), 0);
        bis(all, 0);
    }
    std::vector<int32_t> leaf_of(n);
    for (int64_t v = 0; v < 2 * n - 1; v++)
        if (t.leaf_elem[v] >= 0) leaf_of[t.leaf_elem[v]] = (int32_t)v;

    // arrowhead elements: pair {u, v} -> the endpoint whose leaf comes first in postorder
    std::vector<int32_t> cnt(n, 1);
    for (int64_t u = 0; u < n; u++)
        for (int64_t q = g.ptr[u]; q < g.ptr[u + 1]; q++) {
            const int32_t v = g.adj[q];
            if (v > u) cnt[leaf_of[u] < leaf_of[v] ? u : v]++;
        }
    const int npe = *std::max_element(cnt.begin(), cnt.end());
    if (npe > 64) return MF_ENOTSUP;
    std::vector<int64_t> en((size_t)n * npe);
    std::vector<int32_t> fillc(n, 1);
    for (int64_t w = 0; w < n; w++) en[w * npe] = w;
    for (int64_t u = 0; u < n; u++)
        for (int64_t q = g.ptr[u]; q < g.ptr[u + 1]; q++) {
            const int32_t v = g.adj[q];
            if (v <= u) continue;
            const int64_t w = leaf_of[u] < leaf_of[v] ? u : v;
            const int64_t o = w == u ? v : u;
            en[w * npe + fillc[w]++] = o;
        }
    for (int64_t w = 0; w < n; w++)
        for (int j = fillc[w]; j < npe; j++) en[w * npe + j] = w;  // padding: the element's own vertex

    // destination of every CSR entry in the element array (column-major npe x npe blocks)
    std::vector<int64_t> dest(nnz);
    {
        // local position of each of w's pair partners: search w's short node list
        for (int64_t i = 0; i < n; i++)
            for (int64_t q = rowptr[i]; q < rowptr[i + 1]; q++) {
                const int64_t j = col[q];
                if (j == i) {
                    dest[q] = i * npe * npe;  // (0, 0) of vertex i's element
                    continue;
                }
                const int64_t w = leaf_of[i] < leaf_of[j] ? i : j;
                const int64_t o = w == i ? j : i;
                int lp = -1;
                for (int s = 1; s < fillc[w]; s++)
                    if (en[w * npe + s] == o) {
                        lp = s;
                        break;
                    }
                if (lp < 0) return MF_EINVAL;  // cannot happen: every pair was assigned above
                const int64_t ra = w == i ? 0 : lp, cb = w == i ? lp : 0;
                dest[q] = w * npe * npe + ra + cb * npe;
            }
    }

    mf_mesh_desc d{};
    d.dim = 2;  // no geometry: the tree is given
    d.n_nodes = n;
    d.n_elem = n;
    d.nodes_per_elem = npe;
    d.elem_nodes = en.data();
    rc = mf_symbolic(&d, 1, opt, a, &t);
    if (rc) return rc;
    a->csr_n = n;
    a->csr_nnz = nnz;
    a->csr_dest.swap(dest);
    return MF_OK;
}

extern "C" int mf_analyze_csr(int64_t n, const int64_t* rowptr, const int32_t* col, const mf_options* opt,
                              mf_analysis** out) {
    if (!out) return MF_EINVAL;
    *out = nullptr;
    mf_analysis* a = new (std::nothrow) mf_analysis();
    if (!a) return MF_ENOMEM;
    int rc;
    try {
        rc = mf_symbolic_csr(n, rowptr, col, opt, a);
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
