/*
 * ORACLE -- test infrastructure only.  A plain, slow, FP64 CPU multifrontal
 * solver written from the paper's description, used to check the CUDA path.
 * Only the tests, the smoke check and the benchmark's CPU-baseline leg load
 * it; the product library never links, includes or calls anything here, and
 * this file shares no code with it.
 *
 * What it computes (arXiv 2306.08994):
 *   - Elimination tree built bottom-up from element fronts (Sec. 2.4 steps
 *     1-5, Table 3 `generate_elimination_tree` / `join_adjacent_fronts`), in
 *     two independent forms: (a) recursive longest-axis floor bisection of the
 *     structured element box, (b) the paper's sort-then-pair-adjacent rule on
 *     Morton-ordered elements with the odd front carried up unchanged.
 *   - Symbolic: a dof is a pivot of front v exactly when v is the lowest front
 *     containing every element that touches it (the paper's
 *     "front_membership_count == 1 and not computed", Table 2); each front is
 *     reordered pivots-first, then shared dofs (Sec. 3.2).
 *   - Numeric: fronts processed leaves to root; a leaf front is its element
 *     matrix, a parent front is the extend-add of its children's Schur
 *     complements ("join_fronts", Table 1; composition of a merged front,
 *     Sec. 2.4); then for every fully assembled pivot p: division task
 *     T1 F[p,j] /= F[p,p] for j > p, multiplication T2 t = F[p,j]*F[i,p] and
 *     subtraction T3 F[i,j] -= t for i > p (Sec. 3 task alphabet, Table 2
 *     `compute_front`); the remaining block is the Schur complement
 *     S = F22 - F21 F11^-1 F12 (Sec. 2.2, Eq. Bmat).  The root is factored
 *     completely ("compute_dense_matrix", Table 1).
 *   - Solution (`get_solution`, Table 2): forward substitution with the lower
 *     factor L (non-unit diagonal, the pivot column), then backward
 *     substitution with the unit upper factor U (the divided pivot rows).
 *
 * Readings where the paper is silent or garbled:
 *   loop bounds j, i start at p+1 (the task definitions say j > p, i > p);
 *   the division result is stored back into F[p,j]; no pivoting, with a
 *   static check |F[p,p]| < tau that replaces the pivot by sign*tau (counted)
 *   or fails; extend-add adds child 0 then child 1; the residual used for
 *   refinement is accumulated in double-double (Knuth TwoSum / Dekker-style
 *   TwoProduct via fma) so the refined solution is accurate to about 1 ulp.
 *
 * Layout: every front is a dense column-major m x m array F[i + j*m] while it
 * is processed.  After elimination the oracle keeps, per front, the first k
 * columns (L below/on the diagonal, U strictly above) and the first k rows
 * (U) -- both copied from F -- and the Schur complement until the parent has
 * consumed it.
 */
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_OK 0
#define ORC_EINVAL -1
#define ORC_ENOMEM -2
#define ORC_EZERO_PIVOT -4

/* ------------------------------------------------------------------ trees */
/* Tree arrays, nodes in postorder (left subtree, right subtree, node):
 *   parent[v] (-1 at the root), child[2v], child[2v+1] (-1 if absent),
 *   leaf_elem[v] (element id of a leaf, -1 for internal nodes). */

typedef struct {
    int32_t *parent, *child, *leaf_elem;
    int32_t next;
} tree_out;

static int32_t bisect_rec(tree_out* t, const int32_t nel[3], int32_t lo[3], int32_t hi[3]) {
    int32_t n[3] = {hi[0] - lo[0], hi[1] - lo[1], hi[2] - lo[2]};
    if (n[0] * n[1] * n[2] == 1) {
        int32_t v = t->next++;
        t->leaf_elem[v] = lo[0] + nel[0] * (lo[1] + nel[1] * lo[2]);
        t->child[2 * v] = t->child[2 * v + 1] = -1;
        return v;
    }
    /* longest axis; ties go to the lowest axis (x, then y, then z) */
    int ax = 0;
    for (int a = 1; a < 3; a++)
        if (n[a] > n[ax]) ax = a;
    int32_t mid = lo[ax] + n[ax] / 2;
    int32_t lhi[3] = {hi[0], hi[1], hi[2]}, rlo[3] = {lo[0], lo[1], lo[2]};
    lhi[ax] = mid;
    rlo[ax] = mid;
    int32_t l = bisect_rec(t, nel, lo, lhi);
    int32_t r = bisect_rec(t, nel, rlo, hi);
    int32_t v = t->next++;
    t->leaf_elem[v] = -1;
    t->child[2 * v] = l;
    t->child[2 * v + 1] = r;
    t->parent[l] = v;
    t->parent[r] = v;
    return v;
}

/* Tree (a): recursive floor bisection of the nx*ny*nz element box. */
int orc_tree_bisection(const int32_t nel[3], int32_t* parent, int32_t* child, int32_t* leaf_elem) {
    if (nel[0] < 1 || nel[1] < 1 || nel[2] < 1) return ORC_EINVAL;
    tree_out t = {parent, child, leaf_elem, 0};
    int32_t lo[3] = {0, 0, 0}, hi[3] = {nel[0], nel[1], nel[2]};
    int32_t root = bisect_rec(&t, nel, lo, hi);
    parent[root] = -1;
    return t.next;
}

/* Tree (b): the paper's rule (Table 3).  Elements are sorted by a Morton key
 * (bit-interleaved x,y,z with x the most significant of each group), then
 * adjacent fronts are joined pairwise, an odd last front being carried up
 * unchanged, until one front remains.  The result is renumbered in postorder. */
static int64_t morton_key(int32_t x, int32_t y, int32_t z, int dim) {
    int64_t key = 0;
    for (int b = 20; b >= 0; b--) {
        key = (key << 1) | ((x >> b) & 1);
        key = (key << 1) | ((y >> b) & 1);
        if (dim == 3) key = (key << 1) | ((z >> b) & 1);
    }
    return key;
}

typedef struct { int64_t key; int32_t e; } keyed;
static int cmp_keyed(const void* a, const void* b) {
    const keyed* x = (const keyed*)a;
    const keyed* y = (const keyed*)b;
    if (x->key != y->key) return x->key < y->key ? -1 : 1;
    return x->e - y->e;
}

static void postorder_rec(int32_t v, const int32_t* tl, const int32_t* tr, int32_t* order, int32_t* cnt) {
    if (tl[v] >= 0) postorder_rec(tl[v], tl, tr, order, cnt);
    if (tr[v] >= 0) postorder_rec(tr[v], tl, tr, order, cnt);
    order[(*cnt)++] = v;
}

int orc_tree_pairing(const int32_t nel[3], int32_t* parent, int32_t* child, int32_t* leaf_elem) {
    int dim = nel[2] > 1 ? 3 : 2;
    int32_t ne = nel[0] * nel[1] * nel[2];
    if (ne < 1) return ORC_EINVAL;
    int32_t nn = 2 * ne - 1;
    keyed* ks = (keyed*)malloc(sizeof(keyed) * ne);
    int32_t* tl = (int32_t*)malloc(sizeof(int32_t) * nn);
    int32_t* tr = (int32_t*)malloc(sizeof(int32_t) * nn);
    int32_t* te = (int32_t*)malloc(sizeof(int32_t) * nn);
    int32_t* fronts = (int32_t*)malloc(sizeof(int32_t) * ne);
    int32_t* order = (int32_t*)malloc(sizeof(int32_t) * nn);
    int32_t* newid = (int32_t*)malloc(sizeof(int32_t) * nn);
    for (int32_t e = 0; e < ne; e++) {
        int32_t x = e % nel[0], y = (e / nel[0]) % nel[1], z = e / (nel[0] * nel[1]);
        ks[e].key = morton_key(x, y, z, dim);
        ks[e].e = e;
    }
    qsort(ks, ne, sizeof(keyed), cmp_keyed);
    int32_t nid = 0, nf = ne;
    for (int32_t i = 0; i < ne; i++) {
        te[nid] = ks[i].e;
        tl[nid] = tr[nid] = -1;
        fronts[i] = nid++;
    }
    while (nf > 1) {
        int32_t nnf = 0;
        for (int32_t i = 0; i + 1 < nf; i += 2) {
            te[nid] = -1;
            tl[nid] = fronts[i];
            tr[nid] = fronts[i + 1];
            fronts[nnf++] = nid++;
        }
        if (nf % 2 == 1) fronts[nnf++] = fronts[nf - 1];
        nf = nnf;
    }
    int32_t cnt = 0;
    postorder_rec(fronts[0], tl, tr, order, &cnt);
    for (int32_t i = 0; i < cnt; i++) newid[order[i]] = i;
    for (int32_t i = 0; i < cnt; i++) {
        int32_t o = order[i];
        leaf_elem[i] = te[o];
        child[2 * i] = tl[o] >= 0 ? newid[tl[o]] : -1;
        child[2 * i + 1] = tr[o] >= 0 ? newid[tr[o]] : -1;
        if (tl[o] >= 0) parent[newid[tl[o]]] = i;
        if (tr[o] >= 0) parent[newid[tr[o]]] = i;
    }
    parent[cnt - 1] = -1;
    free(ks); free(tl); free(tr); free(te); free(fronts); free(order); free(newid);
    return cnt;
}

/* ------------------------------------------------------------ the solver */
typedef struct {
    int32_t n_dof, n_elem, npe, n_front;
    const int64_t* elem_nodes; /* borrowed until orc_create returns; copied */
    int64_t* en;
    int32_t *parent, *child, *leaf_elem, *height;
    int32_t *m, *k;
    int64_t* dof_ptr;  /* front dofs: pivots (ascending) then CB (ascending) */
    int32_t* dofs;
    int32_t *cls_ptr, *cls_front, n_cls; /* fronts grouped by height */
    /* numeric */
    double** L;   /* m x k column-major: F[:, 0:k] after elimination */
    double** U;   /* k x m column-major: F[0:k, :] after elimination */
    int64_t n_perturbed;
    int factored;
} orc_mf;

static int cmp_i32(const void* a, const void* b) {
    int32_t x = *(const int32_t*)a, y = *(const int32_t*)b;
    return (x > y) - (x < y);
}

void orc_free(orc_mf* s) {
    if (!s) return;
    if (s->L) for (int32_t v = 0; v < s->n_front; v++) free(s->L[v]);
    if (s->U) for (int32_t v = 0; v < s->n_front; v++) free(s->U[v]);
    free(s->L); free(s->U);
    free(s->en); free(s->parent); free(s->child); free(s->leaf_elem); free(s->height);
    free(s->m); free(s->k); free(s->dof_ptr); free(s->dofs); free(s->cls_ptr); free(s->cls_front);
    free(s);
}

/* Symbolic phase.  Tree nodes must be in postorder (children before parents). */
orc_mf* orc_create(int32_t n_dof, int32_t n_elem, int32_t npe, const int64_t* elem_nodes,
                   int32_t n_front, const int32_t* parent, const int32_t* child, const int32_t* leaf_elem) {
    orc_mf* s = (orc_mf*)calloc(1, sizeof(orc_mf));
    s->n_dof = n_dof; s->n_elem = n_elem; s->npe = npe; s->n_front = n_front;
    s->en = (int64_t*)malloc(sizeof(int64_t) * (size_t)n_elem * npe);
    memcpy(s->en, elem_nodes, sizeof(int64_t) * (size_t)n_elem * npe);
    s->parent = (int32_t*)malloc(sizeof(int32_t) * n_front);
    s->child = (int32_t*)malloc(sizeof(int32_t) * 2 * n_front);
    s->leaf_elem = (int32_t*)malloc(sizeof(int32_t) * n_front);
    memcpy(s->parent, parent, sizeof(int32_t) * n_front);
    memcpy(s->child, child, sizeof(int32_t) * 2 * n_front);
    memcpy(s->leaf_elem, leaf_elem, sizeof(int32_t) * n_front);

    /* subtree of v spans postorder positions [first[v], v] */
    int32_t* first = (int32_t*)malloc(sizeof(int32_t) * n_front);
    int32_t* leaf_of_elem = (int32_t*)malloc(sizeof(int32_t) * n_elem);
    s->height = (int32_t*)malloc(sizeof(int32_t) * n_front);
    for (int32_t v = 0; v < n_front; v++) {
        if (leaf_elem[v] >= 0) {
            first[v] = v;
            s->height[v] = 1;
            leaf_of_elem[leaf_elem[v]] = v;
        } else {
            int32_t c0 = child[2 * v], c1 = child[2 * v + 1];
            first[v] = first[c0];
            int32_t h = s->height[c0];
            if (c1 >= 0) {
                if (first[c1] < first[v]) first[v] = first[c1];
                if (s->height[c1] > h) h = s->height[c1];
            }
            s->height[v] = h + 1;
        }
    }
    /* the lowest front containing all elements of a dof: walk up from the
     * dof's leftmost leaf until the subtree range covers its rightmost leaf */
    int32_t* lo = (int32_t*)malloc(sizeof(int32_t) * n_dof);
    int32_t* hi = (int32_t*)malloc(sizeof(int32_t) * n_dof);
    for (int32_t d = 0; d < n_dof; d++) { lo[d] = INT32_MAX; hi[d] = -1; }
    for (int32_t e = 0; e < n_elem; e++) {
        int32_t lv = leaf_of_elem[e];
        for (int a = 0; a < npe; a++) {
            int64_t d = elem_nodes[(int64_t)e * npe + a];
            if (lv < lo[d]) lo[d] = lv;
            if (lv > hi[d]) hi[d] = lv;
        }
    }
    int32_t* elim = (int32_t*)malloc(sizeof(int32_t) * n_dof);
    for (int32_t d = 0; d < n_dof; d++) {
        if (hi[d] < 0) { elim[d] = -1; continue; } /* dof in no element */
        int32_t v = lo[d];
        while (!(first[v] <= lo[d] && hi[d] <= v)) v = parent[v];
        elim[d] = v;
    }
    /* pivots of every front, ascending */
    int32_t* kcount = (int32_t*)calloc(n_front + 1, sizeof(int32_t));
    for (int32_t d = 0; d < n_dof; d++) if (elim[d] >= 0) kcount[elim[d] + 1]++;
    for (int32_t v = 0; v < n_front; v++) kcount[v + 1] += kcount[v];
    int32_t* piv = (int32_t*)malloc(sizeof(int32_t) * (n_dof > 0 ? n_dof : 1));
    int32_t* fill = (int32_t*)malloc(sizeof(int32_t) * n_front);
    for (int32_t v = 0; v < n_front; v++) fill[v] = kcount[v];
    for (int32_t d = 0; d < n_dof; d++) if (elim[d] >= 0) piv[fill[elim[d]]++] = d; /* ascending d */

    /* contribution-block sets, postorder: leaf = element dofs not eliminated at
     * the leaf; parent = union of the children's CB sets minus its pivots.
     * Front dof list = pivots ascending, then CB ascending (Sec. 3.2 reorder). */
    int32_t** cb = (int32_t**)calloc(n_front, sizeof(int32_t*));
    int32_t* ncb = (int32_t*)calloc(n_front, sizeof(int32_t));
    s->m = (int32_t*)malloc(sizeof(int32_t) * n_front);
    s->k = (int32_t*)malloc(sizeof(int32_t) * n_front);
    s->dof_ptr = (int64_t*)malloc(sizeof(int64_t) * (n_front + 1));
    s->dof_ptr[0] = 0;
    int64_t cap = (int64_t)n_dof + npe + 16;
    s->dofs = (int32_t*)malloc(sizeof(int32_t) * cap);
    int32_t* tmp = (int32_t*)malloc(sizeof(int32_t) * (n_dof + npe + 1));
    for (int32_t v = 0; v < n_front; v++) {
        int32_t nt = 0;
        if (leaf_elem[v] >= 0) {
            int32_t e = leaf_elem[v];
            for (int a = 0; a < npe; a++) tmp[nt++] = (int32_t)elem_nodes[(int64_t)e * npe + a];
        } else {
            for (int c = 0; c < 2; c++) {
                int32_t ch = child[2 * v + c];
                if (ch < 0) continue;
                for (int32_t i = 0; i < ncb[ch]; i++) tmp[nt++] = cb[ch][i];
                free(cb[ch]);
                cb[ch] = NULL;
            }
        }
        qsort(tmp, nt, sizeof(int32_t), cmp_i32);
        int32_t nu = 0;
        for (int32_t i = 0; i < nt; i++)
            if (i == 0 || tmp[i] != tmp[i - 1]) tmp[nu++] = tmp[i];
        int32_t nc = 0;
        cb[v] = (int32_t*)malloc(sizeof(int32_t) * (nu > 0 ? nu : 1));
        for (int32_t i = 0; i < nu; i++)
            if (elim[tmp[i]] != v) cb[v][nc++] = tmp[i];
        ncb[v] = nc;
        s->k[v] = kcount[v + 1] - kcount[v];
        s->m[v] = s->k[v] + nc;
        s->dof_ptr[v + 1] = s->dof_ptr[v] + s->m[v];
        while (s->dof_ptr[v + 1] > cap) {
            cap *= 2;
            s->dofs = (int32_t*)realloc(s->dofs, sizeof(int32_t) * cap);
        }
        int32_t* out = s->dofs + s->dof_ptr[v];
        for (int32_t i = 0; i < s->k[v]; i++) out[i] = piv[kcount[v] + i];
        for (int32_t i = 0; i < nc; i++) out[s->k[v] + i] = cb[v][i];
    }
    for (int32_t v = 0; v < n_front; v++) free(cb[v]);
    free(cb); free(ncb); free(tmp); free(piv); free(fill); free(kcount);
    free(elim); free(lo); free(hi); free(first); free(leaf_of_elem);

    /* Foata classes at front granularity: fronts of equal height */
    int32_t H = 0;
    for (int32_t v = 0; v < n_front; v++) if (s->height[v] > H) H = s->height[v];
    s->n_cls = H;
    s->cls_ptr = (int32_t*)calloc(H + 1, sizeof(int32_t));
    s->cls_front = (int32_t*)malloc(sizeof(int32_t) * n_front);
    for (int32_t v = 0; v < n_front; v++) s->cls_ptr[s->height[v]]++;
    for (int32_t c = 0; c < H; c++) s->cls_ptr[c + 1] += s->cls_ptr[c];
    int32_t* cf = (int32_t*)malloc(sizeof(int32_t) * (H + 1));
    memcpy(cf, s->cls_ptr, sizeof(int32_t) * (H + 1));
    for (int32_t v = 0; v < n_front; v++) s->cls_front[cf[s->height[v] - 1]++] = v;
    free(cf);
    return s;
}

/* Sizes: out[0..7] = n_front, n_classes, max m, sum k, nnz(L+U), sum CB
 * entries, factor flops (paper variant), max k. */
void orc_info(const orc_mf* s, int64_t* out) {
    int64_t mx = 0, sk = 0, nnz = 0, scb = 0, mk = 0;
    double fl = 0;
    for (int32_t v = 0; v < s->n_front; v++) {
        int64_t m = s->m[v], k = s->k[v];
        if (m > mx) mx = m;
        if (k > mk) mk = k;
        sk += k;
        nnz += m * k + k * (m - k);
        scb += (m - k) * (m - k);
        /* per pivot p: (m-p-1) divisions + 2 (m-p-1)^2 mult/sub */
        for (int64_t p = 0; p < k; p++) fl += (double)(m - p - 1) + 2.0 * (double)(m - p - 1) * (m - p - 1);
    }
    out[0] = s->n_front; out[1] = s->n_cls; out[2] = mx; out[3] = sk;
    out[4] = nnz; out[5] = scb; out[6] = (int64_t)fl; out[7] = mk;
}

void orc_fronts(const orc_mf* s, int32_t* m, int32_t* k, int32_t* height, int32_t* parent, int64_t* dof_ptr, int32_t* dofs) {
    memcpy(m, s->m, sizeof(int32_t) * s->n_front);
    memcpy(k, s->k, sizeof(int32_t) * s->n_front);
    memcpy(height, s->height, sizeof(int32_t) * s->n_front);
    memcpy(parent, s->parent, sizeof(int32_t) * s->n_front);
    memcpy(dof_ptr, s->dof_ptr, sizeof(int64_t) * (s->n_front + 1));
    memcpy(dofs, s->dofs, sizeof(int32_t) * s->dof_ptr[s->n_front]);
}

/* position of each front dof inside the front, in a caller scratch array
 * indexed by global dof (entries outside the front are left untouched) */
static void mark_front(const orc_mf* s, int32_t v, int32_t* where) {
    const int32_t* fd = s->dofs + s->dof_ptr[v];
    for (int32_t i = 0; i < s->m[v]; i++) where[fd[i]] = i;
}

/* Numeric factorization.  Ke: n_elem element matrices, each npe x npe
 * column-major.  tau: static pivot threshold (|pivot| < tau is replaced by
 * sign*tau and counted, or an error when fail_small != 0).  Fronts of one
 * height class are independent and may run on nthreads OpenMP threads; the
 * class loop is the barrier.  Returns the number of perturbed pivots or a
 * negative error code. */
int64_t orc_factor(orc_mf* s, const double* Ke, double tau, int fail_small, int nthreads) {
    const int32_t nf = s->n_front, npe = s->npe;
    if (!s->L) {
        s->L = (double**)calloc(nf, sizeof(double*));
        s->U = (double**)calloc(nf, sizeof(double*));
    }
    double** S = (double**)calloc(nf, sizeof(double*)); /* Schur complements awaiting the parent */
    int64_t perturbed = 0;
    int failed = 0;
#ifdef _OPENMP
    if (nthreads < 1) nthreads = 1;
#endif
    for (int32_t c = 0; c < s->n_cls; c++) {
        int32_t f0 = s->cls_ptr[c], f1 = s->cls_ptr[c + 1];
#ifdef _OPENMP
#pragma omp parallel num_threads(nthreads) reduction(+ : perturbed)
#endif
        {
            int32_t* where = (int32_t*)malloc(sizeof(int32_t) * (s->n_dof > 0 ? s->n_dof : 1));
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 1)
#endif
            for (int32_t idx = f0; idx < f1; idx++) {
                int32_t v = s->cls_front[idx];
                int64_t m = s->m[v], k = s->k[v];
                double* F = (double*)calloc((size_t)(m * m > 0 ? m * m : 1), sizeof(double));
                mark_front(s, v, where);
                if (s->leaf_elem[v] >= 0) {
                    /* leaf: the element matrix is the front */
                    int32_t e = s->leaf_elem[v];
                    const double* K = Ke + (int64_t)e * npe * npe;
                    const int64_t* en = s->en + (int64_t)e * npe;
                    for (int b = 0; b < npe; b++)
                        for (int a = 0; a < npe; a++)
                            F[where[en[a]] + where[en[b]] * m] += K[a + b * npe];
                } else {
                    /* extend-add: child 0, then child 1 */
                    for (int ci = 0; ci < 2; ci++) {
                        int32_t ch = s->child[2 * v + ci];
                        if (ch < 0) continue;
                        int64_t kc = s->k[ch], nc = s->m[ch] - kc;
                        const int32_t* cd = s->dofs + s->dof_ptr[ch] + kc;
                        for (int64_t j = 0; j < nc; j++)
                            for (int64_t i = 0; i < nc; i++)
                                F[where[cd[i]] + where[cd[j]] * m] += S[ch][i + j * nc];
                        free(S[ch]);
                        S[ch] = NULL;
                    }
                }
                /* compute_front: eliminate the fully assembled pivots 0..k-1 */
                for (int64_t p = 0; p < k; p++) {
                    double piv = F[p + p * m];
                    if (!(fabs(piv) >= tau)) {
                        if (fail_small) {
#ifdef _OPENMP
#pragma omp atomic write
#endif
                            failed = 1;
                        }
                        piv = (piv < 0) ? -tau : tau;
                        F[p + p * m] = piv;
                        perturbed++;
                    }
                    for (int64_t j = p + 1; j < m; j++) {
                        double t1 = F[p + j * m] / piv; /* T1: division */
                        F[p + j * m] = t1;
                        for (int64_t i = p + 1; i < m; i++) {
                            double t2 = t1 * F[i + p * m]; /* T2: multiplication */
                            F[i + j * m] = F[i + j * m] - t2; /* T3: subtraction */
                        }
                    }
                }
                /* keep the factor: first k columns (L and U11) and first k rows (U) */
                free(s->L[v]);
                free(s->U[v]);
                s->L[v] = (double*)malloc(sizeof(double) * (size_t)(m * k > 0 ? m * k : 1));
                s->U[v] = (double*)malloc(sizeof(double) * (size_t)(m * k > 0 ? m * k : 1));
                for (int64_t j = 0; j < k; j++)
                    for (int64_t i = 0; i < m; i++) s->L[v][i + j * m] = F[i + j * m];
                for (int64_t j = 0; j < m; j++)
                    for (int64_t i = 0; i < k; i++) s->U[v][i + j * k] = F[i + j * m];
                /* Schur complement = trailing block, handed to the parent */
                int64_t nc = m - k;
                if (nc > 0) {
                    S[v] = (double*)malloc(sizeof(double) * (size_t)(nc * nc));
                    for (int64_t j = 0; j < nc; j++)
                        for (int64_t i = 0; i < nc; i++) S[v][i + j * nc] = F[(k + i) + (k + j) * m];
                }
                free(F);
            }
            free(where);
        }
    }
    for (int32_t v = 0; v < nf; v++) free(S[v]);
    free(S);
    s->n_perturbed = perturbed;
    s->factored = 1;
    if (failed) return ORC_EZERO_PIVOT;
    return perturbed;
}

/* Copy front v's factor: Lout m x k (column-major) and Uout k x m (column-major). */
int orc_get_factor(const orc_mf* s, int32_t v, double* Lout, double* Uout) {
    if (!s->factored || v < 0 || v >= s->n_front) return ORC_EINVAL;
    int64_t m = s->m[v], k = s->k[v];
    memcpy(Lout, s->L[v], sizeof(double) * (size_t)(m * k));
    memcpy(Uout, s->U[v], sizeof(double) * (size_t)(m * k));
    return ORC_OK;
}

/* Solve A x = b with the stored factors (get_solution, Table 2).
 * b: n_dof x nrhs column-major, overwritten with x.
 * Forward, leaves to root: gather the front's right-hand side (b at its
 * pivots plus the update vectors of its children), solve with the lower
 * factor (divide by the diagonal), pass w_CB - L21 y to the parent.
 * Backward, root to leaves: x_piv = y - U12 x_CB, then the unit upper
 * triangle of U11 bottom-up. */
static int solve_impl(const orc_mf* s, double* b, int nrhs, int transposed) {
    if (!s->factored) return ORC_EINVAL;
    const int32_t nf = s->n_front;
    int32_t* where = (int32_t*)malloc(sizeof(int32_t) * (s->n_dof > 0 ? s->n_dof : 1));
    double** upd = (double**)calloc(nf, sizeof(double*));
    double* y = (double*)malloc(sizeof(double) * (size_t)s->n_dof);
    for (int r = 0; r < nrhs; r++) {
        double* br = b + (int64_t)r * s->n_dof;
        /* forward */
        for (int32_t v = 0; v < nf; v++) {
            int64_t m = s->m[v], k = s->k[v];
            const int32_t* fd = s->dofs + s->dof_ptr[v];
            const double* L = s->L[v];
            const double* U = s->U[v];
            double* w = (double*)calloc((size_t)(m > 0 ? m : 1), sizeof(double));
            mark_front(s, v, where);
            for (int64_t i = 0; i < k; i++) w[i] = br[fd[i]];
            for (int ci = 0; ci < 2; ci++) {
                int32_t ch = s->child[2 * v + ci];
                if (ch < 0) continue;
                int64_t kc = s->k[ch], nc = s->m[ch] - kc;
                const int32_t* cd = s->dofs + s->dof_ptr[ch] + kc;
                for (int64_t i = 0; i < nc; i++) w[where[cd[i]]] += upd[ch][i];
                free(upd[ch]);
                upd[ch] = NULL;
            }
            for (int64_t p = 0; p < k; p++) {
                double yp;
                if (!transposed) {
                    /* L: column p holds L[p..m-1, p], diagonal included */
                    yp = w[p] / L[p + p * m];
                    for (int64_t i = p + 1; i < m; i++) w[i] -= L[i + p * m] * yp;
                } else {
                    /* U^T: unit diagonal, row p of U becomes column p */
                    yp = w[p];
                    for (int64_t i = p + 1; i < m; i++) w[i] -= U[p + i * k] * yp;
                }
                w[p] = yp;
            }
            for (int64_t i = 0; i < k; i++) y[fd[i]] = w[i];
            if (m - k > 0) {
                upd[v] = (double*)malloc(sizeof(double) * (size_t)(m - k));
                for (int64_t i = 0; i < m - k; i++) upd[v][i] = w[k + i];
            }
            free(w);
        }
        /* backward */
        for (int32_t v = nf - 1; v >= 0; v--) {
            int64_t m = s->m[v], k = s->k[v];
            const int32_t* fd = s->dofs + s->dof_ptr[v];
            const double* L = s->L[v];
            const double* U = s->U[v];
            double* z = (double*)malloc(sizeof(double) * (size_t)(k > 0 ? k : 1));
            for (int64_t i = 0; i < k; i++) z[i] = y[fd[i]];
            /* subtract the already known CB part */
            for (int64_t j = k; j < m; j++) {
                double xj = br[fd[j]];
                for (int64_t i = 0; i < k; i++)
                    z[i] -= (!transposed ? U[i + j * k] : L[j + i * m]) * xj;
            }
            for (int64_t p = k - 1; p >= 0; p--) {
                double xp = !transposed ? z[p] : z[p] / L[p + p * m];
                for (int64_t i = 0; i < p; i++)
                    z[i] -= (!transposed ? U[i + p * k] : L[p + i * m]) * xp;
                z[p] = xp;
            }
            for (int64_t i = 0; i < k; i++) br[fd[i]] = z[i];
            free(z);
        }
    }
    for (int32_t v = 0; v < nf; v++) free(upd[v]);
    free(upd); free(y); free(where);
    return ORC_OK;
}

int orc_solve(const orc_mf* s, double* b, int nrhs) { return solve_impl(s, b, nrhs, 0); }
/* A^T x = g with the same factors: U^T forward (unit), then L^T backward. */
int orc_solve_adjoint(const orc_mf* s, double* b, int nrhs) { return solve_impl(s, b, nrhs, 1); }

/* ----------------------------------------------- double-double residual */
typedef struct { double hi, lo; } dd;
static dd two_sum(double a, double b) {
    double s = a + b, bb = s - a;
    dd r = {s, (a - (s - bb)) + (b - bb)};
    return r;
}
static dd dd_add_prod(dd acc, double a, double b) {
    double p = a * b;
    double pe = fma(a, b, -p); /* exact error of the product */
    dd s = two_sum(acc.hi, p);
    double e = s.lo + acc.lo + pe;
    dd r = two_sum(s.hi, e);
    return r;
}

/* r = b - A x with A given element by element (Ke column-major), every
 * product and sum carried in double-double; elements in ascending order. */
int orc_residual_dd(int32_t n_dof, int32_t n_elem, int32_t npe, const int64_t* en, const double* Ke,
                    const double* x, const double* b, double* r, int nrhs) {
    dd* acc = (dd*)malloc(sizeof(dd) * (size_t)n_dof);
    for (int q = 0; q < nrhs; q++) {
        const double* xq = x + (int64_t)q * n_dof;
        for (int32_t d = 0; d < n_dof; d++) { acc[d].hi = b[(int64_t)q * n_dof + d]; acc[d].lo = 0; }
        for (int32_t e = 0; e < n_elem; e++) {
            const double* K = Ke + (int64_t)e * npe * npe;
            const int64_t* nd = en + (int64_t)e * npe;
            for (int a = 0; a < npe; a++)
                for (int bb = 0; bb < npe; bb++)
                    acc[nd[a]] = dd_add_prod(acc[nd[a]], -K[a + bb * npe], xq[nd[bb]]);
        }
        for (int32_t d = 0; d < n_dof; d++) r[(int64_t)q * n_dof + d] = acc[d].hi + acc[d].lo;
    }
    free(acc);
    return ORC_OK;
}

/* Solve then refine: x = solve(b); repeat r = b - A x (double-double),
 * x += solve(r) until the correction is below 4 ulp of x or maxit.
 * Returns the number of refinement steps taken. */
int orc_solve_refined(const orc_mf* s, const double* Ke, const double* b, double* x, int nrhs, int maxit) {
    int64_t n = s->n_dof;
    double* r = (double*)malloc(sizeof(double) * (size_t)(n * nrhs));
    memcpy(x, b, sizeof(double) * (size_t)(n * nrhs));
    int rc = orc_solve(s, x, nrhs);
    if (rc) { free(r); return rc; }
    int it = 0;
    for (; it < maxit; it++) {
        orc_residual_dd(s->n_dof, s->n_elem, s->npe, s->en, Ke, x, b, r, nrhs);
        orc_solve(s, r, nrhs);
        double dn = 0, xn = 0;
        for (int64_t i = 0; i < n * nrhs; i++) {
            x[i] += r[i];
            if (fabs(r[i]) > dn) dn = fabs(r[i]);
            if (fabs(x[i]) > xn) xn = fabs(x[i]);
        }
        if (dn <= 4.0 * 1.1102230246251565e-16 * xn) { it++; break; }
    }
    free(r);
    return it;
}

/* g_e = -lambda_e^T dK_e x_e for every element (dK column-major). */
void orc_element_grad(int32_t n_elem, int32_t npe, const int64_t* en, const double* dK,
                      const double* lambda, const double* x, double* g) {
    for (int32_t e = 0; e < n_elem; e++) {
        const double* K = dK + (int64_t)e * npe * npe;
        const int64_t* nd = en + (int64_t)e * npe;
        double acc = 0;
        for (int bb = 0; bb < npe; bb++)
            for (int a = 0; a < npe; a++) acc += lambda[nd[a]] * K[a + bb * npe] * x[nd[bb]];
        g[e] = -acc;
    }
}

int32_t orc_n_front(const orc_mf* s) { return s->n_front; }
int orc_max_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
int64_t orc_sum_m(const orc_mf* s) { return s->dof_ptr[s->n_front]; }
