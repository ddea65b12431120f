/*
 * fec_oracle.c -- plain, slow, single-threaded CPU oracle for exact Euclidean
 * clustering (FEC, "Fast Euclidean Clustering for Point Cloud Segmentation").
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the package smoke check and
 * the CPU-baseline leg of the benchmark may load this file.  The product path
 * (the CUDA library) never calls it and shares no code, header, table or helper
 * with it.
 *
 * What it computes (the plain definition, written out):
 *   - Eq. 1 / Section 2.2: two clusters are separated when the closest pair of
 *     points across them is farther than the threshold d.  Equivalently, the
 *     clusters are the connected components of the graph G whose edges join
 *     every pair of points at distance <= d (equality joins; see the readings
 *     below).
 *   - Algorithm 1, input: an unorganised cloud P, the radius d and a size cap;
 *     output: one label per point.  Section 3.1 sets the size bounds like PCL's
 *     EuclideanClusterExtraction, so clusters outside [min_size, max_size] are
 *     dropped (label -1).
 *   - Kept clusters are numbered 0..k-1 in increasing order of their smallest
 *     point index.
 *
 * Exactness: coordinates are quantised to integer units of 1/1024 m with
 * round-half-to-even, q = rint(x * 1024); the join test is the integer test
 * dx^2 + dy^2 + dz^2 <= T2 with T2 = floor((d * 1024)^2) evaluated in double.
 * For d a multiple of 1/1024 this is exactly "distance <= d".
 *
 * Two independent routes to the same components:
 *   fec_oracle_cluster     -- breadth-first search over a kd-tree index (the
 *                             paper's spatial index, Algorithm 1 "Constructing
 *                             kd-tree", complexity in Section 2.2), seeded from
 *                             every unvisited point in increasing index order,
 *                             so each component's seed is its smallest index.
 *   fec_oracle_bruteforce  -- all n(n-1)/2 pairs, union-find.  O(n^2): tiny
 *                             inputs only.
 *
 * Status codes (the oracle's own; the test-suite maps them by name):
 *   0 OK, 1 INVALID_ARG, 2 NONFINITE, 3 OUT_OF_RANGE, 4 OOM.
 * Precedence: argument errors, then any non-finite coordinate, then any
 * coordinate with |rint(x*1024)| >= 2^23.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_OK 0
#define OR_INVALID_ARG 1
#define OR_NONFINITE 2
#define OR_OUT_OF_RANGE 3
#define OR_OOM 4

#define QLIMIT 8388608.0 /* 2^23 units */

/* ------------------------------------------------------------------------ */
/* Quantisation and threshold                                                */
/* ------------------------------------------------------------------------ */

/* q = rint(x * 1024), ties to even (the C default rounding mode).  x * 1024 is
 * an exact power-of-two scaling in float, so the only rounding is rint. */
int fec_oracle_quantize(const float *xyz, int64_t n, int32_t *q)
{
    int nonfinite = 0, outside = 0;
    for (int64_t i = 0; i < 3 * n; ++i) {
        float v = xyz[i];
        if (!isfinite(v)) {
            nonfinite = 1;
            continue;
        }
        double r = rint((double)(v * 1024.0f));
        if (fabs(r) >= QLIMIT) {
            outside = 1;
            continue;
        }
        q[i] = (int32_t)r;
    }
    if (nonfinite) return OR_NONFINITE;
    if (outside) return OR_OUT_OF_RANGE;
    return OR_OK;
}

/* T2 = floor((d*1024)^2).  d*1024 has at most 24 significant bits, so its
 * square is exact in double.  Capped at 2^62: no two valid points are farther
 * apart than 3 * (2^24)^2 < 2^50 squared units. */
int64_t fec_oracle_threshold(float d)
{
    double s = (double)d * 1024.0;
    double t = floor(s * s);
    if (t >= 4611686018427387904.0) return (int64_t)4611686018427387904LL;
    return (int64_t)t;
}

static int64_t sqdist(const int32_t *a, const int32_t *b)
{
    int64_t dx = (int64_t)a[0] - b[0];
    int64_t dy = (int64_t)a[1] - b[1];
    int64_t dz = (int64_t)a[2] - b[2];
    return dx * dx + dy * dy + dz * dz;
}

static int check_args(const float *xyz, int64_t n, float d, int64_t min_size,
                      int64_t max_size, const int32_t *labels, const int32_t *k)
{
    if (n < 0 || n > 2147483647LL) return OR_INVALID_ARG;
    if (!isfinite(d) || !(d > 0.0f)) return OR_INVALID_ARG;
    if (min_size < 0 || max_size < min_size) return OR_INVALID_ARG;
    if (k == NULL) return OR_INVALID_ARG;
    if (n > 0 && (xyz == NULL || labels == NULL)) return OR_INVALID_ARG;
    return OR_OK;
}

/* Turn a component map (comp[i] = smallest index of i's component) into the
 * output: sizes, the [min_size, max_size] filter, and numbering of the kept
 * components 0..k-1 in increasing order of their smallest index. */
static int finish_labels(const int32_t *comp, int64_t n, int64_t min_size,
                         int64_t max_size, int32_t *labels, int32_t *num_clusters)
{
    int64_t *size = (int64_t *)calloc((size_t)(n > 0 ? n : 1), sizeof(int64_t));
    int32_t *number = (int32_t *)malloc((size_t)(n > 0 ? n : 1) * sizeof(int32_t));
    if (!size || !number) {
        free(size);
        free(number);
        return OR_OOM;
    }
    for (int64_t i = 0; i < n; ++i) size[comp[i]] += 1;
    int32_t k = 0;
    for (int64_t s = 0; s < n; ++s) {
        number[s] = -1;
        if (comp[s] == s && size[s] >= min_size && size[s] <= max_size) number[s] = k++;
    }
    for (int64_t i = 0; i < n; ++i) labels[i] = number[comp[i]];
    *num_clusters = k;
    free(size);
    free(number);
    return OR_OK;
}

/* ------------------------------------------------------------------------ */
/* kd-tree                                                                   */
/* ------------------------------------------------------------------------ */

#define LEAF_SIZE 8

typedef struct {
    int32_t lo[3], hi[3];  /* bounding box of the node's points */
    int64_t begin, end;    /* range in perm[] */
    int64_t alive;         /* points of this subtree not yet visited */
    int32_t left, right;   /* children, -1 for a leaf */
    int32_t parent;
} kd_node;

typedef struct {
    const int32_t *q;
    int32_t *perm;
    kd_node *nodes;
    int64_t nnodes, cap;
    int32_t *leaf_of; /* point -> leaf node */
} kd_tree;

/* k-th smallest of perm[lo..hi) by coordinate `axis`; three-way partition so
 * that runs of equal coordinates (flat ground) stay linear. */
static void kd_select(kd_tree *t, int64_t lo, int64_t hi, int64_t kth, int axis)
{
    int32_t *p = t->perm;
    const int32_t *q = t->q;
    while (hi - lo > 1) {
        int64_t mid = lo + (hi - lo) / 2;
        int32_t a = q[3 * (int64_t)p[lo] + axis], b = q[3 * (int64_t)p[mid] + axis],
                c = q[3 * (int64_t)p[hi - 1] + axis];
        int32_t pivot = (a < b) ? ((b < c) ? b : ((a < c) ? c : a))
                                : ((a < c) ? a : ((b < c) ? c : b));
        int64_t lt = lo, i = lo, gt = hi;
        while (i < gt) {
            int32_t v = q[3 * (int64_t)p[i] + axis];
            if (v < pivot) {
                int32_t s = p[lt]; p[lt] = p[i]; p[i] = s;
                ++lt; ++i;
            } else if (v > pivot) {
                --gt;
                int32_t s = p[gt]; p[gt] = p[i]; p[i] = s;
            } else {
                ++i;
            }
        }
        if (kth < lt) hi = lt;
        else if (kth >= gt) lo = gt;
        else return;
    }
}

static int32_t kd_build(kd_tree *t, int64_t begin, int64_t end, int32_t parent)
{
    int32_t id = (int32_t)t->nnodes++;
    kd_node *nd = &t->nodes[id];
    nd->begin = begin;
    nd->end = end;
    nd->alive = end - begin;
    nd->parent = parent;
    nd->left = nd->right = -1;
    for (int a = 0; a < 3; ++a) {
        nd->lo[a] = INT32_MAX;
        nd->hi[a] = INT32_MIN;
    }
    for (int64_t i = begin; i < end; ++i) {
        const int32_t *pt = &t->q[3 * (int64_t)t->perm[i]];
        for (int a = 0; a < 3; ++a) {
            if (pt[a] < nd->lo[a]) nd->lo[a] = pt[a];
            if (pt[a] > nd->hi[a]) nd->hi[a] = pt[a];
        }
    }
    if (end - begin <= LEAF_SIZE) {
        for (int64_t i = begin; i < end; ++i) t->leaf_of[t->perm[i]] = id;
        return id;
    }
    int axis = 0;
    int64_t widest = -1;
    for (int a = 0; a < 3; ++a) {
        int64_t w = (int64_t)nd->hi[a] - nd->lo[a];
        if (w > widest) {
            widest = w;
            axis = a;
        }
    }
    int64_t mid = begin + (end - begin) / 2;
    kd_select(t, begin, end, mid, axis);
    int32_t l = kd_build(t, begin, mid, id);
    int32_t r = kd_build(t, mid, end, id);
    t->nodes[id].left = l; /* nodes[] never moves: it is sized up front */
    t->nodes[id].right = r;
    return id;
}

/* squared distance from point p to the node's box */
static int64_t box_sqdist(const kd_node *nd, const int32_t *p)
{
    int64_t s = 0;
    for (int a = 0; a < 3; ++a) {
        int64_t g = 0;
        if (p[a] < nd->lo[a]) g = (int64_t)nd->lo[a] - p[a];
        else if (p[a] > nd->hi[a]) g = (int64_t)p[a] - nd->hi[a];
        s += g * g;
    }
    return s;
}

static void kd_mark_visited(kd_tree *t, int32_t point)
{
    int32_t id = t->leaf_of[point];
    while (id >= 0) {
        t->nodes[id].alive -= 1;
        id = t->nodes[id].parent;
    }
}

/* Components by BFS over the kd-tree: comp[i] = smallest index of i's
 * component (the BFS seed). */
static int kd_components(const int32_t *q, int64_t n, int64_t T2, int32_t *comp)
{
    if (n == 0) return OR_OK;
    kd_tree t;
    memset(&t, 0, sizeof(t));
    t.q = q;
    t.cap = n / 2 + 64; /* leaves hold >= 4 points, so nodes <= n/2 */
    t.perm = (int32_t *)malloc((size_t)n * sizeof(int32_t));
    t.leaf_of = (int32_t *)malloc((size_t)n * sizeof(int32_t));
    t.nodes = (kd_node *)malloc((size_t)t.cap * sizeof(kd_node));
    unsigned char *visited = (unsigned char *)calloc((size_t)n, 1);
    int32_t *queue = (int32_t *)malloc((size_t)n * sizeof(int32_t));
    int32_t *stack = (int32_t *)malloc((size_t)t.cap * sizeof(int32_t));
    if (!t.perm || !t.leaf_of || !t.nodes || !visited || !queue || !stack) {
        free(t.perm); free(t.leaf_of); free(t.nodes);
        free(visited); free(queue); free(stack);
        return OR_OOM;
    }
    for (int64_t i = 0; i < n; ++i) t.perm[i] = (int32_t)i;
    kd_build(&t, 0, n, -1);

    for (int64_t seed = 0; seed < n; ++seed) {
        if (visited[seed]) continue;
        int64_t head = 0, tail = 0;
        visited[seed] = 1;
        comp[seed] = (int32_t)seed;
        kd_mark_visited(&t, (int32_t)seed);
        queue[tail++] = (int32_t)seed;
        while (head < tail) {
            const int32_t *p = &q[3 * (int64_t)queue[head++]];
            /* radius query: every not-yet-visited point within T2 of p */
            int64_t sp = 0;
            stack[sp++] = 0;
            while (sp > 0) {
                const kd_node *nd = &t.nodes[stack[--sp]];
                if (nd->alive == 0 || box_sqdist(nd, p) > T2) continue;
                if (nd->left < 0) {
                    for (int64_t i = nd->begin; i < nd->end; ++i) {
                        int32_t j = t.perm[i];
                        if (visited[j]) continue;
                        if (sqdist(p, &q[3 * (int64_t)j]) <= T2) {
                            visited[j] = 1;
                            comp[j] = (int32_t)seed;
                            kd_mark_visited(&t, j);
                            queue[tail++] = j;
                        }
                    }
                } else {
                    stack[sp++] = nd->left;
                    stack[sp++] = nd->right;
                }
            }
        }
    }
    free(t.perm); free(t.leaf_of); free(t.nodes);
    free(visited); free(queue); free(stack);
    return OR_OK;
}

/* ------------------------------------------------------------------------ */
/* Brute force: every pair, union-find                                       */
/* ------------------------------------------------------------------------ */

static int32_t uf_find(int32_t *parent, int32_t x)
{
    while (parent[x] != x) {
        parent[x] = parent[parent[x]];
        x = parent[x];
    }
    return x;
}

static int brute_components(const int32_t *q, int64_t n, int64_t T2, int32_t *comp)
{
    int32_t *parent = (int32_t *)malloc((size_t)(n > 0 ? n : 1) * sizeof(int32_t));
    if (!parent) return OR_OOM;
    for (int64_t i = 0; i < n; ++i) parent[i] = (int32_t)i;
    for (int64_t i = 0; i < n; ++i)
        for (int64_t j = i + 1; j < n; ++j)
            if (sqdist(&q[3 * i], &q[3 * j]) <= T2) {
                int32_t a = uf_find(parent, (int32_t)i), b = uf_find(parent, (int32_t)j);
                if (a == b) continue;
                if (a < b) parent[b] = a; /* the smaller index stays the root */
                else parent[a] = b;
            }
    for (int64_t i = 0; i < n; ++i) comp[i] = uf_find(parent, (int32_t)i);
    free(parent);
    return OR_OK;
}

/* ------------------------------------------------------------------------ */
/* Entry points                                                              */
/* ------------------------------------------------------------------------ */

typedef int (*components_fn)(const int32_t *, int64_t, int64_t, int32_t *);

static int run(components_fn fn, const float *xyz, int64_t n, float d, int64_t min_size,
               int64_t max_size, int32_t *labels, int32_t *num_clusters)
{
    int st = check_args(xyz, n, d, min_size, max_size, labels, num_clusters);
    if (st != OR_OK) return st;
    *num_clusters = 0;
    if (n == 0) return OR_OK;
    int32_t *q = (int32_t *)malloc((size_t)n * 3 * sizeof(int32_t));
    int32_t *comp = (int32_t *)malloc((size_t)n * sizeof(int32_t));
    if (!q || !comp) {
        free(q);
        free(comp);
        return OR_OOM;
    }
    st = fec_oracle_quantize(xyz, n, q);
    if (st == OR_OK) st = fn(q, n, fec_oracle_threshold(d), comp);
    if (st == OR_OK) st = finish_labels(comp, n, min_size, max_size, labels, num_clusters);
    free(q);
    free(comp);
    return st;
}

int fec_oracle_cluster(const float *xyz, int64_t n, float d, int64_t min_size,
                       int64_t max_size, int32_t *labels, int32_t *num_clusters)
{
    return run(kd_components, xyz, n, d, min_size, max_size, labels, num_clusters);
}

int fec_oracle_bruteforce(const float *xyz, int64_t n, float d, int64_t min_size,
                          int64_t max_size, int32_t *labels, int32_t *num_clusters)
{
    return run(brute_components, xyz, n, d, min_size, max_size, labels, num_clusters);
}

/* Component map only (comp[i] = smallest index in i's component), from
 * already-quantised coordinates; used by tests of the BFS itself. */
int fec_oracle_components(const int32_t *q, int64_t n, int64_t T2, int32_t *comp)
{
    return kd_components(q, n, T2, comp);
}
