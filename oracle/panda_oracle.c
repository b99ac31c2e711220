/*
 * panda_oracle.c -- plain CPU oracle for PANDA's kd-tree construction and exact
 * k-nearest-neighbour query (Patwary et al., "PANDA: Extreme Scale Parallel
 * K-Nearest Neighbor on Distributed Architectures", arXiv 1607.08220).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg may load this library.  It shares no code,
 * header, table or constant generator with the CUDA path; it is deliberately
 * slow and written to be checked against the paper by eye.
 *
 * Build: gcc -O2 -ffp-contract=off -fno-fast-math -fopenmp -shared -fPIC
 * (no FMA contraction, IEEE round-to-nearest-even, denormals kept), so every
 * float operation below is one correctly rounded FP32 operation.
 *
 * What it computes
 * ----------------
 * Result definition (the thing every implementation must reproduce): for a
 * query q, the k points with the smallest keys (d2(q,x), id) in ascending
 * order, where d2 is the FP32 sum over dimensions 0..d-1, in that order, of
 * fl(fl(q_i - x_i) * fl(q_i - x_i)), each operation rounded separately.  Ids
 * are unique, so the answer is unique.  or_brute_knn() is that definition
 * written out; the kd-tree path (or_build + or_knn) only accelerates it.
 *
 * Tree construction, Sec. III-A (steps ii-iv) and Sec. III-A1:
 *   - a node with count <= B is a leaf (bucket rule, Sec. III-A1 "Choice of
 *     bucket size");
 *   - split dimension = the dimension of maximum variance over a sample of
 *     the node's points (Sec. III-A1 "Choice of split dimension");
 *   - split value = the sample "interval point" closest to 50% of a histogram
 *     of all node points over the sorted samples (Sec. III-A1 "Choice of split
 *     point", 1024 samples for a local tree);
 *   - points are shuffled so each bucket is contiguous (step iv, "SIMD
 *     packing"); here every partition is stable, so the final point order is
 *     the leaf order.
 * Readings where the paper is silent (each also listed in the design notes):
 *   R1 sample: S' = min(1024, n_node) values at positions floor(j*n_node/S'),
 *      j = 0..S'-1, in the node's current (stable) order;
 *   R2 variance in FP32 in a fixed order: element j goes into partial j mod 32
 *      sequentially, then the 32 partials are added pairwise at offsets
 *      16, 8, 4, 2, 1; mean = sum / S', var = sum((x - mean)^2) / S';
 *      argmax by a sequential scan with strict '>' (ties -> lowest dim);
 *   R3 histogram bin of x = #{v_j <= x} over sorted samples v; cumulative
 *      c_j = #{x < v_j}; j* = argmin |2 c_j - n_node| (ties -> smallest j);
 *      s = v_{j*}; left = {x[dim] < s}, right = {x[dim] >= s};
 *   R4 if var[dim*] is not > 0 or c_{j*} == 0 (heavy duplicates): take the
 *      dims in descending-variance order (the same scan repeated) and use the
 *      first one whose node max > node min with s = the smallest node value
 *      greater than the node min; if every dim is constant, split by index:
 *      left = the first ceil(n/2) points in stable order ("index split");
 *   R5 every node stores its tight axis-aligned bounding box.
 *
 * Query, Algorithm 1 (Sec. III-B/III-C) with three corrections:
 *   C1 the bound pushed for a child is its tight box distance (the literal
 *      sqrt(d^2 + d'^2) accumulation over-estimates when a dimension is split
 *      twice and can prune true neighbours);
 *   C2 after a replacement the pruning radius is the new k-th key of H, not
 *      the inserted distance;
 *   C3 keys (d2, id) are compared lexicographically; a subtree is pruned only
 *      when its bound is strictly greater than the current k-th distance.
 * Distances stay squared (no sqrt).  If n < k the tail of a row is
 * (id -1, d2 +inf).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_OK 0
#define OR_ERR_INVALID 1
#define OR_ERR_NONFINITE 2
#define OR_ERR_UNSUPPORTED 3
#define OR_ERR_NOMEM 4
#define OR_ERR_DEPTH 5

#define OR_SAMPLES 1024   /* local-tree sample count, Sec. III-A1 */
#define OR_MAX_DEPTH 64   /* deepest level allowed below the root */
#define OR_MAX_DIM 16

typedef struct {
    int32_t leaf;         /* 1 = bucket */
    int32_t index_split;  /* 1 = split by stable index (all dims constant) */
    int32_t dim;          /* split dimension (inner) */
    int32_t depth;        /* root = 0 */
    float split;          /* split value s: left x[dim] < s, right x[dim] >= s */
    int64_t start, count; /* range of the node in the leaf-order permutation */
    int64_t left, right;  /* child node indices (inner), -1 for a leaf */
} or_node;

typedef struct {
    int64_t n;
    int32_t d, bucket;
    float *pts;           /* copy of the input, row-major [n][d], original order */
    int32_t *perm;        /* leaf order: perm[i] = original row index */
    or_node *nodes;
    float *lo, *hi;       /* tight boxes [cap][d] */
    int64_t n_nodes, cap;
    int32_t depth;        /* deepest node */
    int32_t status;
} or_tree;

/* ---------------------------------------------------------------- helpers */

/* FP32 sum of vals[0..cnt) in the fixed order of reading R2. */
static float fixed_order_sum(const float *vals, int64_t cnt)
{
    float part[32];
    for (int p = 0; p < 32; p++) part[p] = 0.0f;
    for (int64_t j = 0; j < cnt; j++) part[j % 32] = part[j % 32] + vals[j];
    for (int off = 16; off >= 1; off /= 2)
        for (int p = 0; p < off; p++) part[p] = part[p] + part[p + off];
    return part[0];
}

static int cmp_float(const void *a, const void *b)
{
    float x = *(const float *)a, y = *(const float *)b;
    return (x < y) ? -1 : (x > y) ? 1 : 0;
}

/* #{j : v[j] <= x} for sorted v (binary search for the histogram bin). */
static int64_t upper_bound_count(const float *v, int64_t cnt, float x)
{
    int64_t lo = 0, hi = cnt;
    while (lo < hi) {
        int64_t mid = lo + (hi - lo) / 2;
        if (v[mid] <= x) lo = mid + 1; else hi = mid;
    }
    return lo;
}

static int key_less(float da, int32_t ia, float db, int32_t ib)
{
    return (da < db) || (da == db && ia < ib);
}

/* Squared distance, dims in order, each op rounded (no FMA: -ffp-contract=off). */
static float sq_dist(const float *q, const float *x, int d)
{
    float acc = 0.0f;
    for (int i = 0; i < d; i++) {
        float t = q[i] - x[i];
        float sq = t * t;
        acc = acc + sq;
    }
    return acc;
}

/* Squared distance from q to the box [lo, hi], same rounding and order. */
static float box_dist(const float *q, const float *lo, const float *hi, int d)
{
    float acc = 0.0f;
    for (int i = 0; i < d; i++) {
        float g = 0.0f;
        if (q[i] < lo[i]) g = lo[i] - q[i];
        else if (q[i] > hi[i]) g = q[i] - hi[i];
        float sq = g * g;
        acc = acc + sq;
    }
    return acc;
}

/* ------------------------------------------------------------------ build */

typedef struct {
    float *samples;   /* [d][OR_SAMPLES] */
    float *sorted;    /* [OR_SAMPLES] */
    float *dev;       /* [OR_SAMPLES] */
    int64_t *hist;    /* [OR_SAMPLES + 1] */
    int32_t *tmp;     /* [n] partition scratch */
} or_scratch;

static int64_t new_node(or_tree *t)
{
    if (t->n_nodes == t->cap) {
        int64_t cap = t->cap * 2;
        or_node *nn = (or_node *)realloc(t->nodes, (size_t)cap * sizeof(or_node));
        if (!nn) return -1;
        t->nodes = nn;
        float *nlo = (float *)realloc(t->lo, (size_t)cap * t->d * sizeof(float));
        if (!nlo) return -1;
        t->lo = nlo;
        float *nhi = (float *)realloc(t->hi, (size_t)cap * t->d * sizeof(float));
        if (!nhi) return -1;
        t->hi = nhi;
        t->cap = cap;
    }
    return t->n_nodes++;
}

static float coord(const or_tree *t, int64_t pos, int dim)
{
    return t->pts[(int64_t)t->perm[pos] * t->d + dim];
}

/* Index of the largest value by a sequential scan with strict '>' over the
 * dims not yet used (ties keep the lowest dim). */
static int argmax_unused(const float *var, const int *used, int d)
{
    int best = -1;
    for (int k = 0; k < d; k++) {
        if (used[k]) continue;
        if (best < 0 || var[k] > var[best]) best = k;
    }
    return best;
}

/* Stable partition of perm[start..start+count) by pred(position-in-node). */
static void stable_partition(or_tree *t, or_scratch *s, int64_t start, int64_t count,
                             int mode, int dim, float split, int64_t *left_count)
{
    int64_t nl = 0, nr = 0;
    int64_t half = (count + 1) / 2;
    /* left points first, in order */
    for (int64_t i = 0; i < count; i++) {
        int go_left = (mode == 1) ? (i < half) : (coord(t, start + i, dim) < split);
        if (go_left) s->tmp[nl++] = t->perm[start + i];
    }
    for (int64_t i = 0; i < count; i++) {
        int go_left = (mode == 1) ? (i < half) : (coord(t, start + i, dim) < split);
        if (!go_left) s->tmp[nl + nr++] = t->perm[start + i];
    }
    memcpy(t->perm + start, s->tmp, (size_t)count * sizeof(int32_t));
    *left_count = nl;
}

static int64_t build_node(or_tree *t, or_scratch *s, int64_t start, int64_t count, int depth)
{
    const int d = t->d;
    int64_t id = new_node(t);
    if (id < 0) { t->status = OR_ERR_NOMEM; return -1; }
    or_node *nd = &t->nodes[id];
    memset(nd, 0, sizeof(*nd));
    nd->start = start;
    nd->count = count;
    nd->depth = depth;
    nd->left = nd->right = -1;
    if (depth > t->depth) t->depth = depth;

    /* R5: tight box of the node */
    for (int k = 0; k < d; k++) {
        float mn = coord(t, start, k), mx = mn;
        for (int64_t i = 1; i < count; i++) {
            float x = coord(t, start + i, k);
            if (x < mn) mn = x;
            if (x > mx) mx = x;
        }
        t->lo[id * d + k] = mn;
        t->hi[id * d + k] = mx;
    }

    /* bucket rule */
    if (count <= t->bucket) { nd->leaf = 1; return id; }
    if (depth >= OR_MAX_DEPTH) { t->status = OR_ERR_DEPTH; return -1; }

    /* R1: sample at stable strided positions */
    int64_t ns = count < OR_SAMPLES ? count : OR_SAMPLES;
    for (int64_t j = 0; j < ns; j++) {
        int64_t pos = start + (j * count) / ns;
        for (int k = 0; k < d; k++) s->samples[k * OR_SAMPLES + j] = coord(t, pos, k);
    }

    /* R2: per-dimension sample variance, fixed order */
    float var[OR_MAX_DIM];
    for (int k = 0; k < d; k++) {
        const float *col = s->samples + k * OR_SAMPLES;
        float mean = fixed_order_sum(col, ns) / (float)ns;
        for (int64_t j = 0; j < ns; j++) {
            float c = col[j] - mean;
            s->dev[j] = c * c;
        }
        var[k] = fixed_order_sum(s->dev, ns) / (float)ns;
    }
    int used[OR_MAX_DIM] = {0};
    int dim = argmax_unused(var, used, d);

    int mode = 0;          /* 0 value split, 1 index split */
    float split = 0.0f;
    int have_split = 0;

    if (var[dim] > 0.0f) {
        /* R3: sorted interval points, histogram of all node points, closest to 50% */
        memcpy(s->sorted, s->samples + dim * OR_SAMPLES, (size_t)ns * sizeof(float));
        qsort(s->sorted, (size_t)ns, sizeof(float), cmp_float);
        for (int64_t b = 0; b <= ns; b++) s->hist[b] = 0;
        for (int64_t i = 0; i < count; i++)
            s->hist[upper_bound_count(s->sorted, ns, coord(t, start + i, dim))]++;
        int64_t c = 0, best_j = -1, best_c = 0, best_err = 0;
        for (int64_t j = 0; j < ns; j++) {
            c += s->hist[j];                 /* c_j = #{x < v_j} */
            int64_t err = 2 * c - count;
            if (err < 0) err = -err;
            if (best_j < 0 || err < best_err) { best_j = j; best_err = err; best_c = c; }
        }
        if (best_c > 0) { split = s->sorted[best_j]; have_split = 1; }
    }
    if (!have_split) {
        /* R4: first non-constant dim in descending-variance order */
        for (int r = 0; r < d && !have_split; r++) {
            int k = argmax_unused(var, used, d);
            used[k] = 1;
            float mn = t->lo[id * d + k], mx = t->hi[id * d + k];
            if (mx > mn) {
                float nxt = mx;
                for (int64_t i = 0; i < count; i++) {
                    float x = coord(t, start + i, k);
                    if (x > mn && x < nxt) nxt = x;
                }
                dim = k;
                split = nxt;
                have_split = 1;
            }
        }
        if (!have_split) {
            mode = 1;
            dim = 0;
            split = t->lo[id * d + 0];
        }
    }

    int64_t nl = 0;
    stable_partition(t, s, start, count, mode, dim, split, &nl);
    nd = &t->nodes[id];
    nd->dim = dim;
    nd->split = split;
    nd->index_split = mode;

    int64_t l = build_node(t, s, start, nl, depth + 1);
    if (l < 0) return -1;
    int64_t r = build_node(t, s, start + nl, count - nl, depth + 1);
    if (r < 0) return -1;
    t->nodes[id].left = l;
    t->nodes[id].right = r;
    return id;
}

void or_free(or_tree *t)
{
    if (!t) return;
    free(t->pts);
    free(t->perm);
    free(t->nodes);
    free(t->lo);
    free(t->hi);
    free(t);
}

/* Build a kd-tree over pts (host, row-major [n][d]).  Returns OR_* status. */
int or_build(const float *pts, int64_t n, int32_t d, int32_t bucket, or_tree **out)
{
    *out = NULL;
    if (!pts || n < 1 || n >= ((int64_t)1 << 31) || d < 1 || bucket < 1) return OR_ERR_INVALID;
    if (d > OR_MAX_DIM) return OR_ERR_UNSUPPORTED;
    for (int64_t i = 0; i < n * d; i++)
        if (!isfinite(pts[i])) return OR_ERR_NONFINITE;

    or_tree *t = (or_tree *)calloc(1, sizeof(or_tree));
    if (!t) return OR_ERR_NOMEM;
    t->n = n;
    t->d = d;
    t->bucket = bucket;
    t->cap = 1024;
    t->pts = (float *)malloc((size_t)(n * d) * sizeof(float));
    t->perm = (int32_t *)malloc((size_t)n * sizeof(int32_t));
    t->nodes = (or_node *)malloc((size_t)t->cap * sizeof(or_node));
    t->lo = (float *)malloc((size_t)t->cap * d * sizeof(float));
    t->hi = (float *)malloc((size_t)t->cap * d * sizeof(float));
    or_scratch s;
    s.samples = (float *)malloc((size_t)d * OR_SAMPLES * sizeof(float));
    s.sorted = (float *)malloc(OR_SAMPLES * sizeof(float));
    s.dev = (float *)malloc(OR_SAMPLES * sizeof(float));
    s.hist = (int64_t *)malloc((OR_SAMPLES + 1) * sizeof(int64_t));
    s.tmp = (int32_t *)malloc((size_t)n * sizeof(int32_t));
    int st = OR_OK;
    if (!t->pts || !t->perm || !t->nodes || !t->lo || !t->hi || !s.samples || !s.sorted ||
        !s.dev || !s.hist || !s.tmp) {
        st = OR_ERR_NOMEM;
    } else {
        memcpy(t->pts, pts, (size_t)(n * d) * sizeof(float));
        for (int64_t i = 0; i < n; i++) t->perm[i] = (int32_t)i;
        build_node(t, &s, 0, n, 0);
        st = t->status;
    }
    free(s.samples);
    free(s.sorted);
    free(s.dev);
    free(s.hist);
    free(s.tmp);
    if (st != OR_OK) { or_free(t); return st; }
    *out = t;
    return OR_OK;
}

/* ------------------------------------------------------------- inspection */

int64_t or_tree_num_nodes(const or_tree *t) { return t->n_nodes; }
int32_t or_tree_depth(const or_tree *t) { return t->depth; }

/* Copy the node table out (preorder: a node precedes its subtrees).
 * meta[i] = {leaf, index_split, dim, depth}; range[i] = {start, count, left, right};
 * lo/hi [n_nodes][d]; perm [n]. */
void or_tree_export(const or_tree *t, int32_t *meta, float *split, int64_t *range,
                    float *lo, float *hi, int32_t *perm)
{
    for (int64_t i = 0; i < t->n_nodes; i++) {
        const or_node *nd = &t->nodes[i];
        meta[4 * i + 0] = nd->leaf;
        meta[4 * i + 1] = nd->index_split;
        meta[4 * i + 2] = nd->dim;
        meta[4 * i + 3] = nd->depth;
        split[i] = nd->split;
        range[4 * i + 0] = nd->start;
        range[4 * i + 1] = nd->count;
        range[4 * i + 2] = nd->left;
        range[4 * i + 3] = nd->right;
    }
    memcpy(lo, t->lo, (size_t)(t->n_nodes * t->d) * sizeof(float));
    memcpy(hi, t->hi, (size_t)(t->n_nodes * t->d) * sizeof(float));
    memcpy(perm, t->perm, (size_t)t->n * sizeof(int32_t));
}

/* ------------------------------------------------------------------ query */

/* Insert (dv, iv) into the ascending list (hd, hid) of length *cnt <= k.
 * Caller guarantees *cnt < k or (dv, iv) < the k-th key. */
static void heap_insert(float *hd, int32_t *hid, int32_t *cnt, int32_t k, float dv, int32_t iv)
{
    int32_t pos = (*cnt < k) ? *cnt : k - 1;
    while (pos > 0 && key_less(dv, iv, hd[pos - 1], hid[pos - 1])) {
        hd[pos] = hd[pos - 1];
        hid[pos] = hid[pos - 1];
        pos--;
    }
    hd[pos] = dv;
    hid[pos] = iv;
    if (*cnt < k) (*cnt)++;
}

static void write_row(const float *hd, const int32_t *hid, int32_t cnt, int32_t k,
                      int32_t *ids, float *d2)
{
    for (int32_t j = 0; j < k; j++) {
        if (j < cnt) { ids[j] = hid[j]; d2[j] = hd[j]; }
        else { ids[j] = -1; d2[j] = INFINITY; }
    }
}

/* Algorithm 1 (corrected) for one query; visits = {nodes processed, points scanned}.
 * r2: Algorithm 1's search radius r, squared (reading R11: only points with
 * d2 <= r2 are neighbours; +inf = unbounded).  Until k neighbours are held,
 * r' = r2. */
static void find_knn(const or_tree *t, const float *q, int32_t k, float r2, float *hd, int32_t *hid,
                     int32_t *cnt, int64_t *visits)
{
    const int d = t->d;
    int64_t stack_node[2 * OR_MAX_DEPTH + 4];
    float stack_bound[2 * OR_MAX_DEPTH + 4];
    int sp = 0;
    *cnt = 0;
    stack_node[sp] = 0;
    stack_bound[sp] = box_dist(q, t->lo, t->hi, d);
    sp++;
    while (sp > 0) {
        sp--;
        int64_t node = stack_node[sp];
        float bound = stack_bound[sp];
        float rk = (*cnt < k) ? r2 : hd[k - 1];          /* r' */
        if (bound > rk) continue;                        /* C3: prune only if strictly farther */
        const or_node *nd = &t->nodes[node];
        if (visits) visits[0]++;
        if (nd->leaf) {
            for (int64_t i = nd->start; i < nd->start + nd->count; i++) {
                int32_t id = t->perm[i];
                float dv = sq_dist(q, t->pts + (int64_t)id * d, d);
                if (visits) visits[1]++;
                if (!(dv <= r2)) continue;
                if (*cnt < k || key_less(dv, id, hd[k - 1], hid[k - 1]))
                    heap_insert(hd, hid, cnt, k, dv, id);   /* C2: r' = new k-th key */
            }
        } else {
            int64_t near = (q[nd->dim] >= nd->split) ? nd->right : nd->left;
            int64_t far = (near == nd->right) ? nd->left : nd->right;
            float bfar = box_dist(q, t->lo + far * d, t->hi + far * d, d);     /* C1 */
            float bnear = box_dist(q, t->lo + near * d, t->hi + near * d, d);
            if (bfar <= rk) { stack_node[sp] = far; stack_bound[sp] = bfar; sp++; }
            stack_node[sp] = near;
            stack_bound[sp] = bnear;
            sp++;
        }
    }
}

/* KNN of m queries (host [m][d]) against the tree: ids/d2 [m][k], neighbours
 * within squared radius r2 (+inf: unbounded).  visits (optional) [m][2].
 * nthreads <= 0 uses the OpenMP default. */
int or_knn_r(const or_tree *t, const float *q, int64_t m, int32_t k, float r2, int32_t *ids, float *d2,
             int64_t *visits, int32_t nthreads)
{
    if (!t || m < 0 || k < 1 || (m > 0 && (!q || !ids || !d2)) || !(r2 >= 0.0f)) return OR_ERR_INVALID;
    if (k > 4096) return OR_ERR_UNSUPPORTED;
    for (int64_t i = 0; i < m * t->d; i++)
        if (!isfinite(q[i])) return OR_ERR_NONFINITE;
#ifdef _OPENMP
    if (nthreads <= 0) nthreads = omp_get_max_threads();
#else
    nthreads = 1;
#endif
    int failed = 0;
#pragma omp parallel num_threads(nthreads)
    {
        float *hd = (float *)malloc((size_t)k * sizeof(float));
        int32_t *hid = (int32_t *)malloc((size_t)k * sizeof(int32_t));
        if (!hd || !hid) {
#pragma omp atomic write
            failed = 1;
        } else {
#pragma omp for schedule(dynamic, 256)
            for (int64_t i = 0; i < m; i++) {
                int32_t cnt = 0;
                int64_t *v = visits ? visits + 2 * i : NULL;
                if (v) v[0] = v[1] = 0;
                find_knn(t, q + i * t->d, k, r2, hd, hid, &cnt, v);
                write_row(hd, hid, cnt, k, ids + i * k, d2 + i * k);
            }
        }
        free(hd);
        free(hid);
    }
    return failed ? OR_ERR_NOMEM : OR_OK;
}

int or_knn(const or_tree *t, const float *q, int64_t m, int32_t k, int32_t *ids, float *d2,
           int64_t *visits, int32_t nthreads)
{
    return or_knn_r(t, q, m, k, INFINITY, ids, d2, visits, nthreads);
}

/* The plain definition: exhaustive search over all n points, neighbours
 * within squared radius r2 (+inf: unbounded). */
int or_brute_knn_r(const float *pts, int64_t n, int32_t d, const float *q, int64_t m, int32_t k, float r2,
                   int32_t *ids, float *d2, int32_t nthreads)
{
    if (!pts || n < 1 || d < 1 || k < 1 || m < 0 || (m > 0 && (!q || !ids || !d2)) || !(r2 >= 0.0f))
        return OR_ERR_INVALID;
    if (k > 4096) return OR_ERR_UNSUPPORTED;
#ifdef _OPENMP
    if (nthreads <= 0) nthreads = omp_get_max_threads();
#else
    nthreads = 1;
#endif
    int failed = 0;
#pragma omp parallel num_threads(nthreads)
    {
        float *hd = (float *)malloc((size_t)k * sizeof(float));
        int32_t *hid = (int32_t *)malloc((size_t)k * sizeof(int32_t));
        if (!hd || !hid) {
#pragma omp atomic write
            failed = 1;
        } else {
#pragma omp for schedule(dynamic, 16)
            for (int64_t i = 0; i < m; i++) {
                int32_t cnt = 0;
                const float *qi = q + i * d;
                for (int64_t j = 0; j < n; j++) {
                    float dv = sq_dist(qi, pts + j * d, d);
                    if (!(dv <= r2)) continue;
                    if (cnt < k || key_less(dv, (int32_t)j, hd[k - 1], hid[k - 1]))
                        heap_insert(hd, hid, &cnt, k, dv, (int32_t)j);
                }
                write_row(hd, hid, cnt, k, ids + i * k, d2 + i * k);
            }
        }
        free(hd);
        free(hid);
    }
    return failed ? OR_ERR_NOMEM : OR_OK;
}

int or_brute_knn(const float *pts, int64_t n, int32_t d, const float *q, int64_t m, int32_t k,
                 int32_t *ids, float *d2, int32_t nthreads)
{
    return or_brute_knn_r(pts, n, d, q, m, k, INFINITY, ids, d2, nthreads);
}

/* Same as or_brute_knn for a subset of query rows: rows[r] indexes q. */
int or_brute_knn_rows(const float *pts, int64_t n, int32_t d, const float *q, const int64_t *rows,
                      int64_t nrows, int32_t k, int32_t *ids, float *d2, int32_t nthreads)
{
    if (!rows || nrows < 0) return OR_ERR_INVALID;
    if (nrows == 0) return OR_OK;
    float *qs = (float *)malloc((size_t)(nrows * d) * sizeof(float));
    if (!qs) return OR_ERR_NOMEM;
    for (int64_t r = 0; r < nrows; r++) memcpy(qs + r * d, q + rows[r] * d, (size_t)d * sizeof(float));
    int st = or_brute_knn(pts, n, d, qs, nrows, k, ids, d2, nthreads);
    free(qs);
    return st;
}

int32_t or_max_depth(void) { return OR_MAX_DEPTH; }
int32_t or_sample_count(void) { return OR_SAMPLES; }
