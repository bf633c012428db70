/*
 * sf_oracle_kdtree.c -- exact k nearest neighbours of every point of a large
 * cloud, for the oracle's bandwidths at sizes where the all-pairs loop of
 * or_knn (sf_oracle.c) is out of reach (16.8M points: 2.8e14 pairs).
 *
 * TEST INFRASTRUCTURE ONLY, like sf_oracle.c: loaded by the tests alone. It
 * shares no code with the CUDA library and uses no Morton order, no 32-ary
 * index and no histogram selection: a plain binary k-d tree with median
 * splits and a depth-first nearest-first search, the textbook method.
 *
 * Definition (the same as or_knn, and pinned against it by the CPU tests):
 * the neighbours of i are the k points j != i with the smallest
 *   d2 = ((dx*dx) + (dy*dy)) + (dz*dz),  dx = (double)x_i - (double)x_j
 * (separately rounded double operations; build with -ffp-contract=off), ties
 * broken by the smaller original index j, and h_i = (float) sqrt(d2 of the
 * k-th).
 *
 * Why the tree cannot change the answer: a subtree on the far side of a
 * splitting plane at coordinate s holds only points with |y_a - x_a| >=
 * |s - x_a| on the split axis a. Squaring and the rounded sums are monotone,
 * so every such point has d2 >= fl(fl(s - x_a)^2) as computed here. The
 * subtree is skipped only when that bound is strictly larger than the
 * current k-th d2 of a full list, so no point that could enter the list
 * (a smaller d2, or an equal d2 with a smaller index) is ever skipped.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

#define KD_LEAF 16

typedef struct {
    const float *xyz;
    int64_t n;
    int64_t *idx;      /* point order: each node owns a contiguous range */
    int nlevels;       /* inner levels; nodes of level l are 2^l - 1 .. 2^(l+1) - 2 */
    int8_t *axis;      /* per inner node */
    float *split;      /* per inner node: coordinate at the range's middle */
} kd_tree;

static float coord(const kd_tree *t, int64_t i, int a) { return t->xyz[3 * t->idx[i] + a]; }

static void swap_idx(int64_t *v, int64_t a, int64_t b) {
    int64_t x = v[a];
    v[a] = v[b];
    v[b] = x;
}

/* Reorder idx[lo, hi) so that position mid holds the element of rank mid - lo
 * by coordinate a, everything before it is <= and everything after it >=. */
static void select_mid(kd_tree *t, int64_t lo, int64_t hi, int64_t mid, int a) {
    int64_t *v = t->idx;
    while (hi - lo > 1) {
        /* median of three as pivot, moved to hi - 1 */
        int64_t m = lo + (hi - lo) / 2;
        if (coord(t, m, a) < coord(t, lo, a)) swap_idx(v, m, lo);
        if (coord(t, hi - 1, a) < coord(t, lo, a)) swap_idx(v, hi - 1, lo);
        if (coord(t, m, a) < coord(t, hi - 1, a)) swap_idx(v, m, hi - 1);
        const float pv = coord(t, hi - 1, a);
        /* three-way partition: [lo, lt) < pv, [lt, gt) == pv, [gt, hi) > pv */
        int64_t lt = lo, i = lo, gt = hi;
        while (i < gt) {
            const float c = coord(t, i, a);
            if (c < pv) {
                swap_idx(v, lt++, i++);
            } else if (c > pv) {
                swap_idx(v, i, --gt);
            } else {
                ++i;
            }
        }
        if (mid < lt) {
            hi = lt;
        } else if (mid >= gt) {
            lo = gt;
        } else {
            return;
        }
    }
}

/* Range of inner node `node` at level l: ranges halve level by level. */
static void node_range(const kd_tree *t, int64_t node, int64_t *lo, int64_t *hi) {
    int64_t a = 0, b = t->n;
    /* path from the root: bits of (node + 1) below the leading one */
    int depth = 0;
    for (int64_t x = node + 1; x > 1; x >>= 1) ++depth;
    for (int d = depth - 1; d >= 0; --d) {
        const int64_t mid = a + (b - a) / 2;
        if (((node + 1) >> d) & 1) a = mid;
        else b = mid;
    }
    *lo = a;
    *hi = b;
}

static int kd_build(kd_tree *t) {
    const int64_t n = t->n;
    t->idx = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
    if (!t->idx) return -1;
    for (int64_t i = 0; i < n; ++i) t->idx[i] = i;
    int levels = 0;
    while ((n >> levels) > KD_LEAF) ++levels;
    t->nlevels = levels;
    const int64_t ninner = ((int64_t)1 << levels) - 1;
    t->axis = (int8_t *)malloc((size_t)(ninner > 0 ? ninner : 1));
    t->split = (float *)malloc(sizeof(float) * (size_t)(ninner > 0 ? ninner : 1));
    if (!t->axis || !t->split) return -1;
    for (int l = 0; l < levels; ++l) {
        const int64_t first = ((int64_t)1 << l) - 1, count = (int64_t)1 << l;
        int64_t c;
#pragma omp parallel for schedule(dynamic, 1)
        for (c = 0; c < count; ++c) {
            const int64_t node = first + c;
            int64_t lo, hi;
            node_range(t, node, &lo, &hi);
            /* split the widest extent of the range's bounding box */
            float bl[3] = {INFINITY, INFINITY, INFINITY}, bh[3] = {-INFINITY, -INFINITY, -INFINITY};
            for (int64_t i = lo; i < hi; ++i)
                for (int a = 0; a < 3; ++a) {
                    const float v = coord(t, i, a);
                    if (v < bl[a]) bl[a] = v;
                    if (v > bh[a]) bh[a] = v;
                }
            int a = 0;
            for (int b = 1; b < 3; ++b)
                if ((double)bh[b] - (double)bl[b] > (double)bh[a] - (double)bl[a]) a = b;
            const int64_t mid = lo + (hi - lo) / 2;
            select_mid(t, lo, hi, mid, a);
            t->axis[node] = (int8_t)a;
            t->split[node] = coord(t, mid, a);
        }
    }
    return 0;
}

/* Candidate list of one query: ascending (d2, j), at most k entries. */
typedef struct {
    double *d;
    int64_t *j;
    int cnt, k;
} kd_list;

static void list_offer(kd_list *L, double d2, int64_t j) {
    const int k = L->k;
    if (L->cnt == k && (d2 > L->d[k - 1] || (d2 == L->d[k - 1] && j > L->j[k - 1]))) return;
    int pos = (L->cnt < k) ? L->cnt : k - 1;
    while (pos > 0 && (L->d[pos - 1] > d2 || (L->d[pos - 1] == d2 && L->j[pos - 1] > j))) {
        L->d[pos] = L->d[pos - 1];
        L->j[pos] = L->j[pos - 1];
        --pos;
    }
    L->d[pos] = d2;
    L->j[pos] = j;
    if (L->cnt < k) ++L->cnt;
}

static void kd_query(const kd_tree *t, int64_t qi, kd_list *L, int64_t *stack) {
    const double q[3] = {(double)t->xyz[3 * qi], (double)t->xyz[3 * qi + 1], (double)t->xyz[3 * qi + 2]};
    /* stack entries: node index, or ~node for a far child still to be bounded */
    int sp = 0;
    stack[sp++] = 0;
    while (sp > 0) {
        int64_t node = stack[--sp];
        if (node < 0) {
            /* far child of a split: visit only if the plane is not beyond the k-th */
            node = ~node;
            const int64_t parent = (node - 1) / 2;
            const double ds = (double)t->split[parent] - q[t->axis[parent]];
            const double b = ds * ds;
            if (L->cnt == L->k && b > L->d[L->k - 1]) continue;
        }
        int depth = 0;
        for (int64_t x = node + 1; x > 1; x >>= 1) ++depth;
        if (depth == t->nlevels) {
            int64_t lo, hi;
            node_range(t, node, &lo, &hi);
            for (int64_t i = lo; i < hi; ++i) {
                const int64_t j = t->idx[i];
                if (j == qi) continue;
                const double dx = q[0] - (double)t->xyz[3 * j + 0];
                const double dy = q[1] - (double)t->xyz[3 * j + 1];
                const double dz = q[2] - (double)t->xyz[3 * j + 2];
                list_offer(L, ((dx * dx) + (dy * dy)) + (dz * dz), j);
            }
            continue;
        }
        const int a = t->axis[node];
        const int64_t left = 2 * node + 1, right = 2 * node + 2;
        /* the near side first (pushed last), the far side bounded when popped */
        if (q[a] < (double)t->split[node]) {
            stack[sp++] = ~right;
            stack[sp++] = left;
        } else {
            stack[sp++] = ~left;
            stack[sp++] = right;
        }
    }
}

/*
 * h_out[i] (float, n) = bandwidth of every point i; nbr_out (nullable, n*k)
 * = its neighbours ascending by (d2, j). Returns 0, or -1 if k < 1, n <= k,
 * or memory runs out.
 */
int or_knn_tree(const float *xyz, int64_t n, int k, float *h_out, int64_t *nbr_out) {
    if (k < 1 || n <= k) return -1;
    kd_tree t;
    memset(&t, 0, sizeof t);
    t.xyz = xyz;
    t.n = n;
    int rc = kd_build(&t);
    if (rc == 0) {
        int failed = 0;
#pragma omp parallel reduction(| : failed)
        {
            kd_list L;
            L.k = k;
            L.d = (double *)malloc(sizeof(double) * (size_t)k);
            L.j = (int64_t *)malloc(sizeof(int64_t) * (size_t)k);
            int64_t *stack = (int64_t *)malloc(sizeof(int64_t) * (size_t)(2 * t.nlevels + 2));
            if (!L.d || !L.j || !stack) {
                failed = 1;
            } else {
                int64_t i;
#pragma omp for schedule(dynamic, 256)
                for (i = 0; i < n; ++i) {
                    L.cnt = 0;
                    kd_query(&t, i, &L, stack);
                    h_out[i] = (float)sqrt(L.d[k - 1]);
                    if (nbr_out)
                        for (int m = 0; m < k; ++m) nbr_out[i * k + m] = L.j[m];
                }
            }
            free(L.d);
            free(L.j);
            free(stack);
        }
        if (failed) rc = -1;
    }
    free(t.idx);
    free(t.axis);
    free(t.split);
    return rc;
}
