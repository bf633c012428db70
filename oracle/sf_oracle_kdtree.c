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
    float *pts;        /* the points in that order (x, y, z), moved with idx */
    int nlevels;       /* inner levels; nodes of level l are 2^l - 1 .. 2^(l+1) - 2 */
    int8_t *axis;      /* per inner node */
    float *split;      /* per inner node: coordinate at the range's middle */
} kd_tree;

static float coord(const kd_tree *t, int64_t i, int a) { return t->pts[3 * i + a]; }

static void swap_pt(kd_tree *t, int64_t a, int64_t b) {
    int64_t x = t->idx[a];
    t->idx[a] = t->idx[b];
    t->idx[b] = x;
    for (int c = 0; c < 3; ++c) {
        float y = t->pts[3 * a + c];
        t->pts[3 * a + c] = t->pts[3 * b + c];
        t->pts[3 * b + c] = y;
    }
}

/* Reorder [lo, hi) so that position mid holds the element of rank mid - lo
 * by coordinate a, everything before it is <= and everything after it >=. */
static void select_mid(kd_tree *t, int64_t lo, int64_t hi, int64_t mid, int a) {
    while (hi - lo > 1) {
        /* median of three as pivot, moved to hi - 1 */
        int64_t m = lo + (hi - lo) / 2;
        if (coord(t, m, a) < coord(t, lo, a)) swap_pt(t, m, lo);
        if (coord(t, hi - 1, a) < coord(t, lo, a)) swap_pt(t, hi - 1, lo);
        if (coord(t, m, a) < coord(t, hi - 1, a)) swap_pt(t, m, hi - 1);
        const float pv = coord(t, hi - 1, a);
        /* three-way partition: [lo, lt) < pv, [lt, gt) == pv, [gt, hi) > pv */
        int64_t lt = lo, i = lo, gt = hi;
        while (i < gt) {
            const float c = coord(t, i, a);
            if (c < pv) {
                swap_pt(t, lt++, i++);
            } else if (c > pv) {
                swap_pt(t, i, --gt);
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

/* Split a node's range at its middle along the widest extent of its box. */
static void split_node(kd_tree *t, int64_t node, int64_t lo, int64_t hi, const float bl[3],
                       const float bh[3]) {
    int a = 0;
    for (int b = 1; b < 3; ++b)
        if ((double)bh[b] - (double)bl[b] > (double)bh[a] - (double)bl[a]) a = b;
    const int64_t mid = lo + (hi - lo) / 2;
    select_mid(t, lo, hi, mid, a);
    t->axis[node] = (int8_t)a;
    t->split[node] = coord(t, mid, a);
}

static int kd_build(kd_tree *t) {
    const int64_t n = t->n;
    t->idx = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
    t->pts = (float *)malloc(sizeof(float) * 3 * (size_t)n);
    if (!t->idx || !t->pts) return -1;
    int64_t i0;
#pragma omp parallel for schedule(static)
    for (i0 = 0; i0 < n; ++i0) {
        t->idx[i0] = i0;
        t->pts[3 * i0 + 0] = t->xyz[3 * i0 + 0];
        t->pts[3 * i0 + 1] = t->xyz[3 * i0 + 1];
        t->pts[3 * i0 + 2] = t->xyz[3 * i0 + 2];
    }
    int levels = 0;
    while ((n >> levels) > KD_LEAF) ++levels;
    t->nlevels = levels;
    const int64_t ninner = ((int64_t)1 << levels) - 1;
    t->axis = (int8_t *)malloc((size_t)(ninner > 0 ? ninner : 1));
    t->split = (float *)malloc(sizeof(float) * (size_t)(ninner > 0 ? ninner : 1));
    if (!t->axis || !t->split) return -1;
    int nthr = 1;
#ifdef _OPENMP
    nthr = omp_get_max_threads();
#endif
    for (int l = 0; l < levels; ++l) {
        const int64_t first = ((int64_t)1 << l) - 1, count = (int64_t)1 << l;
        int64_t c;
        if (count < nthr) {
            /* few large nodes: the bounding box in parallel, node by node */
            for (c = 0; c < count; ++c) {
                const int64_t node = first + c;
                int64_t lo, hi;
                node_range(t, node, &lo, &hi);
                float b0 = INFINITY, b1 = INFINITY, b2 = INFINITY;
                float e0 = -INFINITY, e1 = -INFINITY, e2 = -INFINITY;
                int64_t i;
#pragma omp parallel for schedule(static) reduction(min : b0, b1, b2) reduction(max : e0, e1, e2)
                for (i = lo; i < hi; ++i) {
                    const float x = coord(t, i, 0), y = coord(t, i, 1), z = coord(t, i, 2);
                    b0 = x < b0 ? x : b0;
                    b1 = y < b1 ? y : b1;
                    b2 = z < b2 ? z : b2;
                    e0 = x > e0 ? x : e0;
                    e1 = y > e1 ? y : e1;
                    e2 = z > e2 ? z : e2;
                }
                const float bl[3] = {b0, b1, b2}, bh[3] = {e0, e1, e2};
                split_node(t, node, lo, hi, bl, bh);
            }
            continue;
        }
#pragma omp parallel for schedule(dynamic, 1)
        for (c = 0; c < count; ++c) {
            const int64_t node = first + c;
            int64_t lo, hi;
            node_range(t, node, &lo, &hi);
            float bl[3] = {INFINITY, INFINITY, INFINITY}, bh[3] = {-INFINITY, -INFINITY, -INFINITY};
            for (int64_t i = lo; i < hi; ++i)
                for (int a = 0; a < 3; ++a) {
                    const float v = coord(t, i, a);
                    if (v < bl[a]) bl[a] = v;
                    if (v > bh[a]) bh[a] = v;
                }
            split_node(t, node, lo, hi, bl, bh);
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

/* The k nearest points other than point qi (which sits at q) into L. */
static void kd_query_at(const kd_tree *t, int64_t qi, const double q[3], kd_list *L, int64_t *stack) {
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
                const double dx = q[0] - (double)t->pts[3 * i + 0];
                const double dy = q[1] - (double)t->pts[3 * i + 1];
                const double dz = q[2] - (double)t->pts[3 * i + 2];
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
                int64_t p;
                /* queries in tree order (neighbouring queries share tree paths) */
#pragma omp for schedule(dynamic, 256)
                for (p = 0; p < n; ++p) {
                    const int64_t i = t.idx[p];
                    const double q[3] = {(double)t.pts[3 * p], (double)t.pts[3 * p + 1],
                                         (double)t.pts[3 * p + 2]};
                    L.cnt = 0;
                    kd_query_at(&t, i, q, &L, stack);
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
    free(t.pts);
    free(t.axis);
    free(t.split);
    return rc;
}

/*
 * Kernel density with kNN bandwidths at m target positions r (m x 3 doubles),
 * for clouds where neither every bandwidth nor every pair can be evaluated:
 * the same numbers as or_density_at(xyz, ell = (h_j, h_j, h_j), ...) with h_j
 * the kNN bandwidth of or_knn, bit for bit (pinned by the CPU tests).
 *
 * The sum of Eq. 7 only has terms with q < 9 (or q < 1), i.e. |r - y_j| < R h_j
 * (R = 3 or 1). Which particles can reach r is decided from upper bounds of
 * their bandwidths, and only those particles get their exact h_j (a k-d tree
 * query as in or_knn_tree); every other particle is provably out of support:
 *
 * - A subtree whose points number at least k + 1 has, for each of its points,
 *   k other points inside its bounding box, so h_j <= the box diagonal D. The
 *   deepest tree level whose nodes all hold at least k + 1 points gives every
 *   point such a box; an upper node takes the largest D below it.
 * - A node is skipped when the distance from r to its box is at least R D
 *   (with a relative margin of 1e-5 + 2 amb_band on the squares, which covers
 *   rounding and the ambiguous band below); a point is skipped when
 *   |r - y_j| >= R F_j, F_j the distance from y_j to the farthest corner of
 *   its box (its k box mates lie no farther), before its kNN query.
 *
 * The surviving terms are then added in ascending j, with the operations of
 * or_density_at, so the result equals its result exactly: rho, wpeak (the sum
 * of in-support peaks), amb (the mass of pairs within amb_band of the cutoff)
 * and pairs (the in-support count), each times inv_neff where or_density_at
 * multiplies. Returns 0, or -1 on bad arguments or memory exhaustion.
 */
typedef struct {
    double lo[3], hi[3];
    double u;  /* bandwidth bound of every point below */
} kd_bound;

typedef struct {
    int64_t j;
    double val, peak;
    int in, amb;
} kd_term;

static int term_cmp(const void *a, const void *b) {
    const int64_t x = ((const kd_term *)a)->j, y = ((const kd_term *)b)->j;
    return (x > y) - (x < y);
}

int or_density_knn_tree(const float *xyz, int64_t n, int k, const double *r, int64_t m,
                        int kernel, double p3, double inv_neff, double *rho, double *wpeak,
                        double *amb, int64_t *pairs, double amb_band) {
    if (k < 1 || n <= k) return -1;
    const double pi = 3.14159265358979323846;
    const double qmax = (kernel == 0) ? 1.0 : 9.0;
    const double cnorm = (kernel == 0) ? 15.0 / (8.0 * pi) : 1.0 / (pow(2.0 * pi, 1.5) * p3);
    kd_tree t;
    memset(&t, 0, sizeof t);
    t.xyz = xyz;
    t.n = n;
    if (kd_build(&t) != 0) {
        free(t.idx);
        free(t.pts);
        free(t.axis);
        free(t.split);
        return -1;
    }
    /* deepest level whose every node holds >= k + 1 points */
    int du = 0;
    while (du < t.nlevels && (n >> (du + 1)) >= (int64_t)k + 1) ++du;
    const int64_t nb = ((int64_t)2 << du) - 1;
    kd_bound *B = (kd_bound *)malloc(sizeof(kd_bound) * (size_t)nb);
    float *hcache = (float *)malloc(sizeof(float) * (size_t)n);
    int rc = (B && hcache) ? 0 : -1;
    if (hcache) {
        int64_t i;
#pragma omp parallel for schedule(static)
        for (i = 0; i < n; ++i) hcache[i] = -1.0f;
    }
    if (rc == 0) {
        const int64_t first = ((int64_t)1 << du) - 1, count = (int64_t)1 << du;
        int64_t c;
#pragma omp parallel for schedule(dynamic, 64)
        for (c = 0; c < count; ++c) {
            kd_bound *b = &B[first + c];
            int64_t lo, hi;
            node_range(&t, first + c, &lo, &hi);
            for (int a = 0; a < 3; ++a) {
                b->lo[a] = INFINITY;
                b->hi[a] = -INFINITY;
            }
            for (int64_t i = lo; i < hi; ++i)
                for (int a = 0; a < 3; ++a) {
                    const double v = (double)coord(&t, i, a);
                    if (v < b->lo[a]) b->lo[a] = v;
                    if (v > b->hi[a]) b->hi[a] = v;
                }
            double d2 = 0.0;
            for (int a = 0; a < 3; ++a) d2 += (b->hi[a] - b->lo[a]) * (b->hi[a] - b->lo[a]);
            /* rounded up: h_j = (float)sqrt(d2_k) may round up by half a float ulp */
            b->u = sqrt(d2) * (1.0 + 1e-6) + 1e-300;
        }
        for (int l = du - 1; l >= 0; --l) {
            const int64_t f = ((int64_t)1 << l) - 1, cnt = (int64_t)1 << l;
            for (c = 0; c < cnt; ++c) {
                kd_bound *b = &B[f + c];
                const kd_bound *x = &B[2 * (f + c) + 1], *y = &B[2 * (f + c) + 2];
                for (int a = 0; a < 3; ++a) {
                    b->lo[a] = x->lo[a] < y->lo[a] ? x->lo[a] : y->lo[a];
                    b->hi[a] = x->hi[a] > y->hi[a] ? x->hi[a] : y->hi[a];
                }
                b->u = x->u > y->u ? x->u : y->u;
            }
        }
        /* (R^2) with the margin: rounding, and the ambiguous band on the far side */
        const double R2 = qmax * (1.0 + 1e-5 + 2.0 * amb_band);
        int failed = 0;
#pragma omp parallel reduction(| : failed)
        {
            kd_list L;
            L.k = k;
            L.d = (double *)malloc(sizeof(double) * (size_t)k);
            L.j = (int64_t *)malloc(sizeof(int64_t) * (size_t)k);
            int64_t *stack = (int64_t *)malloc(sizeof(int64_t) * (size_t)(2 * t.nlevels + 2));
            int64_t *nstack = (int64_t *)malloc(sizeof(int64_t) * (size_t)(2 * du + 4));
            int64_t tcap = 4096, nt = 0;
            kd_term *T = (kd_term *)malloc(sizeof(kd_term) * (size_t)tcap);
            if (!L.d || !L.j || !stack || !nstack || !T) {
                failed = 1;
            } else {
                int64_t q;
#pragma omp for schedule(dynamic, 1)
                for (q = 0; q < m; ++q) {
                    if (failed) continue;
                    const double rx = r[3 * q + 0], ry = r[3 * q + 1], rz = r[3 * q + 2];
                    const double rv[3] = {rx, ry, rz};
                    nt = 0;
                    int sp = 0;
                    nstack[sp++] = 0;
                    while (sp > 0 && !failed) {
                        const int64_t node = nstack[--sp];
                        const kd_bound *b = &B[node];
                        double g2 = 0.0;
                        for (int a = 0; a < 3; ++a) {
                            double g = 0.0;
                            if (rv[a] < b->lo[a]) g = b->lo[a] - rv[a];
                            else if (rv[a] > b->hi[a]) g = rv[a] - b->hi[a];
                            g2 += g * g;
                        }
                        if (!(g2 < R2 * b->u * b->u)) continue;
                        int depth = 0;
                        for (int64_t x = node + 1; x > 1; x >>= 1) ++depth;
                        if (depth < du) {
                            nstack[sp++] = 2 * node + 1;
                            nstack[sp++] = 2 * node + 2;
                            continue;
                        }
                        int64_t lo, hi;
                        node_range(&t, node, &lo, &hi);
                        for (int64_t i = lo; i < hi; ++i) {
                            const int64_t j = t.idx[i];
                            const double px = (double)t.pts[3 * i + 0];
                            const double py = (double)t.pts[3 * i + 1];
                            const double pz = (double)t.pts[3 * i + 2];
                            const double dx = rx - px, dy = ry - py, dz = rz - pz;
                            /* this point's own bound: its k box mates lie no farther
                               than the box corner farthest from it */
                            const double pp[3] = {px, py, pz};
                            double f2 = 0.0;
                            for (int a = 0; a < 3; ++a) {
                                const double e = pp[a] - b->lo[a] > b->hi[a] - pp[a] ? pp[a] - b->lo[a]
                                                                                     : b->hi[a] - pp[a];
                                f2 += e * e;
                            }
                            const double uj2 = f2 * (1.0 + 4e-6) + 1e-300;
                            if (!(((dx * dx) + (dy * dy)) + (dz * dz) < R2 * uj2)) continue;
                            /* h_j once per point, shared by all targets (by tree position) */
                            float hf;
#pragma omp atomic read
                            hf = hcache[i];
                            if (hf < 0.0f) {
                                L.cnt = 0;
                                const double pq[3] = {px, py, pz};
                                kd_query_at(&t, j, pq, &L, stack);
                                hf = (float)sqrt(L.d[k - 1]);
#pragma omp atomic write
                                hcache[i] = hf;
                            }
                            const double h = (double)hf;
                            if (!(h > 0.0)) continue;
                            /* the term exactly as or_density_at evaluates it */
                            const double ux = dx / h, uy = dy / h, uz = dz / h;
                            const double qq = ((ux * ux) + (uy * uy)) + (uz * uz);
                            const int ambiguous = fabs(qq / qmax - 1.0) < amb_band;
                            if (!(qq < qmax) && !ambiguous) continue;
                            const double peak = cnorm / ((h * h) * h);
                            const double val = (kernel == 0) ? peak * (1.0 - qq) : peak * exp(-0.5 * qq);
                            if (nt == tcap) {
                                kd_term *T2 = (kd_term *)realloc(T, sizeof(kd_term) * (size_t)(2 * tcap));
                                if (!T2) {
                                    failed = 1;
                                    break;
                                }
                                T = T2;
                                tcap *= 2;
                            }
                            T[nt].j = j;
                            T[nt].val = val;
                            T[nt].peak = peak;
                            T[nt].in = qq < qmax;
                            T[nt].amb = ambiguous;
                            ++nt;
                        }
                    }
                    qsort(T, (size_t)nt, sizeof(kd_term), term_cmp);
                    double sum = 0.0, wsum = 0.0, asum = 0.0;
                    int64_t np = 0;
                    for (int64_t e = 0; e < nt; ++e) {
                        if (T[e].amb) asum += fabs(T[e].val);
                        if (!T[e].in) continue;
                        sum += T[e].val;
                        wsum += T[e].peak;
                        ++np;
                    }
                    rho[q] = inv_neff * sum;
                    if (wpeak) wpeak[q] = inv_neff * wsum;
                    if (amb) amb[q] = inv_neff * asum;
                    if (pairs) pairs[q] = np;
                }
            }
            free(L.d);
            free(L.j);
            free(stack);
            free(nstack);
            free(T);
        }
        if (failed) rc = -1;
    }
    free(B);
    free(hcache);
    free(t.idx);
    free(t.pts);
    free(t.axis);
    free(t.split);
    return rc;
}
