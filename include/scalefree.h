/*
 * scalefree.h -- C ABI of libscalefree.so: on-the-fly adaptive kernel density
 * estimation over a region of interest (ROI) of a large float32 xyz point
 * cloud, on one NVIDIA GB300 (sm_103a).
 *
 * The method is the one of ScaleFree (arXiv 2601.20758, Sec. 3): a density
 * field on a uniform grid over a box B (Sec. 3.1), from per-particle adaptive
 * smoothing lengths, evaluated by gathering the kernel contributions of the
 * particles near each node (Sec. 3.2.1, Algorithms 1-4), plus density-threshold
 * selection of points (Sec. 4.1).
 *
 * Conventions shared by every call
 * --------------------------------
 * - Pointers named d_* are DEVICE pointers on the current CUDA device; h_* are
 *   HOST pointers. The caller owns every buffer passed in. The library owns
 *   the index (sf_index) and its internal workspaces.
 * - `stream` is a cudaStream_t passed as void* (NULL = the legacy default
 *   stream). Calls are stream-ordered. A call that returns a host scalar
 *   (h_*) synchronises that stream before returning.
 * - Every call returns an sf_status. Invalid arguments are rejected before
 *   any launch. sf_last_error() gives a message for the calling thread.
 * - Float inputs must be finite.
 * - Coordinates are world coordinates in float32; boxes are closed boxes
 *   [lo, hi] in double.
 * - Determinism: results are bit-identical from run to run for the same
 *   inputs (no floating-point atomics anywhere).
 * - One index may be used from several host threads on different streams
 *   once sf_bandwidths has returned; each stream gets its own workspace.
 */
#ifndef SCALEFREE_H
#define SCALEFREE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct sf_index sf_index;

typedef enum {
    SF_OK = 0,
    SF_ERR_INVALID_ARG = 1, /* NULL pointer, bad size, bad enum, dims < 2 ...      */
    SF_ERR_OOM = 2,         /* device allocation failed                              */
    SF_ERR_CUDA = 3,        /* a CUDA call or a kernel launch failed                 */
    SF_ERR_TIMEOUT = 4,     /* a bounded device-side wait gave up                    */
    SF_ERR_DEGENERATE = 5,  /* N <= k, fewer than 2 particles in B, P80 == P20     */
    SF_ERR_EMPTY_ROI = 6,   /* no particle of the scope lies in the ROI              */
    SF_ERR_BUSY = 7,        /* not admitted (serving)                                */
    SF_ERR_CAPACITY = 8     /* an output buffer (or an internal list) is too small   */
} sf_status;

/* Kernels.
 * SF_K_EPAN   (Eqs. 4 and 7): K = 15/(8 pi) / (lx ly lz) * (1 - q) for q < 1, else 0.
 * SF_K_GAUSS3: K = exp(-q/2) / ((2 pi)^(3/2) lx ly lz P3) for q < 9, else 0,
 *             P3 = P(chi^2_3 <= 9), so that the truncated kernel integrates to 1.
 * with q = sum_k ((r_k - y_k) / l_k)^2 (Eq. 8). */
enum { SF_K_EPAN = 0, SF_K_GAUSS3 = 1 };

/* Bandwidth rules.
 * SF_BW_KNN  : l_j = (h_j, h_j, h_j), h_j = distance to the k-th nearest other
 *              point, computed once per cloud by sf_bandwidths.
 * SF_BW_MBE  : the paper's modified Breiman estimator, per ROI (Eqs. 1, 2, 5, 6).
 * SF_BW_FIXED: l_j = fixed_h for every particle. */
enum { SF_BW_KNN = 0, SF_BW_MBE = 1, SF_BW_FIXED = 2 };

/* Which particles enter the sum, and the normaliser N_eff.
 * SF_SCOPE_CLIP  : particles inside the ROI box B, N_eff = N_B (Eq. 2, Sec. 3.1).
 * SF_SCOPE_GLOBAL: all particles, N_eff = N. */
enum { SF_SCOPE_CLIP = 0, SF_SCOPE_GLOBAL = 1 };

/* Precision variants. Point densities (sf_kde_points, DIRECT, kNN bandwidths):
 * the squared-distance cross term on tensor cores in TF32 (one pass), 3xTF32
 * (hi/lo split, three passes) or BF16 (one pass, 8 significant bits); see
 * sf_kde_points. Grids (sf_kde_grid, truncated Gaussian, kNN or fixed lengths):
 * the particles whose support covers a whole 8 x 4 x 8 node tile are summed as
 * a tensor-core product of their per-axis kernel factors in the same three
 * forms (terms off by about 1e-3 relative in TF32, 8e-3 in BF16, 2^-21 in
 * 3xTF32); the other particles stay FP32, and so do batches (sf_batch_create)
 * of Gaussian grids with tile_z 8. FP32 is the default everywhere and the only
 * form of every other call. */
enum { SF_PREC_FP32 = 0, SF_PREC_TF32 = 1, SF_PREC_3XTF32 = 2, SF_PREC_BF16 = 3 };

/* Point densities: DIRECT evaluates the kernel sum at each point (self term
 * included); INTERP interpolates the ROI grid trilinearly (Sec. 3.1, last step);
 * TETLIN takes the selection volume's piecewise-linear field (sf_iso_surface),
 * so that sf_select with the surface's threshold picks the points inside it. */
enum { SF_POINTS_DIRECT = 0, SF_POINTS_INTERP = 1, SF_POINTS_TETLIN = 2 };

/* Exact moment acceleration of grids (sf_kde_grid; Eq. 4 is a polynomial in
 * the offsets inside its support). With the Epanechnikov kernel and one
 * smoothing length for every particle (rule FIXED, and the pilot density of
 * rule MBE, Eq. 2), the sum over the points of an index node that lies wholly
 * inside the support of a grid node r is
 *     c (M0 - sum_k (M0 (r_k - mu_k)^2 + C_k) / l_k^2)
 * from the node's point count M0, centroid mu and central second moments C_k,
 * so only the nodes that straddle the support's edge are summed point by
 * point. The result is the same sum as the pair-by-pair gather up to rounding
 * (FP32 terms, FP64 accumulation). The pair-by-pair gather is faster whenever
 * it can run (the straddling shell holds most of the pairs unless l is many
 * leaf widths), but its per-tile candidate lists are bounded by 2^31 entries;
 * the moment form keeps no lists. SF_ACCEL_AUTO (0, the default): the gather,
 * and the moment form where the gather's lists would exceed that bound;
 * SF_ACCEL_NONE: the gather only (CAPACITY past the bound); SF_ACCEL_MOMENTS:
 * the moment form wherever it applies. The moments (48 bytes per index node,
 * about 1.5 bytes per point) are built with the index. */
enum { SF_ACCEL_AUTO = 0, SF_ACCEL_NONE = 1, SF_ACCEL_MOMENTS = 2 };

typedef struct {
    double lo[3];
    double hi[3];
} sf_box;

/* 80 bytes, fixed layout. */
typedef struct {
    int32_t rule;        /* SF_BW_*                                              */
    int32_t k;           /* kNN neighbours (SF_BW_KNN), 1 <= k <= 256            */
    double fixed_h[3];   /* SF_BW_FIXED smoothing lengths, > 0                   */
    double cap_factor;   /* SF_BW_MBE: l^(j) <= cap_factor * s_k (paper: 5)      */
    double p_lo, p_hi;   /* SF_BW_MBE: percentiles of Eq. 1 (paper: 20, 80)      */
    double log_base;     /* SF_BW_MBE: base of the log in Eq. 1; <= 0 means e    */
    int32_t scope;       /* SF_SCOPE_*                                           */
    int32_t prec;        /* SF_PREC_* (non-FP32: sf_kde_points only)             */
    int32_t points_mode; /* SF_POINTS_*                                          */
    int32_t accel;       /* SF_ACCEL_* (grids; 0 = AUTO)                         */
} sf_params;

/* Fill *p with the defaults: KNN, k = 32, cap 5, percentiles 20/80, natural
 * log, GLOBAL scope, FP32, DIRECT points, ACCEL_AUTO. */
void sf_params_default(sf_params *p);

/*
 * sf_build_index -- copy the cloud and build the spatial index on the device.
 *
 * Replaces the CPU k-d tree of Sec. 3.2 (built on the CPU and uploaded there)
 * by a GPU index: points radix-sorted by 63-bit Morton key (21 bits per axis
 * over the cloud's bounding box), stored as float4 (x, y, z, h) in that
 * order; leaves are runs of 32 consecutive sorted points and every upper
 * level groups 32 nodes; each node keeps its bounding box, the largest
 * smoothing length below it and the moments of its points (count, centroid,
 * central second moments; see SF_ACCEL_AUTO).
 *
 * d_xyz : device float32 [n][3] (x, y, z interleaved); read only, not kept.
 * n     : 1 <= n < 2^31.
 * out   : receives the new index; free it with sf_free_index.
 * Synchronises `stream` (the node count is read back). Errors: INVALID_ARG,
 * OOM, CUDA.
 * The calls' scratch comes from the device's default stream-ordered memory
 * pool (cudaMallocAsync); the first index build sets that pool to keep the
 * memory it has mapped between calls instead of returning it at every
 * synchronisation (a setting of this process only).
 */
sf_status sf_build_index(const float *d_xyz, int64_t n, void *stream, sf_index **out);

/* Number of points in the index. */
int64_t sf_index_size(const sf_index *idx);

/*
 * sf_bandwidths -- per-point smoothing lengths that do not depend on the ROI.
 *
 * SF_BW_KNN  : h_j = Euclidean distance to the k-th nearest other point of the
 *              cloud. The neighbour set is exact with respect to FP64 squared
 *              distances ((dx*dx)+(dy*dy))+(dz*dz) of the float inputs, ties broken
 *              by the smaller original index, and h_j = (float)sqrt(d2_k) -- it
 *              is bit-identical to a brute-force FP64 evaluation. n <= k gives
 *              DEGENERATE.
 * SF_BW_FIXED: stores fixed_h (isotropic only if the three are equal).
 * SF_BW_MBE  : nothing to precompute (the rule is per ROI); returns SF_OK.
 * The result stays resident in the index and is used by later calls with the
 * same rule. The kernels are queued on `stream` and the call returns without
 * waiting for them: a later call on another stream must be ordered after them
 * (an event, or a synchronisation) -- streams created non-blocking do not wait
 * for the legacy default stream.
 */
sf_status sf_bandwidths(sf_index *idx, const sf_params *params, void *stream);

/*
 * sf_get_bandwidths -- copy the kNN bandwidths h_j out, in ORIGINAL point
 * order. d_h: device float [n]. INVALID_ARG if no kNN bandwidths were built.
 */
sf_status sf_get_bandwidths(const sf_index *idx, float *d_h, void *stream);

/*
 * sf_knn_neighbours -- the k nearest other points of every point (for
 * verification): d_nbr device uint32 [n][k], original indices, row i for
 * original point i, in no particular order within a row; d_h device float [n]
 * (nullable). Same exactness contract as sf_bandwidths; does not change the
 * resident bandwidths.
 */
sf_status sf_knn_neighbours(sf_index *idx, int32_t k, uint32_t *d_nbr, float *d_h, void *stream);

/*
 * sf_knn_work_counts -- the work of the kNN bandwidths (SF_BW_KNN with this k)
 * on this index, for issue-rate accounting: one run of the same search with
 * counters, its results discarded (the index's resident bandwidths are not
 * touched). h_counts (host int64[3]): [0] (query, candidate) distance
 * evaluations -- every lane of a query leaf's warp evaluates every candidate
 * staged for the leaf, over all of the search's passes; [1] candidates staged,
 * summed over query leaves and passes; [2] query leaves (of 32 points).
 * Synchronises the stream. Errors: INVALID_ARG, DEGENERATE (n <= k), OOM, CUDA.
 */
sf_status sf_knn_work_counts(sf_index *idx, int32_t k, int64_t *h_counts, void *stream);

/*
 * sf_kde_grid -- density at every node of a dims[0] x dims[1] x dims[2] grid
 * over the ROI box (Sec. 3.1, Eq. 7; Algorithm 4's output).
 *
 * Nodes are vertex-centred: r_k(i) = lo_k + i * s_k, s_k = (hi_k - lo_k) /
 * (dims[k] - 1), so dims[k] >= 2 and hi_k > lo_k. d_out is device float
 * [dims[2]][dims[1]][dims[0]] (x fastest, index i_x + i_y*dims[0] +
 * i_z*dims[0]*dims[1], as in Algorithms 2 and 4).
 * rule KNN needs sf_bandwidths(KNN) first; FIXED uses params->fixed_h; MBE
 * runs the paper's pilot -> adaptive-length -> final pipeline for this ROI
 * (Algorithm 1) with scope CLIP. It finds B's particles through the index (the
 * leaves whose box meets B), so its per-call scratch and time follow the ROI;
 * its adaptive lengths live in two buffers the index allocates at its first
 * MBE call and keeps until sf_free_index (16 bytes per point and per node).
 * MBE calls on one index run one at a time (host lock; the device work of a
 * call is ordered after the previous call's, on any stream).
 * h_mass (nullable, host): FP64 total mass sum_n rho_n s_x s_y s_z; giving it
 * synchronises the stream.
 * Errors: INVALID_ARG, OOM, CUDA, DEGENERATE (MBE with N_B < 2 or P80 == P20),
 * EMPTY_ROI (scope CLIP and no point in B; d_out is zero-filled), CAPACITY (the
 * per-tile candidate lists would exceed 2^31 entries: fewer nodes or a smaller ROI;
 * not where SF_ACCEL_AUTO hands the grid to the moment form).
 * The call synchronises the stream once to size its work lists (before the
 * density kernels run); EMPTY_ROI is returned by the call itself.
 */
sf_status sf_kde_grid(sf_index *idx, const sf_box *roi, const int32_t dims[3], int32_t kernel,
                      const sf_params *params, float *d_out, double *h_mass, void *stream);

/*
 * sf_kde_points -- density at every point inside the ROI box (closed).
 *
 * Output in ascending original index: d_ids[i] (device uint32) is the
 * original index of the i-th ROI point and d_density[i] (device float) its
 * density. capacity = length of both buffers; *h_count (host, required)
 * receives the number of ROI points (the stream is synchronised). If the
 * count exceeds capacity, CAPACITY is returned and nothing is written.
 * The ROI's points are found through the index (the leaves whose bounding box
 * meets the box), so for the kNN and fixed rules the call's time and scratch
 * grow with the ROI's points, not with the cloud: about 24 bytes per ROI point
 * plus 9 bytes per point of the leaves that meet the box (sf_query_workspace
 * gives the exact figure). Rule MBE keeps its resident buffers as for sf_kde_grid.
 * Scope CLIP with no point in B returns EMPTY_ROI with *h_count = 0.
 * DIRECT sums the kernels at each point (the point's own kernel included);
 * INTERP interpolates the grid of the same dims trilinearly.
 * params->prec TF32 / 3XTF32 / BF16 (DIRECT with kNN bandwidths only): the
 * cross term -2 x.y of each squared distance, in coordinates centred on each
 * group of 32 query points, runs on the tensor cores; the relative error of
 * q = d^2/h^2 is about 2^-10 (TF32), 2^-21 (3xTF32) or 2^-8 (BF16) times
 * (|x| + |y|)^2 / d^2, so TF32 densities carry errors of order 1e-2, 3xTF32
 * ones of order 1e-5 and BF16 ones of order 1e-1; near the cutoff a pair may
 * fall on either side. dims is used by
 * INTERP and by rule MBE (whose smoothing lengths depend on the grid spacing);
 * it may be NULL otherwise.
 */
sf_status sf_kde_points(sf_index *idx, const sf_box *roi, const int32_t *dims, int32_t kernel,
                        const sf_params *params, float *d_density, uint32_t *d_ids,
                        int64_t capacity, int64_t *h_count, void *stream);

/*
 * sf_query_workspace -- the device memory a call would allocate, before it is
 * made (admission by memory in a serving loop).
 *
 * what = SF_WS_GRID: sf_kde_grid(idx, roi, dims, kernel, params, ..., h_mass)
 * with h_mass given; SF_WS_POINTS: sf_kde_points(idx, roi, dims, kernel,
 * params, ...). *h_bytes (host) receives the most stream-ordered scratch the
 * call holds at once (each allocation rounded up to 256 bytes; the device's
 * pool may round further). The grid figure is exact: it runs the call's
 * candidate count for this ROI (an index walk per node tile). The points
 * figure counts the ROI's leaves and bounds the ROI's points by 32 per leaf.
 * Synchronises the stream. Rules SF_BW_KNN and SF_BW_FIXED (the MBE rule's
 * workspace depends on its per-ROI lengths: INVALID_ARG). Errors: INVALID_ARG,
 * OOM, CUDA.
 */
enum { SF_WS_GRID = 1, SF_WS_POINTS = 2 };
sf_status sf_query_workspace(sf_index *idx, const sf_box *roi, const int32_t *dims, int32_t kernel,
                             const sf_params *params, int32_t what, int64_t *h_bytes, void *stream);

/* The most stream-ordered scratch (bytes, counted as sf_query_workspace counts
 * it) that the calling thread's most recent library call held at once. */
int64_t sf_last_call_workspace(void);

/*
 * sf_select -- density-threshold selection of points (Sec. 4.1).
 *
 * Inputs: n densities d_density (device float >= 0) of points with original
 * indices d_ids (device uint32, ascending, each < n_total).
 * Threshold t: if `threshold` is not NaN, t = (float)threshold; otherwise t is
 * the nearest-rank `percentile` (0..100) of the n densities: the value at
 * 1-based rank ceil(percentile/100 * n) (at least 1) in ascending order.
 * Selected: every i with density > t (strict).
 * Outputs: d_mask (device uint8 [n_total], nullable): 1 for selected original
 * indices, 0 elsewhere; d_sel_ids (device uint32 [n], nullable): the selected
 * original indices, ascending; *h_nsel (host, nullable) the count and
 * *h_threshold (host, nullable) the t used -- either synchronises the stream.
 * n = 0 selects nothing. Errors: INVALID_ARG, OOM, CUDA.
 */
sf_status sf_select(sf_index *idx, const float *d_density, const uint32_t *d_ids, int64_t n,
                    int64_t n_total, double threshold, double percentile, uint8_t *d_mask,
                    uint32_t *d_sel_ids, int64_t *h_nsel, double *h_threshold, void *stream);

/*
 * sf_iso_surface -- the boundary of the selection volume (Sec. 4.1: a density
 * threshold, an iso-surface of the density field computed on the GPU, the points
 * inside it), as a triangle soup in device memory.
 *
 * d_grid: device float [dims[2]][dims[1]][dims[0]] over the closed box roi (as
 * sf_kde_grid writes it). Every cell is split into the six tetrahedra around its
 * main diagonal (for each ordering a, b, c of the axes: corners 0, e_a,
 * e_a + e_b, (1,1,1), orderings (x,y,z), (x,z,y), (y,x,z), (y,z,x), (z,x,y),
 * (z,y,x)); the grid values are interpolated linearly on each, and the volume is
 * where that field exceeds `threshold`. Its boundary: one triangle for a
 * tetrahedron with one corner on the other side from the three others, two for
 * two and two; corners are "inside" when value > threshold (compared in FP64);
 * the crossing on an edge from corner a to b is P_a + (t - f_a)/(f_b - f_a)
 * (P_b - P_a) in FP64; every triangle is oriented with its normal pointing away
 * from the inside corners (toward lower density). Output d_tris: device float
 * [capacity][9] (three vertices x, y, z), in cell order (x fastest), then
 * tetrahedron order, then the case's triangles. *h_ntri (host, required) gets the
 * number of triangles; more than capacity gives CAPACITY and writes nothing
 * (d_tris may be NULL with capacity 0 to count). Synchronises the stream.
 * Errors: INVALID_ARG, OOM, CUDA, CAPACITY.
 */
sf_status sf_iso_surface(const float *d_grid, const sf_box *roi, const int32_t dims[3], double threshold,
                         float *d_tris, int64_t capacity, int64_t *h_ntri, void *stream);

/*
 * sf_resample_grid -- a finished grid read at the nodes of another grid by
 * trilinear interpolation (Sec. 3.1, last step: the density at any position
 * inside B from the eight nodes around it).
 *
 * d_src: device float [src_dims[2]][src_dims[1]][src_dims[0]] over the closed box
 * src_box (vertex-centred nodes, x fastest, as sf_kde_grid writes it). Every node
 * of the grid (dst_box, dst_dims) gets weight * the interpolated value, stored
 * into d_dst (device float, same layout) or, with accumulate != 0, added to
 * what d_dst holds (so w1 F1 + w2 F2 takes two calls). Node positions and the
 * weighted sum are computed in FP64, rounded once to float. Destination nodes
 * outside src_box get 0 (or nothing added); *h_outside (host, nullable) receives
 * their number and then the stream is synchronised. For view caches (a small pan
 * or zoom answered from a grid over a larger box) and for precomputed global
 * fields read at a view's nodes. Errors: INVALID_ARG, OOM, CUDA.
 */
sf_status sf_resample_grid(const float *d_src, const sf_box *src_box, const int32_t src_dims[3],
                           const sf_box *dst_box, const int32_t dst_dims[3], float weight,
                           int32_t accumulate, float *d_dst, int64_t *h_outside, void *stream);

/*
 * Batched ROI grids: many ROIs of uneven size in one persistent execution.
 *
 * Every (ROI, 8x4xZ node tile) lists its candidate leaves, the lists are cut
 * into work items of similar size, one persistent kernel (one warp per item at
 * a time) drains the items of all ROIs, and each tile adds its items' partial
 * sums in a fixed order: a
 * plan's results are bit-identical from run to run, and equal sf_kde_grid's up
 * to the final rounding to float (the items are cut differently). sf_batch_create sizes the buffers (it synchronises the stream)
 * and, unless tune->no_graph, captures the execution into a CUDA graph that
 * sf_batch_run replays; the index must not change while a batch exists.
 * Rules KNN and FIXED, both scopes (CLIP counts N_B per ROI at creation).
 * params->prec: FP32, or the grid variants TF32 / 3XTF32 / BF16 (Gaussian
 * kernel, tile_z 8; see SF_PREC_*).
 *
 * rois: nroi closed boxes; dims: nroi x 3 int32 (dims[3r..3r+2] for ROI r,
 * each in [2, 4096]). d_outs: nroi device pointers, grid r of
 * dims[3r+2]*dims[3r+1]*dims[3r] floats, x fastest (may change between runs).
 * h_masses (nullable, host double[nroi]): FP64 mass per ROI; synchronises.
 */
typedef struct sf_batch sf_batch;
typedef struct {
    int32_t tile_z;          /* node tile depth in z: 4 or 8 (0: 8)                 */
    int32_t items_per_slot;  /* work items per resident warp, 1..64 (0: 4)          */
    int32_t no_graph;        /* 1: launch the kernels directly instead of a graph   */
    int32_t reserved;        /* must be 0                                           */
} sf_tune;

sf_status sf_batch_create(sf_index *idx, int32_t nroi, const sf_box *rois, const int32_t *dims,
                          int32_t kernel, const sf_params *params, const sf_tune *tune,
                          void *stream, sf_batch **out);
sf_status sf_batch_run(sf_batch *batch, float *const *d_outs, double *h_masses, void *stream);
void sf_batch_free(sf_batch *batch);
/* One-shot: create (without a graph), run, free. */
sf_status sf_batch_kde_grid(sf_index *idx, int32_t nroi, const sf_box *rois, const int32_t *dims,
                            int32_t kernel, const sf_params *params, float *const *d_outs,
                            double *h_masses, void *stream);

/*
 * sf_kde_grid_static -- sf_kde_grid without any device memory allocation.
 *
 * The paper has no counterpart; this entry point exists for callers that
 * cannot allocate device memory while they run: a real-time render or VR frame
 * loop that reserved its device memory up front and cannot let an allocation
 * stall or synchronise the GPU in the middle of a frame, and processes whose
 * device memory is already owned by another allocator (a framework's caching
 * allocator or a pool sized at start-up), where a cudaMalloc from this
 * library would fail or fragment that memory. The caller still passes the
 * inputs (the index) and the output buffer d_out.
 *
 * It computes the same grid as sf_kde_grid, with the same kernels and node
 * coordinates, for rules SF_BW_KNN and SF_BW_FIXED (both scopes); rule
 * SF_BW_MBE needs scratch proportional to the cloud and gives INVALID_ARG.
 * It always sums pair by pair (params->accel may be AUTO or NONE; MOMENTS
 * gives INVALID_ARG), and reports CAPACITY-free sizes only as stated below.
 * All scratch lives in one fixed array of about 0.55 MB in device memory,
 * which every GPU that loads the library holds until the process exits; it
 * limits dims[k] to at most 1024 and the grid to at most 65536 tiles of
 * 16 x 16 x 8 nodes (512^3 nodes fit); larger sizes give INVALID_ARG with a
 * message. The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress) with that device current; make that first call
 * before any stream capture. Every call shares the one array and leaves its
 * contents behind for the next: calls that overlap on the GPU (different
 * streams, or different host threads, at the same time) race on it and must
 * be serialised by the caller. h_mass as for sf_kde_grid; the call
 * synchronises only when h_mass is given, and only then reports EMPTY_ROI
 * (without h_mass an empty clip-scope ROI yields the zero grid and SF_OK).
 */
sf_status sf_kde_grid_static(sf_index *idx, const sf_box *roi, const int32_t dims[3],
                             int32_t kernel, const sf_params *params, float *d_out,
                             double *h_mass, void *stream);

/*
 * sf_count_support_pairs -- the algorithmic work of one ROI recompute: the
 * number of (grid node, particle) pairs (h_grid_pairs, needs dims) and of
 * (ROI point, particle) pairs (h_point_pairs, DIRECT) whose kernel value is
 * non-zero (q < 1 for EPAN, q < 9 for GAUSS3), counted by the same kernels as
 * sf_kde_grid / sf_kde_points in a counting variant (slower; not for timing).
 * Either output may be NULL. Synchronises the stream.
 */
sf_status sf_count_support_pairs(sf_index *idx, const sf_box *roi, const int32_t dims[3],
                                 int32_t kernel, const sf_params *params, int64_t *h_grid_pairs,
                                 int64_t *h_point_pairs, void *stream);

/*
 * sf_grid_work_counts -- where the grid's work goes for one ROI (a diagnostic for
 * tuning and for the roofline's account of wasted evaluations), from the same
 * counting variant as sf_count_support_pairs. h_counts (host int64[5]):
 *   [0] in-support (node, particle) pairs (= h_grid_pairs),
 *   [1] candidate-leaf visits by node tiles,
 *   [2] (particle, tile) pairs staged: particles whose support reaches the tile,
 *   [3] of those, the pairs whose support covers every node of the tile (summed
 *       on the tensor cores),
 *   [4] (node, particle) pairs evaluated (every staged particle against every
 *       node of its tile).
 * Synchronises the stream. Rules kNN and fixed.
 */
sf_status sf_grid_work_counts(sf_index *idx, const sf_box *roi, const int32_t dims[3], int32_t kernel,
                              const sf_params *params, int64_t h_counts[5], void *stream);

/*
 * Kernel timing: when enabled, the main kernels (k_grid, k_points, k_knn,
 * k_radix_sort, and the counting variants) are bracketed by CUDA events on the
 * stream they are launched on. sf_kernel_timing sums the elapsed times and
 * counts the launches recorded under `name` since the last reset (it waits for
 * the recorded events). Off by default; enabling adds event records only.
 */
void sf_kernel_timing_enable(int enable);
void sf_kernel_timing_reset(void);
sf_status sf_kernel_timing(const char *name, double *h_ms_total, int64_t *h_launches);
/* The individual durations (ms, launch order) of up to `cap` launches recorded
 * under `name`; *h_count receives the number recorded (may exceed cap). */
sf_status sf_kernel_timing_list(const char *name, double *h_ms, int64_t cap, int64_t *h_count);

/* Synchronise `stream` and return (then clear) any status a kernel recorded
 * on the device for this index. Every call returns the statuses of its own
 * kernels itself (each call has its own status word), so this reports only
 * CUDA errors of work still queued on the stream. */
sf_status sf_sync_status(sf_index *idx, void *stream);

/* Release the index and all of its device memory, and hand the default pool's
 * unused memory back to the system. Safe on NULL. */
void sf_free_index(sf_index *idx);

/* Message describing the last error of the calling thread ("" if none). */
const char *sf_last_error(void);

/* Number of kernels the library has launched in this process so far. */
uint64_t sf_launch_count(void);

#ifdef __cplusplus
}
#endif

#endif /* SCALEFREE_H */
