// sf_api.cu -- the extern "C" entry points of libscalefree.so (include/scalefree.h).
// Argument checking, per-call device parameters and the order of launches; all
// arithmetic on the data runs in the kernels of the other translation units.
#include <cmath>
#include <cstring>

#include "sf_internal.cuh"

namespace sf {

const char *last_error_cstr();
void clear_error();
sf_status knn_neighbours(sf_index *idx, int k, uint32_t *d_nbr_orig, float *d_h_orig, cudaStream_t s);
sf_status knn_work_counts(sf_index *idx, int k, int64_t *h_counts, cudaStream_t s);
sf_status scatter_bandwidths(const sf_index *idx, float *d_h_orig, cudaStream_t s);
sf_status select_points(const float *d_density, const uint32_t *d_ids, int64_t n, int64_t n_total,
                        double threshold, double percentile, uint8_t *d_mask, uint32_t *d_sel_ids,
                        int64_t *h_nsel, double *h_threshold, cudaStream_t s);
sf_status roi_compact(sf_index *idx, const int *d_leaves, int64_t nslots, const uint8_t *d_inroi,
                      const float *d_rho, float *d_density, uint32_t *d_ids, int64_t capacity,
                      int64_t *h_count, cudaStream_t s);
sf_status grid_workspace(sf_index *idx, const sf_box &roi, const GridSpec &g,
                         const DensityCall &call, int64_t *bytes, cudaStream_t s);
sf_status points_workspace(sf_index *idx, const sf_box &roi, const GridSpec *g,
                           const DensityCall &call, int64_t base_bytes, int64_t *bytes,
                           cudaStream_t s);
int64_t last_call_scratch_peak();
sf_status mbe_prepare(sf_index *idx, const sf_box &roi, const GridSpec &g, int kernel,
                      const sf_params &p, DensityParams *d_dp, float4 *d_ell, float4 *d_nell,
                      float *d_pilot, cudaStream_t s);
sf_status interp_points(sf_index *idx, const sf_box &roi, const GridSpec &g, const float *d_grid,
                        const int *d_leaves, int64_t nslots, float *d_rho_sorted, uint8_t *d_inroi,
                        cudaStream_t s, int tet);

// Count the points of the scope and set N_eff (device); EMPTY_ROI is recorded
// in the status word when the clip scope holds no point.
__global__ void k_count_box(const float4 *__restrict__ pos, int64_t n, float3 lo, float3 hi,
                            unsigned long long *cnt) {
    unsigned long long c = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const float4 p = pos[i];
        c += (p.x >= lo.x && p.x <= hi.x && p.y >= lo.y && p.y <= hi.y && p.z >= lo.z && p.z <= hi.z);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    if ((threadIdx.x & 31) == 0 && c) atomicAdd(cnt, c);
}

__global__ void k_set_params(DensityParams *dp, const unsigned long long *cnt, int64_t n_all,
                             float ex, float ey, float ez, int *status) {
    const int64_t neff = cnt ? (int64_t)*cnt : n_all;
    dp->ell_uniform[0] = ex;
    dp->ell_uniform[1] = ey;
    dp->ell_uniform[2] = ez;
    dp->pad0 = 0.f;
    dp->neff = neff;
    dp->inv_neff = neff > 0 ? 1.0 / (double)neff : 0.0;
    if (neff == 0 && status) *status = ST_EMPTY;
}

sf_status set_density_params(sf_index *idx, bool clip, const sf_box &roi, const float ell[3],
                             DensityParams *d_dp, int *d_status, cudaStream_t s) {
    unsigned long long *cnt = nullptr;
    Scratch sc(s);
    if (clip) {
        cnt = sc.get<unsigned long long>(1);
        SF_TRY_SCRATCH(sc);
        float3 lo, hi;
        float flo[3], fhi[3];
        for (int k = 0; k < 3; ++k) {
            float a = (float)roi.lo[k];
            if ((double)a < roi.lo[k]) a = nextafterf(a, INFINITY);
            float b = (float)roi.hi[k];
            if ((double)b > roi.hi[k]) b = nextafterf(b, -INFINITY);
            flo[k] = a;
            fhi[k] = b;
        }
        lo = make_float3(flo[0], flo[1], flo[2]);
        hi = make_float3(fhi[0], fhi[1], fhi[2]);
        SF_TRY_CUDA(cudaMemsetAsync(cnt, 0, sizeof *cnt, s));
        const unsigned g = std::max(1u, std::min<unsigned>(blocks_for(idx->n, 256), 152 * 8));
        SF_TRY_CUDA(launch(k_count_box, dim3(g), dim3(256), 0, s, (const float4 *)idx->pos, idx->n,
                           lo, hi, cnt));
    }
    SF_TRY_CUDA(launch(k_set_params, dim3(1), dim3(1), 0, s, d_dp,
                       (const unsigned long long *)cnt, idx->n, ell[0], ell[1], ell[2], d_status));
    return SF_OK;
}

static sf_status check_roi(const sf_box *roi, const char *fn) {
    if (!roi) return fail(SF_ERR_INVALID_ARG, "%s: roi is NULL", fn);
    for (int k = 0; k < 3; ++k)
        if (!std::isfinite(roi->lo[k]) || !std::isfinite(roi->hi[k]) || !(roi->hi[k] > roi->lo[k]))
            return fail(SF_ERR_INVALID_ARG, "%s: roi axis %d must satisfy lo < hi (finite)", fn, k);
    return SF_OK;
}

static sf_status check_params(const sf_index *idx, const sf_params *p, int kernel, const char *fn) {
    if (!p) return fail(SF_ERR_INVALID_ARG, "%s: params is NULL", fn);
    if (kernel != SF_K_EPAN && kernel != SF_K_GAUSS3)
        return fail(SF_ERR_INVALID_ARG, "%s: unknown kernel %d", fn, kernel);
    if (p->scope != SF_SCOPE_CLIP && p->scope != SF_SCOPE_GLOBAL)
        return fail(SF_ERR_INVALID_ARG, "%s: unknown scope %d", fn, p->scope);
    if (p->prec != SF_PREC_FP32 && p->prec != SF_PREC_TF32 && p->prec != SF_PREC_3XTF32 &&
        p->prec != SF_PREC_BF16)
        return fail(SF_ERR_INVALID_ARG, "%s: unsupported precision %d", fn, p->prec);
    if (p->points_mode != SF_POINTS_DIRECT && p->points_mode != SF_POINTS_INTERP &&
        p->points_mode != SF_POINTS_TETLIN)
        return fail(SF_ERR_INVALID_ARG, "%s: unknown points_mode %d", fn, p->points_mode);
    if (p->accel != SF_ACCEL_AUTO && p->accel != SF_ACCEL_NONE && p->accel != SF_ACCEL_MOMENTS)
        return fail(SF_ERR_INVALID_ARG, "%s: bad accel %d", fn, p->accel);
    switch (p->rule) {
        case SF_BW_KNN:
            if (idx->bw_rule != SF_BW_KNN || idx->knn_k != p->k)
                return fail(SF_ERR_INVALID_ARG, "%s: kNN bandwidths for k=%d are not built", fn, p->k);
            break;
        case SF_BW_FIXED:
            for (int k = 0; k < 3; ++k)
                if (!(p->fixed_h[k] > 0.0) || !std::isfinite(p->fixed_h[k]))
                    return fail(SF_ERR_INVALID_ARG, "%s: fixed_h must be positive", fn);
            break;
        case SF_BW_MBE:
            if (!(p->cap_factor > 0.0) || !(p->p_lo >= 0.0) || !(p->p_hi <= 100.0) || !(p->p_lo < p->p_hi))
                return fail(SF_ERR_INVALID_ARG, "%s: bad MBE parameters", fn);
            break;
        default:
            return fail(SF_ERR_INVALID_ARG, "%s: unknown rule %d", fn, p->rule);
    }
    return SF_OK;
}

static sf_status make_grid(const sf_box &roi, const int32_t *dims, GridSpec &g, const char *fn) {
    if (!dims) return fail(SF_ERR_INVALID_ARG, "%s: dims is NULL", fn);
    for (int k = 0; k < 3; ++k)
        if (dims[k] < 2 || dims[k] > 4096)
            return fail(SF_ERR_INVALID_ARG, "%s: dims[%d]=%d outside [2, 4096]", fn, k, dims[k]);
    g.nx = dims[0];
    g.ny = dims[1];
    g.nz = dims[2];
    for (int k = 0; k < 3; ++k) {
        g.lo[k] = roi.lo[k];
        g.hi[k] = roi.hi[k];
        g.s[k] = (roi.hi[k] - roi.lo[k]) / (double)(dims[k] - 1);
    }
    return SF_OK;
}

// Bandwidths and density parameters for one call; MBE runs its per-ROI pipeline.
struct Prepared {
    DensityCall call;
    DensityParams *dp = nullptr;
    int *status = nullptr;  // this call's device status word (ST_EMPTY in clip scope)
    float4 *ell = nullptr;
    float4 *nell = nullptr;
    // rule MBE: the index's resident length buffers are this call's until it
    // returns; the device work queued by then is marked for the next call
    std::unique_lock<std::mutex> mbe_lock;
    sf_index *idx = nullptr;
    cudaStream_t stream = nullptr;
    ~Prepared() {
        if (mbe_lock.owns_lock() && idx->mbe_done) cudaEventRecord(idx->mbe_done, stream);
    }
};

// The estimator's resident buffers (16 bytes per point and per node), made at
// its first call on the index; later calls order their device work after the
// previous call's, whatever stream either ran on.
static sf_status mbe_buffers(sf_index *idx, cudaStream_t s) {
    if (!idx->mbe_ell) {
        cudaError_t e;
        if ((e = cudaMalloc(&idx->mbe_ell, sizeof(float4) * idx->n)) != cudaSuccess ||
            (e = cudaMalloc(&idx->mbe_nell, sizeof(float4) * idx->nnodes)) != cudaSuccess ||
            (e = cudaEventCreateWithFlags(&idx->mbe_done, cudaEventDisableTiming)) != cudaSuccess) {
            cudaFree(idx->mbe_ell);
            cudaFree(idx->mbe_nell);
            idx->mbe_ell = idx->mbe_nell = nullptr;
            idx->mbe_done = nullptr;
            return fail(SF_ERR_OOM, "rule MBE: resident length buffers: %s", cudaGetErrorString(e));
        }
        return SF_OK;
    }
    SF_TRY_CUDA(cudaStreamWaitEvent(s, idx->mbe_done, 0));
    return SF_OK;
}

static sf_status prepare(sf_index *idx, const sf_box &roi, const GridSpec *g, int kernel,
                         const sf_params &p, Scratch &sc, Prepared &out, cudaStream_t s) {
    out.dp = sc.get<DensityParams>(1);
    out.status = sc.get<int>(1);
    SF_TRY_SCRATCH(sc);
    SF_TRY_CUDA(cudaMemsetAsync(out.status, 0, sizeof(int), s));
    out.call.kernel = kernel;
    out.call.accel = p.accel;
    out.call.dp = out.dp;
    out.call.ell = nullptr;
    out.call.nell_override = nullptr;
    if (p.rule == SF_BW_MBE) {
        if (!g) return fail(SF_ERR_INVALID_ARG, "rule MBE needs the grid dims");
        KTimer t("mbe_prepare", s);
        out.mbe_lock = std::unique_lock<std::mutex>(idx->mbe_mu);
        out.idx = idx;
        out.stream = s;
        SF_TRY(mbe_buffers(idx, s));
        out.ell = idx->mbe_ell;
        out.nell = idx->mbe_nell;
        SF_TRY(mbe_prepare(idx, roi, *g, kernel, p, out.dp, out.ell, out.nell, nullptr, s));
        out.call.bw = BW_ANISO;
        out.call.clip = 1;
        out.call.ell = out.ell;
        out.call.nell_override = out.nell;
        return SF_OK;
    }
    const bool clip = p.scope == SF_SCOPE_CLIP;
    out.call.clip = clip ? 1 : 0;
    float ell[3] = {0.f, 0.f, 0.f};
    if (p.rule == SF_BW_FIXED) {
        out.call.bw = BW_UNIFORM;
        for (int k = 0; k < 3; ++k) ell[k] = (float)p.fixed_h[k];
    } else {
        out.call.bw = BW_ISO;
    }
    SF_TRY(set_density_params(idx, clip, roi, ell, out.dp, out.status, s));
    return SF_OK;
}

// The status a call's kernels recorded, as the call's return value.
static sf_status call_status(int st) {
    if (st == ST_EMPTY) return fail(SF_ERR_EMPTY_ROI, "no particle of the scope lies in the ROI");
    if (st != ST_OK) return fail((sf_status)st, "device reported status %d", st);
    return SF_OK;
}

}  // namespace sf

using namespace sf;

extern "C" {

void sf_params_default(sf_params *p) {
    if (!p) return;
    memset(p, 0, sizeof *p);
    p->rule = SF_BW_KNN;
    p->k = 32;
    p->fixed_h[0] = p->fixed_h[1] = p->fixed_h[2] = 0.0;
    p->cap_factor = 5.0;
    p->p_lo = 20.0;
    p->p_hi = 80.0;
    p->log_base = 0.0;
    p->scope = SF_SCOPE_GLOBAL;
    p->prec = SF_PREC_FP32;
    p->points_mode = SF_POINTS_DIRECT;
}

int64_t sf_index_size(const sf_index *idx) { return idx ? idx->n : 0; }

sf_status sf_bandwidths(sf_index *idx, const sf_params *p, void *stream) {
    clear_error();
    if (!idx || !p) return fail(SF_ERR_INVALID_ARG, "sf_bandwidths: NULL argument");
    cudaStream_t s = (cudaStream_t)stream;
    std::lock_guard<std::mutex> lk(idx->mu);
    switch (p->rule) {
        case SF_BW_KNN: {
            if (p->k < 1 || p->k > 256) return fail(SF_ERR_INVALID_ARG, "sf_bandwidths: k=%d outside [1, 256]", p->k);
            if (idx->n <= p->k)
                return fail(SF_ERR_DEGENERATE, "sf_bandwidths: n=%lld <= k=%d", (long long)idx->n, p->k);
            idx->bw_rule = -1;
            SF_TRY(knn_bandwidths(idx, p->k, nullptr, nullptr, s));
            idx->bw_rule = SF_BW_KNN;
            idx->knn_k = p->k;
            return SF_OK;
        }
        case SF_BW_FIXED:
            for (int k = 0; k < 3; ++k) {
                if (!(p->fixed_h[k] > 0.0)) return fail(SF_ERR_INVALID_ARG, "sf_bandwidths: fixed_h must be > 0");
                idx->fixed_h[k] = (float)p->fixed_h[k];
            }
            return SF_OK;
        case SF_BW_MBE:
            return SF_OK;
        default:
            return fail(SF_ERR_INVALID_ARG, "sf_bandwidths: unknown rule %d", p->rule);
    }
}

sf_status sf_get_bandwidths(const sf_index *idx, float *d_h, void *stream) {
    clear_error();
    if (!idx || !d_h) return fail(SF_ERR_INVALID_ARG, "sf_get_bandwidths: NULL argument");
    if (idx->bw_rule != SF_BW_KNN) return fail(SF_ERR_INVALID_ARG, "sf_get_bandwidths: no kNN bandwidths built");
    return scatter_bandwidths(idx, d_h, (cudaStream_t)stream);
}

sf_status sf_knn_work_counts(sf_index *idx, int32_t k, int64_t *h_counts, void *stream) {
    clear_error();
    if (!idx || !h_counts) return fail(SF_ERR_INVALID_ARG, "sf_knn_work_counts: NULL argument");
    if (k < 1 || k > 256) return fail(SF_ERR_INVALID_ARG, "sf_knn_work_counts: k=%d outside [1, 256]", k);
    if (idx->n <= k) return fail(SF_ERR_DEGENERATE, "sf_knn_work_counts: n <= k");
    return knn_work_counts(idx, k, h_counts, (cudaStream_t)stream);
}

sf_status sf_knn_neighbours(sf_index *idx, int32_t k, uint32_t *d_nbr, float *d_h, void *stream) {
    clear_error();
    if (!idx || !d_nbr) return fail(SF_ERR_INVALID_ARG, "sf_knn_neighbours: NULL argument");
    if (k < 1 || k > 256) return fail(SF_ERR_INVALID_ARG, "sf_knn_neighbours: k=%d outside [1, 256]", k);
    if (idx->n <= k) return fail(SF_ERR_DEGENERATE, "sf_knn_neighbours: n <= k");
    return knn_neighbours(idx, k, d_nbr, d_h, (cudaStream_t)stream);
}

sf_status sf_kde_grid(sf_index *idx, const sf_box *roi, const int32_t dims[3], int32_t kernel,
                      const sf_params *params, float *d_out, double *h_mass, void *stream) {
    clear_error();
    if (!idx || !d_out) return fail(SF_ERR_INVALID_ARG, "sf_kde_grid: NULL argument");
    SF_TRY(check_roi(roi, "sf_kde_grid"));
    SF_TRY(check_params(idx, params, kernel, "sf_kde_grid"));
    if (params->prec != SF_PREC_FP32 && (kernel != SF_K_GAUSS3 || params->rule == SF_BW_MBE))
        return fail(SF_ERR_INVALID_ARG,
                    "sf_kde_grid: TF32 / 3xTF32 / BF16 grids need the Gaussian kernel and rule KNN or FIXED");
    GridSpec g;
    SF_TRY(make_grid(*roi, dims, g, "sf_kde_grid"));
    cudaStream_t s = (cudaStream_t)stream;
    Scratch sc(s);
    double *d_mass = h_mass ? sc.get<double>(1) : nullptr;
    SF_TRY_SCRATCH(sc);
    Prepared pr;
    SF_TRY(prepare(idx, *roi, &g, kernel, *params, sc, pr, s));
    pr.call.prec = params->prec;
    StatusPeek peek;
    peek.d_src = pr.status;
    SF_TRY(density_grid(idx, *roi, g, pr.call, d_out, d_mass, s, nullptr, &peek));
    if (h_mass) {
        SF_TRY_CUDA(cudaMemcpyAsync(h_mass, d_mass, sizeof(double), cudaMemcpyDeviceToHost, s));
        SF_TRY_CUDA(cudaStreamSynchronize(s));
    }
    return call_status(peek.value);
}

sf_status sf_kde_points(sf_index *idx, const sf_box *roi, const int32_t *dims, int32_t kernel,
                        const sf_params *params, float *d_density, uint32_t *d_ids,
                        int64_t capacity, int64_t *h_count, void *stream) {
    clear_error();
    if (!idx || !d_density || !d_ids || !h_count)
        return fail(SF_ERR_INVALID_ARG, "sf_kde_points: NULL argument");
    if (capacity < 0) return fail(SF_ERR_INVALID_ARG, "sf_kde_points: negative capacity");
    SF_TRY(check_roi(roi, "sf_kde_points"));
    SF_TRY(check_params(idx, params, kernel, "sf_kde_points"));
    if (params->prec != SF_PREC_FP32 &&
        (params->rule != SF_BW_KNN || params->points_mode != SF_POINTS_DIRECT))
        return fail(SF_ERR_INVALID_ARG, "sf_kde_points: TF32 / 3xTF32 / BF16 need rule KNN and DIRECT");
    GridSpec g;
    const bool interp = params->points_mode != SF_POINTS_DIRECT;
    const bool need_grid = params->rule == SF_BW_MBE || interp;
    if (need_grid) SF_TRY(make_grid(*roi, dims, g, "sf_kde_points"));
    cudaStream_t s = (cudaStream_t)stream;
    *h_count = 0;
    Scratch sc(s);
    Prepared pr;
    SF_TRY(prepare(idx, *roi, need_grid ? &g : nullptr, kernel, *params, sc, pr, s));
    // the leaves that can hold an ROI point (one synchronisation)
    StatusPeek peek;
    peek.d_src = pr.status;
    int *leaves = nullptr;
    int64_t nleaf = 0;
    SF_TRY(roi_leaf_list(idx, *roi, sc, &leaves, &nleaf, &peek, s));
    if (peek.value != ST_OK || nleaf == 0) return call_status(peek.value);
    float *rho = sc.get<float>(nleaf * kLeaf);
    uint8_t *inroi = sc.get<uint8_t>(nleaf * kLeaf);
    SF_TRY_SCRATCH(sc);
    if (params->prec != SF_PREC_FP32) {
        SF_TRY(density_points_tc(idx, *roi, pr.call, params->prec, leaves, nleaf, rho, inroi, s));
    } else if (interp) {
        Scratch gs(s);
        float *grid = gs.get<float>((int64_t)g.nx * g.ny * g.nz);
        SF_TRY_SCRATCH(gs);
        SF_TRY(density_grid(idx, *roi, g, pr.call, grid, nullptr, s));
        SF_TRY(interp_points(idx, *roi, g, grid, leaves, nleaf, rho, inroi, s,
                             params->points_mode == SF_POINTS_TETLIN));
    } else {
        SF_TRY(density_points(idx, *roi, pr.call, leaves, nleaf, rho, inroi, s));
    }
    SF_TRY(roi_compact(idx, leaves, nleaf, inroi, rho, d_density, d_ids, capacity, h_count, s));
    return SF_OK;
}

sf_status sf_query_workspace(sf_index *idx, const sf_box *roi, const int32_t *dims, int32_t kernel,
                             const sf_params *params, int32_t what, int64_t *h_bytes, void *stream) {
    clear_error();
    if (!idx || !h_bytes) return fail(SF_ERR_INVALID_ARG, "sf_query_workspace: NULL argument");
    *h_bytes = 0;
    if (what != SF_WS_GRID && what != SF_WS_POINTS)
        return fail(SF_ERR_INVALID_ARG, "sf_query_workspace: what=%d is not SF_WS_GRID or SF_WS_POINTS", what);
    SF_TRY(check_roi(roi, "sf_query_workspace"));
    SF_TRY(check_params(idx, params, kernel, "sf_query_workspace"));
    if (params->rule == SF_BW_MBE)
        return fail(SF_ERR_INVALID_ARG,
                    "sf_query_workspace: rule MBE's workspace depends on its adaptive lengths (kNN and fixed rules only)");
    GridSpec g;
    const bool need_grid = what == SF_WS_GRID || params->points_mode != SF_POINTS_DIRECT;
    if (need_grid) SF_TRY(make_grid(*roi, dims, g, "sf_query_workspace"));
    cudaStream_t s = (cudaStream_t)stream;
    Scratch sc(s);
    Prepared pr;
    SF_TRY(prepare(idx, *roi, need_grid ? &g : nullptr, kernel, *params, sc, pr, s));
    // what the entry point itself holds: its parameters and status word
    const int64_t base = scratch_round(sizeof(DensityParams)) + scratch_round(sizeof(int));
    int64_t b = 0;
    if (what == SF_WS_GRID) {
        SF_TRY(grid_workspace(idx, *roi, g, pr.call, &b, s));
        b += base + scratch_round(sizeof(double));  // the mass word (h_mass given)
    } else {
        const bool interp = params->points_mode != SF_POINTS_DIRECT && params->prec == SF_PREC_FP32;
        SF_TRY(points_workspace(idx, *roi, interp ? &g : nullptr, pr.call, base, &b, s));
    }
    *h_bytes = b;
    return SF_OK;
}

int64_t sf_last_call_workspace(void) { return last_call_scratch_peak(); }

sf_status sf_select(sf_index *idx, const float *d_density, const uint32_t *d_ids, int64_t n,
                    int64_t n_total, double threshold, double percentile, uint8_t *d_mask,
                    uint32_t *d_sel_ids, int64_t *h_nsel, double *h_threshold, void *stream) {
    clear_error();
    (void)idx;
    if (n < 0 || n_total < 0 || n > n_total || n_total >= (int64_t(1) << 32))
        return fail(SF_ERR_INVALID_ARG, "sf_select: bad sizes n=%lld n_total=%lld", (long long)n,
                    (long long)n_total);
    if (n > 0 && (!d_density || !d_ids)) return fail(SF_ERR_INVALID_ARG, "sf_select: NULL inputs");
    if (std::isnan(threshold) && !(percentile >= 0.0 && percentile <= 100.0))
        return fail(SF_ERR_INVALID_ARG, "sf_select: percentile must be in [0, 100]");
    return select_points(d_density, d_ids, n, n_total, threshold, percentile, d_mask, d_sel_ids,
                         h_nsel, h_threshold, (cudaStream_t)stream);
}

static sf_status count_pairs_impl(sf_index *idx, const sf_box *roi, const int32_t dims[3],
                                  int32_t kernel, const sf_params *params, int64_t *h_grid_pairs,
                                  int64_t *h_point_pairs, int64_t *h_work, void *stream) {
    if (!idx || (!h_grid_pairs && !h_point_pairs))
        return fail(SF_ERR_INVALID_ARG, "sf_count_support_pairs: NULL argument");
    SF_TRY(check_roi(roi, "sf_count_support_pairs"));
    SF_TRY(check_params(idx, params, kernel, "sf_count_support_pairs"));
    GridSpec g;
    const bool need_grid = h_grid_pairs || params->rule == SF_BW_MBE;
    if (need_grid) SF_TRY(make_grid(*roi, dims, g, "sf_count_support_pairs"));
    cudaStream_t s = (cudaStream_t)stream;
    Scratch sc(s);
    // [0..4]: grid pairs and the grid's work accounting (sf_grid_work_counts); [5]: points
    unsigned long long *cnt = sc.get<unsigned long long>(6);
    SF_TRY_SCRATCH(sc);
    SF_TRY_CUDA(cudaMemsetAsync(cnt, 0, 6 * sizeof(unsigned long long), s));
    Prepared pr;
    SF_TRY(prepare(idx, *roi, need_grid ? &g : nullptr, kernel, *params, sc, pr, s));
    if (h_grid_pairs) {
        float *grid = sc.get<float>((int64_t)g.nx * g.ny * g.nz);
        SF_TRY_SCRATCH(sc);
        SF_TRY(density_grid(idx, *roi, g, pr.call, grid, nullptr, s, cnt));
    }
    if (h_point_pairs) {
        int *leaves = nullptr;
        int64_t nleaf = 0;
        SF_TRY(roi_leaf_list(idx, *roi, sc, &leaves, &nleaf, nullptr, s));
        float *rho = sc.get<float>(nleaf * kLeaf);
        uint8_t *inroi = sc.get<uint8_t>(nleaf * kLeaf);
        SF_TRY_SCRATCH(sc);
        if (nleaf > 0)
            SF_TRY(density_points(idx, *roi, pr.call, leaves, nleaf, rho, inroi, s, cnt + 5));
    }
    unsigned long long h[6] = {0, 0, 0, 0, 0, 0};
    int h_st = 0;
    SF_TRY_CUDA(cudaMemcpyAsync(h, cnt, sizeof h, cudaMemcpyDeviceToHost, s));
    SF_TRY_CUDA(cudaMemcpyAsync(&h_st, pr.status, sizeof h_st, cudaMemcpyDeviceToHost, s));
    SF_TRY_CUDA(cudaStreamSynchronize(s));
    if (h_grid_pairs) *h_grid_pairs = (int64_t)h[0];
    if (h_point_pairs) *h_point_pairs = (int64_t)h[5];
    if (h_work)
        for (int k = 0; k < 5; ++k) h_work[k] = (int64_t)h[k];
    return call_status(h_st);
}

sf_status sf_count_support_pairs(sf_index *idx, const sf_box *roi, const int32_t dims[3],
                                 int32_t kernel, const sf_params *params, int64_t *h_grid_pairs,
                                 int64_t *h_point_pairs, void *stream) {
    clear_error();
    return count_pairs_impl(idx, roi, dims, kernel, params, h_grid_pairs, h_point_pairs, nullptr,
                            stream);
}

sf_status sf_grid_work_counts(sf_index *idx, const sf_box *roi, const int32_t dims[3], int32_t kernel,
                              const sf_params *params, int64_t h_counts[5], void *stream) {
    clear_error();
    if (!h_counts) return fail(SF_ERR_INVALID_ARG, "sf_grid_work_counts: NULL argument");
    int64_t pairs = 0;
    return count_pairs_impl(idx, roi, dims, kernel, params, &pairs, nullptr, h_counts, stream);
}

struct sf_batch {
    sf::BatchPlan *plan = nullptr;
    int nroi = 0;
};

sf_status sf_batch_create(sf_index *idx, int32_t nroi, const sf_box *rois, const int32_t *dims,
                          int32_t kernel, const sf_params *params, const sf_tune *tune,
                          void *stream, sf_batch **out) {
    clear_error();
    if (!out) return fail(SF_ERR_INVALID_ARG, "sf_batch_create: out is NULL");
    *out = nullptr;
    if (!idx || !rois || !dims || nroi < 1 || nroi > 65536)
        return fail(SF_ERR_INVALID_ARG, "sf_batch_create: bad arguments (nroi=%d)", nroi);
    SF_TRY(check_params(idx, params, kernel, "sf_batch_create"));
    if (params->rule == SF_BW_MBE)
        return fail(SF_ERR_INVALID_ARG, "sf_batch_create: rule MBE is per ROI; use sf_kde_grid");
    if (params->prec != SF_PREC_FP32 && kernel != SF_K_GAUSS3)
        return fail(SF_ERR_INVALID_ARG,
                    "sf_batch_create: TF32 / 3xTF32 / BF16 grids need the Gaussian kernel");
    int tz = 8, ips = 4;
    bool graph = true;
    if (tune) {
        if (tune->tile_z != 0 && tune->tile_z != 4 && tune->tile_z != 8)
            return fail(SF_ERR_INVALID_ARG, "sf_batch_create: tile_z must be 4 or 8");
        if (tune->tile_z) tz = tune->tile_z;
        if (tz != 8 && params->prec != SF_PREC_FP32)
            return fail(SF_ERR_INVALID_ARG, "sf_batch_create: the tensor-core variants need tile_z 8");
        if (tune->items_per_slot < 0 || tune->items_per_slot > 64)
            return fail(SF_ERR_INVALID_ARG, "sf_batch_create: items_per_slot outside [0, 64]");
        if (tune->items_per_slot) ips = tune->items_per_slot;
        graph = tune->no_graph == 0;
    }
    std::vector<GridSpec> grids(nroi);
    for (int r = 0; r < nroi; ++r) {
        SF_TRY(check_roi(&rois[r], "sf_batch_create"));
        SF_TRY(make_grid(rois[r], dims + 3 * r, grids[r], "sf_batch_create"));
    }
    cudaStream_t s = (cudaStream_t)stream;
    Scratch sc(s);
    int *d_st = sc.get<int>(1);
    SF_TRY_SCRATCH(sc);
    SF_TRY_CUDA(cudaMemsetAsync(d_st, 0, sizeof(int), s));
    DensityParams *dps = nullptr;
    SF_TRY_CUDA(cudaMalloc(&dps, sizeof(DensityParams) * nroi));
    const bool clip = params->scope == SF_SCOPE_CLIP;
    float ell[3] = {0.f, 0.f, 0.f};
    const int bw = params->rule == SF_BW_FIXED ? BW_UNIFORM : BW_ISO;
    if (bw == BW_UNIFORM)
        for (int k = 0; k < 3; ++k) ell[k] = (float)params->fixed_h[k];
    for (int r = 0; r < nroi; ++r) {
        sf_status st = set_density_params(idx, clip, rois[r], ell, dps + r, d_st, s);
        if (st != SF_OK) {
            cudaFree(dps);
            return st;
        }
    }
    sf::BatchPlan *plan = nullptr;
    SF_TRY(batch_create(idx, nroi, rois, grids.data(), kernel, bw, clip, dps, tz, ips, graph, s, &plan,
                        params->prec));
    sf_batch *b = new sf_batch();
    b->plan = plan;
    b->nroi = nroi;
    *out = b;
    int h_st = 0;
    SF_TRY_CUDA(cudaMemcpyAsync(&h_st, d_st, sizeof h_st, cudaMemcpyDeviceToHost, s));
    SF_TRY_CUDA(cudaStreamSynchronize(s));
    return call_status(h_st);  // EMPTY_ROI: some clip-scope ROI holds no particle (the plan is kept)
}

sf_status sf_batch_run(sf_batch *b, float *const *d_outs, double *h_masses, void *stream) {
    clear_error();
    if (!b || !d_outs) return fail(SF_ERR_INVALID_ARG, "sf_batch_run: NULL argument");
    for (int r = 0; r < b->nroi; ++r)
        if (!d_outs[r]) return fail(SF_ERR_INVALID_ARG, "sf_batch_run: output %d is NULL", r);
    return batch_run(b->plan, d_outs, h_masses, (cudaStream_t)stream);
}

void sf_batch_free(sf_batch *b) {
    if (!b) return;
    batch_free(b->plan);
    delete b;
}

sf_status sf_batch_kde_grid(sf_index *idx, int32_t nroi, const sf_box *rois, const int32_t *dims,
                            int32_t kernel, const sf_params *params, float *const *d_outs,
                            double *h_masses, void *stream) {
    sf_tune t;
    memset(&t, 0, sizeof t);
    t.no_graph = 1;  // a one-shot batch gains nothing from a graph
    sf_batch *b = nullptr;
    const sf_status cs = sf_batch_create(idx, nroi, rois, dims, kernel, params, &t, stream, &b);
    if (cs != SF_OK && cs != SF_ERR_EMPTY_ROI) return cs;
    // an empty clip-scope ROI still gets its (zero) grid
    sf_status st = sf_batch_run(b, d_outs, h_masses, stream);
    sf_batch_free(b);
    if (st != SF_OK) return st;
    return cs == SF_OK ? SF_OK : fail(cs, "sf_batch_kde_grid: a clip-scope ROI holds no particle");
}

sf_status sf_sync_status(sf_index *idx, void *stream) {
    if (!idx) return fail(SF_ERR_INVALID_ARG, "sf_sync_status: NULL index");
    cudaStream_t s = (cudaStream_t)stream;
    int st = 0;
    SF_TRY_CUDA(cudaMemcpyAsync(&st, idx->d_status, sizeof st, cudaMemcpyDeviceToHost, s));
    SF_TRY_CUDA(cudaStreamSynchronize(s));
    if (st != 0) {
        SF_TRY_CUDA(cudaMemsetAsync(idx->d_status, 0, sizeof(int), s));
        SF_TRY_CUDA(cudaStreamSynchronize(s));
        return fail((sf_status)st, "device reported status %d", st);
    }
    return SF_OK;
}

void sf_free_index(sf_index *idx) {
    if (!idx) return;
    cudaFree(idx->pos);
    cudaFree(idx->perm);
    cudaFree(idx->nlo);
    cudaFree(idx->nhi);
    cudaFree(idx->nell);
    cudaFree(idx->d_status);
    cudaFree(idx->mom);
    cudaFree(idx->mbe_ell);
    cudaFree(idx->mbe_nell);
    if (idx->mbe_done) cudaEventDestroy(idx->mbe_done);
    const int dev = idx->device;
    delete idx;
    trim_pool_memory(dev);
}

const char *sf_last_error(void) { return last_error_cstr(); }

uint64_t sf_launch_count(void) { return g_launches.load(); }

}  // extern "C"
