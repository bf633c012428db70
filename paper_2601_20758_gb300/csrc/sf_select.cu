// sf_select.cu -- density-threshold selection (Sec. 4.1: a density threshold
// decides which points are selected).
//
// The nearest-rank threshold is an exact order statistic of the float32
// densities, found by radix selection on their bit patterns (integer work,
// bit-exact); compaction is a prefix sum, so the selected indices come out
// ascending.
#include <cmath>

#include "sf_internal.cuh"

namespace sf {

__global__ void k_ordered_keys(const float *__restrict__ v, int64_t n, uint32_t *__restrict__ keys) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        keys[i] = float_to_ordered(v[i]);
}

__global__ void k_sel_flags(const float *__restrict__ v, int64_t n, const uint32_t *__restrict__ tkey,
                            float tconst, int use_key, uint32_t *__restrict__ flags,
                            float *__restrict__ t_out) {
    const float t = use_key ? ordered_to_float(*tkey) : tconst;
    if (blockIdx.x == 0 && threadIdx.x == 0 && t_out) *t_out = t;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        flags[i] = v[i] > t ? 1u : 0u;
}

__global__ void k_sel_write(const uint32_t *__restrict__ flags, const uint32_t *__restrict__ pos,
                            const uint32_t *__restrict__ ids, int64_t n, int64_t n_total,
                            uint8_t *__restrict__ mask, uint32_t *__restrict__ sel) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        if (flags[i]) {
            const uint32_t id = ids[i];
            if (sel) sel[pos[i]] = id;
            if (mask && (int64_t)id < n_total) mask[id] = 1;
        }
    }
}

static unsigned stride_grid(int64_t n) {
    return std::max(1u, std::min<unsigned>(blocks_for(n, 256), 152 * 16));
}

sf_status select_points(const float *d_density, const uint32_t *d_ids, int64_t n, int64_t n_total,
                        double threshold, double percentile, uint8_t *d_mask, uint32_t *d_sel_ids,
                        int64_t *h_nsel, double *h_threshold, cudaStream_t s) {
    if (d_mask && n_total > 0) SF_TRY_CUDA(cudaMemsetAsync(d_mask, 0, (size_t)n_total, s));
    if (n == 0) {
        if (h_nsel) *h_nsel = 0;
        if (h_threshold) *h_threshold = std::isnan(threshold) ? NAN : (double)(float)threshold;
        return SF_OK;
    }
    Scratch sc(s);
    uint32_t *flags = sc.get<uint32_t>(n);
    uint32_t *pos = sc.get<uint32_t>(n);
    uint32_t *total = sc.get<uint32_t>(1);
    float *tval = sc.get<float>(1);
    uint32_t *tkey = nullptr;
    const bool by_rank = std::isnan(threshold);
    if (by_rank) {
        uint32_t *keys = sc.get<uint32_t>(n);
        int64_t *rank = sc.get<int64_t>(1);
        tkey = sc.get<uint32_t>(1);
        SF_TRY_SCRATCH(sc);
        int64_t r = (int64_t)std::ceil(percentile / 100.0 * (double)n);
        if (r < 1) r = 1;
        if (r > n) r = n;
        const int64_t r0 = r - 1;
        SF_TRY_CUDA(cudaMemcpyAsync(rank, &r0, sizeof r0, cudaMemcpyHostToDevice, s));
        SF_TRY_CUDA(launch(k_ordered_keys, dim3(stride_grid(n)), dim3(256), 0, s, d_density, n, keys));
        SF_TRY(radix_select_u32(keys, n, rank, tkey, s));
    }
    SF_TRY_SCRATCH(sc);
    SF_TRY_CUDA(launch(k_sel_flags, dim3(stride_grid(n)), dim3(256), 0, s, d_density, n,
                       (const uint32_t *)tkey, (float)threshold, by_rank ? 1 : 0, flags, tval));
    SF_TRY(scan_u32(flags, pos, n, total, s));
    SF_TRY_CUDA(launch(k_sel_write, dim3(stride_grid(n)), dim3(256), 0, s, (const uint32_t *)flags,
                       (const uint32_t *)pos, d_ids, n, n_total, d_mask, d_sel_ids));
    if (h_nsel || h_threshold) {
        uint32_t ht = 0;
        float tv = 0.f;
        SF_TRY_CUDA(cudaMemcpyAsync(&ht, total, sizeof ht, cudaMemcpyDeviceToHost, s));
        SF_TRY_CUDA(cudaMemcpyAsync(&tv, tval, sizeof tv, cudaMemcpyDeviceToHost, s));
        SF_TRY_CUDA(cudaStreamSynchronize(s));
        if (h_nsel) *h_nsel = ht;
        if (h_threshold) *h_threshold = tv;
    }
    return SF_OK;
}

}  // namespace sf
