// sf_roi.cu -- the points of one ROI, found through the index, and their
// densities compacted into ascending original-index order (sf_kde_points).
//
// The ROI's points are those inside the closed box B (Sec. 3.1). The index
// keeps every leaf's bounding box, so the leaves that can hold a point of B
// are found by testing the level-1 nodes and then their 32 leaves: one warp
// per level-1 node, no walk over the points. Everything after that -- the
// densities of the leaves' points, the compaction and the sort into original
// order -- is sized by the leaves found, not by the cloud: a small ROI of a
// billion-point cloud costs what its few thousand points cost.
//
// The same sizes give the call's device workspace before the call is made
// (sf_query_workspace), for admission by memory in a serving loop.
#include <cmath>

#include "sf_internal.cuh"

namespace sf {

sf_status grid_workspace(sf_index *idx, const sf_box &roi, const GridSpec &g,
                         const DensityCall &call, int64_t *bytes, cudaStream_t s);

namespace {

__device__ __forceinline__ bool box_meets(const float4 &lo, const float4 &hi, const float3 &blo,
                                          const float3 &bhi) {
    return !(lo.x > bhi.x || hi.x < blo.x || lo.y > bhi.y || hi.y < blo.y || lo.z > bhi.z ||
             hi.z < blo.z);
}

constexpr int kRoiWarps = 8;

// One warp per level-1 node: the node's leaves whose bounding box meets the box
// [blo, bhi]. Count pass: cnt[node] = how many; emit pass: their indices at
// list[off[node] ...], ascending.
template <bool EMIT>
__global__ void __launch_bounds__(kRoiWarps * 32)
    k_roi_leaves(TreeView tv, float3 blo, float3 bhi, uint32_t *__restrict__ cnt,
                 const uint32_t *__restrict__ off, int *__restrict__ list) {
    const int lane = threadIdx.x & 31;
    const int64_t node = (int64_t)blockIdx.x * kRoiWarps + (threadIdx.x >> 5);
    if (node >= tv.cnt[1]) return;
    const float4 plo = __ldg(&tv.nlo[tv.off[1] + node]);
    const float4 phi = __ldg(&tv.nhi[tv.off[1] + node]);
    unsigned m = 0;
    if (box_meets(plo, phi, blo, bhi)) {  // warp-uniform
        const int64_t c = node * kFanout + lane;
        bool ok = false;
        if (c < tv.cnt[0]) ok = box_meets(__ldg(&tv.nlo[tv.off[0] + c]), __ldg(&tv.nhi[tv.off[0] + c]), blo, bhi);
        m = __ballot_sync(0xffffffffu, ok);
        if (EMIT && ok) list[off[node] + __popc(m & ((1u << lane) - 1u))] = (int)c;
    }
    if (!EMIT && lane == 0) cnt[node] = __popc(m);
}

// flags[i] = inroi[i] (the scan's input).
__global__ void k_roi_flags(const uint8_t *__restrict__ inroi, int64_t n, uint32_t *__restrict__ flags) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        flags[i] = inroi[i];
}

// The ROI points as (original index, density bits) pairs at their scan positions.
__global__ void k_roi_pairs(const int *__restrict__ leaves, int64_t nslot_pts,
                            const uint8_t *__restrict__ inroi, const uint32_t *__restrict__ pos,
                            const float *__restrict__ rho, const uint32_t *__restrict__ perm,
                            uint64_t *__restrict__ keys, uint32_t *__restrict__ vals) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nslot_pts;
         i += (int64_t)gridDim.x * blockDim.x) {
        if (!inroi[i]) continue;
        const int64_t j = (int64_t)leaves[i / kLeaf] * kLeaf + (i % kLeaf);
        const uint32_t p = pos[i];
        keys[p] = perm[j];
        vals[p] = __float_as_uint(rho[i]);
    }
}

__global__ void k_roi_out(const uint64_t *__restrict__ keys, const uint32_t *__restrict__ vals,
                          int64_t m, float *__restrict__ dens, uint32_t *__restrict__ ids) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m;
         i += (int64_t)gridDim.x * blockDim.x) {
        ids[i] = (uint32_t)keys[i];
        dens[i] = __uint_as_float(vals[i]);
    }
}

unsigned sgrid(int64_t n) { return std::max(1u, std::min<unsigned>(blocks_for(n, 256), 152 * 16)); }

// Exact float bounds of the closed double box.
void roi_bounds(const sf_box &roi, float3 &lo, float3 &hi) {
    float l[3], h[3];
    for (int k = 0; k < 3; ++k) {
        float a = (float)roi.lo[k];
        if ((double)a < roi.lo[k]) a = nextafterf(a, INFINITY);
        float b = (float)roi.hi[k];
        if ((double)b > roi.hi[k]) b = nextafterf(b, -INFINITY);
        l[k] = a;
        h[k] = b;
    }
    lo = make_float3(l[0], l[1], l[2]);
    hi = make_float3(h[0], h[1], h[2]);
}

int64_t scan_parts_bytes(int64_t n) { return n > 0 ? scratch_round(4 * ((n + 2047) / 2048)) : 0; }

}  // namespace

// Leaves whose bounding box meets the ROI: *d_list (in sc, ascending), *h_nleaf.
// Synchronises the stream once (the count); peek is read at that point.
sf_status roi_leaf_list(sf_index *idx, const sf_box &roi, Scratch &sc, int **d_list,
                        int64_t *h_nleaf, StatusPeek *peek, cudaStream_t s) {
    float3 lo, hi;
    roi_bounds(roi, lo, hi);
    const TreeView tv = idx->view();
    if (idx->nlevels < 2) {  // a single leaf (n <= 32)
        int *list = sc.get<int>(1);
        SF_TRY_SCRATCH(sc);
        SF_TRY_CUDA(cudaMemsetAsync(list, 0, sizeof(int), s));
        if (peek && peek->d_src) {
            SF_TRY_CUDA(cudaMemcpyAsync(&peek->value, peek->d_src, sizeof(int), cudaMemcpyDeviceToHost, s));
            SF_TRY_CUDA(cudaStreamSynchronize(s));
        }
        *d_list = list;
        *h_nleaf = 1;
        return SF_OK;
    }
    const int64_t n1 = tv.cnt[1];
    uint32_t *cnt = sc.get<uint32_t>(n1);
    uint32_t *off = sc.get<uint32_t>(n1);
    uint32_t *tot = sc.get<uint32_t>(1);
    SF_TRY_SCRATCH(sc);
    const unsigned nb = blocks_for(n1, kRoiWarps);
    SF_TRY_CUDA(launch(k_roi_leaves<false>, dim3(nb), dim3(kRoiWarps * 32), 0, s, tv, lo, hi, cnt,
                       (const uint32_t *)nullptr, (int *)nullptr));
    SF_TRY(scan_u32(cnt, off, n1, tot, s));
    uint32_t h = 0;
    SF_TRY_CUDA(cudaMemcpyAsync(&h, tot, sizeof h, cudaMemcpyDeviceToHost, s));
    if (peek && peek->d_src)
        SF_TRY_CUDA(cudaMemcpyAsync(&peek->value, peek->d_src, sizeof(int), cudaMemcpyDeviceToHost, s));
    SF_TRY_CUDA(cudaStreamSynchronize(s));
    int *list = sc.get<int>(std::max<int64_t>(1, h));
    SF_TRY_SCRATCH(sc);
    if (h > 0)
        SF_TRY_CUDA(launch(k_roi_leaves<true>, dim3(nb), dim3(kRoiWarps * 32), 0, s, tv, lo, hi,
                           (uint32_t *)nullptr, (const uint32_t *)off, list));
    *d_list = list;
    *h_nleaf = h;
    return SF_OK;
}

// Bytes roi_leaf_list holds when it returns (the list included), and its peak.
static int64_t leaf_list_bytes(const sf_index *idx, int64_t nleaf, int64_t *peak) {
    if (idx->nlevels < 2) {
        *peak = scratch_round(4);
        return *peak;
    }
    const int64_t n1 = idx->cnt[1];
    const int64_t held = 2 * scratch_round(4 * n1) + scratch_round(4);
    *peak = held + std::max(scan_parts_bytes(n1), scratch_round(4 * std::max<int64_t>(1, nleaf)));
    return held + scratch_round(4 * std::max<int64_t>(1, nleaf));
}

// The ROI points of the slots (rho, inroi over nslots * 32 slot points) in
// ascending original index: d_density / d_ids, *h_count. CAPACITY if more than
// capacity. Synchronises once (the count).
sf_status roi_compact(sf_index *idx, const int *d_leaves, int64_t nslots, const uint8_t *d_inroi,
                      const float *d_rho, float *d_density, uint32_t *d_ids, int64_t capacity,
                      int64_t *h_count, cudaStream_t s) {
    const int64_t np = nslots * kLeaf;
    *h_count = 0;
    if (np == 0) return SF_OK;
    Scratch sc(s);
    uint32_t *flags = sc.get<uint32_t>(np);
    uint32_t *pos = sc.get<uint32_t>(np);
    uint32_t *total = sc.get<uint32_t>(1);
    SF_TRY_SCRATCH(sc);
    SF_TRY_CUDA(launch(k_roi_flags, dim3(sgrid(np)), dim3(256), 0, s, d_inroi, np, flags));
    SF_TRY(scan_u32(flags, pos, np, total, s));
    uint32_t m = 0;
    SF_TRY_CUDA(cudaMemcpyAsync(&m, total, sizeof m, cudaMemcpyDeviceToHost, s));
    SF_TRY_CUDA(cudaStreamSynchronize(s));
    *h_count = m;
    if ((int64_t)m > capacity)
        return fail(SF_ERR_CAPACITY, "sf_kde_points: %u ROI points exceed capacity %lld", m,
                    (long long)capacity);
    if (m == 0) return SF_OK;
    uint64_t *keys = sc.get<uint64_t>(m);
    uint32_t *vals = sc.get<uint32_t>(m);
    uint64_t *ktmp = sc.get<uint64_t>(m);
    uint32_t *vtmp = sc.get<uint32_t>(m);
    SF_TRY_SCRATCH(sc);
    SF_TRY_CUDA(launch(k_roi_pairs, dim3(sgrid(np)), dim3(256), 0, s, d_leaves, np, d_inroi,
                       (const uint32_t *)pos, d_rho, (const uint32_t *)idx->perm, keys, vals));
    // original indices are < 2^31: 32 key bits, four 8-bit passes (stable)
    SF_TRY(radix_sort_pairs(keys, vals, ktmp, vtmp, m, 32, s));
    SF_TRY_CUDA(launch(k_roi_out, dim3(sgrid(m)), dim3(256), 0, s, (const uint64_t *)keys,
                       (const uint32_t *)vals, (int64_t)m, d_density, d_ids));
    return SF_OK;
}

// Peak bytes of roi_compact for np slot points of which at most m are in the ROI.
static int64_t compact_peak(int64_t np, int64_t m) {
    if (np == 0) return 0;
    const int64_t base = 2 * scratch_round(4 * np) + scratch_round(4);
    int64_t peak = base + scan_parts_bytes(np);
    if (m > 0) {
        const int64_t pairs = 2 * scratch_round(8 * m) + 2 * scratch_round(4 * m);
        const int64_t counts = scratch_round(4 * 256 * ((m + 4095) / 4096));
        peak = std::max(peak, base + pairs + counts + scan_parts_bytes(256 * ((m + 4095) / 4096)));
    }
    return peak;
}

// Workspace of sf_kde_points (rules kNN and fixed) for `roi`: counts the ROI's
// leaves (one synchronisation) and sizes every buffer the call allocates; the
// point count is bounded by 32 per leaf. grid: the INTERP grid's spec (or null).
sf_status points_workspace(sf_index *idx, const sf_box &roi, const GridSpec *g,
                           const DensityCall &call, int64_t base_bytes, int64_t *bytes,
                           cudaStream_t s) {
    int64_t nleaf = 0;
    {
        Scratch sc(s);
        int *list = nullptr;
        SF_TRY(roi_leaf_list(idx, roi, sc, &list, &nleaf, nullptr, s));
    }
    int64_t list_peak = 0;
    const int64_t list_held = leaf_list_bytes(idx, nleaf, &list_peak);
    const int64_t np = nleaf * kLeaf;
    const int64_t slots = scratch_round(4 * std::max<int64_t>(1, np)) + scratch_round(std::max<int64_t>(1, np));
    int64_t during = 0;
    if (g) {  // INTERP: the grid first
        int64_t gb = 0;
        SF_TRY(grid_workspace(idx, roi, *g, call, &gb, s));
        during = scratch_round(4 * (int64_t)g->nx * g->ny * g->nz) + gb;
    }
    const int64_t peak = std::max(list_peak, list_held + slots + std::max(during, compact_peak(np, np)));
    *bytes = base_bytes + peak;
    return SF_OK;
}

}  // namespace sf
