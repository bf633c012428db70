// sf_index.cu -- GPU spatial index over the point cloud.
//
// Stands in for the CPU-built k-d tree of Sec. 3.2 (used there by the range
// queries of Algorithm 2): the points are sorted by 63-bit Morton key over
// their bounding box, leaves are runs of 32 consecutive sorted points (one
// warp), and each upper level groups 32 consecutive nodes, so a warp tests all
// children of a node at once during traversal. Nodes keep a bounding box and
// the largest smoothing length per axis below them.
#include "sf_internal.cuh"

namespace sf {

// ---------------------------------------------------------------------------
// Bounding box (exact: min/max of float bit patterns in a monotone integer order)
// ---------------------------------------------------------------------------
__device__ __forceinline__ int ord_i(float f) {
    int i = __float_as_int(f);
    return i >= 0 ? i : i ^ 0x7fffffff;
}
__device__ __forceinline__ float ord_f(int i) { return __int_as_float(i >= 0 ? i : i ^ 0x7fffffff); }

__global__ void k_bbox_init(int *bb) {
    if (threadIdx.x < 3) bb[threadIdx.x] = 0x7fffffff;
    else if (threadIdx.x < 6) bb[threadIdx.x] = (int)0x80000000;
}

__global__ void k_bbox(const float *__restrict__ xyz, int64_t n, int *bb) {
    int mn[3] = {0x7fffffff, 0x7fffffff, 0x7fffffff};
    int mx[3] = {(int)0x80000000, (int)0x80000000, (int)0x80000000};
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            int v = ord_i(xyz[3 * i + k]);
            mn[k] = min(mn[k], v);
            mx[k] = max(mx[k], v);
        }
    }
#pragma unroll
    for (int k = 0; k < 3; ++k) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            mn[k] = min(mn[k], __shfl_xor_sync(0xffffffffu, mn[k], o));
            mx[k] = max(mx[k], __shfl_xor_sync(0xffffffffu, mx[k], o));
        }
    }
    if ((threadIdx.x & 31) == 0) {
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            atomicMin(&bb[k], mn[k]);
            atomicMax(&bb[3 + k], mx[k]);
        }
    }
}

// ---------------------------------------------------------------------------
// Morton keys: 21 bits per axis, x in bit 0, y in bit 1, z in bit 2.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint64_t spread3(uint32_t v) {
    uint64_t x = v & 0x1fffffu;
    x = (x | x << 32) & 0x1f00000000ffffull;
    x = (x | x << 16) & 0x1f0000ff0000ffull;
    x = (x | x << 8) & 0x100f00f00f00f00full;
    x = (x | x << 4) & 0x10c30c30c30c30c3ull;
    x = (x | x << 2) & 0x1249249249249249ull;
    return x;
}

__device__ __forceinline__ uint32_t quant21(float v, float lo, float scale) {
    float t = (v - lo) * scale;
    t = fminf(fmaxf(t, 0.0f), 2097151.0f);
    return (uint32_t)t;
}

__global__ void k_morton(const float *__restrict__ xyz, int64_t n, const int *__restrict__ bb,
                         uint64_t *__restrict__ keys, uint32_t *__restrict__ vals) {
    float lo[3], sc[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        lo[k] = ord_f(bb[k]);
        float ext = ord_f(bb[3 + k]) - lo[k];
        sc[k] = ext > 0.0f ? 2097152.0f / ext : 0.0f;
    }
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        uint64_t key = spread3(quant21(xyz[3 * i + 0], lo[0], sc[0])) |
                       (spread3(quant21(xyz[3 * i + 1], lo[1], sc[1])) << 1) |
                       (spread3(quant21(xyz[3 * i + 2], lo[2], sc[2])) << 2);
        keys[i] = key;
        vals[i] = (uint32_t)i;
    }
}

__global__ void k_gather(const float *__restrict__ xyz, const uint32_t *__restrict__ perm,
                         int64_t n, float4 *__restrict__ pos) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t o = perm[i];
        pos[i] = make_float4(xyz[3 * o + 0], xyz[3 * o + 1], xyz[3 * o + 2], 0.0f);
    }
}

// ---------------------------------------------------------------------------
// Node boxes: one warp per node; lane c holds child c (a point for leaves).
// ---------------------------------------------------------------------------
__device__ __forceinline__ void warp_minmax(float3 &lo, float3 &hi) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        lo.x = fminf(lo.x, __shfl_xor_sync(0xffffffffu, lo.x, o));
        lo.y = fminf(lo.y, __shfl_xor_sync(0xffffffffu, lo.y, o));
        lo.z = fminf(lo.z, __shfl_xor_sync(0xffffffffu, lo.z, o));
        hi.x = fmaxf(hi.x, __shfl_xor_sync(0xffffffffu, hi.x, o));
        hi.y = fmaxf(hi.y, __shfl_xor_sync(0xffffffffu, hi.y, o));
        hi.z = fmaxf(hi.z, __shfl_xor_sync(0xffffffffu, hi.z, o));
    }
}

__global__ void k_leaf_boxes(const float4 *__restrict__ pos, int64_t n, int64_t nleaf,
                             float4 *__restrict__ nlo, float4 *__restrict__ nhi) {
    const int lane = threadIdx.x & 31;
    const int64_t leaf = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (leaf >= nleaf) return;
    const int64_t i = leaf * kLeaf + lane;
    float3 lo = make_float3(INFINITY, INFINITY, INFINITY), hi = make_float3(-INFINITY, -INFINITY, -INFINITY);
    if (i < n) {
        float4 p = pos[i];
        lo = make_float3(p.x, p.y, p.z);
        hi = lo;
    }
    warp_minmax(lo, hi);
    if (lane == 0) {
        nlo[leaf] = make_float4(lo.x, lo.y, lo.z, 0.0f);
        nhi[leaf] = make_float4(hi.x, hi.y, hi.z, 0.0f);
    }
}

__global__ void k_inner_boxes(float4 *__restrict__ nlo, float4 *__restrict__ nhi,
                              int64_t child_off, int64_t child_cnt, int64_t off, int64_t cnt) {
    const int lane = threadIdx.x & 31;
    const int64_t node = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (node >= cnt) return;
    const int64_t c = node * kFanout + lane;
    float3 lo = make_float3(INFINITY, INFINITY, INFINITY), hi = make_float3(-INFINITY, -INFINITY, -INFINITY);
    if (c < child_cnt) {
        float4 a = nlo[child_off + c], b = nhi[child_off + c];
        lo = make_float3(a.x, a.y, a.z);
        hi = make_float3(b.x, b.y, b.z);
    }
    warp_minmax(lo, hi);
    if (lane == 0) {
        nlo[off + node] = make_float4(lo.x, lo.y, lo.z, 0.0f);
        nhi[off + node] = make_float4(hi.x, hi.y, hi.z, 0.0f);
    }
}

// ---------------------------------------------------------------------------
// Node maximum smoothing length per axis.
//   BW_ISO  : l = (h, h, h) from pos.w
//   BW_ANISO: l from the per-point array, only points inside the clip box count
// A leaf with no contributing point gets 0 (never accepted by traversal).
// ---------------------------------------------------------------------------
__global__ void k_leaf_ell(const float4 *__restrict__ pos, const float4 *__restrict__ ell,
                           int64_t n, int64_t nleaf, int clip, double3 blo, double3 bhi,
                           float4 *__restrict__ nell, const int *__restrict__ list) {
    const int lane = threadIdx.x & 31;
    const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (w >= nleaf) return;
    const int64_t leaf = list ? (int64_t)list[w] : w;
    const int64_t i = leaf * kLeaf + lane;
    float3 m = make_float3(0.f, 0.f, 0.f);
    float hmin = INFINITY;  // smallest positive length of the leaf (any axis)
    if (i < n) {
        float4 p = pos[i];
        bool in = true;
        if (clip)
            in = (double)p.x >= blo.x && (double)p.x <= bhi.x && (double)p.y >= blo.y &&
                 (double)p.y <= bhi.y && (double)p.z >= blo.z && (double)p.z <= bhi.z;
        if (in) {
            if (ell) {
                float4 e = ell[i];
                m = make_float3(e.x, e.y, e.z);
            } else {
                m = make_float3(p.w, p.w, p.w);
            }
            if (m.x > 0.f && m.y > 0.f && m.z > 0.f) hmin = fminf(m.x, fminf(m.y, m.z));
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        m.x = fmaxf(m.x, __shfl_xor_sync(0xffffffffu, m.x, o));
        m.y = fmaxf(m.y, __shfl_xor_sync(0xffffffffu, m.y, o));
        m.z = fmaxf(m.z, __shfl_xor_sync(0xffffffffu, m.z, o));
        hmin = fminf(hmin, __shfl_xor_sync(0xffffffffu, hmin, o));
    }
    if (lane == 0) nell[leaf] = make_float4(m.x, m.y, m.z, hmin);
}

__global__ void k_inner_ell(float4 *__restrict__ nell, int64_t child_off, int64_t child_cnt,
                            int64_t off, int64_t cnt) {
    const int lane = threadIdx.x & 31;
    const int64_t node = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (node >= cnt) return;
    const int64_t c = node * kFanout + lane;
    float3 m = make_float3(0.f, 0.f, 0.f);
    if (c < child_cnt) {
        float4 a = nell[child_off + c];
        m = make_float3(a.x, a.y, a.z);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        m.x = fmaxf(m.x, __shfl_xor_sync(0xffffffffu, m.x, o));
        m.y = fmaxf(m.y, __shfl_xor_sync(0xffffffffu, m.y, o));
        m.z = fmaxf(m.z, __shfl_xor_sync(0xffffffffu, m.z, o));
    }
    if (lane == 0) nell[off + node] = make_float4(m.x, m.y, m.z, 0.0f);
}

// The calls' scratch comes from the device's stream-ordered pool; by default the
// pool returns freed memory to the system at every synchronisation, so each
// call would map its scratch afresh. From the first index build on, the pool
// keeps the memory it has mapped (the attribute lives with this process);
// sf_free_index hands the pool's unused memory back.
void keep_pool_memory(int device) {
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, device) != cudaSuccess) return;
    uint64_t keep = UINT64_MAX;
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
}

void trim_pool_memory(int device) {
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, device) != cudaSuccess) return;
    cudaMemPoolTrimTo(pool, 0);
}

sf_status build_node_ell(sf_index *idx, int bw, const float4 *ell, const sf_box *clip_roi,
                         float4 *d_nell, cudaStream_t s, const int *d_leaves, int64_t nleaf) {
    double3 blo = make_double3(0, 0, 0), bhi = make_double3(0, 0, 0);
    if (clip_roi) {
        blo = make_double3(clip_roi->lo[0], clip_roi->lo[1], clip_roi->lo[2]);
        bhi = make_double3(clip_roi->hi[0], clip_roi->hi[1], clip_roi->hi[2]);
    }
    const float4 *e = (bw == BW_ANISO) ? ell : nullptr;
    const int64_t nl = d_leaves ? nleaf : idx->cnt[0];
    if (d_leaves)  // leaves off the list hold no contributing point
        SF_TRY_CUDA(cudaMemsetAsync(d_nell, 0, sizeof(float4) * idx->cnt[0], s));
    SF_TRY_CUDA(launch(k_leaf_ell, dim3(blocks_for(nl * 32, 256)), dim3(256), 0, s,
                       (const float4 *)idx->pos, e, idx->n, nl, clip_roi ? 1 : 0, blo,
                       bhi, d_nell, d_leaves));
    for (int l = 1; l < idx->nlevels; ++l)
        SF_TRY_CUDA(launch(k_inner_ell, dim3(blocks_for(idx->cnt[l] * 32, 256)), dim3(256), 0, s,
                           d_nell, idx->off[l - 1], idx->cnt[l - 1], idx->off[l], idx->cnt[l]));
    return SF_OK;
}

}  // namespace sf

using namespace sf;

extern "C" sf_status sf_build_index(const float *d_xyz, int64_t n, void *stream, sf_index **out) {
    if (!out) return fail(SF_ERR_INVALID_ARG, "sf_build_index: out is NULL");
    *out = nullptr;
    if (!d_xyz) return fail(SF_ERR_INVALID_ARG, "sf_build_index: d_xyz is NULL");
    if (n < 1 || n >= (int64_t(1) << 31))
        return fail(SF_ERR_INVALID_ARG, "sf_build_index: n=%lld out of range [1, 2^31)", (long long)n);
    cudaStream_t s = (cudaStream_t)stream;
    sf_index *idx = new sf_index();
    idx->n = n;
    cudaGetDevice(&idx->device);
    keep_pool_memory(idx->device);

    // level sizes are a function of n alone
    int64_t c = (n + kLeaf - 1) / kLeaf, total = 0;
    int L = 0;
    while (true) {
        if (L >= kMaxLevels) {
            delete idx;
            return fail(SF_ERR_INVALID_ARG, "sf_build_index: too many tree levels");
        }
        idx->off[L] = total;
        idx->cnt[L] = c;
        total += c;
        ++L;
        if (c == 1) break;
        c = (c + kFanout - 1) / kFanout;
    }
    idx->nlevels = L;
    idx->nnodes = total;

    auto cleanup = [&](sf_status st) {
        sf_free_index(idx);
        return st;
    };
    cudaError_t e;
    if ((e = cudaMalloc(&idx->pos, n * sizeof(float4))) != cudaSuccess ||
        (e = cudaMalloc(&idx->perm, n * sizeof(uint32_t))) != cudaSuccess ||
        (e = cudaMalloc(&idx->nlo, total * sizeof(float4))) != cudaSuccess ||
        (e = cudaMalloc(&idx->nhi, total * sizeof(float4))) != cudaSuccess ||
        (e = cudaMalloc(&idx->nell, total * sizeof(float4))) != cudaSuccess ||
        (e = cudaMalloc(&idx->d_status, sizeof(int))) != cudaSuccess ||
        (e = cudaMalloc(&idx->mom, 3 * total * sizeof(float4))) != cudaSuccess)
        return cleanup(fail(SF_ERR_OOM, "sf_build_index: cudaMalloc: %s", cudaGetErrorString(e)));
    if ((e = cudaMemsetAsync(idx->d_status, 0, sizeof(int), s)) != cudaSuccess ||
        (e = cudaMemsetAsync(idx->nell, 0, total * sizeof(float4), s)) != cudaSuccess)
        return cleanup(fail(SF_ERR_CUDA, "sf_build_index: memset: %s", cudaGetErrorString(e)));

    sf_status st = [&]() -> sf_status {
        Scratch sc(s);
        int *bb = sc.get<int>(6);
        uint64_t *ka = sc.get<uint64_t>(n), *kb = sc.get<uint64_t>(n);
        uint32_t *vb = sc.get<uint32_t>(n);
        SF_TRY_SCRATCH(sc);
        const unsigned g = std::min<unsigned>(blocks_for(n, 256), 152 * 16);
        SF_TRY_CUDA(launch(k_bbox_init, dim3(1), dim3(32), 0, s, bb));
        SF_TRY_CUDA(launch(k_bbox, dim3(g), dim3(256), 0, s, d_xyz, n, bb));
        SF_TRY_CUDA(launch(k_morton, dim3(g), dim3(256), 0, s, d_xyz, n, (const int *)bb, ka, idx->perm));
        SF_TRY(radix_sort_pairs(ka, idx->perm, kb, vb, n, 63, s));
        SF_TRY_CUDA(launch(k_gather, dim3(g), dim3(256), 0, s, d_xyz, (const uint32_t *)idx->perm, n, idx->pos));
        SF_TRY_CUDA(launch(k_leaf_boxes, dim3(blocks_for(idx->cnt[0] * 32, 256)), dim3(256), 0, s,
                           (const float4 *)idx->pos, n, idx->cnt[0], idx->nlo, idx->nhi));
        for (int l = 1; l < idx->nlevels; ++l)
            SF_TRY_CUDA(launch(k_inner_boxes, dim3(blocks_for(idx->cnt[l] * 32, 256)), dim3(256), 0, s,
                               idx->nlo, idx->nhi, idx->off[l - 1], idx->cnt[l - 1], idx->off[l],
                               idx->cnt[l]));
        SF_TRY(build_moments(idx, s));
        int hb[6];
        SF_TRY_CUDA(cudaMemcpyAsync(hb, bb, sizeof hb, cudaMemcpyDeviceToHost, s));
        SF_TRY_CUDA(cudaStreamSynchronize(s));
        for (int k = 0; k < 3; ++k) {
            int a = hb[k] >= 0 ? hb[k] : hb[k] ^ 0x7fffffff;
            int b = hb[3 + k] >= 0 ? hb[3 + k] : hb[3 + k] ^ 0x7fffffff;
            memcpy(&idx->bbox_lo[k], &a, 4);
            memcpy(&idx->bbox_hi[k], &b, 4);
        }
        return SF_OK;
    }();
    if (st != SF_OK) return cleanup(st);
    *out = idx;
    return SF_OK;
}
