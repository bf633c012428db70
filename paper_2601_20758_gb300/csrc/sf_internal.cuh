// sf_internal.cuh -- internal declarations shared by the CUDA translation units
// of libscalefree.so. Not part of the C ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <map>
#include <mutex>
#include <vector>

#include "scalefree.h"

namespace sf {

// ---------------------------------------------------------------------------
// Errors and launches
// ---------------------------------------------------------------------------
extern std::atomic<uint64_t> g_launches;

// Records a message for sf_last_error() and returns st.
sf_status fail(sf_status st, const char *fmt, ...);

#define SF_TRY_CUDA(expr)                                                                    \
    do {                                                                                     \
        cudaError_t _e = (expr);                                                             \
        if (_e != cudaSuccess)                                                               \
            return ::sf::fail(_e == cudaErrorMemoryAllocation ? SF_ERR_OOM : SF_ERR_CUDA,    \
                              "%s: %s (%s:%d)", #expr, cudaGetErrorString(_e), __FILE__,     \
                              __LINE__);                                                     \
    } while (0)

#define SF_TRY(expr)                                                                         \
    do {                                                                                     \
        sf_status _s = (expr);                                                               \
        if (_s != SF_OK) return _s;                                                          \
    } while (0)

// Launch a kernel, count it, and return the launch error (empty grids are skipped).
template <typename... KArgs, typename... Args>
inline cudaError_t launch(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem,
                          cudaStream_t s, Args... args) {
    if (grid.x == 0 || grid.y == 0 || grid.z == 0) return cudaSuccess;
    kernel<<<grid, block, smem, s>>>(static_cast<KArgs>(args)...);
    g_launches.fetch_add(1, std::memory_order_relaxed);
    return cudaGetLastError();
}

// Optional CUDA-event timing of named kernels on their launching stream
// (enabled with sf_kernel_timing_enable; off by default, then a no-op).
struct KTimer {
    const char *name;
    cudaStream_t s;
    cudaEvent_t a = nullptr, b = nullptr;
    KTimer(const char *n, cudaStream_t st);
    ~KTimer();
};

inline unsigned blocks_for(int64_t n, int per_block) {
    return (unsigned)((n + per_block - 1) / per_block);
}

// ---------------------------------------------------------------------------
// Stream-ordered scratch memory (cudaMallocAsync from the device's default
// pool, released at scope exit with cudaFreeAsync on the same stream).
// ---------------------------------------------------------------------------
struct Scratch {
    cudaStream_t s;
    std::vector<void *> ptrs;
    cudaError_t err = cudaSuccess;
    explicit Scratch(cudaStream_t st) : s(st) {}
    ~Scratch() {
        for (void *p : ptrs) cudaFreeAsync(p, s);
    }
    template <typename T>
    T *get(int64_t count) {
        if (count <= 0) count = 1;
        void *p = nullptr;
        cudaError_t e = cudaMallocAsync(&p, (size_t)count * sizeof(T), s);
        if (e != cudaSuccess) {
            err = e;
            return nullptr;
        }
        ptrs.push_back(p);
        return static_cast<T *>(p);
    }
};

#define SF_TRY_SCRATCH(sc)                                                                   \
    do {                                                                                     \
        if ((sc).err != cudaSuccess)                                                         \
            return ::sf::fail((sc).err == cudaErrorMemoryAllocation ? SF_ERR_OOM             \
                                                                    : SF_ERR_CUDA,           \
                              "scratch allocation: %s", cudaGetErrorString((sc).err));       \
    } while (0)

// ---------------------------------------------------------------------------
// Index layout
// ---------------------------------------------------------------------------
constexpr int kLeaf = 32;    // points per leaf (one warp)
constexpr int kFanout = 32;  // children per inner node (one warp)
constexpr int kMaxLevels = 8;

// Device status word codes (mirrors sf_status values).
enum : int { ST_OK = 0, ST_TIMEOUT = SF_ERR_TIMEOUT, ST_DEGENERATE = SF_ERR_DEGENERATE,
             ST_EMPTY = SF_ERR_EMPTY_ROI };

struct TreeView {
    const float4 *pos;   // sorted points (x, y, z, h)
    const float4 *nlo;   // node bbox min (w unused)
    const float4 *nhi;   // node bbox max (w unused)
    const float4 *nell;  // node max smoothing length per axis (w unused)
    int64_t n;           // points
    int nlevels;         // level 0 = leaves; level nlevels-1 = root (1 node)
    int64_t off[kMaxLevels];
    int64_t cnt[kMaxLevels];
};

}  // namespace sf

struct sf_index {
    int64_t n = 0;
    int device = 0;
    float4 *pos = nullptr;     // sorted (x, y, z, h)
    uint32_t *perm = nullptr;  // sorted position -> original index
    float4 *nlo = nullptr, *nhi = nullptr, *nell = nullptr;
    int nlevels = 0;
    int64_t off[sf::kMaxLevels] = {0};
    int64_t cnt[sf::kMaxLevels] = {0};
    int64_t nnodes = 0;
    float bbox_lo[3] = {0, 0, 0}, bbox_hi[3] = {0, 0, 0};
    int bw_rule = -1;  // rule whose bandwidths are resident (-1: none)
    int knn_k = 0;
    float fixed_h[3] = {0, 0, 0};
    int *d_status = nullptr;  // device status word
    std::mutex mu;

    sf::TreeView view() const {
        sf::TreeView v;
        v.pos = pos;
        v.nlo = nlo;
        v.nhi = nhi;
        v.nell = nell;
        v.n = n;
        v.nlevels = nlevels;
        for (int l = 0; l < sf::kMaxLevels; ++l) {
            v.off[l] = off[l];
            v.cnt[l] = cnt[l];
        }
        return v;
    }
};

namespace sf {

// Packed FP32 pairs (two IEEE single-precision lanes per 64-bit register,
// one instruction for both; each lane rounds exactly like the scalar op).
typedef unsigned long long f32x2;
__device__ __forceinline__ f32x2 f2_pack(float a, float b) {
    f32x2 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
    return r;
}
__device__ __forceinline__ void f2_unpack(f32x2 v, float &a, float &b) {
    asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(v));
}
__device__ __forceinline__ f32x2 f2_sub(f32x2 a, f32x2 b) {
    f32x2 r;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ f32x2 f2_mul(f32x2 a, f32x2 b) {
    f32x2 r;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ f32x2 f2_fma(f32x2 a, f32x2 b, f32x2 c) {
    f32x2 r;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
    return r;
}
__device__ __forceinline__ f32x2 f2_ld(const float *p) {  // 8-byte aligned
    return *reinterpret_cast<const f32x2 *>(p);
}

// ---------------------------------------------------------------------------
// Primitives (sf_prims.cu)
// ---------------------------------------------------------------------------
// Exclusive prefix sum of n uint32 values; *d_total (device, nullable) gets the sum.
sf_status scan_u32(const uint32_t *d_in, uint32_t *d_out, int64_t n, uint32_t *d_total,
                   cudaStream_t s);
// Stable LSD radix sort of (key, val) pairs over the low `bits` bits of key.
// Result ends in (keys, vals); keys_tmp / vals_tmp are n-element scratch.
sf_status radix_sort_pairs(uint64_t *keys, uint32_t *vals, uint64_t *keys_tmp,
                           uint32_t *vals_tmp, int64_t n, int bits, cudaStream_t s);
// Order-preserving map of float bits to uint32 (total order on non-NaN floats).
__host__ __device__ inline uint32_t float_to_ordered(float f) {
#ifdef __CUDA_ARCH__
    uint32_t u = __float_as_uint(f);
#else
    union { float f; uint32_t u; } c;
    c.f = f;
    uint32_t u = c.u;
#endif
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__host__ __device__ inline float ordered_to_float(uint32_t o) {
    uint32_t u = (o & 0x80000000u) ? (o & 0x7fffffffu) : ~o;
#ifdef __CUDA_ARCH__
    return __uint_as_float(u);
#else
    union { float f; uint32_t u; } c;
    c.u = u;
    return c.f;
#endif
}
// k-th smallest (0-based rank read from d_rank) of n ordered-uint32 keys; the
// key is written to *d_result. d_keys may be gathered through d_idx (nullable).
sf_status radix_select_u32(const uint32_t *d_keys, int64_t n, const int64_t *d_rank,
                           uint32_t *d_result, cudaStream_t s);

// ---------------------------------------------------------------------------
// Density engine (sf_density.cu)
// ---------------------------------------------------------------------------
enum BwMode : int { BW_ISO = 0, BW_UNIFORM = 1, BW_ANISO = 2 };

// Per-call constants living in device memory (filled by earlier kernels when
// they depend on the data, e.g. N_B and l of the paper's estimator).
struct DensityParams {
    float ell_uniform[3];  // BW_UNIFORM smoothing lengths
    float pad0;
    double inv_neff;       // 1 / N_eff
    int64_t neff;
};

struct GridSpec {
    int nx, ny, nz;
    double lo[3], hi[3], s[3];
};

struct DensityCall {
    int kernel;       // SF_K_*
    int bw;           // BwMode
    int clip;         // 1: only points inside roi count
    const float4 *ell;  // BW_ANISO per sorted point (lx, ly, lz, unused); else null
    const DensityParams *dp;  // device
    float4 *nell_override;     // node max-ell array to use (null: the index's own)
};

sf_status density_grid(sf_index *idx, const sf_box &roi, const GridSpec &g,
                       const DensityCall &call, float *d_out, double *d_mass, cudaStream_t s,
                       unsigned long long *d_pairs = nullptr);

// Density at the sorted points inside roi (DIRECT). d_rho_sorted[i] for sorted
// i in roi, d_inroi[i] = 1/0. d_count receives the number of roi points.
sf_status density_points(sf_index *idx, const sf_box &roi, const DensityCall &call,
                         float *d_rho_sorted, uint8_t *d_inroi, cudaStream_t s,
                         unsigned long long *d_pairs = nullptr);

// Node max smoothing length per axis for BW_ISO (from pos.w) or BW_ANISO (from ell,
// only points inside roi when clip) into d_nell.
sf_status build_node_ell(sf_index *idx, int bw, const float4 *ell, const sf_box *clip_roi,
                         float4 *d_nell, cudaStream_t s);

// Batched grids over many ROIs (sf_density.cu).
struct BatchPlan;
sf_status batch_create(sf_index *idx, int nroi, const sf_box *rois, const GridSpec *grids,
                       int kernel, int bw, bool clip, DensityParams *d_dps, int tz, int ips,
                       bool use_graph, cudaStream_t s, BatchPlan **out);
sf_status batch_run(BatchPlan *P, float *const *outs, double *h_mass, cudaStream_t s);
void batch_free(BatchPlan *P);

// ---------------------------------------------------------------------------
// kNN (sf_knn.cu)
// ---------------------------------------------------------------------------
sf_status knn_bandwidths(sf_index *idx, int k, uint32_t *d_nbr_orig, float *d_h_sorted,
                         cudaStream_t s);

}  // namespace sf
