// sf_internal.cuh -- internal declarations shared by the CUDA translation units
// of libscalefree.so. Not part of the C ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
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
// Every entry point starts with this: clears the message, opens the scratch count.
void clear_error();

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

// Raise a kernel's dynamic shared-memory limit once per device (the attribute
// is per device; the flag word is per kernel, one bit per device ordinal < 64).
template <typename K>
inline cudaError_t smem_attr_once(K kernel, size_t smem, std::atomic<uint64_t> &done) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const uint64_t bit = dev < 64 ? (uint64_t(1) << dev) : 0;
    if (bit && (done.load(std::memory_order_acquire) & bit)) return cudaSuccess;
    e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess && bit) done.fetch_or(bit, std::memory_order_release);
    return e;
}

// A device status word to read back at a synchronisation the call makes anyway
// (the copy is queued just before that synchronisation).
struct StatusPeek {
    const int *d_src = nullptr;  // per-call device status word (ST_*)
    int value = 0;               // host copy, valid after the synchronisation
};

// ---------------------------------------------------------------------------
// Stream-ordered scratch memory (cudaMallocAsync from the device's default
// pool, released at scope exit with cudaFreeAsync on the same stream).
// ---------------------------------------------------------------------------
// Bytes of scratch the calling thread holds, and the most it has held since the
// start of its current library call (each allocation counted rounded up to 256 B).
struct ScratchStats {
    int64_t live = 0;
    int64_t peak = 0;
};
ScratchStats &scratch_stats();  // thread-local
constexpr int64_t kScratchAlign = 256;
inline int64_t scratch_round(int64_t bytes) {
    return (std::max<int64_t>(bytes, 1) + kScratchAlign - 1) / kScratchAlign * kScratchAlign;
}

struct Scratch {
    cudaStream_t s;
    std::vector<void *> ptrs;
    int64_t held = 0;
    cudaError_t err = cudaSuccess;
    explicit Scratch(cudaStream_t st) : s(st) {}
    ~Scratch() {
        for (void *p : ptrs) cudaFreeAsync(p, s);
        scratch_stats().live -= held;
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
        const int64_t b = scratch_round(count * (int64_t)sizeof(T));
        held += b;
        ScratchStats &st = scratch_stats();
        st.live += b;
        if (st.live > st.peak) st.peak = st.live;
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
    float4 *mom = nullptr;    // per node: (mu_hi, M0), (mu_lo, -), (C, -); see build_moments
    // The estimator's per-point adaptive lengths and per-node maxima (rule MBE),
    // allocated at its first call and kept; calls take mbe_mu for their whole
    // duration and order their device work after the previous call's (mbe_done).
    float4 *mbe_ell = nullptr, *mbe_nell = nullptr;
    cudaEvent_t mbe_done = nullptr;
    std::mutex mbe_mu;
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

// Reciprocal of the hardware approximation (relative error below 2^-22). Used
// for the conservative support filters and for u_k = s / l_k and c / prod l_k,
// where a few ulps stay far inside the 1e-5 density tolerance.
__device__ __forceinline__ float rcp_approx(float x) {
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Squared-support slack of the filters (covers the reciprocal's error and the
// rounding of the gap terms; the filters only ever admit too much).
constexpr float kFilterSlack = 3.0e-5f;

// The box [lo, hi] widened by a margin that covers the float rounding of box
// and node coordinates (relative 1e-6 of the coordinates).
__device__ __forceinline__ void widen_box(const float lo[3], const float hi[3], float wlo[3],
                                          float whi[3]) {
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const float m = 1.0e-6f * (fabsf(lo[k]) + fabsf(hi[k])) + 1.0e-30f;
        wlo[k] = lo[k] - m;
        whi[k] = hi[k] + m;
    }
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

// Count the points of a sorted cloud inside [lo, hi] (closed, float bounds) into *cnt.
__global__ void k_count_box(const float4 *__restrict__ pos, int64_t n, float3 lo, float3 hi,
                            unsigned long long *cnt);
// N_eff = *cnt (clip scope) or n_all (cnt == NULL), 1/N_eff and the uniform lengths
// into *dp; ST_EMPTY into *status (nullable) when N_eff = 0.
__global__ void k_set_params(DensityParams *dp, const unsigned long long *cnt, int64_t n_all,
                             float ex, float ey, float ez, int *status);
// Launches the two above for one ROI; d_status (nullable) is the call's own status word.
sf_status set_density_params(sf_index *idx, bool clip, const sf_box &roi, const float ell[3],
                             DensityParams *d_dp, int *d_status, cudaStream_t s);

// Exact float bounds of a closed double box: x >= lo_f <=> (double)x >= lo.
void float_bounds(const double lo[3], const double hi[3], float flo[3], float fhi[3]);
// Normalisation constant of the kernel: 15/(8 pi) or 1/((2 pi)^1.5 P3).
float kernel_cnorm(int kernel);
// Node coordinates r_k(i) = lo_k + i s_k in double, split into float (hi, lo), x then y then z.
void node_axes(const GridSpec &g, float2 *ax);

struct DensityCall {
    int kernel;       // SF_K_*
    int bw;           // BwMode
    int clip;         // 1: only points inside roi count
    const float4 *ell;  // BW_ANISO per sorted point (lx, ly, lz, unused); else null
    const DensityParams *dp;  // device
    float4 *nell_override;     // node max-ell array to use (null: the index's own)
    int prec = SF_PREC_FP32;   // grids: SF_PREC_* (non-FP32: Gaussian with kNN or fixed lengths)
    int accel = SF_ACCEL_AUTO; // grids: SF_ACCEL_* (the moment form: Epanechnikov, uniform lengths)
};

// Per-node moments of the index (sf_moments.cu), built once with the index:
// for node g, mom[3g] = (mu_hi, M0), mom[3g+1] = (mu_lo, 0), mom[3g+2] = (C, 0)
// with M0 the point count, mu = centroid (mu_hi + mu_lo in float pairs) and
// C_k = sum (y_k - mu_k)^2 (leaves: FP32 sums of offsets within the leaf; inner
// nodes: FP64 parallel-axis combine of their children, rounded once).
sf_status build_moments(sf_index *idx, cudaStream_t s);
// Grid density by exact moments (Epanechnikov, BW_UNIFORM only); same contract
// as density_grid. ws_bytes (nullable): return the call's bytes instead of running.
sf_status density_grid_moments(sf_index *idx, const sf_box &roi, const GridSpec &g,
                               const DensityCall &call, float *d_out, double *d_mass,
                               cudaStream_t s, int64_t *ws_bytes, StatusPeek *peek);
// Sum of n per-tile (or per-block) FP64 partial masses times cell, into *out.
__global__ void k_mass_final(const double *__restrict__ part, int64_t n, double cell, double *out);
// True when the moment form applies to this call (Epanechnikov, one length per axis).
inline bool moments_apply(const DensityCall &c) {
    return c.kernel == SF_K_EPAN && c.bw == BW_UNIFORM && c.accel != SF_ACCEL_NONE;
}

// peek (nullable): a status word read back at the call's sizing synchronisation.
sf_status density_grid(sf_index *idx, const sf_box &roi, const GridSpec &g,
                       const DensityCall &call, float *d_out, double *d_mass, cudaStream_t s,
                       unsigned long long *d_pairs = nullptr, StatusPeek *peek = nullptr);

// Density (DIRECT) at the points of the query leaves d_leaves[0..nslots) that lie
// inside roi: for slot t and lane l (the point of sorted index d_leaves[t] * 32 + l),
// d_inroi[t * 32 + l] = 1/0 and, if 1, d_rho_sorted[t * 32 + l] = its density.
// d_leaves == NULL: every leaf in order (slot = leaf; nslots ignored).
sf_status density_points(sf_index *idx, const sf_box &roi, const DensityCall &call,
                         const int *d_leaves, int64_t nslots, float *d_rho_sorted,
                         uint8_t *d_inroi, cudaStream_t s, unsigned long long *d_pairs = nullptr);
// The same with the tensor-core cross term (prec = SF_PREC_TF32 / 3XTF32 / BF16).
sf_status density_points_tc(sf_index *idx, const sf_box &roi, const DensityCall &call, int prec,
                            const int *d_leaves, int64_t nslots, float *d_rho_sorted,
                            uint8_t *d_inroi, cudaStream_t s);

// Node max smoothing length per axis for BW_ISO (from pos.w) or BW_ANISO (from ell,
// only points inside roi when clip) into d_nell. d_leaves (nullable): only these
// nleaf leaves can hold a contributing point; every other leaf gets 0.
sf_status build_node_ell(sf_index *idx, int bw, const float4 *ell, const sf_box *clip_roi,
                         float4 *d_nell, cudaStream_t s, const int *d_leaves = nullptr,
                         int64_t nleaf = 0);

// The device's stream-ordered pool keeps freed scratch while indexes exist / is trimmed.
void keep_pool_memory(int device);
void trim_pool_memory(int device);

// Leaves whose bounding box meets the ROI: *d_list (in sc, ascending), *h_nleaf.
// Synchronises the stream once (the count); peek (nullable) is read at that point.
sf_status roi_leaf_list(sf_index *idx, const sf_box &roi, Scratch &sc, int **d_list,
                        int64_t *h_nleaf, StatusPeek *peek, cudaStream_t s);

// Batched grids over many ROIs (sf_density.cu).
struct BatchPlan;
sf_status batch_create(sf_index *idx, int nroi, const sf_box *rois, const GridSpec *grids,
                       int kernel, int bw, bool clip, DensityParams *d_dps, int tz, int ips,
                       bool use_graph, cudaStream_t s, BatchPlan **out, int prec = SF_PREC_FP32);
sf_status batch_run(BatchPlan *P, float *const *outs, double *h_mass, cudaStream_t s);
void batch_free(BatchPlan *P);

// ---------------------------------------------------------------------------
// kNN (sf_knn.cu)
// ---------------------------------------------------------------------------
sf_status knn_bandwidths(sf_index *idx, int k, uint32_t *d_nbr_orig, float *d_h_sorted,
                         cudaStream_t s);

}  // namespace sf
