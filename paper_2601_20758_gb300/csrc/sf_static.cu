// sf_static.cu -- sf_kde_grid_static: the ROI grid density without any device
// memory allocation, for callers that cannot allocate (see scalefree.h).
//
// All scratch the call needs lives in one file-scope __device__ array of
// fixed size (kStaticBytes, about 0.55 MB), held by every GPU that loads the
// library until the process exits. The call computes the same numbers as
// sf_kde_grid (same kernels, same node coordinates), for the kNN and fixed
// bandwidth rules; the paper's estimator (rule MBE) needs per-point scratch
// proportional to the cloud and is rejected here.
#include <cmath>
#include <cstddef>
#include <mutex>

#include "sf_internal.cuh"

namespace sf {

sf_status density_grid_prealloc(sf_index *idx, const sf_box &roi, const GridSpec &g,
                                const DensityCall &call, const float2 *d_axis,
                                double *d_mass_part, float *d_out, double *d_mass, cudaStream_t s);
int64_t grid_tile_count(const GridSpec &g);
const char *last_error_cstr();
void clear_error();

namespace {

constexpr int kStaticMaxDim = 1024;          // nodes per axis
constexpr int64_t kStaticMaxTiles = 65536;   // 16 x 16 x 8 node tiles (e.g. 512^3)

struct StaticScratch {
    float2 axis[3 * kStaticMaxDim];     // node coordinates, (hi, lo) float pairs
    DensityParams dp;                   // N_eff and the fixed lengths
    unsigned long long count;           // particles in the ROI (clip scope)
    int status;                         // this call's status word (ST_EMPTY)
    double mass;                        // FP64 total mass
    double mass_part[kStaticMaxTiles];  // per-tile partial sums
};

constexpr size_t kStaticBytes = sizeof(StaticScratch);

}  // namespace

// The scratch itself. In host code this name is only a handle for
// cudaGetSymbolAddress: its device address is looked up per device below.
static __device__ __align__(256) unsigned char g_static_scratch[kStaticBytes];

namespace {

std::mutex g_static_mu;
constexpr int kMaxDevices = 64;
void *g_static_addr[kMaxDevices] = {nullptr};

// Device address of the scratch on the current device (looked up once per
// device, on the first call made with that device current).
sf_status static_scratch(StaticScratch **out) {
    int dev = 0;
    SF_TRY_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) return fail(SF_ERR_INVALID_ARG, "device ordinal %d", dev);
    std::lock_guard<std::mutex> lk(g_static_mu);
    if (g_static_addr[dev]) {
        // a context torn down since (cudaDeviceReset) leaves a stale address: check it
        cudaPointerAttributes at;
        const cudaError_t e = cudaPointerGetAttributes(&at, g_static_addr[dev]);
        if (e != cudaSuccess || at.type != cudaMemoryTypeDevice || at.device != dev) {
            (void)cudaGetLastError();  // the query's error must not surface at the next launch
            g_static_addr[dev] = nullptr;
        }
    }
    if (!g_static_addr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
        if (e != cudaSuccess || !p)
            return fail(SF_ERR_CUDA, "cudaGetSymbolAddress(static scratch): %s", cudaGetErrorString(e));
        g_static_addr[dev] = p;
    }
    *out = static_cast<StaticScratch *>(g_static_addr[dev]);
    return SF_OK;
}

}  // namespace

// r_k(i) = lo_k + i s_k in FP64 (separately rounded product and sum, as the
// host computes it for sf_kde_grid), split into a float (hi, lo) pair.
__global__ void k_static_axis(float2 *axis, int nx, int ny, int nz, double3 lo, double3 s) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    const int n = nx + ny + nz;
    if (t >= n) return;
    int i;
    double l, sp;
    if (t < nx) {
        i = t; l = lo.x; sp = s.x;
    } else if (t < nx + ny) {
        i = t - nx; l = lo.y; sp = s.y;
    } else {
        i = t - nx - ny; l = lo.z; sp = s.z;
    }
    const double r = __dadd_rn(l, __dmul_rn((double)i, sp));
    const float h = (float)r;
    axis[t] = make_float2(h, (float)__dsub_rn(r, (double)h));
}

}  // namespace sf

using namespace sf;

extern "C" sf_status sf_kde_grid_static(sf_index *idx, const sf_box *roi, const int32_t dims[3],
                                        int32_t kernel, const sf_params *p, float *d_out,
                                        double *h_mass, void *stream) {
    clear_error();
    if (!idx || !d_out || !roi || !dims || !p)
        return fail(SF_ERR_INVALID_ARG, "sf_kde_grid_static: NULL argument");
    for (int k = 0; k < 3; ++k)
        if (!std::isfinite(roi->lo[k]) || !std::isfinite(roi->hi[k]) || !(roi->hi[k] > roi->lo[k]))
            return fail(SF_ERR_INVALID_ARG, "sf_kde_grid_static: roi axis %d must satisfy lo < hi", k);
    if (kernel != SF_K_EPAN && kernel != SF_K_GAUSS3)
        return fail(SF_ERR_INVALID_ARG, "sf_kde_grid_static: unknown kernel %d", kernel);
    if ((p->scope != SF_SCOPE_CLIP && p->scope != SF_SCOPE_GLOBAL) || p->prec != SF_PREC_FP32 ||
        (p->accel != SF_ACCEL_AUTO && p->accel != SF_ACCEL_NONE))
        return fail(SF_ERR_INVALID_ARG, "sf_kde_grid_static: bad scope, precision or accel field");
    float ell[3] = {0.f, 0.f, 0.f};
    int bw;
    if (p->rule == SF_BW_KNN) {
        if (idx->bw_rule != SF_BW_KNN || idx->knn_k != p->k)
            return fail(SF_ERR_INVALID_ARG, "sf_kde_grid_static: kNN bandwidths for k=%d are not built", p->k);
        bw = BW_ISO;
    } else if (p->rule == SF_BW_FIXED) {
        for (int k = 0; k < 3; ++k) {
            if (!(p->fixed_h[k] > 0.0) || !std::isfinite(p->fixed_h[k]))
                return fail(SF_ERR_INVALID_ARG, "sf_kde_grid_static: fixed_h must be positive");
            ell[k] = (float)p->fixed_h[k];
        }
        bw = BW_UNIFORM;
    } else {
        return fail(SF_ERR_INVALID_ARG,
                    "sf_kde_grid_static: rule %d not supported without allocation (kNN or fixed only)",
                    p->rule);
    }
    GridSpec g;
    for (int k = 0; k < 3; ++k) {
        if (dims[k] < 2 || dims[k] > kStaticMaxDim)
            return fail(SF_ERR_INVALID_ARG,
                        "sf_kde_grid_static: dims[%d]=%d outside [2, %d] (static scratch limit)", k,
                        dims[k], kStaticMaxDim);
        g.lo[k] = roi->lo[k];
        g.hi[k] = roi->hi[k];
        g.s[k] = (roi->hi[k] - roi->lo[k]) / (double)(dims[k] - 1);
    }
    g.nx = dims[0];
    g.ny = dims[1];
    g.nz = dims[2];
    const int64_t tiles = grid_tile_count(g);
    if (tiles > kStaticMaxTiles)
        return fail(SF_ERR_INVALID_ARG,
                    "sf_kde_grid_static: %lld node tiles exceed the static scratch limit of %lld "
                    "(at most 512^3 nodes)", (long long)tiles, (long long)kStaticMaxTiles);
    StaticScratch *S = nullptr;
    SF_TRY(static_scratch(&S));
    cudaStream_t s = (cudaStream_t)stream;
    const bool clip = p->scope == SF_SCOPE_CLIP;
    if (clip) {
        float lo[3], hi[3];
        for (int k = 0; k < 3; ++k) {
            float a = (float)roi->lo[k];
            if ((double)a < roi->lo[k]) a = nextafterf(a, INFINITY);
            float b = (float)roi->hi[k];
            if ((double)b > roi->hi[k]) b = nextafterf(b, -INFINITY);
            lo[k] = a;
            hi[k] = b;
        }
        // the count is left over from the previous call: clear it first
        SF_TRY_CUDA(cudaMemsetAsync(&S->count, 0, sizeof(unsigned long long), s));
        const unsigned gb = std::max(1u, std::min<unsigned>(blocks_for(idx->n, 256), 152 * 8));
        SF_TRY_CUDA(launch(k_count_box, dim3(gb), dim3(256), 0, s, (const float4 *)idx->pos, idx->n,
                           make_float3(lo[0], lo[1], lo[2]), make_float3(hi[0], hi[1], hi[2]),
                           &S->count));
    }
    // so is the status word
    SF_TRY_CUDA(cudaMemsetAsync(&S->status, 0, sizeof(int), s));
    SF_TRY_CUDA(launch(k_set_params, dim3(1), dim3(1), 0, s, &S->dp,
                       clip ? (const unsigned long long *)&S->count : nullptr, idx->n, ell[0],
                       ell[1], ell[2], &S->status));
    SF_TRY_CUDA(launch(k_static_axis, dim3(blocks_for(g.nx + g.ny + g.nz, 256)), dim3(256), 0, s,
                       S->axis, g.nx, g.ny, g.nz, make_double3(g.lo[0], g.lo[1], g.lo[2]),
                       make_double3(g.s[0], g.s[1], g.s[2])));
    DensityCall call;
    call.kernel = kernel;
    call.bw = bw;
    call.clip = clip ? 1 : 0;
    call.ell = nullptr;
    call.dp = &S->dp;
    call.nell_override = nullptr;
    SF_TRY(density_grid_prealloc(idx, *roi, g, call, S->axis, S->mass_part, d_out,
                                 h_mass ? &S->mass : nullptr, s));
    if (h_mass) {
        // the status is read only here, where the call synchronises anyway
        int st = 0;
        SF_TRY_CUDA(cudaMemcpyAsync(h_mass, &S->mass, sizeof(double), cudaMemcpyDeviceToHost, s));
        SF_TRY_CUDA(cudaMemcpyAsync(&st, &S->status, sizeof st, cudaMemcpyDeviceToHost, s));
        SF_TRY_CUDA(cudaStreamSynchronize(s));
        if (st == ST_EMPTY)
            return fail(SF_ERR_EMPTY_ROI, "sf_kde_grid_static: no particle of the scope lies in the ROI");
    }
    return SF_OK;
}
