// sf_fields.cu -- a density grid sampled at the nodes of another grid by
// trilinear interpolation (Sec. 3.1: the density at any position inside B from
// the eight nodes around it), scaled and optionally added to the destination.
//
// This serves the consumers of finished grids rather than the estimator: a
// view cache that answers a small pan or zoom from a grid computed over a
// larger box, and the precomputed-field conditions of the paper's study
// (Sec. 5: one fixed 64^3 field, or 64^3 and 128^3 fields blended by the
// scale), which read a global field at the nodes of the current view.
//
// One thread per destination node; the node's position and its cell in the
// source grid are computed in FP64 (the source grid's node coordinates as
// lo + i s, like every grid of the library), the eight-point weighted sum in
// FP64, one rounding to float at the end.
#include <cmath>

#include "sf_internal.cuh"

namespace sf {

namespace {

struct Axes {
    double lo[3], s[3], inv[3];  // source: origin, spacing, 1 / spacing
    int n[3];                    // source nodes per axis
    double dlo[3], ds[3];        // destination: origin and spacing
    int dn[3];                   // destination nodes per axis
    double blo[3], bhi[3];       // the source box (closed)
};

__global__ void k_resample(const float *__restrict__ src, Axes A, float weight, int accumulate,
                           float *__restrict__ dst, unsigned long long *outside) {
    const int64_t total = (int64_t)A.dn[0] * A.dn[1] * A.dn[2];
    unsigned long long out_cnt = 0;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t ix = t % A.dn[0], iy = (t / A.dn[0]) % A.dn[1], iz = t / ((int64_t)A.dn[0] * A.dn[1]);
        const int64_t id[3] = {ix, iy, iz};
        double u[3];
        int c[3];
        bool in = true;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const double r = __dadd_rn(A.dlo[k], __dmul_rn((double)id[k], A.ds[k]));
            in = in && r >= A.blo[k] && r <= A.bhi[k];
            const double v = (r - A.lo[k]) * A.inv[k];
            int ci = (int)floor(v);
            ci = ci < 0 ? 0 : (ci > A.n[k] - 2 ? A.n[k] - 2 : ci);
            c[k] = ci;
            u[k] = v - (double)ci;
        }
        double val = 0.0;
        if (in) {
#pragma unroll
            for (int dz = 0; dz < 2; ++dz)
#pragma unroll
                for (int dy = 0; dy < 2; ++dy)
#pragma unroll
                    for (int dx = 0; dx < 2; ++dx) {
                        const double w = (dx ? u[0] : 1.0 - u[0]) * (dy ? u[1] : 1.0 - u[1]) *
                                         (dz ? u[2] : 1.0 - u[2]);
                        const int64_t o = ((int64_t)(c[2] + dz) * A.n[1] + (c[1] + dy)) * A.n[0] + (c[0] + dx);
                        val += w * (double)__ldg(&src[o]);
                    }
        } else {
            ++out_cnt;
        }
        const float res = (float)((double)weight * val);
        dst[t] = accumulate ? dst[t] + res : res;
    }
    if (outside) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) out_cnt += __shfl_xor_sync(0xffffffffu, out_cnt, o);
        if ((threadIdx.x & 31) == 0 && out_cnt) atomicAdd(outside, out_cnt);
    }
}

}  // namespace

}  // namespace sf

using namespace sf;

extern "C" sf_status sf_resample_grid(const float *d_src, const sf_box *src_box, const int32_t src_dims[3],
                                      const sf_box *dst_box, const int32_t dst_dims[3], float weight,
                                      int32_t accumulate, float *d_dst, int64_t *h_outside,
                                      void *stream) {
    clear_error();
    if (!d_src || !src_box || !src_dims || !dst_box || !dst_dims || !d_dst)
        return fail(SF_ERR_INVALID_ARG, "sf_resample_grid: NULL argument");
    if (!std::isfinite(weight)) return fail(SF_ERR_INVALID_ARG, "sf_resample_grid: weight must be finite");
    Axes A;
    for (int k = 0; k < 3; ++k) {
        const double lo = src_box->lo[k], hi = src_box->hi[k], dlo = dst_box->lo[k], dhi = dst_box->hi[k];
        if (!std::isfinite(lo) || !std::isfinite(hi) || !(hi > lo) || !std::isfinite(dlo) ||
            !std::isfinite(dhi) || !(dhi > dlo))
            return fail(SF_ERR_INVALID_ARG, "sf_resample_grid: axis %d boxes must satisfy lo < hi", k);
        if (src_dims[k] < 2 || src_dims[k] > 4096 || dst_dims[k] < 2 || dst_dims[k] > 4096)
            return fail(SF_ERR_INVALID_ARG, "sf_resample_grid: dims[%d] outside [2, 4096]", k);
        A.lo[k] = lo;
        A.n[k] = src_dims[k];
        A.s[k] = (hi - lo) / (double)(src_dims[k] - 1);
        A.inv[k] = 1.0 / A.s[k];
        A.dlo[k] = dlo;
        A.dn[k] = dst_dims[k];
        A.ds[k] = (dhi - dlo) / (double)(dst_dims[k] - 1);
        A.blo[k] = lo;
        A.bhi[k] = hi;
    }
    cudaStream_t s = (cudaStream_t)stream;
    Scratch sc(s);
    unsigned long long *cnt = nullptr;
    if (h_outside) {
        cnt = sc.get<unsigned long long>(1);
        SF_TRY_SCRATCH(sc);
        SF_TRY_CUDA(cudaMemsetAsync(cnt, 0, sizeof *cnt, s));
    }
    const int64_t total = (int64_t)A.dn[0] * A.dn[1] * A.dn[2];
    const unsigned blocks = (unsigned)std::max<int64_t>(1, std::min<int64_t>((total + 255) / 256, 152 * 16));
    SF_TRY_CUDA(launch(k_resample, dim3(blocks), dim3(256), 0, s, d_src, A, weight, accumulate ? 1 : 0,
                       d_dst, cnt));
    if (h_outside) {
        unsigned long long h = 0;
        SF_TRY_CUDA(cudaMemcpyAsync(&h, cnt, sizeof h, cudaMemcpyDeviceToHost, s));
        SF_TRY_CUDA(cudaStreamSynchronize(s));
        *h_outside = (int64_t)h;
    }
    return SF_OK;
}
