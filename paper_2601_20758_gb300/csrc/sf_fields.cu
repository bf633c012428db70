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

// ---------------------------------------------------------------------------
// Selection volume boundary (sf_iso_surface)
// ---------------------------------------------------------------------------
namespace sf {

namespace {

struct IsoGrid {
    int n[3];
    double lo[3], s[3];
    double t;
};

// Corner c (0..3) of the tetrahedron of ordering o (0..5), as 0/1 offsets in a bitmask
// x | y << 1 | z << 2: corners 0, e_a, e_a + e_b, (1,1,1) for the orderings
// (x,y,z), (x,z,y), (y,x,z), (y,z,x), (z,x,y), (z,y,x).
__device__ __forceinline__ int tet_corner(int o, int c) {
    const int a = o >> 1;                                            // first axis: 0,0,1,1,2,2
    const int b = (o == 0 || o == 5) ? 1 : ((o == 1 || o == 3) ? 2 : 0);  // second axis
    if (c == 0) return 0;
    if (c == 1) return 1 << a;
    if (c == 2) return (1 << a) | (1 << b);
    return 7;
}

// Triangles of one tetrahedron: 0, 1 or 2 (count only when out == nullptr).
__device__ int tet_triangles(const IsoGrid &G, const float *__restrict__ grid, int cx, int cy, int cz,
                             int o, float *out) {
    double P[4][3], f[4];
    bool in[4];
    int nin = 0;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        const int m = tet_corner(o, c);
        const int ix = cx + (m & 1), iy = cy + ((m >> 1) & 1), iz = cz + (m >> 2);
        f[c] = (double)grid[((int64_t)iz * G.n[1] + iy) * G.n[0] + ix];
        P[c][0] = G.lo[0] + (double)ix * G.s[0];
        P[c][1] = G.lo[1] + (double)iy * G.s[1];
        P[c][2] = G.lo[2] + (double)iz * G.s[2];
        in[c] = f[c] > G.t;
        nin += in[c];
    }
    if (nin == 0 || nin == 4) return 0;
    const int ntri = nin == 2 ? 2 : 1;
    if (!out) return ntri;
    auto cross = [&](int a, int b, double *r) {
        const double w = (G.t - f[a]) / (f[b] - f[a]);
#pragma unroll
        for (int k = 0; k < 3; ++k) r[k] = P[a][k] + w * (P[b][k] - P[a][k]);
    };
    double cen[3] = {0.0, 0.0, 0.0};
#pragma unroll
    for (int c = 0; c < 4; ++c)
        if (in[c])
#pragma unroll
            for (int k = 0; k < 3; ++k) cen[k] += P[c][k];
#pragma unroll
    for (int k = 0; k < 3; ++k) cen[k] /= (double)nin;
    double V[2][3][3];
    if (ntri == 1) {
        int lone = -1;
#pragma unroll
        for (int c = 0; c < 4; ++c)
            if (in[c] == (nin == 1)) lone = c;   // the corner on its own side
        int j = 0;
#pragma unroll
        for (int c = 0; c < 4; ++c)
            if (c != lone) cross(lone, c, V[0][j++]);
    } else {
        int I = -1, J = -1, K = -1, Lc = -1;
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            if (in[c]) {
                if (I < 0) I = c; else J = c;
            } else {
                if (K < 0) K = c; else Lc = c;
            }
        }
        cross(I, K, V[0][0]);
        cross(I, Lc, V[0][1]);
        cross(J, Lc, V[0][2]);
        cross(I, K, V[1][0]);
        cross(J, Lc, V[1][1]);
        cross(J, K, V[1][2]);
    }
    for (int q = 0; q < ntri; ++q) {
        double *a = V[q][0], *b = V[q][1], *c = V[q][2];
        const double e1[3] = {b[0] - a[0], b[1] - a[1], b[2] - a[2]};
        const double e2[3] = {c[0] - a[0], c[1] - a[1], c[2] - a[2]};
        const double n[3] = {e1[1] * e2[2] - e1[2] * e2[1], e1[2] * e2[0] - e1[0] * e2[2],
                             e1[0] * e2[1] - e1[1] * e2[0]};
        const double dn = n[0] * (a[0] - cen[0]) + n[1] * (a[1] - cen[1]) + n[2] * (a[2] - cen[2]);
        const int ib = dn < 0.0 ? 2 : 1, ic = dn < 0.0 ? 1 : 2;   // toward the inside: flip
        float *w = out + 9 * q;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            w[k] = (float)a[k];
            w[3 + k] = (float)V[q][ib][k];
            w[6 + k] = (float)V[q][ic][k];
        }
    }
    return ntri;
}

// One thread per cell: its triangle count (pass 1) or its triangles at off[cell] (pass 2).
template <bool EMIT>
__global__ void k_iso(const float *__restrict__ grid, IsoGrid G, uint32_t *__restrict__ cnt,
                      const uint32_t *__restrict__ off, float *__restrict__ tris) {
    const int64_t nc = (int64_t)(G.n[0] - 1) * (G.n[1] - 1) * (G.n[2] - 1);
    for (int64_t cell = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; cell < nc;
         cell += (int64_t)gridDim.x * blockDim.x) {
        const int cx = (int)(cell % (G.n[0] - 1));
        const int cy = (int)((cell / (G.n[0] - 1)) % (G.n[1] - 1));
        const int cz = (int)(cell / ((int64_t)(G.n[0] - 1) * (G.n[1] - 1)));
        if (!EMIT) {
            uint32_t t = 0;
            for (int o = 0; o < 6; ++o) t += (uint32_t)tet_triangles(G, grid, cx, cy, cz, o, nullptr);
            cnt[cell] = t;
        } else {
            float *w = tris + 9 * (int64_t)off[cell];
            for (int o = 0; o < 6; ++o) w += 9 * tet_triangles(G, grid, cx, cy, cz, o, w);
        }
    }
}

}  // namespace

}  // namespace sf

extern "C" sf_status sf_iso_surface(const float *d_grid, const sf_box *roi, const int32_t dims[3],
                                    double threshold, float *d_tris, int64_t capacity, int64_t *h_ntri,
                                    void *stream) {
    clear_error();
    if (!d_grid || !roi || !dims || !h_ntri) return fail(SF_ERR_INVALID_ARG, "sf_iso_surface: NULL argument");
    if (!std::isfinite(threshold)) return fail(SF_ERR_INVALID_ARG, "sf_iso_surface: threshold must be finite");
    if (capacity < 0 || (capacity > 0 && !d_tris))
        return fail(SF_ERR_INVALID_ARG, "sf_iso_surface: bad capacity / output");
    IsoGrid G;
    for (int k = 0; k < 3; ++k) {
        if (!std::isfinite(roi->lo[k]) || !std::isfinite(roi->hi[k]) || !(roi->hi[k] > roi->lo[k]))
            return fail(SF_ERR_INVALID_ARG, "sf_iso_surface: roi axis %d must satisfy lo < hi", k);
        if (dims[k] < 2 || dims[k] > 4096)
            return fail(SF_ERR_INVALID_ARG, "sf_iso_surface: dims[%d] outside [2, 4096]", k);
        G.n[k] = dims[k];
        G.lo[k] = roi->lo[k];
        G.s[k] = (roi->hi[k] - roi->lo[k]) / (double)(dims[k] - 1);
    }
    G.t = threshold;
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t nc = (int64_t)(G.n[0] - 1) * (G.n[1] - 1) * (G.n[2] - 1);
    Scratch sc(s);
    uint32_t *cnt = sc.get<uint32_t>(nc);
    uint32_t *off = sc.get<uint32_t>(nc);
    uint32_t *tot = sc.get<uint32_t>(1);
    SF_TRY_SCRATCH(sc);
    const unsigned blocks = (unsigned)std::max<int64_t>(1, std::min<int64_t>((nc + 255) / 256, 152 * 16));
    SF_TRY_CUDA(launch(k_iso<false>, dim3(blocks), dim3(256), 0, s, d_grid, G, cnt,
                       (const uint32_t *)nullptr, (float *)nullptr));
    SF_TRY(scan_u32(cnt, off, nc, tot, s));
    uint32_t h = 0;
    SF_TRY_CUDA(cudaMemcpyAsync(&h, tot, sizeof h, cudaMemcpyDeviceToHost, s));
    SF_TRY_CUDA(cudaStreamSynchronize(s));
    *h_ntri = h;
    if ((int64_t)h > capacity) {
        if (capacity == 0 && !d_tris) return SF_OK;   // counting only
        return fail(SF_ERR_CAPACITY, "sf_iso_surface: %u triangles exceed capacity %lld", h, (long long)capacity);
    }
    if (h > 0)
        SF_TRY_CUDA(launch(k_iso<true>, dim3(blocks), dim3(256), 0, s, d_grid, G, (uint32_t *)nullptr,
                           (const uint32_t *)off, d_tris));
    return SF_OK;
}
