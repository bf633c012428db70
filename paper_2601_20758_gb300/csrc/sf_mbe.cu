// sf_mbe.cu -- the paper's modified Breiman estimator for one ROI (Sec. 3.1,
// Algorithm 1), ahead of the final gather:
//   1. the particles of the box B and their count N_B, found through the index
//      (the points of the leaves whose bounding box meets B), so that this and
//      every later step scale with the ROI's leaves, not with the cloud;
//   2. per-axis percentiles P^(20), P^(80) of their coordinates (exact order
//      statistics by radix selection) and l_k = 2 (P80 - P20) / log N_B (Eq. 1);
//   3. pilot density at the grid nodes with the constant l (Eq. 2; Algorithm 2);
//   4. pilot density at each particle by trilinear interpolation, the mean
//      aveDen in FP64 (Eq. 5; Algorithm 3's reduction, done as deterministic
//      per-block FP64 partial sums), and l_k^(j) = min(l_k (aveDen/pDen)^(1/3),
//      cap s_k) (Eq. 6), with pDen = 0 giving the cap;
//   5. per-node maxima of l^(j) for the traversal of the final gather (Eq. 7),
//      from the leaves that meet B (every other leaf gets 0).
// Also: trilinear interpolation of a grid at the ROI points (density "at any
// position", the last step of Sec. 3.1).
#include <cmath>
#include <memory>

#include "sf_internal.cuh"

namespace sf {

struct InterpGrid {
    int nx, ny, nz;
    double lo[3], inv_s[3];
};

static InterpGrid interp_grid(const GridSpec &g) {
    InterpGrid ig;
    ig.nx = g.nx;
    ig.ny = g.ny;
    ig.nz = g.nz;
    for (int k = 0; k < 3; ++k) {
        ig.lo[k] = g.lo[k];
        ig.inv_s[k] = 1.0 / g.s[k];
    }
    return ig;
}

// The position in the grid is formed in FP64 (three subtractions and products
// per point) so that the weights carry no cancellation from large coordinates.
__device__ __forceinline__ float trilinear(const float *__restrict__ grid, const InterpGrid &g,
                                           float x, float y, float z) {
    const double u[3] = {((double)x - g.lo[0]) * g.inv_s[0], ((double)y - g.lo[1]) * g.inv_s[1],
                         ((double)z - g.lo[2]) * g.inv_s[2]};
    const int n[3] = {g.nx, g.ny, g.nz};
    int i[3];
    float t[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        int c = (int)floor(u[k]);
        c = min(max(c, 0), n[k] - 2);
        i[k] = c;
        t[k] = (float)(u[k] - (double)c);
    }
    const int64_t sx = 1, sy = g.nx, sz = (int64_t)g.nx * g.ny;
    const float *b = grid + i[2] * sz + i[1] * sy + i[0] * sx;
    const float c00 = b[0] * (1.f - t[0]) + b[1] * t[0];
    const float c10 = b[sy] * (1.f - t[0]) + b[sy + 1] * t[0];
    const float c01 = b[sz] * (1.f - t[0]) + b[sz + 1] * t[0];
    const float c11 = b[sz + sy] * (1.f - t[0]) + b[sz + sy + 1] * t[0];
    const float c0 = c00 * (1.f - t[1]) + c10 * t[1];
    const float c1 = c01 * (1.f - t[1]) + c11 * t[1];
    return c0 * (1.f - t[2]) + c1 * t[2];
}

// The piecewise-linear field of the selection volume at (x, y, z): the cell as for
// trilinear, the tetrahedron of the axis ordering with u_a >= u_b >= u_c (ties by
// the lower axis first) around the cell's main diagonal, and
// f = f0 + u_a (f1 - f0) + u_b (f2 - f1) + u_c (f3 - f2) along its corners
// 0, e_a, e_a + e_b, (1, 1, 1). FP64 throughout, one rounding at the end.
__device__ __forceinline__ float tet_linear(const float *__restrict__ grid, const InterpGrid &g,
                                            float x, float y, float z) {
    const double v[3] = {((double)x - g.lo[0]) * g.inv_s[0], ((double)y - g.lo[1]) * g.inv_s[1],
                         ((double)z - g.lo[2]) * g.inv_s[2]};
    const int n[3] = {g.nx, g.ny, g.nz};
    int c[3];
    double u[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        int ci = (int)floor(v[k]);
        ci = min(max(ci, 0), n[k] - 2);
        c[k] = ci;
        u[k] = v[k] - (double)ci;
    }
    // the axis order, descending u, ties to the lower axis
    int a = 0, b = 1, d = 2;
    if (u[b] > u[a]) { const int t = a; a = b; b = t; }
    if (u[d] > u[b]) { const int t = b; b = d; d = t; }
    if (u[b] > u[a]) { const int t = a; a = b; b = t; }
    const int64_t st[3] = {1, g.nx, (int64_t)g.nx * g.ny};
    const float *base = grid + c[2] * st[2] + c[1] * st[1] + c[0];
    const double f0 = base[0];
    const double f1 = base[st[a]];
    const double f2 = base[st[a] + st[b]];
    const double f3 = base[st[0] + st[1] + st[2]];
    return (float)(f0 + u[a] * (f1 - f0) + u[b] * (f2 - f1) + u[d] * (f3 - f2));
}

// Slot t of the listed leaves = point leaves[t / 32] * 32 + t % 32: flags[t] = 1
// when that point exists and lies in the closed box [lo, hi] (float bounds).
__global__ void k_box_flags(const float4 *__restrict__ pos, int64_t n, const int *__restrict__ leaves,
                            int64_t nslots, float3 lo, float3 hi, uint32_t *__restrict__ flags) {
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < nslots;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = (int64_t)leaves[t / kLeaf] * kLeaf + (t % kLeaf);
        uint32_t f = 0u;
        if (i < n) {
            const float4 p = pos[i];
            f = (p.x >= lo.x && p.x <= hi.x && p.y >= lo.y && p.y <= hi.y && p.z >= lo.z &&
                 p.z <= hi.z) ? 1u : 0u;
        }
        flags[t] = f;
    }
}

// The members' sorted positions at their scan positions (ascending, as the
// leaves are listed in ascending order).
__global__ void k_box_list(const uint32_t *__restrict__ flags, const uint32_t *__restrict__ pos_,
                           const int *__restrict__ leaves, int64_t nslots, uint32_t *__restrict__ list) {
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < nslots;
         t += (int64_t)gridDim.x * blockDim.x)
        if (flags[t]) list[pos_[t]] = (uint32_t)((int64_t)leaves[t / kLeaf] * kLeaf + (t % kLeaf));
}

__global__ void k_axis_keys(const float4 *__restrict__ pos, const uint32_t *__restrict__ list,
                            int64_t m, int axis, uint32_t *__restrict__ keys) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m;
         i += (int64_t)gridDim.x * blockDim.x) {
        const float4 p = pos[list[i]];
        keys[i] = float_to_ordered(axis == 0 ? p.x : (axis == 1 ? p.y : p.z));
    }
}

__global__ void k_pden(const float4 *__restrict__ pos, const uint32_t *__restrict__ list, int64_t m,
                       const float *__restrict__ pilot, InterpGrid g, float *__restrict__ pden,
                       double *__restrict__ part) {
    __shared__ double red[32];
    double acc = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m;
         i += (int64_t)gridDim.x * blockDim.x) {
        const float4 p = pos[list[i]];
        const float v = trilinear(pilot, g, p.x, p.y, p.z);
        pden[i] = v;
        acc += (double)v;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
        part[blockIdx.x] = t;
    }
}

__global__ void k_aveden(const double *__restrict__ part, int nparts, int64_t m, double *ave) {
    __shared__ double red[32];
    double t = 0.0;
    for (int i = threadIdx.x; i < nparts; i += blockDim.x) t += part[i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = t;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
        *ave = s / (double)m;
    }
}

__global__ void k_asl(const uint32_t *__restrict__ list, int64_t m, const float *__restrict__ pden,
                      const double *__restrict__ ave, float3 ell0, float3 cap,
                      float4 *__restrict__ ell) {
    const float a = (float)*ave;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m;
         i += (int64_t)gridDim.x * blockDim.x) {
        const float pd = pden[i];
        float3 l = cap;
        if (pd > 0.f) {
            const float g = cbrtf(a / pd);
            l = make_float3(fminf(ell0.x * g, cap.x), fminf(ell0.y * g, cap.y), fminf(ell0.z * g, cap.z));
        }
        ell[list[i]] = make_float4(l.x, l.y, l.z, 0.f);
    }
}

// Slot i = t * 32 + l is the point of sorted index leaves[t] * 32 + l.
// tet: the selection volume's piecewise-linear field instead of trilinear.
__global__ void k_interp(const float4 *__restrict__ pos, int64_t n, const int *__restrict__ leaves,
                         int64_t nslots, float3 lo, float3 hi, const float *__restrict__ grid,
                         InterpGrid g, int tet, float *__restrict__ rho, uint8_t *__restrict__ inroi) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nslots * kLeaf;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t j = (int64_t)leaves[i / kLeaf] * kLeaf + (i % kLeaf);
        bool in = false;
        if (j < n) {
            const float4 p = pos[j];
            in = p.x >= lo.x && p.x <= hi.x && p.y >= lo.y && p.y <= hi.y && p.z >= lo.z &&
                 p.z <= hi.z;
            if (in) rho[i] = tet ? tet_linear(grid, g, p.x, p.y, p.z) : trilinear(grid, g, p.x, p.y, p.z);
        }
        inroi[i] = in ? 1 : 0;
    }
}

static void box_bounds(const sf_box &roi, float3 &lo, float3 &hi) {
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

static unsigned sgrid(int64_t n) {
    return std::max(1u, std::min<unsigned>(blocks_for(n, 256), 152 * 16));
}

sf_status mbe_prepare(sf_index *idx, const sf_box &roi, const GridSpec &g, int kernel,
                      const sf_params &p, DensityParams *d_dp, float4 *d_ell, float4 *d_nell,
                      float *d_pilot_out, cudaStream_t s) {
    const int64_t n = idx->n;
    float3 blo, bhi;
    box_bounds(roi, blo, bhi);
    Scratch sc(s);
    // phase timers (recorded only while sf_kernel_timing_enable is on)
    auto phase = std::make_unique<KTimer>("mbe_members", s);
    // 1. members of B, through the index: the leaves whose box meets B, then their points
    int *leaves = nullptr;
    int64_t nleaf = 0;
    SF_TRY(roi_leaf_list(idx, roi, sc, &leaves, &nleaf, nullptr, s));
    const int64_t slots = nleaf * kLeaf;
    uint32_t *flags = sc.get<uint32_t>(slots);
    uint32_t *posn = sc.get<uint32_t>(slots);
    uint32_t *total = sc.get<uint32_t>(1);
    SF_TRY_SCRATCH(sc);
    SF_TRY_CUDA(launch(k_box_flags, dim3(sgrid(slots)), dim3(256), 0, s, (const float4 *)idx->pos, n,
                       (const int *)leaves, slots, blo, bhi, flags));
    SF_TRY(scan_u32(flags, posn, slots, total, s));
    uint32_t hnb = 0;
    SF_TRY_CUDA(cudaMemcpyAsync(&hnb, total, sizeof hnb, cudaMemcpyDeviceToHost, s));
    SF_TRY_CUDA(cudaStreamSynchronize(s));
    const int64_t nb = hnb;
    if (nb < 2) return fail(SF_ERR_DEGENERATE, "MBE: %lld particles in the ROI (need >= 2)", (long long)nb);
    uint32_t *list = sc.get<uint32_t>(nb);
    uint32_t *keys = sc.get<uint32_t>(nb);
    int64_t *ranks = sc.get<int64_t>(12);
    uint32_t *sel = sc.get<uint32_t>(12);
    SF_TRY_SCRATCH(sc);
    SF_TRY_CUDA(launch(k_box_list, dim3(sgrid(slots)), dim3(256), 0, s, (const uint32_t *)flags,
                       (const uint32_t *)posn, (const int *)leaves, slots, list));
    phase = std::make_unique<KTimer>("mbe_lengths", s);
    // 2. percentiles: order statistics at floor(pos) and floor(pos) + 1
    const double q[2] = {p.p_lo, p.p_hi};
    int64_t hr[12];
    double frac[2];
    int64_t ilo[2];
    for (int t = 0; t < 2; ++t) {
        const double pq = (q[t] / 100.0) * (double)(nb - 1);
        ilo[t] = (int64_t)std::floor(pq);
        frac[t] = pq - (double)ilo[t];
    }
    for (int axis = 0; axis < 3; ++axis)
        for (int t = 0; t < 2; ++t) {
            hr[axis * 4 + t * 2 + 0] = ilo[t];
            hr[axis * 4 + t * 2 + 1] = std::min<int64_t>(ilo[t] + 1, nb - 1);
        }
    SF_TRY_CUDA(cudaMemcpyAsync(ranks, hr, sizeof hr, cudaMemcpyHostToDevice, s));
    for (int axis = 0; axis < 3; ++axis) {
        SF_TRY_CUDA(launch(k_axis_keys, dim3(sgrid(nb)), dim3(256), 0, s, (const float4 *)idx->pos,
                           (const uint32_t *)list, nb, axis, keys));
        for (int r = 0; r < 4; ++r)
            SF_TRY(radix_select_u32(keys, nb, ranks + axis * 4 + r, sel + axis * 4 + r, s));
    }
    uint32_t hs[12];
    SF_TRY_CUDA(cudaMemcpyAsync(hs, sel, sizeof hs, cudaMemcpyDeviceToHost, s));
    SF_TRY_CUDA(cudaStreamSynchronize(s));
    const double lg = (p.log_base > 0.0) ? std::log((double)nb) / std::log(p.log_base)
                                         : std::log((double)nb);
    double ell0[3];
    for (int axis = 0; axis < 3; ++axis) {
        double P[2];
        for (int t = 0; t < 2; ++t) {
            const double v0 = (double)ordered_to_float(hs[axis * 4 + t * 2 + 0]);
            const double v1 = (double)ordered_to_float(hs[axis * 4 + t * 2 + 1]);
            P[t] = (ilo[t] + 1 >= nb) ? v0 : v0 + frac[t] * (v1 - v0);
        }
        ell0[axis] = 2.0 * (P[1] - P[0]) / lg;
        if (!(ell0[axis] > 0.0))
            return fail(SF_ERR_DEGENERATE, "MBE: percentile spread is zero on axis %d", axis);
    }
    phase = std::make_unique<KTimer>("mbe_pilot", s);
    // 3. pilot density with the constant l (Eq. 2), clip scope
    const int64_t G = (int64_t)g.nx * g.ny * g.nz;
    float *pilot = d_pilot_out ? d_pilot_out : sc.get<float>(G);
    SF_TRY_SCRATCH(sc);
    const float ellf[3] = {(float)ell0[0], (float)ell0[1], (float)ell0[2]};
    // N_B >= 2 here, so the scope is never empty: no status word is needed
    SF_TRY(set_density_params(idx, true, roi, ellf, d_dp, nullptr, s));
    DensityCall pc;
    pc.kernel = kernel;
    pc.bw = BW_UNIFORM;
    pc.clip = 1;
    pc.ell = nullptr;
    pc.dp = d_dp;
    pc.nell_override = nullptr;
    pc.accel = p.accel;  // Epanechnikov: the pilot's one length makes it a moment sum
    SF_TRY(density_grid(idx, roi, g, pc, pilot, nullptr, s));
    phase = std::make_unique<KTimer>("mbe_asl", s);
    // 4. pilot at the particles, aveDen, adaptive lengths
    const InterpGrid ig = interp_grid(g);
    const unsigned gb = sgrid(nb);
    float *pden = sc.get<float>(nb);
    double *part = sc.get<double>(gb);
    double *ave = sc.get<double>(1);
    SF_TRY_SCRATCH(sc);
    SF_TRY_CUDA(launch(k_pden, dim3(gb), dim3(256), 0, s, (const float4 *)idx->pos,
                       (const uint32_t *)list, nb, (const float *)pilot, ig, pden, part));
    SF_TRY_CUDA(launch(k_aveden, dim3(1), dim3(1024), 0, s, (const double *)part, (int)gb, nb, ave));
    const float3 l0 = make_float3(ellf[0], ellf[1], ellf[2]);
    const float3 cap = make_float3((float)(p.cap_factor * g.s[0]), (float)(p.cap_factor * g.s[1]),
                                   (float)(p.cap_factor * g.s[2]));
    SF_TRY_CUDA(launch(k_asl, dim3(gb), dim3(256), 0, s, (const uint32_t *)list, nb,
                       (const float *)pden, (const double *)ave, l0, cap, d_ell));
    // 5. node maxima over the members
    phase = std::make_unique<KTimer>("mbe_node_ell", s);
    SF_TRY(build_node_ell(idx, BW_ANISO, d_ell, &roi, d_nell, s, leaves, nleaf));
    return SF_OK;
}

sf_status interp_points(sf_index *idx, const sf_box &roi, const GridSpec &g, const float *d_grid,
                        const int *d_leaves, int64_t nslots, float *d_rho_sorted, uint8_t *d_inroi,
                        cudaStream_t s, int tet) {
    float3 lo, hi;
    box_bounds(roi, lo, hi);
    SF_TRY_CUDA(launch(k_interp, dim3(sgrid(nslots * kLeaf)), dim3(256), 0, s,
                       (const float4 *)idx->pos, idx->n, d_leaves, nslots, lo, hi, d_grid,
                       interp_grid(g), tet, d_rho_sorted, d_inroi));
    return SF_OK;
}

}  // namespace sf
