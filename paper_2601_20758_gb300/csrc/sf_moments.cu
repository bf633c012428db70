// sf_moments.cu -- exact moment form of the Epanechnikov sum for particles
// that share one smoothing length per axis (rule FIXED, and the pilot density
// of the paper's estimator, Eq. 2).
//
// Inside its support the Epanechnikov kernel (Eq. 4) is a quadratic polynomial
// of the offset. For a grid node r and a set P of particles that all lie
// strictly inside r's support,
//     sum_{j in P} (1 - sum_k (r_k - y_jk)^2 / l_k^2)
//       = M0 - sum_k (M0 (r_k - mu_k)^2 + C_k) / l_k^2,
// with M0 = |P|, mu its centroid and C_k = sum_j (y_jk - mu_k)^2: the offsets
// e_j = y_j - mu sum to zero, so sum_j (d - e_j)^2 = M0 d^2 + sum_j e_j^2 with
// no cancellation between the terms. Every index node carries (M0, mu, C).
//
// The grid kernel gives each warp a 2 x 2 x 2 block of grid nodes and walks
// the index once for the block, testing each node three ways: out of reach of
// all 8 grid nodes (skipped); wholly inside the support of all 8 (and, with
// the clip scope, inside the ROI box): its moments are added, one lane per
// node; otherwise it is descended, and the leaves met this way are summed
// point by point, one point per lane against the 8 grid nodes. The walk order
// is fixed, each lane adds its terms in that order (FP32 terms, FP32 partial
// sums folded every 32 steps into a compensated (hi, lo) FP32 pair, about 48
// significant bits) and the lanes are combined by a fixed shuffle tree, so the
// result is deterministic. FP64 is kept out of the loops: its rate on this GPU
// is a small fraction of FP32's.
//
// Why blocks of 2 x 2 x 2: a node can take the moment form only if it lies
// inside the support of every grid node its warp serves, so the straddling
// shell, summed point by point, is as thick as the block plus a leaf. With
// the pilot's lengths (about 10 to 30 node spacings at 256^3) an 8 x 4 x 8
// tile would leave only about a tenth of the support to the moments. Even so
// the shell (thickness ~ block + leaf, relative volume ~ 3 x thickness / l)
// holds most pairs unless l spans many leaf widths, and each block pays its
// own walk, so the tile gather is faster wherever it can run; this form has no
// candidate lists and takes the grids whose lists would not fit.
#include <cmath>
#include <vector>

#include "sf_internal.cuh"

namespace sf {

// --------------------------------------------------------------------------
// Moments of the index nodes
// --------------------------------------------------------------------------
// s = a + b rounded, e = the exact error (a + b = s + e; Knuth's two-sum, no
// ordering of |a| and |b| needed).
__device__ __forceinline__ float two_sum(float a, float b, float &e) {
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return s;
}

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ void store_moments(float4 *mom, int64_t g, double m, const double mu[3],
                                              const double c[3]) {
    float h[3], l[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        h[k] = (float)mu[k];
        l[k] = (float)(mu[k] - (double)h[k]);
    }
    mom[3 * g + 0] = make_float4(h[0], h[1], h[2], (float)m);
    mom[3 * g + 1] = make_float4(l[0], l[1], l[2], 0.f);
    mom[3 * g + 2] = make_float4((float)c[0], (float)c[1], (float)c[2], 0.f);
}

__device__ __forceinline__ float warp_sum_f(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// One warp per leaf: count, centroid and central second moments, two passes over
// the offsets e = y - y0 from the leaf's first point (FP32: the offsets are as
// small as the leaf, so their sums keep about 24 bits relative to the leaf's
// size); the centroid y0 + mean(e) is kept as the exact float pair of a two-sum.
// No FP64: its rate on this GPU is a small fraction of FP32's, and even one
// lane's FP64 instructions hold the pipe for a whole warp's worth of cycles.
__global__ void k_mom_leaf(const float4 *__restrict__ pos, int64_t n, int64_t nleaf,
                           float4 *__restrict__ mom) {
    const int lane = threadIdx.x & 31;
    const int64_t leaf = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (leaf >= nleaf) return;
    const int64_t i = leaf * kLeaf + lane;
    const bool v = i < n;
    const float4 p0 = pos[leaf * kLeaf];
    float e[3] = {0.f, 0.f, 0.f};
    if (v) {
        const float4 p = pos[i];
        e[0] = p.x - p0.x;
        e[1] = p.y - p0.y;
        e[2] = p.z - p0.z;
    }
    const int m = __popc(__ballot_sync(0xffffffffu, v));
    float eb[3], c[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) eb[k] = warp_sum_f(e[k]) / (float)m;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const float d = v ? e[k] - eb[k] : 0.f;
        c[k] = warp_sum_f(d * d);
    }
    if (lane == 0) {  // centroid p0 + mean(e) as an exact (hi, lo) float pair: no FP64
        const float y0[3] = {p0.x, p0.y, p0.z};
        float h[3], l[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) h[k] = two_sum(y0[k], eb[k], l[k]);
        mom[3 * leaf + 0] = make_float4(h[0], h[1], h[2], (float)m);
        mom[3 * leaf + 1] = make_float4(l[0], l[1], l[2], 0.f);
        mom[3 * leaf + 2] = make_float4(c[0], c[1], c[2], 0.f);
    }
}

// One warp per inner node, one lane per child: M = sum M_c, mu = sum M_c mu_c / M,
// C = sum (C_c + M_c (mu_c - mu)^2) (parallel-axis identity, all terms >= 0).
// The counts are exact: node i of level L (leaves: L = 0) holds
// min(32^(L+1), n - i 32^(L+1)) points.
__global__ void k_mom_inner(float4 *__restrict__ mom, int64_t n, int level, int64_t child_off,
                            int64_t child_cnt, int64_t off, int64_t cnt) {
    const int lane = threadIdx.x & 31;
    const int64_t node = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (node >= cnt) return;
    const int64_t c = node * kFanout + lane;
    const bool v = c < child_cnt;
    const int64_t span = (int64_t)1 << (5 * level);  // points under a full child (32^level)
    double m = 0.0, mu[3] = {0.0, 0.0, 0.0}, cc[3] = {0.0, 0.0, 0.0};
    if (v) {
        m = (double)min(span, n - c * span);
        const float4 a = mom[3 * (child_off + c) + 0];
        const float4 b = mom[3 * (child_off + c) + 1];
        const float4 q = mom[3 * (child_off + c) + 2];
        mu[0] = (double)a.x + (double)b.x;
        mu[1] = (double)a.y + (double)b.y;
        mu[2] = (double)a.z + (double)b.z;
        cc[0] = q.x;
        cc[1] = q.y;
        cc[2] = q.z;
    }
    const double M = warp_sum_d(m);
    double MU[3], C[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) MU[k] = warp_sum_d(m * mu[k]) / M;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const double d = mu[k] - MU[k];
        C[k] = warp_sum_d(v ? cc[k] + m * d * d : 0.0);
    }
    if (lane == 0) store_moments(mom, off + node, M, MU, C);
}

sf_status build_moments(sf_index *idx, cudaStream_t s) {
    SF_TRY_CUDA(launch(k_mom_leaf, dim3(blocks_for(idx->cnt[0] * 32, 256)), dim3(256), 0, s,
                       (const float4 *)idx->pos, idx->n, idx->cnt[0], idx->mom));
    for (int l = 1; l < idx->nlevels; ++l)
        SF_TRY_CUDA(launch(k_mom_inner, dim3(blocks_for(idx->cnt[l] * 32, 256)), dim3(256), 0, s,
                           idx->mom, idx->n, l, idx->off[l - 1], idx->cnt[l - 1], idx->off[l],
                           idx->cnt[l]));
    return SF_OK;
}

// --------------------------------------------------------------------------
// Grid by moments
// --------------------------------------------------------------------------
constexpr int kMomWarps = 8;
constexpr int kMomFlush = 32;       // FP32 partial sums are folded every 32 steps
constexpr int kMomStack = 32 * kMaxLevels;
constexpr int kMomLeaves = 64;      // straddling leaves gathered before they are summed
// A node takes the moment form only if its largest q over the block is below
// 1 - kFullSlack: every pair it stands for is then inside the support by a
// margin far beyond the rounding of q (and of the oracle's own test).
constexpr float kFullSlack = 1.0e-4f;

struct MomArgs {
    TreeView tv;
    const float4 *mom;
    const DensityParams *dp;
    const float2 *axis;  // node coordinates as (hi, lo): x[nx], y[ny], z[nz]
    int nx, ny, nz;
    int bx, by, bz;      // 2 x 2 x 2 blocks per axis
    float *out;
    double *mass_part;   // per block
    float cnorm;
    float blo[3], bhi[3];  // clip box (float bounds of the closed double box)
};

struct MomWarpSmem {
    int stack[kMomStack];
    int leaves[kMomLeaves];
};

// 0: no point of node g reaches the block; 2: every point of g lies inside the
// support of every node of the block (and inside the clip box); 1: otherwise.
template <bool CLIP>
__device__ __forceinline__ int mom_classify(const MomArgs &a, int64_t g, const float wlo[3],
                                            const float whi[3], const float rl[3]) {
    const float4 lo = __ldg(&a.tv.nlo[g]);
    const float4 hi = __ldg(&a.tv.nhi[g]);
    const float nl[3] = {lo.x, lo.y, lo.z}, nh[3] = {hi.x, hi.y, hi.z};
    bool inside = true;
    if (CLIP) {
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            if (nl[k] > a.bhi[k] || nh[k] < a.blo[k]) return 0;
            inside = inside && nl[k] >= a.blo[k] && nh[k] <= a.bhi[k];
        }
    }
    float qmin = 0.f, qmax = 0.f;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const float gap = fmaxf(fmaxf(nl[k] - whi[k], wlo[k] - nh[k]), 0.f);
        const float far = fmaxf(whi[k] - nl[k], nh[k] - wlo[k]);
        const float t = gap * rl[k], u = far * rl[k];
        qmin = fmaf(t, t, qmin);
        qmax = fmaf(u, u, qmax);
    }
    if (!(qmin < 1.0f + kFilterSlack)) return 0;
    return (inside && qmax < 1.0f - kFullSlack) ? 2 : 1;
}

template <bool CLIP>
__global__ void __launch_bounds__(kMomWarps * 32) k_mom_grid(MomArgs a) {
    __shared__ MomWarpSmem W[kMomWarps];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const unsigned lt = (1u << lane) - 1u;
    const int64_t blk = (int64_t)blockIdx.x * kMomWarps + warp;
    if (blk >= (int64_t)a.bx * a.by * a.bz) return;
    MomWarpSmem &S = W[warp];
    const int bi[3] = {(int)(blk % a.bx), (int)((blk / a.bx) % a.by),
                       (int)(blk / ((int64_t)a.bx * a.by))};
    const int nd[3] = {a.nx, a.ny, a.nz};
    const int aoff[3] = {0, a.nx, a.nx + a.ny};
    int g0[3], nv[3];
    float rh[3][2], rlo[3][2], tlo[3], thi[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        g0[k] = 2 * bi[k];
        nv[k] = min(2, nd[k] - g0[k]);
#pragma unroll
        for (int t = 0; t < 2; ++t) {
            const float2 v = a.axis[aoff[k] + g0[k] + min(t, nv[k] - 1)];
            rh[k][t] = v.x;
            rlo[k][t] = v.y;
        }
        tlo[k] = rh[k][0];
        thi[k] = rh[k][1];
    }
    float wlo[3], whi[3];
    widen_box(tlo, thi, wlo, whi);
    const DensityParams dp = *a.dp;
    float rl[3], rl2[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        rl[k] = rcp_approx(dp.ell_uniform[k]);
        rl2[k] = rl[k] * rl[k];
    }
    const float c = a.cnorm * ((rl[0] * rl[1]) * rl[2]);

    // acc: the current partial sums; (hi, lo): the compensated running sums
    float acc[8], hi[8], lo[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) acc[j] = hi[j] = lo[j] = 0.f;
    int steps = 0;
    auto fold = [&]() {
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            float e;
            hi[j] = two_sum(hi[j], acc[j], e);
            lo[j] += e;
            acc[j] = 0.f;
        }
        steps = 0;
    };

    // the walk starts from a virtual entry whose only child is the root
    const int top = a.tv.nlevels - 1;
    int sp = 1, nl = 0;
    if (lane == 0) S.stack[0] = (top + 1) << 27;
    __syncwarp();
    while (true) {
        if (sp > 0 && nl <= kMomLeaves - 32) {
            const int e = S.stack[sp - 1];
            __syncwarp();
            sp -= 1;
            const int cl = (e >> 27) - 1;
            const int64_t ci = (int64_t)(e & ((1 << 27) - 1)) * kFanout + lane;
            int state = 0;
            if (ci < a.tv.cnt[cl]) {
                const int64_t g = a.tv.off[cl] + ci;
                state = mom_classify<CLIP>(a, g, wlo, whi, rl);
                if (state == 2) {
                    const float4 m0 = __ldg(&a.mom[3 * g + 0]);
                    const float4 m1 = __ldg(&a.mom[3 * g + 1]);
                    const float4 m2 = __ldg(&a.mom[3 * g + 2]);
                    const float M = m0.w;
                    const float mh[3] = {m0.x, m0.y, m0.z}, ml[3] = {m1.x, m1.y, m1.z};
                    const float C[3] = {m2.x, m2.y, m2.z};
                    float q[3][2];
#pragma unroll
                    for (int k = 0; k < 3; ++k)
#pragma unroll
                        for (int t = 0; t < 2; ++t) {
                            const float d = (rh[k][t] - mh[k]) + (rlo[k][t] - ml[k]);
                            q[k][t] = fmaf(M * d, d, C[k]) * rl2[k];
                        }
#pragma unroll
                    for (int j = 0; j < 8; ++j)
                        acc[j] = fmaf(c, M - ((q[0][j & 1] + q[1][(j >> 1) & 1]) + q[2][j >> 2]), acc[j]);
                }
            }
            const unsigned m = __ballot_sync(0xffffffffu, state == 1);
            const int r = __popc(m & lt), k = __popc(m);
            if (cl == 0) {
                if (state == 1) S.leaves[nl + r] = (int)ci;
                nl += k;
            } else {
                if (state == 1) S.stack[sp + (k - 1 - r)] = (cl << 27) | (int)ci;
                sp += k;
            }
            __syncwarp();
            if (++steps >= kMomFlush) fold();
        } else if (nl > 0) {
            for (int t = 0; t < nl; ++t) {
                const int64_t i = (int64_t)S.leaves[t] * kLeaf + lane;
                if (i < a.tv.n) {
                    const float4 p = __ldg(&a.tv.pos[i]);
                    bool in = true;
                    if (CLIP)
                        in = p.x >= a.blo[0] && p.x <= a.bhi[0] && p.y >= a.blo[1] &&
                             p.y <= a.bhi[1] && p.z >= a.blo[2] && p.z <= a.bhi[2];
                    if (in) {
                        const float y[3] = {p.x, p.y, p.z};
                        float q[3][2];
#pragma unroll
                        for (int k = 0; k < 3; ++k)
#pragma unroll
                            for (int tt = 0; tt < 2; ++tt) {
                                const float u = ((rh[k][tt] - y[k]) + rlo[k][tt]) * rl[k];
                                q[k][tt] = u * u;
                            }
#pragma unroll
                        for (int j = 0; j < 8; ++j) {
                            const float qq = (q[0][j & 1] + q[1][(j >> 1) & 1]) + q[2][j >> 2];
                            if (qq < 1.0f) acc[j] = fmaf(c, 1.0f - qq, acc[j]);
                        }
                    }
                }
                if (++steps >= kMomFlush) fold();
            }
            __syncwarp();
            nl = 0;
        } else {
            break;
        }
    }
    fold();
    // lanes combined by a fixed xor tree of compensated sums; lane j < 8 then
    // scales node j of the block (the only FP64 arithmetic of the kernel)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const float h2 = __shfl_xor_sync(0xffffffffu, hi[j], o);
            const float l2 = __shfl_xor_sync(0xffffffffu, lo[j], o);
            float e;
            hi[j] = two_sum(hi[j], h2, e);
            lo[j] += l2 + e;
        }
    }
    float mh = hi[0], ml = lo[0];
#pragma unroll
    for (int j = 1; j < 8; ++j)
        if (lane == j) {
            mh = hi[j];
            ml = lo[j];
        }
    const int ox = lane & 1, oy = (lane >> 1) & 1, oz = (lane >> 2) & 1;
    const bool mine = lane < 8 && ox < nv[0] && oy < nv[1] && oz < nv[2];
    const float fv = (float)(((double)mh + (double)ml) * dp.inv_neff);
    if (mine) a.out[((int64_t)(g0[2] + oz) * a.ny + (g0[1] + oy)) * a.nx + (g0[0] + ox)] = fv;
    const double msum = warp_sum_d(mine ? (double)fv : 0.0);
    if (lane == 0 && a.mass_part) a.mass_part[blk] = msum;
}

sf_status density_grid_moments(sf_index *idx, const sf_box &roi, const GridSpec &g,
                               const DensityCall &call, float *d_out, double *d_mass,
                               cudaStream_t s, int64_t *ws_bytes, StatusPeek *peek) {
    if (!idx->mom) return fail(SF_ERR_INVALID_ARG, "grid by moments: the index has no moments");
    std::vector<float2> ax((size_t)g.nx + g.ny + g.nz);
    node_axes(g, ax.data());
    const int bx = (g.nx + 1) / 2, by = (g.ny + 1) / 2, bz = (g.nz + 1) / 2;
    const int64_t nblk = (int64_t)bx * by * bz;
    if (ws_bytes) {
        *ws_bytes = scratch_round((int64_t)sizeof(float2) * (int64_t)ax.size()) +
                    (d_mass ? scratch_round(8 * nblk) : 0);
        return SF_OK;
    }
    Scratch sc(s);
    float2 *d_axis = sc.get<float2>((int64_t)ax.size());
    double *mass_part = d_mass ? sc.get<double>(nblk) : nullptr;
    SF_TRY_SCRATCH(sc);
    SF_TRY_CUDA(cudaMemcpyAsync(d_axis, ax.data(), ax.size() * sizeof(float2),
                                cudaMemcpyHostToDevice, s));
    if (peek && peek->d_src) {  // the call's status, read at its one synchronisation
        SF_TRY_CUDA(cudaMemcpyAsync(&peek->value, peek->d_src, sizeof(int), cudaMemcpyDeviceToHost, s));
        SF_TRY_CUDA(cudaStreamSynchronize(s));
    }
    MomArgs a;
    a.tv = idx->view();
    a.mom = idx->mom;
    a.dp = call.dp;
    a.axis = d_axis;
    a.nx = g.nx;
    a.ny = g.ny;
    a.nz = g.nz;
    a.bx = bx;
    a.by = by;
    a.bz = bz;
    a.out = d_out;
    a.mass_part = mass_part;
    a.cnorm = kernel_cnorm(SF_K_EPAN);
    float_bounds(roi.lo, roi.hi, a.blo, a.bhi);
    {
        KTimer t("k_mom_grid", s);
        const unsigned grid = blocks_for(nblk, kMomWarps);
        if (call.clip)
            SF_TRY_CUDA(launch(k_mom_grid<true>, dim3(grid), dim3(kMomWarps * 32), 0, s, a));
        else
            SF_TRY_CUDA(launch(k_mom_grid<false>, dim3(grid), dim3(kMomWarps * 32), 0, s, a));
    }
    if (d_mass) {
        const double cell = g.s[0] * g.s[1] * g.s[2];
        SF_TRY_CUDA(launch(k_mass_final, dim3(1), dim3(1024), 0, s, (const double *)mass_part, nblk,
                           cell, d_mass));
    }
    return SF_OK;
}

}  // namespace sf
