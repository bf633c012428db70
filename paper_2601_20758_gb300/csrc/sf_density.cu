// sf_density.cu -- the gather engine: kernel density at grid nodes and at points.
//
// What is computed (Sec. 3.1, Eq. 7; gather formulation of Sec. 3.2.1):
//   rho(r) = inv_neff * sum_j K(r - y_j ; l_j)
// over the particles of the scope, with K the Epanechnikov (Eq. 4) or the
// truncated Gaussian kernel and l_j the per-particle smoothing lengths. Every
// output is written by exactly one thread, in a fixed summation order: no
// atomics, results are deterministic.
//
// Grid, split pipeline (sf_kde_grid, batches): the ROI's nodes are cut into
// 8 x 4 x Z tiles, one warp each. A walk kernel lists every tile's candidate
// leaves (leaves whose support reaches the tile); the lists are cut into work
// items of similar length; persistent warps drain the items, each lane owning
// one (x, y) column of Z nodes in registers. Per candidate leaf the warp
// refines its points (footprint in the tile, ROI clip), stages them in its own
// shared memory with per-axis tables of the kernel factors at the tile's node
// coordinates, so the inner loop per (point, node) pair is two instructions
// (Gaussian: exp(a+b+c) = e^a e^b e^c with the truncation test on
// q_x + q_y < 9 - q_z) or three (Epanechnikov). A last kernel adds each tile's
// item partials in item order (deterministic). The allocation-free entry point
// keeps the older monolithic form: one CTA per 16 x 16 x 8 tile walking and
// summing in one launch.
//
// Points: one warp per leaf of 32 query points; the warp walks the index for
// leaves whose support reaches the query points' box, stages the candidates
// in a shared-memory ring and every lane sums over them for its own point,
// two candidates per instruction (packed FP32x2 arithmetic).
#include <cmath>
#include <vector>

#include "sf_internal.cuh"

namespace sf {

constexpr float kBig = 1.0e30f;
constexpr int kTileX = 16, kTileY = 16, kTileZ = 8;
constexpr int kGridThreads = 256;
constexpr int kStage = 128;       // staged points per chunk (4 leaves)
constexpr int kBatch = 64;        // candidate leaves per traversal batch
constexpr int kStack = 32 * kMaxLevels;
constexpr float kHalfLog2e = 0.72134752044448170368f;  // log2(e) / 2

__device__ __forceinline__ float ex2_approx(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}


// Kernel-specific constants, in the units of q' used on the device:
//   EPAN : q' = sum (d_k / l_k)^2,           support q' < 1,  weight c (1 - q')
//   GAUSS: q' = sum (d_k / l_k)^2 log2(e)/2, support q' < 9 log2(e)/2, weight c 2^-q'
template <int KER>
struct KDef;
template <>
struct KDef<SF_K_EPAN> {
    static constexpr float qmax = 1.0f;   // in q'
    static constexpr float rmul = 1.0f;   // support radius / l
    static constexpr float uscale = 1.0f; // u_k = uscale / l_k
};
template <>
struct KDef<SF_K_GAUSS3> {
    static constexpr float qmax = 9.0f * kHalfLog2e;
    static constexpr float rmul = 3.0f;
    static constexpr float uscale = 0.84932180028801904272f;  // sqrt(log2(e)/2)
};

struct EngineArgs {
    TreeView tv;
    const float4 *ell;       // BW_ANISO per sorted point
    const float4 *nell;      // node max smoothing lengths (BW_ISO / BW_ANISO)
    const DensityParams *dp; // device params (uniform l, inv_neff)
    float cnorm;             // 15/(8 pi) or 1/((2 pi)^1.5 P3)
    float blo[3], bhi[3];    // clip box, float bounds equivalent to the closed double box
};

// Does node i possibly hold a particle whose support reaches the box [wlo, whi]?
// Conservative: the box comes widened by widen_box (a margin covering float
// rounding of the box), and the squared-support test carries kFilterSlack.
template <int KER, int BW, bool CLIP>
__device__ __forceinline__ bool node_reaches(const EngineArgs &a, const float *uni, int64_t i,
                                             const float wlo[3], const float whi[3]) {
    const float4 lo = __ldg(&a.tv.nlo[i]);
    const float4 hi = __ldg(&a.tv.nhi[i]);
    float e[3];
    if (BW == BW_UNIFORM) {
        e[0] = uni[0];
        e[1] = uni[1];
        e[2] = uni[2];
    } else {
        const float4 ne = __ldg(&a.nell[i]);
        e[0] = ne.x;
        e[1] = ne.y;
        e[2] = ne.z;
    }
    if (!(e[0] > 0.f) || !(e[1] > 0.f) || !(e[2] > 0.f)) return false;
    if (CLIP) {
        if (lo.x > a.bhi[0] || hi.x < a.blo[0] || lo.y > a.bhi[1] || hi.y < a.blo[1] ||
            lo.z > a.bhi[2] || hi.z < a.blo[2])
            return false;
    }
    const float nl[3] = {lo.x, lo.y, lo.z}, nh[3] = {hi.x, hi.y, hi.z};
    float q = 0.f;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const float gap = fmaxf(fmaxf(nl[k] - whi[k], wlo[k] - nh[k]), 0.f);
        const float t = gap * rcp_approx(e[k]);
        q = fmaf(t, t, q);
    }
    return q < KDef<KER>::rmul * KDef<KER>::rmul * (1.0f + kFilterSlack);
}


// Warp-cooperative resumable depth-first walk. Emits accepted leaf indices in
// ascending order into out[0..), stopping once fewer than 32 slots remain.
// Stack entries encode (level << 27) | index-in-level; sp is warp-uniform.
template <typename Test>
__device__ int warp_walk(const TreeView &tv, const Test &test, int *stack, int &sp, int *out,
                         int cap) {
    const int lane = threadIdx.x & 31;
    const unsigned lt = (1u << lane) - 1u;
    int nout = 0;
    while (sp > 0 && nout <= cap - 32) {
        const int e = stack[sp - 1];
        __syncwarp();
        sp -= 1;
        const int cl = (e >> 27) - 1;
        const int64_t c = (int64_t)(e & ((1 << 27) - 1)) * kFanout + lane;
        const bool ok = (c < tv.cnt[cl]) && test(tv.off[cl] + c);
        const unsigned m = __ballot_sync(0xffffffffu, ok);
        const int r = __popc(m & lt), k = __popc(m);
        if (cl == 0) {
            if (ok) out[nout + r] = (int)c;
            nout += k;
        } else {
            if (ok) stack[sp + (k - 1 - r)] = (cl << 27) | (int)c;
            sp += k;
        }
        __syncwarp();
    }
    return nout;
}

// Start a walk: test the root (lane 0) and push it, or emit it if it is a leaf.
template <typename Test>
__device__ int warp_walk_start(const TreeView &tv, const Test &test, int *stack, int &sp,
                               int *out) {
    const int lane = threadIdx.x & 31;
    const int top = tv.nlevels - 1;
    const bool ok = __shfl_sync(0xffffffffu, lane == 0 ? (int)test(tv.off[top]) : 0, 0) != 0;
    sp = 0;
    if (!ok) return 0;
    if (top == 0) {
        if (lane == 0) out[0] = 0;
        __syncwarp();
        return 1;
    }
    if (lane == 0) stack[0] = top << 27;
    __syncwarp();
    sp = 1;
    return 0;
}

// Exact float bounds of a closed double box: x >= lo_f <=> (double)x >= lo.
void float_bounds(const double lo[3], const double hi[3], float flo[3], float fhi[3]) {
    for (int k = 0; k < 3; ++k) {
        float a = (float)lo[k];
        if ((double)a < lo[k]) a = nextafterf(a, INFINITY);
        float b = (float)hi[k];
        if ((double)b > hi[k]) b = nextafterf(b, -INFINITY);
        flo[k] = a;
        fhi[k] = b;
    }
}

// Per-point smoothing lengths for the three bandwidth modes.
template <int BW>
__device__ __forceinline__ void point_ell(const EngineArgs &a, const float *uni, int64_t i,
                                          float4 p, float l[3]) {
    if (BW == BW_ISO) {
        l[0] = l[1] = l[2] = p.w;
    } else if (BW == BW_UNIFORM) {
        l[0] = uni[0];
        l[1] = uni[1];
        l[2] = uni[2];
    } else {
        const float4 e = __ldg(&a.ell[i]);
        l[0] = e.x;
        l[1] = e.y;
        l[2] = e.z;
    }
}

// ===========================================================================
// Grid
// ===========================================================================
// Geometry and outputs of one ROI grid (device-side descriptor).
struct RoiDesc {
    const float2 *axis;  // node coordinates as (hi, lo) float pairs: x[nx], y[ny], z[nz]
    int nx, ny, nz;
    int tiles_x, tiles_y, tiles_z;
    int tile_base;       // first global tile index of this ROI
    float *out;          // dims[2] x dims[1] x dims[0], x fastest
    double *mass_part;   // per tile of this ROI
    const DensityParams *dp;
    float blo[3], bhi[3];  // clip box (float bounds of the closed double box)
};

template <int TZ>
struct GridSmemT {
    float2 tx[kStage][kTileX];   // Gauss: (c e^{-qx'}, qx'); Epan: (qx', -)
    float2 ty[kStage][kTileY];   // Gauss: (e^{-qy'}, qy');   Epan: (qy', -)
    float2 tz[kStage][TZ];       // Gauss: (e^{-qz'}, qmax - qz'); Epan: (c (1 - qz'), -)
    float4 sp[kStage];           // staged (x, y, z, c)
    float4 su[kStage];           // staged (u_x, u_y, u_z, -)
    int2 sf[kStage];             // staged footprint: x0|x1<<8|y0<<16|y1<<24, z0|z1<<8
    float2 axt[kTileX + kTileY + TZ];  // the tile's node coordinates
    uint8_t wlist[kGridThreads / 32][kStage];  // per warp: staged candidates touching its rows
    int stack[kStack];
    int leaves[kBatch];
    int wcnt[kGridThreads / 32];
    int nleaves, sp_top, item;
    float uni[3];
    double inv_neff;
    double red[kGridThreads / 32];
    EngineArgs e;                // the call's engine arguments with this ROI's clip box and params
    RoiDesc roi;
};

struct TileGeom {
    int gx0, gy0, gz0;
    int nv[3];
    float tlo[3], thi[3], sp3[3];
};

template <int TZ, int WX = kTileX, int WY = kTileY>
__device__ __forceinline__ void tile_origin(const RoiDesc &r, int tile, int &gx0, int &gy0, int &gz0,
                                            int nv[3]) {
    const int tix = tile % r.tiles_x, tiy = (tile / r.tiles_x) % r.tiles_y,
              tiz = tile / (r.tiles_x * r.tiles_y);
    gx0 = tix * WX;
    gy0 = tiy * WY;
    gz0 = tiz * TZ;
    nv[0] = min(WX, r.nx - gx0);
    nv[1] = min(WY, r.ny - gy0);
    nv[2] = min(TZ, r.nz - gz0);
}

// The tile's node coordinates and the call's parameters into shared memory
// (S.roi and S.e must be set). Block-wide: it contains a barrier.
template <int TZ>
__device__ TileGeom tile_setup(GridSmemT<TZ> &S, int tile) {
    const int tid = threadIdx.x;
    const RoiDesc &r = S.roi;
    TileGeom g;
    tile_origin<TZ>(r, tile, g.gx0, g.gy0, g.gz0, g.nv);
    if (tid < kTileX + kTileY + TZ) {
        float2 v = make_float2(0.f, 0.f);
        if (tid < kTileX) {
            if (tid < g.nv[0]) v = r.axis[g.gx0 + tid];
        } else if (tid < kTileX + kTileY) {
            const int j = tid - kTileX;
            if (j < g.nv[1]) v = r.axis[r.nx + g.gy0 + j];
        } else {
            const int j = tid - kTileX - kTileY;
            if (j < g.nv[2]) v = r.axis[r.nx + r.ny + g.gz0 + j];
        }
        S.axt[tid] = v;
    }
    if (tid == 0) {
        const DensityParams dp = *S.e.dp;
        S.uni[0] = dp.ell_uniform[0];
        S.uni[1] = dp.ell_uniform[1];
        S.uni[2] = dp.ell_uniform[2];
        S.inv_neff = dp.inv_neff;
    }
    __syncthreads();
    const int off[3] = {0, kTileX, kTileX + kTileY};
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        g.tlo[k] = S.axt[off[k]].x;
        g.thi[k] = S.axt[off[k] + g.nv[k] - 1].x;
        // node spacing, for footprints (approximate; footprints are widened by 1)
        g.sp3[k] = g.nv[k] > 1 ? (S.axt[off[k] + 1].x - S.axt[off[k]].x) : 1.f;
    }
    return g;
}

// One chunk: the points of up to four candidate leaves are refined (support
// footprint inside the tile, ROI clip), staged, tabulated per axis and added
// into acc. Block-wide; ends with a barrier so shared memory can be reused.
template <int KER, int BW, bool CLIP, bool CNT, int TZ>
__device__ void grid_chunk(GridSmemT<TZ> &S, const TileGeom &g, const int *leaves, int nl,
                           float acc[TZ], unsigned long long &npairs) {
    const EngineArgs &E = S.e;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int cx = lane & 15, cy = warp * 2 + (lane >> 4);
    // ---- load and refine up to 128 candidate points (threads 0..127)
    bool acc_pt = false;
    float4 p = make_float4(0.f, 0.f, 0.f, 0.f);
    float l[3] = {0.f, 0.f, 0.f};
    int2 fp = make_int2(0, 0);
    if (tid < kStage) {
        const int li = tid >> 5;
        if (li < nl) {
            const int64_t i = (int64_t)leaves[li] * kLeaf + lane;
            if (i < E.tv.n) {
                p = __ldg(&E.tv.pos[i]);
                point_ell<BW>(E, S.uni, i, p, l);
                acc_pt = l[0] > 0.f && l[1] > 0.f && l[2] > 0.f;
                if (CLIP)
                    acc_pt = acc_pt && p.x >= E.blo[0] && p.x <= E.bhi[0] && p.y >= E.blo[1] &&
                             p.y <= E.bhi[1] && p.z >= E.blo[2] && p.z <= E.bhi[2];
                const float pc[3] = {p.x, p.y, p.z};
                int f0[3], f1[3];
                float qlb = 0.f;
#pragma unroll
                for (int k = 0; k < 3; ++k) {
                    const float R = l[k] * KDef<KER>::rmul;
                    if (g.sp3[k] > 0.f) {
                        const float a0 = fminf(fmaxf(ceilf((pc[k] - R - g.tlo[k]) / g.sp3[k]) - 1.f, -1.f), 64.f);
                        const float a1 = fminf(fmaxf(floorf((pc[k] + R - g.tlo[k]) / g.sp3[k]) + 1.f, -1.f), 64.f);
                        f0[k] = max(0, (int)a0);
                        f1[k] = min(g.nv[k] - 1, (int)a1);
                    } else {
                        f0[k] = 0;
                        f1[k] = g.nv[k] - 1;
                    }
                    if (f0[k] > f1[k]) acc_pt = false;
                    float gap = fmaxf(fmaxf(g.tlo[k] - pc[k], pc[k] - g.thi[k]), 0.f);
                    gap = fmaxf(gap - 1.0e-6f * (fabsf(g.tlo[k]) + fabsf(g.thi[k])), 0.f);
                    const float t = gap / R;
                    qlb += t * t;
                }
                if (!(qlb < 1.0f + 1.0e-5f)) acc_pt = false;
                if (acc_pt) {
                    fp.x = f0[0] | (f1[0] << 8) | (f0[1] << 16) | (f1[1] << 24);
                    fp.y = f0[2] | (f1[2] << 8);
                }
            }
        }
    }
    // ---- compact accepted points (stable: leaf order, then lane order)
    const unsigned bal = __ballot_sync(0xffffffffu, acc_pt);
    if (lane == 0) S.wcnt[warp] = __popc(bal);
    __syncthreads();
    int base = 0, ns = 0;
#pragma unroll
    for (int w = 0; w < kStage / 32; ++w) {
        const int c = S.wcnt[w];
        if (w < warp) base += c;
        ns += c;
    }
    if (acc_pt) {
        const int s = base + __popc(bal & ((1u << lane) - 1u));
        const float c = E.cnorm / ((l[0] * l[1]) * l[2]);
        S.sp[s] = make_float4(p.x, p.y, p.z, c);
        S.su[s] = make_float4(KDef<KER>::uscale / l[0], KDef<KER>::uscale / l[1],
                              KDef<KER>::uscale / l[2], 0.f);
        S.sf[s] = fp;
    }
    __syncthreads();
    // ---- per-warp lists: the staged candidates whose rows reach this warp's rows
    {
        int nw = 0;
        for (int g0 = 0; g0 < ns; g0 += 32) {
            const int sidx = g0 + lane;
            bool hit = false;
            if (sidx < ns) {
                const int fx = S.sf[sidx].x;
                const int y0 = (fx >> 16) & 255, y1 = (fx >> 24) & 255;
                hit = !(warp * 2 + 1 < y0 || warp * 2 > y1);
            }
            const unsigned m = __ballot_sync(0xffffffffu, hit);
            if (hit) S.wlist[warp][nw + __popc(m & ((1u << lane) - 1u))] = (uint8_t)sidx;
            nw += __popc(m);
        }
        __syncwarp();
        if (lane == 0) S.wcnt[warp] = nw;
    }
    // ---- per-axis tables: the entries inside each staged point's footprint
    constexpr int kEnt = kTileX + kTileY + TZ;
    for (int e = tid; e < ns * kEnt; e += kGridThreads) {
        const int s = e / kEnt;
        const int j = e - s * kEnt;
        const int2 F = S.sf[s];
        int axis, i, lo_i, hi_i;
        if (j < kTileX) {
            axis = 0; i = j; lo_i = F.x & 255; hi_i = (F.x >> 8) & 255;
        } else if (j < kTileX + kTileY) {
            axis = 1; i = j - kTileX; lo_i = (F.x >> 16) & 255; hi_i = (F.x >> 24) & 255;
        } else {
            axis = 2; i = j - kTileX - kTileY; lo_i = F.y & 255; hi_i = (F.y >> 8) & 255;
        }
        if (i < lo_i || i > hi_i) continue;  // never read by the accumulation
        const float4 P = S.sp[s];
        const float4 U = S.su[s];
        const float pc = axis == 0 ? P.x : (axis == 1 ? P.y : P.z);
        const float u = axis == 0 ? U.x : (axis == 1 ? U.y : U.z);
        const float2 nc = S.axt[j];
        const float d = (nc.x - pc) + nc.y;
        const float t = d * u;
        const float q = t * t;
        const bool sup = q < KDef<KER>::qmax;
        float2 v;
        if (KER == SF_K_GAUSS3) {
            const float w = sup ? ex2_approx(-q) : 0.f;
            if (axis == 0) v = make_float2(w * P.w, sup ? q : kBig);
            else if (axis == 1) v = make_float2(w, sup ? q : kBig);
            else v = make_float2(w, sup ? KDef<KER>::qmax - q : -1.f);
        } else {
            if (axis < 2) v = make_float2(sup ? q : kBig, 0.f);
            else v = make_float2(sup ? P.w * (1.0f - q) : -kBig, 0.f);
        }
        if (axis == 0) S.tx[s][i] = v;
        else if (axis == 1) S.ty[s][i] = v;
        else S.tz[s][i] = v;
    }
    __syncthreads();
    // ---- accumulate: warp owns rows 2w, 2w+1; lane owns column cx
    const int nw = S.wcnt[warp];
    for (int li = 0; li < nw; ++li) {
        const int s = S.wlist[warp][li];
        const int2 F = S.sf[s];
        const int x0 = F.x & 255, x1 = (F.x >> 8) & 255;
        const int y0 = (F.x >> 16) & 255, y1 = (F.x >> 24) & 255;
        const int z0 = F.y & 255, z1 = (F.y >> 8) & 255;
        const bool in = cx >= x0 && cx <= x1 && cy >= y0 && cy <= y1;
        // outside the footprint: no contribution (Gauss: q = BIG; Epan: q in .x = BIG)
        float2 ex = KER == SF_K_GAUSS3 ? make_float2(0.f, kBig) : make_float2(kBig, 0.f);
        float2 ey = ex;
        if (in) {
            ex = S.tx[s][cx];
            ey = S.ty[s][cy];
        }
        if (KER == SF_K_GAUSS3) {
            const float bse = ex.x * ey.x;
            const float qij = ex.y + ey.y;
#pragma unroll
            for (int k = 0; k < TZ; ++k) {
                if (k >= z0 && k <= z1) {
                    const float2 ez = S.tz[s][k];
                    if (qij < ez.y) {
                        acc[k] = fmaf(bse, ez.x, acc[k]);
                        if (CNT) ++npairs;
                    }
                }
            }
        } else {
            const float b = S.sp[s].w * (ex.x + ey.x);
#pragma unroll
            for (int k = 0; k < TZ; ++k) {
                if (k >= z0 && k <= z1) {
                    const float t = S.tz[s][k].x - b;
                    acc[k] += fmaxf(t, 0.f);
                    if (CNT) npairs += (t > 0.f);
                }
            }
        }
    }
    __syncthreads();
}

// Fold a chunk's FP32 sums into the compensated per-voxel sums (TwoSum).
// One per-axis table entry of the split pipeline for a particle at coordinate pc
// (scale u = uscale / l, weight c) and a node nc (hi, lo): q = ((nc - pc) u)^2 and
//   Gauss axis 0: (c e^{-q}, q)   axis 1: (e^{-q}, q)   axis 2: (e^{-q}, qmax - q)
//   Epan  axis 0/1: (q, -)        axis 2: (c (1 - q), -)
// with "no support" values (kBig / -1 / -kBig) where q >= qmax or outside.
template <int KER>
__device__ __forceinline__ float2 kentry(int axis, bool inside, float pc, float u, float c, float2 nc) {
    const float d = (nc.x - pc) + nc.y;
    const float t = d * u;
    const float q = t * t;
    const bool sup = inside && q < KDef<KER>::qmax;
    if (KER == SF_K_GAUSS3) {
        const float w = sup ? ex2_approx(-q) : 0.f;
        if (axis == 0) return make_float2(w * c, sup ? q : kBig);
        if (axis == 1) return make_float2(w, sup ? q : kBig);
        return make_float2(w, sup ? KDef<KER>::qmax - q : -1.f);
    }
    if (axis < 2) return make_float2(sup ? q : kBig, 0.f);
    return make_float2(sup ? c * (1.0f - q) : -kBig, 0.f);
}

template <int TZ>
__device__ __forceinline__ void fold(float acc[TZ], float sum[TZ], float cmp[TZ]) {
#pragma unroll
    for (int k = 0; k < TZ; ++k) {
        const float t = sum[k] + acc[k];
        const float bp = t - sum[k];
        cmp[k] += (sum[k] - (t - bp)) + (acc[k] - bp);
        sum[k] = t;
        acc[k] = 0.f;
    }
}

__device__ __forceinline__ void count_pairs_out(unsigned long long *dst, unsigned long long npairs) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) npairs += __shfl_xor_sync(0xffffffffu, npairs, o);
    if ((threadIdx.x & 31) == 0 && npairs) atomicAdd(dst, npairs);
}

// EngineArgs of one ROI: the call's common arguments with the ROI's params and clip box.
__device__ __forceinline__ void set_roi_engine(EngineArgs &e, const EngineArgs &common, const RoiDesc &r) {
    e = common;
    e.dp = r.dp;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        e.blo[k] = r.blo[k];
        e.bhi[k] = r.bhi[k];
    }
}

// ---------------------------------------------------------------------------
// Monolithic variant (used by the allocation-free entry point): one CTA per
// tile walks the index for its tile and sums everything, 8 nodes deep in z.
// ---------------------------------------------------------------------------
struct GridArgs {
    EngineArgs e;
    RoiDesc roi;
    unsigned long long *pairs;
};

template <int KER, int BW, bool CLIP, bool CNT>
__global__ void __launch_bounds__(kGridThreads, 3) k_grid(GridArgs a) {
    constexpr int TZ = kTileZ;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    GridSmemT<TZ> &S = *reinterpret_cast<GridSmemT<TZ> *>(smem_raw);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int tile = blockIdx.x;
    if (tid == 0) {
        S.e = a.e;
        S.roi = a.roi;
    }
    __syncthreads();
    const TileGeom g = tile_setup<TZ>(S, tile);
    float wlo[3], whi[3];
    widen_box(g.tlo, g.thi, wlo, whi);
    auto test = [&](int64_t node) { return node_reaches<KER, BW, CLIP>(S.e, S.uni, node, wlo, whi); };
    const int cx = lane & 15, cy = warp * 2 + (lane >> 4);
    unsigned long long npairs = 0;
    float acc[TZ], sum[TZ], cmp[TZ];
#pragma unroll
    for (int k = 0; k < TZ; ++k) acc[k] = sum[k] = cmp[k] = 0.f;

    if (warp == 0) {
        int spv;
        int n0 = warp_walk_start(S.e.tv, test, S.stack, spv, S.leaves);
        if (lane == 0) {
            S.sp_top = spv;
            S.nleaves = n0;
        }
    }
    __syncthreads();
    bool first = true;
    while (true) {
        if (warp == 0 && !(first && S.nleaves > 0)) {
            int spv = S.sp_top;
            int n = warp_walk(S.e.tv, test, S.stack, spv, S.leaves, kBatch);
            if (lane == 0) {
                S.sp_top = spv;
                S.nleaves = n;
            }
        }
        first = false;
        __syncthreads();
        const int nl = S.nleaves;
        const bool more = S.sp_top > 0;
        if (nl == 0 && !more) break;
        for (int cb = 0; cb < nl; cb += kStage / kLeaf) {
            grid_chunk<KER, BW, CLIP, CNT, TZ>(S, g, S.leaves + cb, min(kStage / kLeaf, nl - cb), acc,
                                               npairs);
            fold<TZ>(acc, sum, cmp);
        }
        if (!more) break;
    }
    if (CNT) count_pairs_out(a.pairs, (cx < g.nv[0] && cy < g.nv[1]) ? npairs : 0ull);
    // ---- write the tile and its mass
    double msum = 0.0;
    const double inv_neff = S.inv_neff;
    const RoiDesc &r = S.roi;
    if (cx < g.nv[0] && cy < g.nv[1]) {
        float *o = r.out + ((int64_t)g.gz0 * r.ny + (g.gy0 + cy)) * r.nx + (g.gx0 + cx);
        const int64_t zs = (int64_t)r.nx * r.ny;
#pragma unroll
        for (int k = 0; k < TZ; ++k) {
            if (k < g.nv[2]) {
                const double v = ((double)sum[k] + (double)cmp[k]) * inv_neff;
                const float fv = (float)v;
                o[k * zs] = fv;
                msum += (double)fv;
            }
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) msum += __shfl_xor_sync(0xffffffffu, msum, o);
    if (lane == 0) S.red[warp] = msum;
    __syncthreads();
    if (tid == 0) {
        double t = 0.0;
        for (int w = 0; w < kGridThreads / 32; ++w) t += S.red[w];
        r.mass_part[tile] = t;
    }
}

// ---------------------------------------------------------------------------
// Split pipeline over one or many ROIs. Tiles over dense regions hold far more
// candidates than others, so each (ROI, tile)'s candidate leaves are listed
// first and cut into balanced work items; persistent CTAs sum the items into
// per-item partial grids, and a per-tile reduction adds the partials in item
// order (deterministic). Global tile index = roi.tile_base + local tile.
// ---------------------------------------------------------------------------
struct MrArgs {
    EngineArgs e;               // common part (index, bandwidths, kernel constant)
    int prec;                   // SF_PREC_* of the work kernel (host-side choice)
    const RoiDesc *rois;        // device array
    const int *tile_roi;        // global tile -> ROI index
    int ntiles;
    unsigned long long *pairs;  // counting variant
    // count walk only (nullable): candidate leaves whose largest support radius on
    // every axis is below twice the ROI's node spacing (sizes the tile depth)
    unsigned long long *small_leaves = nullptr;
};

constexpr int kWalkWarps = 8;
constexpr int kWX = 8, kWY = 4;  // node tile of one warp in the split pipeline (x, y)
constexpr int kLaneTables = 10;   // staged points from which each lane fills its own tables

struct WalkWarpSmem {
    int stack[kStack];
    int leaves[kBatch];
    EngineArgs e;
};

// One warp per (ROI, tile): count (EMIT = false) or list (EMIT = true) its candidate leaves.
template <int KER, int BW, bool CLIP, bool EMIT, int TZ>
__global__ void __launch_bounds__(kWalkWarps * 32) k_mr_walk(MrArgs a, uint32_t *cnt,
                                                             const uint32_t *off, int *list) {
    __shared__ WalkWarpSmem W[kWalkWarps];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int gt = blockIdx.x * kWalkWarps + warp;
    if (gt >= a.ntiles) return;
    WalkWarpSmem &S = W[warp];
    const RoiDesc &r = a.rois[a.tile_roi[gt]];
    if (lane == 0) set_roi_engine(S.e, a.e, r);
    __syncwarp();
    int gx0, gy0, gz0, nv[3];
    tile_origin<TZ, kWX, kWY>(r, gt - r.tile_base, gx0, gy0, gz0, nv);
    float tlo[3], thi[3];
    tlo[0] = r.axis[gx0].x;
    thi[0] = r.axis[gx0 + nv[0] - 1].x;
    tlo[1] = r.axis[r.nx + gy0].x;
    thi[1] = r.axis[r.nx + gy0 + nv[1] - 1].x;
    tlo[2] = r.axis[r.nx + r.ny + gz0].x;
    thi[2] = r.axis[r.nx + r.ny + gz0 + nv[2] - 1].x;
    float uni[3] = {r.dp->ell_uniform[0], r.dp->ell_uniform[1], r.dp->ell_uniform[2]};
    float wlo[3], whi[3];
    widen_box(tlo, thi, wlo, whi);
    auto test = [&](int64_t node) { return node_reaches<KER, BW, CLIP>(S.e, uni, node, wlo, whi); };
    int spv;
    int nl = warp_walk_start(S.e.tv, test, S.stack, spv, S.leaves);
    uint32_t total = 0, nsmall = 0;
    const uint32_t base = EMIT ? off[gt] : 0u;
    // the ROI's node spacing per axis (dims >= 2), for the small-support count
    const float sp[3] = {r.axis[1].x - r.axis[0].x, r.axis[r.nx + 1].x - r.axis[r.nx].x,
                         r.axis[r.nx + r.ny + 1].x - r.axis[r.nx + r.ny].x};
    while (true) {
        if (nl == 0) {
            if (spv == 0) break;
            nl = warp_walk(S.e.tv, test, S.stack, spv, S.leaves, kBatch);
            if (nl == 0) break;
        }
        if (EMIT)
            for (int i = lane; i < nl; i += 32) list[base + total + i] = S.leaves[i];
        if (!EMIT && a.small_leaves) {
            for (int i0 = 0; i0 < nl; i0 += 32) {
                bool sm = false;
                if (i0 + lane < nl) {
                    float e[3] = {uni[0], uni[1], uni[2]};
                    if (BW != BW_UNIFORM) {
                        const float4 ne = __ldg(&S.e.nell[S.e.tv.off[0] + S.leaves[i0 + lane]]);
                        e[0] = ne.x;
                        e[1] = ne.y;
                        e[2] = ne.z;
                    }
                    sm = KDef<KER>::rmul * e[0] < 2.f * sp[0] && KDef<KER>::rmul * e[1] < 2.f * sp[1] &&
                         KDef<KER>::rmul * e[2] < 2.f * sp[2];
                }
                nsmall += __popc(__ballot_sync(0xffffffffu, sm));
            }
        }
        total += nl;
        __syncwarp();
        nl = 0;
    }
    if (!EMIT && lane == 0) {
        cnt[gt] = total;
        if (a.small_leaves && nsmall) atomicAdd(a.small_leaves, (unsigned long long)nsmall);
    }
}

__global__ void k_total64(const uint32_t *__restrict__ cnt, int n, unsigned long long *out) {
    unsigned long long t = 0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) t += cnt[i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if ((threadIdx.x & 31) == 0 && t) atomicAdd(out, t);
}

__global__ void k_grid_item_counts(const uint32_t *__restrict__ cnt, int ntiles, uint32_t lpw,
                                   uint32_t *__restrict__ ic) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < ntiles) ic[t] = max(1u, (cnt[t] + lpw - 1) / lpw);
}

__global__ void k_grid_items(const uint32_t *__restrict__ cnt, const uint32_t *__restrict__ off,
                             const uint32_t *__restrict__ ic, const uint32_t *__restrict__ ioff,
                             int ntiles, uint32_t lpw, int4 *__restrict__ items) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= ntiles) return;
    const uint32_t n = cnt[t], b = off[t];
    for (uint32_t i = 0; i < ic[t]; ++i)
        items[ioff[t] + i] = make_int4(t, (int)(b + i * lpw), (int)(b + min(n, (i + 1) * lpw)), 0);
}

// ---- tensor-core sums of particles whose support covers the whole tile ------
// For such a particle every node (x, y, z) of the 8 x 4 x TZ tile is in support
// and its Gaussian term is the product tx[x] ty[y] tz[z] of its table entries,
// so the tile's sum over these particles is a matrix product:
//   rho[(x, y), z] += sum_s A[(x, y), s] B[s, z],  A = tx ty (32 x S),  B = tz (S x 8).
// It runs as mma.sync m16n8k8 (TF32) or m16n8k16 (BF16) blocks with FP32
// accumulators; 3xTF32 splits every operand into TF32 hi + lo parts and adds the
// three products hi*hi + hi*lo + lo*hi (about 2^-21 relative). These are the
// grid's precision variants; the FP32 path keeps every particle on the FP32
// pipes, which measured faster on this GPU than these mma.sync blocks.
__device__ __forceinline__ uint32_t tf32_of(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return r;
}

__device__ __forceinline__ void mma_k8_tf32(float d[4], uint32_t a0, uint32_t a1, uint32_t a2,
                                            uint32_t a3, uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
        "{%8,%9}, {%0,%1,%2,%3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

__device__ __forceinline__ void mma_k16_bf16(float d[4], uint32_t a0, uint32_t a1, uint32_t a2,
                                             uint32_t a3, uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
        "{%8,%9}, {%0,%1,%2,%3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

// Two floats as a bf16 pair: `first` in the low half (the lower column / row index).
__device__ __forceinline__ uint32_t bf16x2_of(float first, float second) {
    uint32_t r;
    asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(second), "f"(first));
    return r;
}

// A (x = g, y) (TF32 fragment values) times B; PREC 3XTF32 adds the three split products.
template <int PREC>
__device__ __forceinline__ void mma_k8(float d[4], float a0, float a1, float a2, float a3, float b0,
                                       float b1) {
    const uint32_t A0 = tf32_of(a0), A1 = tf32_of(a1), A2 = tf32_of(a2), A3 = tf32_of(a3);
    const uint32_t B0 = tf32_of(b0), B1 = tf32_of(b1);
    if (PREC != SF_PREC_3XTF32) {
        mma_k8_tf32(d, A0, A1, A2, A3, B0, B1);
        return;
    }
    const uint32_t L0 = tf32_of(a0 - __uint_as_float(A0)), L1 = tf32_of(a1 - __uint_as_float(A1));
    const uint32_t L2 = tf32_of(a2 - __uint_as_float(A2)), L3 = tf32_of(a3 - __uint_as_float(A3));
    const uint32_t M0 = tf32_of(b0 - __uint_as_float(B0)), M1 = tf32_of(b1 - __uint_as_float(B1));
    mma_k8_tf32(d, L0, L1, L2, L3, B0, B1);
    mma_k8_tf32(d, A0, A1, A2, A3, M0, M1);
    mma_k8_tf32(d, A0, A1, A2, A3, B0, B1);
}

// Shared memory of one warp of the split pipeline: its 8 x 4 x TZ node tile.
template <int TZ>
struct WTileSmem {
    float2 tx[kLeaf][kWX];   // Gauss: (c e^{-qx'}, qx'); Epan: (qx', -)
    float2 ty[kLeaf][kWY];   // Gauss: (e^{-qy'}, qy');   Epan: (qy', -)
    float2 tz[kLeaf][TZ];    // Gauss: (e^{-qz'}, qmax - qz'); Epan: (c (1 - qz'), -)
    float4 sp[kLeaf];        // staged (x, y, z, c)
    float4 su[kLeaf];        // staged (u_x, u_y, u_z, -)
    int2 sf[kLeaf];          // footprint: x0|x1<<8|y0<<16|y1<<24, z0|z1<<8
    float2 axt[kWX + kWY + TZ];
    float uni[3];
    EngineArgs e;
    RoiDesc roi;
};

// Persistent warps: each takes (ROI, tile, leaf range) items from a counter and
// sums them into the item's partial grid. No block barriers: a warp owns its
// tile, its staging and its tables.
template <int KER, int BW, bool CLIP, bool CNT, int TZ, int PREC = SF_PREC_FP32>
__global__ void __launch_bounds__(kGridThreads, 4)
    k_mr_work(MrArgs a, const int4 *__restrict__ items, const uint32_t *__restrict__ n_items,
              const int *__restrict__ list, double *__restrict__ part, unsigned int *next) {
    // the tensor-core path of the precision variants: Gaussian, 8 nodes deep (the
    // B operand's 8 columns); the FP32 path sums every particle in FP32
    constexpr bool kMma = KER == SF_K_GAUSS3 && TZ == 8 && PREC != SF_PREC_FP32;
    constexpr bool kFull = KER == SF_K_GAUSS3 && TZ == 8 && (PREC != SF_PREC_FP32 || CNT);
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    WTileSmem<TZ> &S = reinterpret_cast<WTileSmem<TZ> *>(smem_raw)[warp];
    const int cx = lane & (kWX - 1), cy = lane / kWX;
    const uint32_t nitems = *n_items;
    unsigned long long npairs = 0;
    int cur_roi = -1;
    while (true) {
        unsigned int item = 0;
        if (lane == 0) item = atomicAdd(next, 1u);
        item = __shfl_sync(0xffffffffu, item, 0);
        if (item >= nitems) break;
        const int4 it = items[item];
        const int ri = a.tile_roi[it.x];
        if (ri != cur_roi) {
            if (lane == 0) {
                S.roi = a.rois[ri];
                set_roi_engine(S.e, a.e, S.roi);
            }
            cur_roi = ri;
            __syncwarp();
        }
        const EngineArgs &E = S.e;
        const RoiDesc &r = S.roi;
        // ---- the tile's node coordinates
        TileGeom g;
        float isp[3], mcen[3], mhw[3];  // 1 / node spacing; tile box widened by the rounding margin
        tile_origin<TZ, kWX, kWY>(r, it.x - r.tile_base, g.gx0, g.gy0, g.gz0, g.nv);
        if (lane < kWX + kWY + TZ) {
            float2 v = make_float2(0.f, 0.f);
            if (lane < kWX) {
                if (lane < g.nv[0]) v = r.axis[g.gx0 + lane];
            } else if (lane < kWX + kWY) {
                const int j = lane - kWX;
                if (j < g.nv[1]) v = r.axis[r.nx + g.gy0 + j];
            } else {
                const int j = lane - kWX - kWY;
                if (j < g.nv[2]) v = r.axis[r.nx + r.ny + g.gz0 + j];
            }
            S.axt[lane] = v;
        }
        if (lane == 0) {
            S.uni[0] = E.dp->ell_uniform[0];
            S.uni[1] = E.dp->ell_uniform[1];
            S.uni[2] = E.dp->ell_uniform[2];
        }
        __syncwarp();
        {
            const int off[3] = {0, kWX, kWX + kWY};
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                g.tlo[k] = S.axt[off[k]].x;
                g.thi[k] = S.axt[off[k] + g.nv[k] - 1].x;
                g.sp3[k] = g.nv[k] > 1 ? (S.axt[off[k] + 1].x - S.axt[off[k]].x) : 1.f;
                isp[k] = g.sp3[k] > 0.f ? 1.0f / g.sp3[k] : 0.f;
                const float mg = 1.0e-6f * (fabsf(g.tlo[k]) + fabsf(g.thi[k]));
                const float lo_m = g.tlo[k] - mg, hi_m = g.thi[k] + mg;
                mcen[k] = 0.5f * (lo_m + hi_m);
                mhw[k] = 0.5f * (hi_m - lo_m);
            }
        }
        float acc[TZ], sum[TZ], cmp[TZ];
#pragma unroll
        for (int k = 0; k < TZ; ++k) acc[k] = sum[k] = cmp[k] = 0.f;
        unsigned long long np = 0;
        unsigned long long st_leaves = 0, st_staged = 0, st_full = 0, st_tested = 0;
        for (int lb = it.y; lb < it.z; ++lb) {
            // ---- one candidate leaf: refine (footprint in this tile, clip) and stage
            const int64_t i = (int64_t)list[lb] * kLeaf + lane;
            bool acc_pt = false;
            float4 p = make_float4(0.f, 0.f, 0.f, 0.f);
            float l[3] = {0.f, 0.f, 0.f}, rl[3] = {0.f, 0.f, 0.f};
            int2 fp = make_int2(0, 0);
            bool full = false;  // the support covers every node of the tile
            if (i < E.tv.n) {
                p = __ldg(&E.tv.pos[i]);
                point_ell<BW>(E, S.uni, i, p, l);
                acc_pt = l[0] > 0.f && l[1] > 0.f && l[2] > 0.f;
                if (CLIP)
                    acc_pt = acc_pt && p.x >= E.blo[0] && p.x <= E.bhi[0] && p.y >= E.blo[1] &&
                             p.y <= E.bhi[1] && p.z >= E.blo[2] && p.z <= E.bhi[2];
                const float pc[3] = {p.x, p.y, p.z};
                int f0[3], f1[3];
                float qlb = 0.f;
#pragma unroll
                for (int k = 0; k < 3; ++k) {
                    rl[k] = BW == BW_ISO && k > 0 ? rl[0] : rcp_approx(l[k]);
                    const float R = l[k] * KDef<KER>::rmul;
                    if (g.sp3[k] > 0.f) {
                        const float a0 = fminf(fmaxf(ceilf((pc[k] - R - g.tlo[k]) * isp[k]) - 1.f, -1.f), 64.f);
                        const float a1 = fminf(fmaxf(floorf((pc[k] + R - g.tlo[k]) * isp[k]) + 1.f, -1.f), 64.f);
                        f0[k] = max(0, (int)a0);
                        f1[k] = min(g.nv[k] - 1, (int)a1);
                    } else {
                        f0[k] = 0;
                        f1[k] = g.nv[k] - 1;
                    }
                    if (f0[k] > f1[k]) acc_pt = false;
                    const float t = fmaxf(fabsf(pc[k] - mcen[k]) - mhw[k], 0.f) * rl[k];
                    qlb = fmaf(t, t, qlb);
                }
                if (!(qlb < KDef<KER>::rmul * KDef<KER>::rmul * (1.0f + kFilterSlack))) acc_pt = false;
                // Small supports: exact footprints. The widened ranges shrink to the nodes whose
                // per-axis q (computed exactly as the tables compute it) is below
                // qmax -- a contiguous run, since q is unimodal along the axis. Then
                // the smallest per-axis q bounds every node's test (the float sums and
                // differences are monotone): a particle that fails it adds nothing to
                // any node of the tile (a dense cluster between the nodes of a coarse
                // grid) and is not staged.
                if (acc_pt && f1[0] - f0[0] < 4 && f1[1] - f0[1] < 4 && f1[2] - f0[2] < 4) {
                    float mq[3];
                    const int aoff[3] = {0, kWX, kWX + kWY};
#pragma unroll
                    for (int k = 0; k < 3; ++k) {
                        const float u = KDef<KER>::uscale * rl[k];
                        auto qat = [&](int ii) {
                            const float2 nc = S.axt[aoff[k] + ii];
                            const float d = (nc.x - pc[k]) + nc.y;
                            const float t = d * u;
                            return t * t;
                        };
                        while (f0[k] <= f1[k] && !(qat(f0[k]) < KDef<KER>::qmax)) ++f0[k];
                        while (f1[k] >= f0[k] && !(qat(f1[k]) < KDef<KER>::qmax)) --f1[k];
                        float m = kBig;
                        if (f0[k] <= f1[k]) {
                            const int ic = min(max((int)rintf((pc[k] - g.tlo[k]) * isp[k]), f0[k]), f1[k]);
#pragma unroll
                            for (int dd = -1; dd <= 1; ++dd) {
                                const int ii = ic + dd;
                                if (ii >= f0[k] && ii <= f1[k]) m = fminf(m, qat(ii));
                            }
                        }
                        mq[k] = m;
                    }
                    if (KER == SF_K_GAUSS3) {
                        if (!(mq[0] + mq[1] < KDef<KER>::qmax - mq[2])) acc_pt = false;
                    } else {
                        const float c = E.cnorm * ((rl[0] * rl[1]) * rl[2]);
                        if (!(c * (1.0f - mq[2]) - c * (mq[0] + mq[1]) > 0.f)) acc_pt = false;
                    }
                }
                if (acc_pt) {
                    fp.x = f0[0] | (f1[0] << 8) | (f0[1] << 16) | (f1[1] << 24);
                    fp.y = f0[2] | (f1[2] << 8);
                }
                // Full coverage: q is convex along each axis, so its largest value over the
                // tile is at a corner node; the node test fl(qx + qy) < fl(qmax - qz) is
                // monotone in each q, so passing it with the per-axis maxima passes it
                // at every node (as the table path would evaluate it).
                if (kFull && acc_pt && f0[0] == 0 && f1[0] == g.nv[0] - 1 && f0[1] == 0 &&
                    f1[1] == g.nv[1] - 1 && f0[2] == 0 && f1[2] == g.nv[2] - 1) {
                    const int aoff[3] = {0, kWX, kWX + kWY};
                    float qm[3];
#pragma unroll
                    for (int k = 0; k < 3; ++k) {
                        const float u = KDef<KER>::uscale * rl[k];
                        float m = 0.f;
#pragma unroll
                        for (int e = 0; e < 2; ++e) {
                            const float2 nc = S.axt[aoff[k] + (e ? g.nv[k] - 1 : 0)];
                            const float d = (nc.x - pc[k]) + nc.y;
                            const float t = d * u;
                            m = fmaxf(m, t * t);
                        }
                        qm[k] = m;
                    }
                    full = qm[0] + qm[1] < KDef<KER>::qmax - qm[2];
                }
            }
            const unsigned bal = __ballot_sync(0xffffffffu, acc_pt);
            const int ns = __popc(bal);
            if (ns == 0) continue;  // warp-uniform
            // staged slots: the full-coverage particles first, [0, nf); the others [nf, ns)
            const unsigned balf = __ballot_sync(0xffffffffu, acc_pt && full);
            const int nf = kMma ? __popc(balf) : 0;
            if (CNT && lane == 0) {
                ++st_leaves;
                st_staged += ns;
                st_full += __popc(balf);
                st_tested += (unsigned long long)ns * (kWX * kWY * TZ);
            }
            const unsigned lt = (1u << lane) - 1u;
            const int my_slot = !kMma ? __popc(bal & lt)
                                      : (full ? __popc(balf & lt) : nf + __popc(bal & ~balf & lt));
            if (acc_pt) {
                const int s = my_slot;
                S.sp[s] = make_float4(p.x, p.y, p.z, E.cnorm * ((rl[0] * rl[1]) * rl[2]));
                S.su[s] = make_float4(KDef<KER>::uscale * rl[0], KDef<KER>::uscale * rl[1],
                                      KDef<KER>::uscale * rl[2], 0.f);
                S.sf[s] = fp;
            }
            __syncwarp();
            // ---- per-axis tables: factors inside the footprint, "no support" values
            // outside it (so the accumulation needs no range tests). Many staged points:
            // each staging lane fills its own point's entries, in an order rotated by
            // its row so that the lanes' stores spread over the banks; few: the entries
            // are spread over all lanes. Same values either way.
            constexpr int kEnt = kWX + kWY + TZ;
            auto entry = [&](int axis, int ii, bool inside, float pc, float u, float c, float2 nc) {
                return kentry<KER>(axis, inside, pc, u, c, nc);
            };
            if (ns >= kLaneTables) {
                if (acc_pt) {
                    const int s = my_slot;
                    const float c = E.cnorm * ((rl[0] * rl[1]) * rl[2]);
                    const float u0 = KDef<KER>::uscale * rl[0], u1 = KDef<KER>::uscale * rl[1],
                                u2 = KDef<KER>::uscale * rl[2];
                    const int x0 = fp.x & 255, x1 = (fp.x >> 8) & 255;
                    const int y0 = (fp.x >> 16) & 255, y1 = (fp.x >> 24) & 255;
                    const int z0 = fp.y & 255, z1 = (fp.y >> 8) & 255;
                    {
#pragma unroll
                        for (int t = 0; t < kWX; ++t) {
                            const int i = (t + (s >> 1)) & (kWX - 1);
                            S.tx[s][i] = entry(0, i, i >= x0 && i <= x1, p.x, u0, c, S.axt[i]);
                        }
#pragma unroll
                        for (int t = 0; t < kWY; ++t) {
                            const int i = (t + (s >> 2)) & (kWY - 1);
                            S.ty[s][i] = entry(1, i, i >= y0 && i <= y1, p.y, u1, c, S.axt[kWX + i]);
                        }
#pragma unroll
                        for (int t = 0; t < TZ; ++t) {
                            const int i = (t + (s >> (TZ == 8 ? 1 : 2))) & (TZ - 1);
                            S.tz[s][i] = entry(2, i, i >= z0 && i <= z1, p.z, u2, c, S.axt[kWX + kWY + i]);
                        }
                    }
                }
            } else
            for (int e = lane; e < ns * kEnt; e += 32) {
                const int s = e / kEnt;
                const int j = e - s * kEnt;
                const int2 F = S.sf[s];
                int axis, ii, lo_i, hi_i;
                if (j < kWX) {
                    axis = 0; ii = j; lo_i = F.x & 255; hi_i = (F.x >> 8) & 255;
                } else if (j < kWX + kWY) {
                    axis = 1; ii = j - kWX; lo_i = (F.x >> 16) & 255; hi_i = (F.x >> 24) & 255;
                } else {
                    axis = 2; ii = j - kWX - kWY; lo_i = F.y & 255; hi_i = (F.y >> 8) & 255;
                }
                const bool inside = ii >= lo_i && ii <= hi_i;
                const float4 P = S.sp[s];
                const float4 U = S.su[s];
                const float pc = axis == 0 ? P.x : (axis == 1 ? P.y : P.z);
                const float u = axis == 0 ? U.x : (axis == 1 ? U.y : U.z);
                const float2 v = entry(axis, ii, inside, pc, u, P.w, S.axt[j]);
                if (axis == 0) S.tx[s][ii] = v;
                else if (axis == 1) S.ty[s][ii] = v;
                else S.tz[s][ii] = v;
            }
            __syncwarp();
            {
            // ---- accumulate: lane owns column (cx, cy) and TZ nodes in z
            for (int s = nf; s < ns; ++s) {
                const float2 ex = S.tx[s][cx];
                const float2 ey = S.ty[s][cy];
                if (KER == SF_K_GAUSS3) {
                    const float bse = ex.x * ey.x;
                    const float qij = ex.y + ey.y;
#pragma unroll
                    for (int k = 0; k < TZ; ++k) {
                        const float2 ez = S.tz[s][k];
                        if (qij < ez.y) {
                            acc[k] = fmaf(bse, ez.x, acc[k]);
                            if (CNT) ++np;
                        }
                    }
                } else {
                    const float b = S.sp[s].w * (ex.x + ey.x);
#pragma unroll
                    for (int k = 0; k < TZ; ++k) {
                        const float t = S.tz[s][k].x - b;
                        acc[k] += fmaxf(t, 0.f);
                        if (CNT) np += (t > 0.f);
                    }
                }
            }
            }
            if (kMma && nf > 0) {  // warp-uniform: the full-coverage particles on the tensor cores
                const int gq = lane >> 2, tig = lane & 3;
                float d0[4] = {0.f, 0.f, 0.f, 0.f}, d1[4] = {0.f, 0.f, 0.f, 0.f};
                if (PREC == SF_PREC_BF16) {
                    for (int s0 = 0; s0 < nf; s0 += 16) {
                        float ax[4], ay[4][4], bz[4];  // particles s0 + 2 tig + {0, 1, 8, 9}
#pragma unroll
                        for (int e = 0; e < 4; ++e) {
                            const int sp = s0 + 2 * tig + (e & 1) + 8 * (e >> 1);
                            const bool v = sp < nf;
                            ax[e] = v ? S.tx[sp][gq].x : 0.f;
                            bz[e] = v ? S.tz[sp][gq].x : 0.f;
#pragma unroll
                            for (int y = 0; y < 4; ++y) ay[e][y] = v ? S.ty[sp][y].x : 0.f;
                        }
                        const uint32_t b0 = bf16x2_of(bz[0], bz[1]), b1 = bf16x2_of(bz[2], bz[3]);
#pragma unroll
                        for (int mb = 0; mb < 2; ++mb) {
                            float *d = mb ? d1 : d0;
                            const int y0 = 2 * mb, y1 = 2 * mb + 1;
                            mma_k16_bf16(d, bf16x2_of(ax[0] * ay[0][y0], ax[1] * ay[1][y0]),
                                         bf16x2_of(ax[0] * ay[0][y1], ax[1] * ay[1][y1]),
                                         bf16x2_of(ax[2] * ay[2][y0], ax[3] * ay[3][y0]),
                                         bf16x2_of(ax[2] * ay[2][y1], ax[3] * ay[3][y1]), b0, b1);
                        }
                    }
                } else {
                    for (int s0 = 0; s0 < nf; s0 += 8) {
                        const int sa = s0 + tig, sb = s0 + tig + 4;
                        const bool va = sa < nf, vb = sb < nf;
                        const float txa = va ? S.tx[sa][gq].x : 0.f, txb = vb ? S.tx[sb][gq].x : 0.f;
                        const float tza = va ? S.tz[sa][gq].x : 0.f, tzb = vb ? S.tz[sb][gq].x : 0.f;
#pragma unroll
                        for (int mb = 0; mb < 2; ++mb) {
                            const float ya0 = va ? S.ty[sa][2 * mb].x : 0.f, ya1 = va ? S.ty[sa][2 * mb + 1].x : 0.f;
                            const float yb0 = vb ? S.ty[sb][2 * mb].x : 0.f, yb1 = vb ? S.ty[sb][2 * mb + 1].x : 0.f;
                            mma_k8<PREC>(mb ? d1 : d0, txa * ya0, txa * ya1, txb * yb0, txb * yb1, tza, tzb);
                        }
                    }
                }
                // to the column owners: row r = x + 8 y of the product is lane r's column
                float *cb = reinterpret_cast<float *>(S.tx);  // the tables are no longer read
                __syncwarp();
#pragma unroll
                for (int mb = 0; mb < 2; ++mb) {
                    const float *d = mb ? d1 : d0;
                    const int r0 = 16 * mb + gq;
                    cb[r0 * 8 + 2 * tig] = d[0];
                    cb[r0 * 8 + 2 * tig + 1] = d[1];
                    cb[(r0 + 8) * 8 + 2 * tig] = d[2];
                    cb[(r0 + 8) * 8 + 2 * tig + 1] = d[3];
                }
                __syncwarp();
#pragma unroll
                for (int k = 0; k < TZ; ++k) acc[k] += cb[lane * 8 + k];
                if (CNT && cx < g.nv[0] && cy < g.nv[1]) np += (unsigned long long)nf * g.nv[2];
            }
            __syncwarp();
            fold<TZ>(acc, sum, cmp);
        }
        if (CNT && cx < g.nv[0] && cy < g.nv[1]) npairs += np;
        if (CNT && lane == 0) {  // work accounting of the counting variant
            atomicAdd(a.pairs + 1, st_leaves);
            atomicAdd(a.pairs + 2, st_staged);
            atomicAdd(a.pairs + 3, st_full);
            atomicAdd(a.pairs + 4, st_tested);
        }
        double *o = part + ((int64_t)item * 32 + lane) * TZ;
#pragma unroll
        for (int k = 0; k < TZ; ++k) o[k] = (double)sum[k] + (double)cmp[k];
    }
    if (CNT) count_pairs_out(a.pairs, npairs);
}

// One warp per (ROI, tile): sum the items' partial grids in item order, scale,
// write, and the tile's mass.
template <int TZ>
__global__ void __launch_bounds__(kGridThreads) k_mr_reduce(MrArgs a, const uint32_t *__restrict__ ic,
                                                            const uint32_t *__restrict__ ioff,
                                                            const double *__restrict__ part) {
    const int lane = threadIdx.x & 31;
    const int gt = blockIdx.x * (kGridThreads / 32) + (threadIdx.x >> 5);
    if (gt >= a.ntiles) return;
    const int cx = lane & (kWX - 1), cy = lane / kWX;
    const RoiDesc &r = a.rois[a.tile_roi[gt]];
    const int tile = gt - r.tile_base;
    int gx0, gy0, gz0, nv[3];
    tile_origin<TZ, kWX, kWY>(r, tile, gx0, gy0, gz0, nv);
    const double inv_neff = r.dp->inv_neff;
    double v[TZ];
#pragma unroll
    for (int k = 0; k < TZ; ++k) v[k] = 0.0;
    const uint32_t i0 = ioff[gt], ni = ic[gt];
    for (uint32_t i = 0; i < ni; ++i) {
        const double *pp = part + ((int64_t)(i0 + i) * 32 + lane) * TZ;
#pragma unroll
        for (int k = 0; k < TZ; ++k) v[k] += pp[k];
    }
    double msum = 0.0;
    if (cx < nv[0] && cy < nv[1]) {
        float *o = r.out + ((int64_t)gz0 * r.ny + (gy0 + cy)) * r.nx + (gx0 + cx);
        const int64_t zs = (int64_t)r.nx * r.ny;
#pragma unroll
        for (int k = 0; k < TZ; ++k) {
            if (k < nv[2]) {
                const float fv = (float)(v[k] * inv_neff);
                o[k * zs] = fv;
                msum += (double)fv;
            }
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) msum += __shfl_xor_sync(0xffffffffu, msum, o);
    if (lane == 0) r.mass_part[tile] = msum;
}

__global__ void k_mass_final(const double *__restrict__ part, int64_t n, double cell,
                             double *out) {
    __shared__ double red[32];
    double t = 0.0;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) t += part[i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = t;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
        *out = s * cell;
    }
}

// One block per ROI: its tiles' masses in order, times its cell volume.
__global__ void k_mr_mass(const RoiDesc *__restrict__ rois, const double *__restrict__ cells,
                          int nroi, double *__restrict__ mass) {
    __shared__ double red[32];
    const int ri = blockIdx.x;
    if (ri >= nroi) return;
    const RoiDesc &r = rois[ri];
    const int nt = r.tiles_x * r.tiles_y * r.tiles_z;
    double t = 0.0;
    for (int i = threadIdx.x; i < nt; i += blockDim.x) t += r.mass_part[i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = t;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
        mass[ri] = s * cells[ri];
    }
}

// ---- monolithic dispatch (allocation-free path) ----------------------------
template <int KER, int BW, bool CLIP, bool CNT>
static cudaError_t launch_grid_t(const GridArgs &a, unsigned tiles, cudaStream_t s) {
    const size_t smem = sizeof(GridSmemT<kTileZ>);
    static std::atomic<uint64_t> attr{0};
    cudaError_t e = smem_attr_once(k_grid<KER, BW, CLIP, CNT>, smem, attr);
    if (e != cudaSuccess) return e;
    KTimer t(CNT ? "k_grid_count" : "k_grid", s);
    return launch(k_grid<KER, BW, CLIP, CNT>, dim3(tiles), dim3(kGridThreads), smem, s, a);
}

template <int KER, int BW, bool CLIP>
static cudaError_t launch_grid(const GridArgs &a, unsigned tiles, cudaStream_t s) {
    return a.pairs ? launch_grid_t<KER, BW, CLIP, true>(a, tiles, s)
                   : launch_grid_t<KER, BW, CLIP, false>(a, tiles, s);
}

template <int KER>
static cudaError_t dispatch_grid(int bw, bool clip, const GridArgs &a, unsigned tiles,
                                 cudaStream_t s) {
    switch (bw * 2 + (clip ? 1 : 0)) {
        case BW_ISO * 2 + 0: return launch_grid<KER, BW_ISO, false>(a, tiles, s);
        case BW_ISO * 2 + 1: return launch_grid<KER, BW_ISO, true>(a, tiles, s);
        case BW_UNIFORM * 2 + 0: return launch_grid<KER, BW_UNIFORM, false>(a, tiles, s);
        case BW_UNIFORM * 2 + 1: return launch_grid<KER, BW_UNIFORM, true>(a, tiles, s);
        case BW_ANISO * 2 + 0: return launch_grid<KER, BW_ANISO, false>(a, tiles, s);
        default: return launch_grid<KER, BW_ANISO, true>(a, tiles, s);
    }
}

// ---- split pipeline ---------------------------------------------------------
// Sizing: count candidate leaves of every (ROI, tile); returns the total (syncs).
template <int KER, int BW, bool CLIP, int TZ>
// tot: 16 bytes -- [0] the 32-bit scan total, [1] the item count of mr_exec,
// bytes 8..15 the same total summed in 64 bits (guards the 32-bit offsets).
// h_small (with a.small_leaves set): the count of small-support candidate leaves.
static sf_status mr_count(const MrArgs &a, uint32_t *cnt, uint32_t *off, uint32_t *tot,
                          uint32_t *h_total, StatusPeek *peek, cudaStream_t s,
                          unsigned long long *h_small = nullptr) {
    const unsigned wb = blocks_for(a.ntiles, kWalkWarps);
    if (a.small_leaves) SF_TRY_CUDA(cudaMemsetAsync(a.small_leaves, 0, sizeof(unsigned long long), s));
    SF_TRY_CUDA(launch(k_mr_walk<KER, BW, CLIP, false, TZ>, dim3(wb), dim3(kWalkWarps * 32), 0, s, a,
                       cnt, (const uint32_t *)nullptr, (int *)nullptr));
    SF_TRY(scan_u32(cnt, off, a.ntiles, tot, s));
    unsigned long long *tot64 = reinterpret_cast<unsigned long long *>(tot + 2);
    SF_TRY_CUDA(cudaMemsetAsync(tot64, 0, sizeof(unsigned long long), s));
    SF_TRY_CUDA(launch(k_total64, dim3(std::min(blocks_for(a.ntiles, 256), 152u * 4u)), dim3(256), 0, s,
                       (const uint32_t *)cnt, a.ntiles, tot64));
    unsigned long long h64 = 0;
    SF_TRY_CUDA(cudaMemcpyAsync(&h64, tot64, sizeof h64, cudaMemcpyDeviceToHost, s));
    if (peek && peek->d_src)
        SF_TRY_CUDA(cudaMemcpyAsync(&peek->value, peek->d_src, sizeof(int), cudaMemcpyDeviceToHost, s));
    if (a.small_leaves && h_small)
        SF_TRY_CUDA(cudaMemcpyAsync(h_small, a.small_leaves, sizeof(unsigned long long),
                                    cudaMemcpyDeviceToHost, s));
    SF_TRY_CUDA(cudaStreamSynchronize(s));
    if (h64 > 0x7fffffffull)
        return fail(SF_ERR_CAPACITY, "grid candidate lists of %llu entries exceed 2^31; use fewer nodes or a smaller ROI",
                    h64);
    *h_total = (uint32_t)h64;
    return SF_OK;
}

template <int TZ>
static size_t mr_work_smem() {
    return sizeof(WTileSmem<TZ>) * (kGridThreads / 32);
}

template <int KER, int BW, bool CLIP, bool CNT, int TZ>
static sf_status mr_work_attr(int *per_sm) {
    const size_t smem = mr_work_smem<TZ>();
    static std::atomic<uint64_t> attr{0};
    SF_TRY_CUDA(smem_attr_once(k_mr_work<KER, BW, CLIP, CNT, TZ>, smem, attr));
    SF_TRY_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, k_mr_work<KER, BW, CLIP, CNT, TZ>,
                                                              kGridThreads, smem));
    if (*per_sm < 1) *per_sm = 1;
    return SF_OK;
}

// Buffers of the execution phase, sized from the count.
struct MrBuffers {
    uint32_t *cnt, *off, *tot, *ic, *ioff;
    int *list;
    int4 *items;
    double *part;
    unsigned int *next;
    uint32_t lpw;
    int64_t slots;        // resident blocks of k_mr_work
};

template <int KER, int BW, bool CLIP, bool CNT, int TZ, int PREC>
static sf_status launch_work(const MrArgs &a, const MrBuffers &b, cudaStream_t s) {
    static std::atomic<uint64_t> attr{0};
    SF_TRY_CUDA(smem_attr_once(k_mr_work<KER, BW, CLIP, CNT, TZ, PREC>, mr_work_smem<TZ>(), attr));
    SF_TRY_CUDA(launch(k_mr_work<KER, BW, CLIP, CNT, TZ, PREC>, dim3((unsigned)b.slots), dim3(kGridThreads),
                       mr_work_smem<TZ>(), s, a, (const int4 *)b.items, (const uint32_t *)(b.tot + 1),
                       (const int *)b.list, b.part, b.next));
    return SF_OK;
}

// Execution: list, items, persistent work, ordered reduce (no host sync; capturable).
template <int KER, int BW, bool CLIP, bool CNT, int TZ>
static sf_status mr_exec(const MrArgs &a, const MrBuffers &b, cudaStream_t s) {
    const unsigned wb = blocks_for(a.ntiles, kWalkWarps);
    SF_TRY_CUDA(launch(k_mr_walk<KER, BW, CLIP, true, TZ>, dim3(wb), dim3(kWalkWarps * 32), 0, s, a,
                       (uint32_t *)nullptr, (const uint32_t *)b.off, b.list));
    SF_TRY_CUDA(launch(k_grid_item_counts, dim3(blocks_for(a.ntiles, 256)), dim3(256), 0, s,
                       (const uint32_t *)b.cnt, a.ntiles, b.lpw, b.ic));
    SF_TRY(scan_u32(b.ic, b.ioff, a.ntiles, b.tot + 1, s));
    SF_TRY_CUDA(launch(k_grid_items, dim3(blocks_for(a.ntiles, 256)), dim3(256), 0, s,
                       (const uint32_t *)b.cnt, (const uint32_t *)b.off, (const uint32_t *)b.ic,
                       (const uint32_t *)b.ioff, a.ntiles, b.lpw, b.items));
    SF_TRY_CUDA(cudaMemsetAsync(b.next, 0, sizeof(unsigned int), s));
    {
        KTimer t(CNT ? "k_grid_work_count" : "k_grid_work", s);
        bool done = false;
        if constexpr (KER == SF_K_GAUSS3 && TZ == 8 && !CNT && BW != BW_ANISO) {
            done = true;
            switch (a.prec) {
                case SF_PREC_TF32: SF_TRY((launch_work<KER, BW, CLIP, CNT, TZ, SF_PREC_TF32>(a, b, s))); break;
                case SF_PREC_3XTF32: SF_TRY((launch_work<KER, BW, CLIP, CNT, TZ, SF_PREC_3XTF32>(a, b, s))); break;
                case SF_PREC_BF16: SF_TRY((launch_work<KER, BW, CLIP, CNT, TZ, SF_PREC_BF16>(a, b, s))); break;
                default: done = false;
            }
        }
        if (!done) SF_TRY((launch_work<KER, BW, CLIP, CNT, TZ, SF_PREC_FP32>(a, b, s)));
    }
    SF_TRY_CUDA(launch(k_mr_reduce<TZ>, dim3(blocks_for(a.ntiles, kGridThreads / 32)), dim3(kGridThreads), 0, s, a,
                       (const uint32_t *)b.ic, (const uint32_t *)b.ioff, (const double *)b.part));
    return SF_OK;
}

// Sizes of an execution from the candidate total: resident blocks, leaves per
// work item, the item bound.
template <int KER, int BW, bool CLIP, bool CNT, int TZ>
static sf_status mr_sizes(const MrArgs &a, uint32_t total, int items_per_slot, int64_t *slots,
                          uint32_t *lpw, int64_t *max_items) {
    int dev = 0, sms = 0, per_sm = 0;
    SF_TRY_CUDA(cudaGetDevice(&dev));
    SF_TRY_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    SF_TRY((mr_work_attr<KER, BW, CLIP, CNT, TZ>(&per_sm)));
    *slots = (int64_t)sms * per_sm;  // resident blocks of 8 persistent warps
    const int64_t warps = *slots * (kGridThreads / 32);
    const int64_t ips = std::max(1, items_per_slot);
    *lpw = (uint32_t)std::max<int64_t>(8, (total + ips * warps - 1) / (ips * warps));
    *max_items = a.ntiles + total / *lpw + 1;
    return SF_OK;
}

// Bytes of the execution buffers mr_plan allocates (each rounded as Scratch counts it).
template <int TZ>
static int64_t mr_plan_bytes(int64_t ntiles, uint32_t total, int64_t max_items) {
    return scratch_round(4 * std::max<int64_t>(1, total)) + 2 * scratch_round(4 * ntiles) +
           scratch_round(16 * max_items) + scratch_round(8 * max_items * 32 * TZ) + scratch_round(4);
}

static int64_t scan_parts_bytes_(int64_t n) { return n > 0 ? scratch_round(4 * ((n + 2047) / 2048)) : 0; }

// Plan the buffers of an execution from the candidate total.
template <int KER, int BW, bool CLIP, bool CNT, int TZ>
static sf_status mr_plan(const MrArgs &a, uint32_t total, int items_per_slot, MrBuffers &b,
                         Scratch *sc, std::vector<void *> *owned, cudaStream_t s) {
    int64_t max_items = 0;
    SF_TRY((mr_sizes<KER, BW, CLIP, CNT, TZ>(a, total, items_per_slot, &b.slots, &b.lpw, &max_items)));
    auto get = [&](size_t bytes) -> void * {
        void *p = nullptr;
        if (sc) {
            p = sc->get<unsigned char>((int64_t)bytes);
        } else if (cudaMalloc(&p, bytes) == cudaSuccess) {
            owned->push_back(p);
        } else {
            p = nullptr;
        }
        return p;
    };
    b.list = (int *)get(sizeof(int) * std::max<int64_t>(1, total));
    b.ic = (uint32_t *)get(sizeof(uint32_t) * a.ntiles);
    b.ioff = (uint32_t *)get(sizeof(uint32_t) * a.ntiles);
    b.items = (int4 *)get(sizeof(int4) * max_items);
    b.part = (double *)get(sizeof(double) * max_items * 32 * TZ);
    b.next = (unsigned int *)get(sizeof(unsigned int));
    if (!b.list || !b.ic || !b.ioff || !b.items || !b.part || !b.next)
        return fail(SF_ERR_OOM, "grid work buffers (%lld items)", (long long)max_items);
    return SF_OK;
}

// ws_bytes (nullable): size the execution and return its bytes instead of running it.
template <int KER, int BW, bool CLIP, int TZ>
// shallow (non-null): if most candidate leaves have supports below twice the node
// spacing, set *shallow and return after the count (the caller re-plans with
// 8 x 4 x 4 tiles); otherwise *shallow = false and the call runs.
static sf_status mr_once(const MrArgs &a_in, int items_per_slot, StatusPeek *peek, int64_t *ws_bytes,
                         cudaStream_t s, bool *shallow = nullptr) {
    Scratch sc(s);
    MrBuffers b;
    MrArgs a = a_in;
    b.cnt = sc.get<uint32_t>(a.ntiles);
    b.off = sc.get<uint32_t>(a.ntiles);
    b.tot = sc.get<uint32_t>(4);
    if (shallow) a.small_leaves = sc.get<unsigned long long>(1);
    SF_TRY_SCRATCH(sc);
    uint32_t total = 0;
    unsigned long long nsmall = 0;
    SF_TRY((mr_count<KER, BW, CLIP, TZ>(a, b.cnt, b.off, b.tot, &total, peek, s, &nsmall)));
    a.small_leaves = nullptr;
    if (shallow) {
        *shallow = 2 * nsmall > (unsigned long long)total;
        if (*shallow) return SF_OK;
    }
    if (ws_bytes) {
        int64_t slots = 0, max_items = 0;
        uint32_t lpw = 0;
        SF_TRY((mr_sizes<KER, BW, CLIP, false, TZ>(a, total, items_per_slot, &slots, &lpw, &max_items)));
        *ws_bytes = 2 * scratch_round(4 * (int64_t)a.ntiles) + scratch_round(16) +
                    (shallow ? scratch_round(8) : 0) +
                    mr_plan_bytes<TZ>(a.ntiles, total, max_items) + scan_parts_bytes_(a.ntiles);
        return SF_OK;
    }
    if (a.pairs) {
        SF_TRY((mr_plan<KER, BW, CLIP, true, TZ>(a, total, items_per_slot, b, &sc, nullptr, s)));
        SF_TRY_SCRATCH(sc);
        return mr_exec<KER, BW, CLIP, true, TZ>(a, b, s);
    }
    SF_TRY((mr_plan<KER, BW, CLIP, false, TZ>(a, total, items_per_slot, b, &sc, nullptr, s)));
    SF_TRY_SCRATCH(sc);
    return mr_exec<KER, BW, CLIP, false, TZ>(a, b, s);
}

template <int KER, int TZ>
static sf_status dispatch_once(int bw, bool clip, const MrArgs &a, int ips, StatusPeek *pk,
                               int64_t *ws, cudaStream_t s, bool *sh = nullptr) {
    switch (bw * 2 + (clip ? 1 : 0)) {
        case BW_ISO * 2 + 0: return mr_once<KER, BW_ISO, false, TZ>(a, ips, pk, ws, s, sh);
        case BW_ISO * 2 + 1: return mr_once<KER, BW_ISO, true, TZ>(a, ips, pk, ws, s, sh);
        case BW_UNIFORM * 2 + 0: return mr_once<KER, BW_UNIFORM, false, TZ>(a, ips, pk, ws, s, sh);
        case BW_UNIFORM * 2 + 1: return mr_once<KER, BW_UNIFORM, true, TZ>(a, ips, pk, ws, s, sh);
        case BW_ANISO * 2 + 0: return mr_once<KER, BW_ANISO, false, TZ>(a, ips, pk, ws, s, sh);
        default: return mr_once<KER, BW_ANISO, true, TZ>(a, ips, pk, ws, s, sh);
    }
}

float kernel_cnorm(int kernel) {
    const double pi = 3.14159265358979323846;
    if (kernel == SF_K_EPAN) return (float)(15.0 / (8.0 * pi));
    const double p3 = std::erf(3.0 / std::sqrt(2.0)) - std::sqrt(2.0 / pi) * 3.0 * std::exp(-4.5);
    return (float)(1.0 / (std::pow(2.0 * pi, 1.5) * p3));
}

static EngineArgs engine_args(sf_index *idx, const sf_box &roi, const DensityCall &call) {
    EngineArgs e;
    e.tv = idx->view();
    e.ell = call.ell;
    e.nell = call.nell_override ? call.nell_override : idx->nell;
    e.dp = call.dp;
    e.cnorm = kernel_cnorm(call.kernel);
    float_bounds(roi.lo, roi.hi, e.blo, e.bhi);
    return e;
}

// Node coordinates r_k(i) = lo_k + i s_k in double, split into float (hi, lo).
void node_axes(const GridSpec &g, float2 *ax) {
    const int nd[3] = {g.nx, g.ny, g.nz};
    size_t o = 0;
    for (int k = 0; k < 3; ++k)
        for (int i = 0; i < nd[k]; ++i) {
            const double r = g.lo[k] + (double)i * g.s[k];
            const float h = (float)r;
            ax[o++] = make_float2(h, (float)(r - (double)h));
        }
}

static RoiDesc roi_desc(const GridSpec &g, int tz, const float2 *axis, int tile_base, float *out,
                        double *mass_part, const DensityParams *dp, const sf_box &roi,
                        int wx = kTileX, int wy = kTileY) {
    RoiDesc r;
    r.axis = axis;
    r.nx = g.nx;
    r.ny = g.ny;
    r.nz = g.nz;
    r.tiles_x = (g.nx + wx - 1) / wx;
    r.tiles_y = (g.ny + wy - 1) / wy;
    r.tiles_z = (g.nz + tz - 1) / tz;
    r.tile_base = tile_base;
    r.out = out;
    r.mass_part = mass_part;
    r.dp = dp;
    float_bounds(roi.lo, roi.hi, r.blo, r.bhi);
    return r;
}

// The tile gather with TZ-deep tiles and ips work items per resident warp (8:
// measured equal or up to 7% faster than 4 on the zoom grids of the 1.07B cloud);
// shallow (non-null): see mr_once (returns early, nothing written, when set).
template <int TZ>
static sf_status grid_gather(sf_index *idx, const sf_box &roi, const GridSpec &g,
                             const DensityCall &call, float *d_out, double *d_mass, cudaStream_t s,
                             unsigned long long *d_pairs, StatusPeek *peek, int64_t *ws_bytes,
                             int ips, bool *shallow) {
    std::vector<float2> ax((size_t)g.nx + g.ny + g.nz);
    node_axes(g, ax.data());
    const int64_t tiles = (int64_t)((g.nx + kWX - 1) / kWX) * ((g.ny + kWY - 1) / kWY) *
                          ((g.nz + TZ - 1) / TZ);
    if (tiles >= (int64_t(1) << 30)) return fail(SF_ERR_INVALID_ARG, "grid too large");
    Scratch sc(s);
    float2 *d_axis = sc.get<float2>((int64_t)ax.size());
    double *mass_part = sc.get<double>(tiles);
    RoiDesc *d_roi = sc.get<RoiDesc>(1);
    int *tile_roi = sc.get<int>(tiles);
    SF_TRY_SCRATCH(sc);
    SF_TRY_CUDA(cudaMemcpyAsync(d_axis, ax.data(), ax.size() * sizeof(float2),
                                cudaMemcpyHostToDevice, s));
    const RoiDesc r = roi_desc(g, TZ, d_axis, 0, d_out, mass_part, call.dp, roi, kWX, kWY);
    SF_TRY_CUDA(cudaMemcpyAsync(d_roi, &r, sizeof r, cudaMemcpyHostToDevice, s));
    SF_TRY_CUDA(cudaMemsetAsync(tile_roi, 0, sizeof(int) * tiles, s));
    MrArgs a;
    a.e = engine_args(idx, roi, call);
    a.rois = d_roi;
    a.tile_roi = tile_roi;
    a.ntiles = (int)tiles;
    a.pairs = d_pairs;
    a.prec = call.prec;
    {
        KTimer t(d_pairs ? "k_grid_count" : "k_grid", s);
        if (call.kernel == SF_K_EPAN)
            SF_TRY((dispatch_once<SF_K_EPAN, TZ>(call.bw, call.clip != 0, a, ips, peek, ws_bytes, s, shallow)));
        else
            SF_TRY((dispatch_once<SF_K_GAUSS3, TZ>(call.bw, call.clip != 0, a, ips, peek, ws_bytes, s, shallow)));
    }
    if (shallow && *shallow) return SF_OK;
    if (ws_bytes) {  // this function's own buffers on top of the execution's
        *ws_bytes += scratch_round(sizeof(float2) * ax.size()) + scratch_round(8 * tiles) +
                     scratch_round(sizeof(RoiDesc)) + scratch_round(4 * tiles);
        return SF_OK;
    }
    if (d_mass) {
        const double cell = g.s[0] * g.s[1] * g.s[2];
        SF_TRY_CUDA(launch(k_mass_final, dim3(1), dim3(1024), 0, s, (const double *)mass_part,
                           tiles, cell, d_mass));
    }
    return SF_OK;
}

// Tile depth: 8 x 4 x 8 node tiles by default; when most of a grid's candidate
// leaves have supports below twice the node spacing on every axis (each particle
// reaches a few nodes: a whole billion-point cloud at 256^3, whose supports are
// about one spacing), 8 x 4 x 4 tiles with 32 work items per warp: fewer nodes
// swept per staged particle (measured 17% faster there, 45% slower on dense zoom
// grids, whose supports span 8 to 150 spacings; the finer items balance the
// cube's uneven tiles, 4% more). The decision costs the 8-deep count walk. The
// tensor-core variants need 8-deep tiles and keep them.
static sf_status density_grid_gather(sf_index *idx, const sf_box &roi, const GridSpec &g,
                                     const DensityCall &call, float *d_out, double *d_mass,
                                     cudaStream_t s, unsigned long long *d_pairs, StatusPeek *peek,
                                     int64_t *ws_bytes) {
    bool shallow = false;
    SF_TRY(grid_gather<kTileZ>(idx, roi, g, call, d_out, d_mass, s, d_pairs, peek, ws_bytes, 8,
                               call.prec == SF_PREC_FP32 ? &shallow : nullptr));
    if (!shallow) return SF_OK;
    if (ws_bytes) *ws_bytes = 0;
    const sf_status st = grid_gather<4>(idx, roi, g, call, d_out, d_mass, s, d_pairs, peek, ws_bytes,
                                        32, nullptr);
    if (st != SF_ERR_CAPACITY) return st;
    // the shallow tiles' lists would pass 2^31 entries where the 8-deep ones fit: keep those
    clear_error();
    if (ws_bytes) *ws_bytes = 0;
    return grid_gather<kTileZ>(idx, roi, g, call, d_out, d_mass, s, d_pairs, peek, ws_bytes, 8, nullptr);
}

// The pair-by-pair gather, or the exact moment form (sf_moments.cu) when the
// call asks for it, or, under SF_ACCEL_AUTO, when the gather's candidate lists
// would pass 2^31 entries (the gather stops at its sizing step, before any
// density kernel has run). The pair count always takes the gather.
static sf_status density_grid_impl(sf_index *idx, const sf_box &roi, const GridSpec &g,
                                   const DensityCall &call, float *d_out, double *d_mass,
                                   cudaStream_t s, unsigned long long *d_pairs, StatusPeek *peek,
                                   int64_t *ws_bytes) {
    if (!d_pairs && moments_apply(call)) {
        if (call.accel == SF_ACCEL_MOMENTS)
            return density_grid_moments(idx, roi, g, call, d_out, d_mass, s, ws_bytes, peek);
        const sf_status st = density_grid_gather(idx, roi, g, call, d_out, d_mass, s, nullptr, peek, ws_bytes);
        if (st != SF_ERR_CAPACITY) return st;
        clear_error();
        return density_grid_moments(idx, roi, g, call, d_out, d_mass, s, ws_bytes, peek);
    }
    return density_grid_gather(idx, roi, g, call, d_out, d_mass, s, d_pairs, peek, ws_bytes);
}

sf_status density_grid(sf_index *idx, const sf_box &roi, const GridSpec &g,
                       const DensityCall &call, float *d_out, double *d_mass, cudaStream_t s,
                       unsigned long long *d_pairs, StatusPeek *peek) {
    return density_grid_impl(idx, roi, g, call, d_out, d_mass, s, d_pairs, peek, nullptr);
}

// Device bytes density_grid holds at its peak for this ROI (it runs the
// candidate count, which synchronises the stream).
sf_status grid_workspace(sf_index *idx, const sf_box &roi, const GridSpec &g,
                         const DensityCall &call, int64_t *bytes, cudaStream_t s) {
    *bytes = 0;
    return density_grid_impl(idx, roi, g, call, nullptr, nullptr, s, nullptr, nullptr, bytes);
}

// Same result as density_grid with the monolithic kernel, on node coordinates
// and per-tile partial sums that the caller has already placed in device
// memory (no allocation here).
sf_status density_grid_prealloc(sf_index *idx, const sf_box &roi, const GridSpec &g,
                                const DensityCall &call, const float2 *d_axis,
                                double *d_mass_part, float *d_out, double *d_mass, cudaStream_t s) {
    GridArgs a;
    a.e = engine_args(idx, roi, call);
    a.roi = roi_desc(g, kTileZ, d_axis, 0, d_out, d_mass_part, call.dp, roi);
    a.pairs = nullptr;
    const int64_t tiles = (int64_t)a.roi.tiles_x * a.roi.tiles_y * a.roi.tiles_z;
    cudaError_t e = (call.kernel == SF_K_EPAN)
                        ? dispatch_grid<SF_K_EPAN>(call.bw, call.clip != 0, a, (unsigned)tiles, s)
                        : dispatch_grid<SF_K_GAUSS3>(call.bw, call.clip != 0, a, (unsigned)tiles, s);
    SF_TRY_CUDA(e);
    if (d_mass) {
        const double cell = g.s[0] * g.s[1] * g.s[2];
        SF_TRY_CUDA(launch(k_mass_final, dim3(1), dim3(1024), 0, s, (const double *)d_mass_part,
                           tiles, cell, d_mass));
    }
    return SF_OK;
}

int64_t grid_tile_count(const GridSpec &g) {
    return (int64_t)((g.nx + kTileX - 1) / kTileX) * ((g.ny + kTileY - 1) / kTileY) *
           ((g.nz + kTileZ - 1) / kTileZ);
}

// ===========================================================================
// Batched grids: many ROIs in one persistent execution, replayed from a graph
// ===========================================================================
struct BatchPlan {
    sf_index *idx = nullptr;
    int nroi = 0;
    int kernel = 0, bw = 0;
    bool clip = false;
    int tz = 8, ips = 4;
    bool use_graph = true;
    std::vector<RoiDesc> h_rois;       // host copy (out pointers updated per run)
    std::vector<void *> owned;         // cudaMalloc'ed buffers
    RoiDesc *d_rois = nullptr;
    double *d_mass = nullptr;
    MrArgs a;
    MrBuffers b;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
};

template <int KER, int BW, bool CLIP, int TZ>
static sf_status batch_build(BatchPlan &P, cudaStream_t s) {
    uint32_t total = 0;
    SF_TRY((mr_count<KER, BW, CLIP, TZ>(P.a, P.b.cnt, P.b.off, P.b.tot, &total, nullptr, s)));
    SF_TRY((mr_plan<KER, BW, CLIP, false, TZ>(P.a, total, P.ips, P.b, nullptr, &P.owned, s)));
    if (!P.use_graph) return SF_OK;
    // capture the execution once, on a private stream (the caller's may be the
    // legacy default stream, which cannot be captured); runs replay it on theirs
    cudaStream_t cs = nullptr;
    SF_TRY_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    cudaError_t ce = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (ce != cudaSuccess) {
        cudaStreamDestroy(cs);
        return fail(SF_ERR_CUDA, "cudaStreamBeginCapture: %s", cudaGetErrorString(ce));
    }
    sf_status st = mr_exec<KER, BW, CLIP, false, TZ>(P.a, P.b, cs);
    cudaGraph_t g = nullptr;
    ce = cudaStreamEndCapture(cs, &g);
    cudaStreamDestroy(cs);
    if (st != SF_OK) {
        if (g) cudaGraphDestroy(g);
        return st;
    }
    SF_TRY_CUDA(ce);
    P.graph = g;
    SF_TRY_CUDA(cudaGraphInstantiate(&P.exec, g, 0));
    return SF_OK;
}

template <int KER, int BW, bool CLIP, int TZ>
static sf_status batch_exec(BatchPlan &P, cudaStream_t s) {
    if (P.exec) {
        KTimer t("k_batch_graph", s);
        SF_TRY_CUDA(cudaGraphLaunch(P.exec, s));
        g_launches.fetch_add(8, std::memory_order_relaxed);  // kernels inside the graph
        return SF_OK;
    }
    return mr_exec<KER, BW, CLIP, false, TZ>(P.a, P.b, s);
}

template <int KER, int TZ>
static sf_status batch_dispatch(BatchPlan &P, bool build, cudaStream_t s) {
    switch (P.bw * 2 + (P.clip ? 1 : 0)) {
        case BW_ISO * 2 + 0: return build ? batch_build<KER, BW_ISO, false, TZ>(P, s) : batch_exec<KER, BW_ISO, false, TZ>(P, s);
        case BW_ISO * 2 + 1: return build ? batch_build<KER, BW_ISO, true, TZ>(P, s) : batch_exec<KER, BW_ISO, true, TZ>(P, s);
        case BW_UNIFORM * 2 + 0: return build ? batch_build<KER, BW_UNIFORM, false, TZ>(P, s) : batch_exec<KER, BW_UNIFORM, false, TZ>(P, s);
        default: return build ? batch_build<KER, BW_UNIFORM, true, TZ>(P, s) : batch_exec<KER, BW_UNIFORM, true, TZ>(P, s);
    }
}

static sf_status batch_call(BatchPlan &P, bool build, cudaStream_t s) {
    if (P.kernel == SF_K_EPAN)
        return P.tz == 4 ? batch_dispatch<SF_K_EPAN, 4>(P, build, s) : batch_dispatch<SF_K_EPAN, 8>(P, build, s);
    return P.tz == 4 ? batch_dispatch<SF_K_GAUSS3, 4>(P, build, s) : batch_dispatch<SF_K_GAUSS3, 8>(P, build, s);
}

void batch_free(BatchPlan *P) {
    if (!P) return;
    if (P->exec) cudaGraphExecDestroy(P->exec);
    if (P->graph) cudaGraphDestroy(P->graph);
    for (void *p : P->owned) cudaFree(p);
    delete P;
}

// rois/grids: nroi boxes and GridSpecs; dps: device DensityParams per ROI (owned by the plan)
sf_status batch_create(sf_index *idx, int nroi, const sf_box *rois, const GridSpec *grids,
                       int kernel, int bw, bool clip, DensityParams *d_dps, int tz, int ips,
                       bool use_graph, cudaStream_t s, BatchPlan **out, int prec) {
    BatchPlan *P = new BatchPlan();
    P->idx = idx;
    P->nroi = nroi;
    P->kernel = kernel;
    P->bw = bw;
    P->clip = clip;
    P->tz = (tz == 4) ? 4 : 8;
    P->ips = ips;
    P->use_graph = use_graph;
    auto bail = [&](sf_status st) {
        batch_free(P);
        return st;
    };
    P->owned.push_back(d_dps);
    int64_t naxis = 0, ntiles = 0;
    std::vector<int64_t> tb(nroi);
    for (int r = 0; r < nroi; ++r) {
        naxis += grids[r].nx + grids[r].ny + grids[r].nz;
        tb[r] = ntiles;
        ntiles += (int64_t)((grids[r].nx + kWX - 1) / kWX) * ((grids[r].ny + kWY - 1) / kWY) *
                  ((grids[r].nz + P->tz - 1) / P->tz);
    }
    if (ntiles >= (int64_t(1) << 30)) return bail(fail(SF_ERR_INVALID_ARG, "batch too large"));
    std::vector<float2> ax(naxis);
    std::vector<int> tile_roi(ntiles);
    void *p_axis = nullptr, *p_rois = nullptr, *p_tr = nullptr, *p_mp = nullptr, *p_mass = nullptr,
         *p_cnt = nullptr, *p_off = nullptr, *p_tot = nullptr;
    cudaError_t e;
    if ((e = cudaMalloc(&p_axis, sizeof(float2) * naxis)) != cudaSuccess ||
        (e = cudaMalloc(&p_rois, sizeof(RoiDesc) * nroi)) != cudaSuccess ||
        (e = cudaMalloc(&p_tr, sizeof(int) * ntiles)) != cudaSuccess ||
        (e = cudaMalloc(&p_mp, sizeof(double) * ntiles)) != cudaSuccess ||
        (e = cudaMalloc(&p_mass, sizeof(double) * 2 * nroi)) != cudaSuccess ||
        (e = cudaMalloc(&p_cnt, sizeof(uint32_t) * ntiles)) != cudaSuccess ||
        (e = cudaMalloc(&p_off, sizeof(uint32_t) * ntiles)) != cudaSuccess ||
        (e = cudaMalloc(&p_tot, sizeof(uint32_t) * 4)) != cudaSuccess) {
        for (void *q : {p_axis, p_rois, p_tr, p_mp, p_mass, p_cnt, p_off, p_tot})
            if (q) cudaFree(q);
        return bail(fail(SF_ERR_OOM, "batch plan: %s", cudaGetErrorString(e)));
    }
    for (void *q : {p_axis, p_rois, p_tr, p_mp, p_mass, p_cnt, p_off, p_tot}) P->owned.push_back(q);
    float2 *d_axis = (float2 *)p_axis;
    double *d_mp = (double *)p_mp;
    P->d_rois = (RoiDesc *)p_rois;
    P->d_mass = (double *)p_mass;
    int64_t ao = 0;
    P->h_rois.resize(nroi);
    std::vector<double> cells(nroi);
    for (int r = 0; r < nroi; ++r) {
        node_axes(grids[r], ax.data() + ao);
        P->h_rois[r] = roi_desc(grids[r], P->tz, d_axis + ao, (int)tb[r], nullptr, d_mp + tb[r],
                                d_dps + r, rois[r], kWX, kWY);
        const int64_t nt = (r + 1 < nroi ? tb[r + 1] : ntiles) - tb[r];
        for (int64_t t = 0; t < nt; ++t) tile_roi[tb[r] + t] = r;
        ao += grids[r].nx + grids[r].ny + grids[r].nz;
        cells[r] = grids[r].s[0] * grids[r].s[1] * grids[r].s[2];
    }
    if ((e = cudaMemcpyAsync(d_axis, ax.data(), sizeof(float2) * naxis, cudaMemcpyHostToDevice, s)) != cudaSuccess ||
        (e = cudaMemcpyAsync(P->d_rois, P->h_rois.data(), sizeof(RoiDesc) * nroi, cudaMemcpyHostToDevice, s)) != cudaSuccess ||
        (e = cudaMemcpyAsync(p_tr, tile_roi.data(), sizeof(int) * ntiles, cudaMemcpyHostToDevice, s)) != cudaSuccess ||
        (e = cudaMemcpyAsync(P->d_mass + nroi, cells.data(), sizeof(double) * nroi, cudaMemcpyHostToDevice, s)) != cudaSuccess)
        return bail(fail(SF_ERR_CUDA, "batch plan upload: %s", cudaGetErrorString(e)));
    sf_box any = rois[0];
    DensityCall call;
    call.kernel = kernel;
    call.bw = bw;
    call.clip = clip ? 1 : 0;
    call.ell = nullptr;
    call.dp = d_dps;
    call.nell_override = nullptr;
    P->a.e = engine_args(idx, any, call);
    P->a.rois = P->d_rois;
    P->a.tile_roi = (const int *)p_tr;
    P->a.ntiles = (int)ntiles;
    P->a.pairs = nullptr;
    P->a.prec = prec;  // the work kernel's form (tensor-core variants: Gaussian, 8-deep tiles)
    P->b.cnt = (uint32_t *)p_cnt;
    P->b.off = (uint32_t *)p_off;
    P->b.tot = (uint32_t *)p_tot;
    sf_status st = batch_call(*P, true, s);
    if (st != SF_OK) return bail(st);
    *out = P;
    return SF_OK;
}

sf_status batch_run(BatchPlan *P, float *const *outs, double *h_mass, cudaStream_t s) {
    bool changed = false;
    for (int r = 0; r < P->nroi; ++r)
        if (P->h_rois[r].out != outs[r]) {
            P->h_rois[r].out = outs[r];
            changed = true;
        }
    if (changed)
        SF_TRY_CUDA(cudaMemcpyAsync(P->d_rois, P->h_rois.data(), sizeof(RoiDesc) * P->nroi,
                                    cudaMemcpyHostToDevice, s));
    SF_TRY(batch_call(*P, false, s));
    if (h_mass) {
        SF_TRY_CUDA(launch(k_mr_mass, dim3(P->nroi), dim3(256), 0, s, (const RoiDesc *)P->d_rois,
                           (const double *)(P->d_mass + P->nroi), P->nroi, P->d_mass));
        SF_TRY_CUDA(cudaMemcpyAsync(h_mass, P->d_mass, sizeof(double) * P->nroi, cudaMemcpyDeviceToHost, s));
        SF_TRY_CUDA(cudaStreamSynchronize(s));
    }
    return SF_OK;
}

// ===========================================================================
// Points (DIRECT)
// ===========================================================================
constexpr int kPtWarps = 4;

struct PointsArgs {
    EngineArgs e;
    const int *leaves;          // query leaves (null: every leaf, slot = leaf)
    int64_t nslots;             // number of query leaves
    float *rho_sorted;          // [nslots * 32]: density of slot point (slot * 32 + lane)
    uint8_t *inroi;             // [nslots * 32]: 1 if that point lies in the ROI
    unsigned long long *pairs;  // counting variant
};

constexpr int kPtRing = 2 * kLeaf;  // staged candidates: two halves of 32

struct __align__(16) PtWarpSmem {
    // staged candidates as structure of arrays (pairs of entries load as one 64-bit word)
    float sx[kPtRing], sy[kPtRing], sz[kPtRing], sc[kPtRing];
    float su[3][kPtRing];  // BW_ISO: su[0] = u^2; else u_x, u_y, u_z
    int stack[kStack];
    int leaves[kBatch];
};

template <int KER, int BW, bool CLIP, bool CNT>
__global__ void __launch_bounds__(kPtWarps * 32) k_points(PointsArgs a) {
    __shared__ PtWarpSmem W[kPtWarps];
    __shared__ float s_uni[3];
    __shared__ float s_runi[4];  // 1 / uniform l_k, and whether all l_k > 0
    __shared__ double s_inv;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (threadIdx.x == 0) {
        const DensityParams dp = *a.e.dp;
        s_uni[0] = dp.ell_uniform[0];
        s_uni[1] = dp.ell_uniform[1];
        s_uni[2] = dp.ell_uniform[2];
        s_runi[0] = 1.0f / s_uni[0];
        s_runi[1] = 1.0f / s_uni[1];
        s_runi[2] = 1.0f / s_uni[2];
        s_runi[3] = (s_uni[0] > 0.f && s_uni[1] > 0.f && s_uni[2] > 0.f) ? 1.f : 0.f;
        s_inv = dp.inv_neff;
    }
    __syncthreads();
    PtWarpSmem &S = W[warp];
    const int64_t slot = (int64_t)blockIdx.x * kPtWarps + warp;
    if (slot >= a.nslots) return;
    const int64_t leaf = a.leaves ? (int64_t)a.leaves[slot] : slot;
    const int64_t qi = leaf * kLeaf + lane;
    const int64_t oi = slot * kLeaf + lane;
    const bool valid = qi < a.e.tv.n;
    float4 q = make_float4(0.f, 0.f, 0.f, 0.f);
    if (valid) q = __ldg(&a.e.tv.pos[qi]);
    // query points: those inside the ROI box (closed)
    const bool active = valid && q.x >= a.e.blo[0] && q.x <= a.e.bhi[0] && q.y >= a.e.blo[1] &&
                        q.y <= a.e.bhi[1] && q.z >= a.e.blo[2] && q.z <= a.e.bhi[2];
    a.inroi[oi] = active ? 1 : 0;
    const unsigned am = __ballot_sync(0xffffffffu, active);
    if (am == 0) return;
    float tlo[3] = {active ? q.x : INFINITY, active ? q.y : INFINITY, active ? q.z : INFINITY};
    float thi[3] = {active ? q.x : -INFINITY, active ? q.y : -INFINITY, active ? q.z : -INFINITY};
#pragma unroll
    for (int k = 0; k < 3; ++k)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            tlo[k] = fminf(tlo[k], __shfl_xor_sync(0xffffffffu, tlo[k], o));
            thi[k] = fmaxf(thi[k], __shfl_xor_sync(0xffffffffu, thi[k], o));
        }
    // the query box widened by the rounding margin (node test and per-point filter),
    // the latter as centre and half-width
    float mlo[3], mhi[3], mcen[3], mhw[3];
    widen_box(tlo, thi, mlo, mhi);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        mcen[k] = 0.5f * (mlo[k] + mhi[k]);
        mhw[k] = 0.5f * (mhi[k] - mlo[k]);
    }
    auto test = [&](int64_t node) { return node_reaches<KER, BW, CLIP>(a.e, s_uni, node, mlo, mhi); };

    float sum = 0.f, cmp = 0.f;
    unsigned long long npairs = 0;
    const f32x2 QX = f2_pack(q.x, q.x), QY = f2_pack(q.y, q.y), QZ = f2_pack(q.z, q.z);
    // entries s and s + 1 (s even) against this lane's query
    auto pair2 = [&](int s, float &acc0, float &acc1) {
        const f32x2 dx = f2_sub(QX, f2_ld(&S.sx[s]));
        const f32x2 dy = f2_sub(QY, f2_ld(&S.sy[s]));
        const f32x2 dz = f2_sub(QZ, f2_ld(&S.sz[s]));
        f32x2 qq;
        if (BW == BW_ISO) {
            qq = f2_mul(f2_fma(dz, dz, f2_fma(dy, dy, f2_mul(dx, dx))), f2_ld(&S.su[0][s]));
        } else {
            const f32x2 tx = f2_mul(dx, f2_ld(&S.su[0][s]));
            const f32x2 ty = f2_mul(dy, f2_ld(&S.su[1][s]));
            const f32x2 tz = f2_mul(dz, f2_ld(&S.su[2][s]));
            qq = f2_fma(tz, tz, f2_fma(ty, ty, f2_mul(tx, tx)));
        }
        float q0, q1, c0, c1;
        f2_unpack(qq, q0, q1);
        f2_unpack(f2_ld(&S.sc[s]), c0, c1);
        const bool in0 = q0 < KDef<KER>::qmax, in1 = q1 < KDef<KER>::qmax;
        if (KER == SF_K_GAUSS3) {
            if (in0) acc0 = fmaf(c0, ex2_approx(-q0), acc0);
            if (in1) acc1 = fmaf(c1, ex2_approx(-q1), acc1);
        } else {
            if (in0) acc0 = fmaf(c0, 1.0f - q0, acc0);
            if (in1) acc1 = fmaf(c1, 1.0f - q1, acc1);
        }
        if (CNT) npairs += (unsigned)in0 + (unsigned)in1;
    };
    auto add = [&](float v) {  // compensated running sum (TwoSum)
        const float t = sum + v;
        const float bp = t - sum;
        cmp += (sum - (t - bp)) + (v - bp);
        sum = t;
    };
    int head = 0, cnt = 0;  // ring of staged candidates: first entry, count (warp-uniform)
    int spv;
    int nl = warp_walk_start(a.e.tv, test, S.stack, spv, S.leaves);
    while (true) {
        if (nl == 0) {
            if (spv == 0) break;
            nl = warp_walk(a.e.tv, test, S.stack, spv, S.leaves, kBatch);
            if (nl == 0) break;
        }
        // software pipeline: the next candidate leaf's point is loaded one step ahead
        float4 pn = make_float4(0.f, 0.f, 0.f, 0.f);
        float4 en = pn;
        {
            const int64_t j0 = (int64_t)S.leaves[0] * kLeaf + lane;
            if (j0 < a.e.tv.n) {
                pn = __ldg(&a.e.tv.pos[j0]);
                if (BW == BW_ANISO) en = __ldg(&a.e.ell[j0]);
            }
        }
        for (int li = 0; li < nl; ++li) {
            const int64_t j = (int64_t)S.leaves[li] * kLeaf + lane;
            const float4 p = pn;
            const float4 pe = en;
            if (li + 1 < nl) {
                const int64_t jn = (int64_t)S.leaves[li + 1] * kLeaf + lane;
                if (jn < a.e.tv.n) {
                    pn = __ldg(&a.e.tv.pos[jn]);
                    if (BW == BW_ANISO) en = __ldg(&a.e.ell[jn]);
                }
            }
            bool ok = false;
            float r[3] = {0.f, 0.f, 0.f};  // 1 / l_k
            if (j < a.e.tv.n) {
                if (BW == BW_ISO) {
                    ok = p.w > 0.f;
                    r[0] = r[1] = r[2] = rcp_approx(p.w);
                } else if (BW == BW_UNIFORM) {
                    ok = s_runi[3] > 0.f;
                    r[0] = s_runi[0]; r[1] = s_runi[1]; r[2] = s_runi[2];
                } else {
                    ok = pe.x > 0.f && pe.y > 0.f && pe.z > 0.f;
                    r[0] = rcp_approx(pe.x); r[1] = rcp_approx(pe.y); r[2] = rcp_approx(pe.z);
                }
                if (CLIP)
                    ok = ok && p.x >= a.e.blo[0] && p.x <= a.e.bhi[0] && p.y >= a.e.blo[1] &&
                         p.y <= a.e.bhi[1] && p.z >= a.e.blo[2] && p.z <= a.e.bhi[2];
                const float pc[3] = {p.x, p.y, p.z};
                float qlb = 0.f;
#pragma unroll
                for (int k = 0; k < 3; ++k) {
                    const float t = fmaxf(fabsf(pc[k] - mcen[k]) - mhw[k], 0.f) * r[k];
                    qlb = fmaf(t, t, qlb);
                }
                ok = ok && qlb < KDef<KER>::rmul * KDef<KER>::rmul * (1.0f + kFilterSlack);
            }
            const unsigned m = __ballot_sync(0xffffffffu, ok);
            if (ok) {
                const int s = (head + cnt + __popc(m & ((1u << lane) - 1u))) & (kPtRing - 1);
                S.sx[s] = p.x;
                S.sy[s] = p.y;
                S.sz[s] = p.z;
                S.sc[s] = a.e.cnorm * ((r[0] * r[1]) * r[2]);
                const float u0 = KDef<KER>::uscale * r[0];
                if (BW == BW_ISO) {
                    S.su[0][s] = u0 * u0;
                } else {
                    S.su[0][s] = u0;
                    S.su[1][s] = KDef<KER>::uscale * r[1];
                    S.su[2][s] = KDef<KER>::uscale * r[2];
                }
            }
            cnt += __popc(m);
            if (cnt >= kLeaf) {  // warp-uniform: a full half of the ring is staged
                __syncwarp();
                float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f;
#pragma unroll
                for (int e = 0; e < kLeaf; e += 4) {
                    pair2(head + e, a0, a1);
                    pair2(head + e + 2, a2, a3);
                }
                head ^= kLeaf;
                cnt -= kLeaf;
                add((a0 + a1) + (a2 + a3));
                __syncwarp();
            }
        }
        nl = 0;
    }
    // the staged remainder (cnt < 32 entries from head), padded to an even
    // count with an entry of zero weight
    if (cnt & 1) {
        if (lane == 0) {
            const int s = (head + cnt) & (kPtRing - 1);
            S.sx[s] = S.sy[s] = S.sz[s] = S.sc[s] = 0.f;
            S.su[0][s] = S.su[1][s] = S.su[2][s] = 0.f;
        }
    }
    __syncwarp();
    if (cnt > 0) {
        float a0 = 0.f, a1 = 0.f;
        for (int e = 0; e < cnt; e += 2) pair2(head + e, a0, a1);
        if (CNT && (cnt & 1)) --npairs;  // the padding entry is "in support" (q = 0)
        add(a0 + a1);
    }
    if (active) a.rho_sorted[oi] = (float)(((double)sum + (double)cmp) * s_inv);
    if (CNT) {
        if (!active) npairs = 0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) npairs += __shfl_xor_sync(0xffffffffu, npairs, o);
        if (lane == 0 && npairs) atomicAdd(a.pairs, npairs);
    }
}

template <int KER, int BW, bool CLIP>
static cudaError_t launch_points(const PointsArgs &a, int64_t nleaf, cudaStream_t s) {
    if (a.pairs) {
        KTimer t("k_points_count", s);
        return launch(k_points<KER, BW, CLIP, true>, dim3(blocks_for(nleaf, kPtWarps)),
                      dim3(kPtWarps * 32), 0, s, a);
    }
    KTimer t("k_points", s);
    return launch(k_points<KER, BW, CLIP, false>, dim3(blocks_for(nleaf, kPtWarps)),
                  dim3(kPtWarps * 32), 0, s, a);
}

template <int KER>
static cudaError_t dispatch_points(int bw, bool clip, const PointsArgs &a, int64_t nleaf,
                                   cudaStream_t s) {
    switch (bw * 2 + (clip ? 1 : 0)) {
        case BW_ISO * 2 + 0: return launch_points<KER, BW_ISO, false>(a, nleaf, s);
        case BW_ISO * 2 + 1: return launch_points<KER, BW_ISO, true>(a, nleaf, s);
        case BW_UNIFORM * 2 + 0: return launch_points<KER, BW_UNIFORM, false>(a, nleaf, s);
        case BW_UNIFORM * 2 + 1: return launch_points<KER, BW_UNIFORM, true>(a, nleaf, s);
        case BW_ANISO * 2 + 0: return launch_points<KER, BW_ANISO, false>(a, nleaf, s);
        default: return launch_points<KER, BW_ANISO, true>(a, nleaf, s);
    }
}

// ---------------------------------------------------------------------------
// Tensor-core cross term (precision variants of the point densities)
//
// With coordinates taken relative to the query leaf's centre, the squared
// distance of query i and candidate j is |x_i|^2 + |y_j|^2 - 2 x_i . y_j; the
// cross term of a 32 x 32 block is a [32 x 8] . [8 x 32] product (features x,
// y, z, zero-padded) done by mma.sync m16n8k8 in TF32 (or as the 3-pass
// hi/lo split, "3xTF32", accurate to about 2^-21 of |x||y|), or m16n8k16 in
// BF16 (8 significant bits); the squared norms,
// the scaling by 1/h^2, the cutoff, the kernel and the compensated sums stay
// in FP32. Isotropic bandwidths only (the kNN rule).
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t to_tf32(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return r;
}

__device__ __forceinline__ void mma_tf32(float d[4], uint32_t a0, uint32_t a1, uint32_t b0) {
    // A rows (groupID, groupID + 8) x cols (tig, tig + 4): cols >= 4 are zero padding
    const uint32_t z = 0u;
    asm volatile(
        "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
        "{%8,%9}, {%0,%1,%2,%3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a0), "r"(a1), "r"(z), "r"(z), "r"(b0), "r"(z));
}

// BF16: m16n8k16 with the features in k = 0..3 (pairs (x, y), (z, 0) in the
// lanes with tig 0 and 1), k = 4..15 zero. a0 / a1: rows g / g + 8, b0: column g.
__device__ __forceinline__ void mma_bf16(float d[4], uint32_t a0, uint32_t a1, uint32_t b0) {
    const uint32_t z = 0u;
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
        "{%8,%9}, {%0,%1,%2,%3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a0), "r"(a1), "r"(z), "r"(z), "r"(b0), "r"(z));
}

// The TF32 fragment layout holds feature tig of a row in lane (g, tig); the BF16
// one wants features (2 tig, 2 tig + 1) packed in that lane (zero for tig >= 2).
__device__ __forceinline__ uint32_t bf16_pair_from_tf32_layout(float f) {
    const int lane = threadIdx.x & 31, tig = lane & 3;
    const float lo = __shfl_sync(0xffffffffu, f, (lane & ~3) | ((2 * tig) & 3));
    const float hi = __shfl_sync(0xffffffffu, f, (lane & ~3) | ((2 * tig + 1) & 3));
    uint32_t r;
    asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(tig < 2 ? hi : 0.f), "f"(tig < 2 ? lo : 0.f));
    return r;
}

template <int PREC>
__device__ __forceinline__ void cross_mma(float d[4], float a0f, float a1f, float b0f) {
    const uint32_t a0h = to_tf32(a0f), a1h = to_tf32(a1f), b0h = to_tf32(b0f);
    mma_tf32(d, a0h, a1h, b0h);
    if (PREC == SF_PREC_3XTF32) {
        const uint32_t a0l = to_tf32(a0f - __uint_as_float(a0h));
        const uint32_t a1l = to_tf32(a1f - __uint_as_float(a1h));
        const uint32_t b0l = to_tf32(b0f - __uint_as_float(b0h));
        mma_tf32(d, a0h, a1h, b0l);
        mma_tf32(d, a0l, a1l, b0h);
    }
}

struct TcWarpSmem {
    int stack[kStack];
    int leaves[kBatch];
    float4 yp[kLeaf];   // candidate relative position (x', y', z', -)
    float4 yk[kLeaf];   // (|y'|^2, u^2, c, -)
};

template <int KER, bool CLIP, int PREC>
__global__ void __launch_bounds__(kPtWarps * 32) k_points_tc(PointsArgs a) {
    __shared__ TcWarpSmem W[kPtWarps];
    __shared__ double s_inv;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int g = lane >> 2, tig = lane & 3;
    if (threadIdx.x == 0) s_inv = a.e.dp->inv_neff;
    __syncthreads();
    TcWarpSmem &S = W[warp];
    const int64_t slot = (int64_t)blockIdx.x * kPtWarps + warp;
    if (slot >= a.nslots) return;
    const int64_t leaf = a.leaves ? (int64_t)a.leaves[slot] : slot;
    const int64_t qi = leaf * kLeaf + lane;
    const int64_t oi = slot * kLeaf + lane;
    const bool valid = qi < a.e.tv.n;
    float4 q = make_float4(0.f, 0.f, 0.f, 0.f);
    if (valid) q = __ldg(&a.e.tv.pos[qi]);
    const bool active = valid && q.x >= a.e.blo[0] && q.x <= a.e.bhi[0] && q.y >= a.e.blo[1] &&
                        q.y <= a.e.bhi[1] && q.z >= a.e.blo[2] && q.z <= a.e.bhi[2];
    a.inroi[oi] = active ? 1 : 0;
    const unsigned am = __ballot_sync(0xffffffffu, active);
    if (am == 0) return;
    float tlo[3] = {active ? q.x : INFINITY, active ? q.y : INFINITY, active ? q.z : INFINITY};
    float thi[3] = {active ? q.x : -INFINITY, active ? q.y : -INFINITY, active ? q.z : -INFINITY};
#pragma unroll
    for (int k = 0; k < 3; ++k)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            tlo[k] = fminf(tlo[k], __shfl_xor_sync(0xffffffffu, tlo[k], o));
            thi[k] = fmaxf(thi[k], __shfl_xor_sync(0xffffffffu, thi[k], o));
        }
    const float cen[3] = {0.5f * (tlo[0] + thi[0]), 0.5f * (tlo[1] + thi[1]), 0.5f * (tlo[2] + thi[2])};
    // this lane's four rows (queries g, g+8, g+16, g+24) relative to the centre
    const float xq[3] = {q.x - cen[0], q.y - cen[1], q.z - cen[2]};
    float feat[4], xsq[4];
#pragma unroll
    for (int sl = 0; sl < 4; ++sl) {
        const int r = g + 8 * sl;
        const float rx = __shfl_sync(0xffffffffu, xq[0], r);
        const float ry = __shfl_sync(0xffffffffu, xq[1], r);
        const float rz = __shfl_sync(0xffffffffu, xq[2], r);
        feat[sl] = tig == 0 ? rx : (tig == 1 ? ry : (tig == 2 ? rz : 0.f));
        xsq[sl] = fmaf(rz, rz, fmaf(ry, ry, rx * rx));
    }
    uint32_t fa16[4] = {0u, 0u, 0u, 0u};  // BF16 A fragments of the four rows
    if (PREC == SF_PREC_BF16) {
#pragma unroll
        for (int sl = 0; sl < 4; ++sl) fa16[sl] = bf16_pair_from_tf32_layout(feat[sl]);
    }
    float uni[3] = {0.f, 0.f, 0.f};
    float wlo[3], whi[3];
    widen_box(tlo, thi, wlo, whi);
    auto test = [&](int64_t node) { return node_reaches<KER, BW_ISO, CLIP>(a.e, uni, node, wlo, whi); };

    float acc[4] = {0.f, 0.f, 0.f, 0.f}, sum[4] = {0.f, 0.f, 0.f, 0.f}, cmp[4] = {0.f, 0.f, 0.f, 0.f};
    int spv;
    int nl = warp_walk_start(a.e.tv, test, S.stack, spv, S.leaves);
    while (true) {
        if (nl == 0) {
            if (spv == 0) break;
            nl = warp_walk(a.e.tv, test, S.stack, spv, S.leaves, kBatch);
            if (nl == 0) break;
        }
        for (int li = 0; li < nl; ++li) {
            const int64_t j = (int64_t)S.leaves[li] * kLeaf + lane;
            bool ok = false;
            float4 p = make_float4(0.f, 0.f, 0.f, 0.f);
            if (j < a.e.tv.n) {
                p = __ldg(&a.e.tv.pos[j]);
                ok = p.w > 0.f;
                if (CLIP)
                    ok = ok && p.x >= a.e.blo[0] && p.x <= a.e.bhi[0] && p.y >= a.e.blo[1] &&
                         p.y <= a.e.bhi[1] && p.z >= a.e.blo[2] && p.z <= a.e.bhi[2];
                const float pc[3] = {p.x, p.y, p.z};
                float qlb = 0.f;
#pragma unroll
                for (int k = 0; k < 3; ++k) {
                    float gap = fmaxf(fmaxf(tlo[k] - pc[k], pc[k] - thi[k]), 0.f);
                    gap = fmaxf(gap - 1.0e-6f * (fabsf(tlo[k]) + fabsf(thi[k])), 0.f);
                    const float t = gap / (p.w * KDef<KER>::rmul);
                    qlb += t * t;
                }
                ok = ok && qlb < 1.0f + 1.0e-5f;
            }
            const unsigned m = __ballot_sync(0xffffffffu, ok);
            if (ok) {
                const int s = __popc(m & ((1u << lane) - 1u));
                const float y0 = p.x - cen[0], y1 = p.y - cen[1], y2 = p.z - cen[2];
                const float u = KDef<KER>::uscale / p.w;
                S.yp[s] = make_float4(y0, y1, y2, 0.f);
                S.yk[s] = make_float4(fmaf(y2, y2, fmaf(y1, y1, y0 * y0)), u * u,
                                      a.e.cnorm / ((p.w * p.w) * p.w), 0.f);
            }
            __syncwarp();
            const int ns = __popc(m);
            for (int nt = 0; nt * 8 < ns; ++nt) {
                // B column g = candidate nt*8 + g, feature row tig: -2 y'
                const int cb = nt * 8 + g;
                float bf = 0.f;
                if (cb < ns && tig < 3) {
                    const float4 y = S.yp[cb];
                    bf = -2.f * (tig == 0 ? y.x : (tig == 1 ? y.y : y.z));
                }
                float d0[4] = {0.f, 0.f, 0.f, 0.f}, d1[4] = {0.f, 0.f, 0.f, 0.f};
                if (PREC == SF_PREC_BF16) {
                    const uint32_t b16 = bf16_pair_from_tf32_layout(bf);
                    mma_bf16(d0, fa16[0], fa16[1], b16);     // rows g, g+8
                    mma_bf16(d1, fa16[2], fa16[3], b16);     // rows g+16, g+24
                } else {
                    cross_mma<PREC>(d0, feat[0], feat[1], bf);   // rows g, g+8
                    cross_mma<PREC>(d1, feat[2], feat[3], bf);   // rows g+16, g+24
                }
                // epilogue: columns 2 tig, 2 tig + 1 of this n-tile
#pragma unroll
                for (int cc = 0; cc < 2; ++cc) {
                    const int jc = nt * 8 + 2 * tig + cc;
                    if (jc < ns) {
                        const float4 yk = S.yk[jc];
                        const float dv[4] = {d0[cc], d0[2 + cc], d1[cc], d1[2 + cc]};
#pragma unroll
                        for (int sl = 0; sl < 4; ++sl) {
                            const float d2 = (xsq[sl] + yk.x) + dv[sl];
                            const float qq = fmaxf(d2, 0.f) * yk.y;
                            if (qq < KDef<KER>::qmax) {
                                if (KER == SF_K_GAUSS3) acc[sl] = fmaf(yk.z, ex2_approx(-qq), acc[sl]);
                                else acc[sl] = fmaf(yk.z, 1.0f - qq, acc[sl]);
                            }
                        }
                    }
                }
            }
            __syncwarp();
#pragma unroll
            for (int sl = 0; sl < 4; ++sl) {
                const float t = sum[sl] + acc[sl];
                const float bp = t - sum[sl];
                cmp[sl] += (sum[sl] - (t - bp)) + (acc[sl] - bp);
                sum[sl] = t;
                acc[sl] = 0.f;
            }
        }
        nl = 0;
    }
    // rows are spread over the four lanes of a group: add them up, then route row L to lane L
    double v[4];
#pragma unroll
    for (int sl = 0; sl < 4; ++sl) {
        v[sl] = (double)sum[sl] + (double)cmp[sl];
        v[sl] += __shfl_xor_sync(0xffffffffu, v[sl], 1);
        v[sl] += __shfl_xor_sync(0xffffffffu, v[sl], 2);
    }
    const int src = 4 * (lane & 7), mysl = lane >> 3;
    double mine = 0.0;
#pragma unroll
    for (int sl = 0; sl < 4; ++sl) {
        const double t = __shfl_sync(0xffffffffu, v[sl], src);
        if (sl == mysl) mine = t;
    }
    if (active) a.rho_sorted[oi] = (float)(mine * s_inv);
}

template <int KER, bool CLIP>
static cudaError_t launch_points_tc(int prec, const PointsArgs &a, int64_t nleaf, cudaStream_t s) {
    KTimer t("k_points_tc", s);
    if (prec == SF_PREC_BF16)
        return launch(k_points_tc<KER, CLIP, SF_PREC_BF16>, dim3(blocks_for(nleaf, kPtWarps)),
                      dim3(kPtWarps * 32), 0, s, a);
    if (prec == SF_PREC_3XTF32)
        return launch(k_points_tc<KER, CLIP, SF_PREC_3XTF32>, dim3(blocks_for(nleaf, kPtWarps)),
                      dim3(kPtWarps * 32), 0, s, a);
    return launch(k_points_tc<KER, CLIP, SF_PREC_TF32>, dim3(blocks_for(nleaf, kPtWarps)),
                  dim3(kPtWarps * 32), 0, s, a);
}

sf_status density_points_tc(sf_index *idx, const sf_box &roi, const DensityCall &call, int prec,
                            const int *d_leaves, int64_t nslots, float *d_rho_sorted,
                            uint8_t *d_inroi, cudaStream_t s) {
    if (call.bw != BW_ISO)
        return fail(SF_ERR_INVALID_ARG, "tensor-core point densities need isotropic (kNN) bandwidths");
    PointsArgs a;
    a.e = engine_args(idx, roi, call);
    a.leaves = d_leaves;
    a.nslots = d_leaves ? nslots : idx->cnt[0];
    a.rho_sorted = d_rho_sorted;
    a.inroi = d_inroi;
    a.pairs = nullptr;
    const int64_t nl = a.nslots;
    cudaError_t e;
    if (call.kernel == SF_K_EPAN)
        e = call.clip ? launch_points_tc<SF_K_EPAN, true>(prec, a, nl, s) : launch_points_tc<SF_K_EPAN, false>(prec, a, nl, s);
    else
        e = call.clip ? launch_points_tc<SF_K_GAUSS3, true>(prec, a, nl, s) : launch_points_tc<SF_K_GAUSS3, false>(prec, a, nl, s);
    SF_TRY_CUDA(e);
    return SF_OK;
}

sf_status density_points(sf_index *idx, const sf_box &roi, const DensityCall &call,
                         const int *d_leaves, int64_t nslots, float *d_rho_sorted,
                         uint8_t *d_inroi, cudaStream_t s, unsigned long long *d_pairs) {
    PointsArgs a;
    a.e = engine_args(idx, roi, call);
    a.leaves = d_leaves;
    a.nslots = d_leaves ? nslots : idx->cnt[0];
    a.rho_sorted = d_rho_sorted;
    a.inroi = d_inroi;
    a.pairs = d_pairs;
    cudaError_t e = (call.kernel == SF_K_EPAN)
                        ? dispatch_points<SF_K_EPAN>(call.bw, call.clip != 0, a, a.nslots, s)
                        : dispatch_points<SF_K_GAUSS3>(call.bw, call.clip != 0, a, a.nslots, s);
    SF_TRY_CUDA(e);
    return SF_OK;
}

}  // namespace sf
