// sf_density.cu -- the gather engine: kernel density at grid nodes and at points.
//
// What is computed (Sec. 3.1, Eq. 7; gather formulation of Sec. 3.2.1):
//   rho(r) = inv_neff * sum_j K(r - y_j ; l_j)
// over the particles of the scope, with K the Epanechnikov (Eq. 4) or the
// truncated Gaussian kernel and l_j the per-particle smoothing lengths. Every
// output is written by exactly one thread, in a fixed summation order: no
// atomics, results are deterministic.
//
// Grid: one CTA per 16 x 16 x 8 voxel tile; each thread owns one (x, y) column
// of 8 voxels in registers. Warp 0 walks the index for leaves whose support
// reaches the tile; their points are refined (footprint in the tile, ROI
// clip) and staged in shared memory, together with per-axis tables of the
// kernel factors at the tile's node coordinates, so the inner loop per
// (point, voxel) pair is two instructions (Gaussian: exp(a+b+c) = e^a e^b e^c
// with the truncation test on q_x + q_y < 9 - q_z) or three (Epanechnikov).
//
// Points: one warp per leaf of 32 query points; the warp walks the index for
// leaves whose support reaches the query points' box, stages the candidates
// in shared memory and every lane sums over them for its own point.
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

// Does node i possibly hold a particle whose support reaches the box [tlo, thi]?
// Conservative: gaps are shrunk by a margin covering float rounding of the box.
template <int KER, int BW, bool CLIP>
__device__ __forceinline__ bool node_reaches(const EngineArgs &a, const float *uni, int64_t i,
                                             const float tlo[3], const float thi[3]) {
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
        float gap = fmaxf(fmaxf(nl[k] - thi[k], tlo[k] - nh[k]), 0.f);
        float margin = 1.0e-6f * (fabsf(tlo[k]) + fabsf(thi[k])) + 1.0e-30f;
        gap = fmaxf(gap - margin, 0.f);
        float t = gap / (e[k] * KDef<KER>::rmul);
        q += t * t;
    }
    return q < 1.0f + 1.0e-5f;
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
static void float_bounds(const double lo[3], const double hi[3], float flo[3], float fhi[3]) {
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
struct GridArgs {
    EngineArgs e;
    const float2 *axis;  // node coordinates as (hi, lo) float pairs: x[nx], y[ny], z[nz]
    int nx, ny, nz;
    int tiles_x, tiles_y, tiles_z;
    float *out;
    double *mass_part;          // per tile, sum of rho (before the cell volume)
    unsigned long long *pairs;  // counting variant: in-support (voxel, particle) pairs
};

struct GridSmem {
    float2 tx[kStage][kTileX];   // Gauss: (c e^{-qx'}, qx'); Epan: (qx', -)
    float2 ty[kStage][kTileY];   // Gauss: (e^{-qy'}, qy');   Epan: (qy', -)
    float2 tz[kStage][kTileZ];   // Gauss: (e^{-qz'}, qmax - qz'); Epan: (c (1 - qz'), -)
    float4 sp[kStage];           // staged (x, y, z, c)
    float4 su[kStage];           // staged (u_x, u_y, u_z, -)
    int2 sf[kStage];             // staged footprint: x0|x1<<8|y0<<16|y1<<24, z0|z1<<8
    float2 axt[kTileX + kTileY + kTileZ];  // the tile's node coordinates
    uint8_t wlist[kGridThreads / 32][kStage];  // per warp: staged candidates touching its rows
    int stack[kStack];
    int leaves[kBatch];
    int wcnt[kGridThreads / 32];
    int nleaves, sp_top, item;
    float uni[3];
    double inv_neff;
    double red[kGridThreads / 32];
};

struct TileGeom {
    int gx0, gy0, gz0;
    int nv[3];
    float tlo[3], thi[3], sp3[3];
};

__device__ __forceinline__ void tile_origin(const GridArgs &a, int tile, int &gx0, int &gy0, int &gz0,
                                            int nv[3]) {
    const int tix = tile % a.tiles_x, tiy = (tile / a.tiles_x) % a.tiles_y,
              tiz = tile / (a.tiles_x * a.tiles_y);
    gx0 = tix * kTileX;
    gy0 = tiy * kTileY;
    gz0 = tiz * kTileZ;
    nv[0] = min(kTileX, a.nx - gx0);
    nv[1] = min(kTileY, a.ny - gy0);
    nv[2] = min(kTileZ, a.nz - gz0);
}

// The tile's node coordinates and the call's parameters into shared memory.
// Block-wide: every thread must call it (it contains a barrier).
__device__ TileGeom tile_setup(const GridArgs &a, GridSmem &S, int tile) {
    const int tid = threadIdx.x;
    TileGeom g;
    tile_origin(a, tile, g.gx0, g.gy0, g.gz0, g.nv);
    if (tid < kTileX + kTileY + kTileZ) {
        float2 v = make_float2(0.f, 0.f);
        if (tid < kTileX) {
            if (tid < g.nv[0]) v = a.axis[g.gx0 + tid];
        } else if (tid < kTileX + kTileY) {
            const int j = tid - kTileX;
            if (j < g.nv[1]) v = a.axis[a.nx + g.gy0 + j];
        } else {
            const int j = tid - kTileX - kTileY;
            if (j < g.nv[2]) v = a.axis[a.nx + a.ny + g.gz0 + j];
        }
        S.axt[tid] = v;
    }
    if (tid == 0) {
        const DensityParams dp = *a.e.dp;
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
template <int KER, int BW, bool CLIP, bool CNT>
__device__ void grid_chunk(const GridArgs &a, GridSmem &S, const TileGeom &g, const int *leaves,
                           int nl, float acc[kTileZ], unsigned long long &npairs) {
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
            if (i < a.e.tv.n) {
                p = __ldg(&a.e.tv.pos[i]);
                point_ell<BW>(a.e, S.uni, i, p, l);
                acc_pt = l[0] > 0.f && l[1] > 0.f && l[2] > 0.f;
                if (CLIP)
                    acc_pt = acc_pt && p.x >= a.e.blo[0] && p.x <= a.e.bhi[0] && p.y >= a.e.blo[1] &&
                             p.y <= a.e.bhi[1] && p.z >= a.e.blo[2] && p.z <= a.e.bhi[2];
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
        const float c = a.e.cnorm / ((l[0] * l[1]) * l[2]);
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
    for (int e = tid; e < ns * (kTileX + kTileY + kTileZ); e += kGridThreads) {
        const int s = e / (kTileX + kTileY + kTileZ);
        const int j = e - s * (kTileX + kTileY + kTileZ);
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
            for (int k = 0; k < kTileZ; ++k) {
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
            for (int k = 0; k < kTileZ; ++k) {
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
__device__ __forceinline__ void fold(float acc[kTileZ], float sum[kTileZ], float cmp[kTileZ]) {
#pragma unroll
    for (int k = 0; k < kTileZ; ++k) {
        const float t = sum[k] + acc[k];
        const float bp = t - sum[k];
        cmp[k] += (sum[k] - (t - bp)) + (acc[k] - bp);
        sum[k] = t;
        acc[k] = 0.f;
    }
}

__device__ __forceinline__ void count_pairs_out(const GridArgs &a, unsigned long long npairs) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) npairs += __shfl_xor_sync(0xffffffffu, npairs, o);
    if ((threadIdx.x & 31) == 0 && npairs) atomicAdd(a.pairs, npairs);
}

// Monolithic variant: one CTA walks the index for its tile and sums everything.
template <int KER, int BW, bool CLIP, bool CNT>
__global__ void __launch_bounds__(kGridThreads, 3) k_grid(GridArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    GridSmem &S = *reinterpret_cast<GridSmem *>(smem_raw);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int tile = blockIdx.x;
    const TileGeom g = tile_setup(a, S, tile);
    auto test = [&](int64_t node) { return node_reaches<KER, BW, CLIP>(a.e, S.uni, node, g.tlo, g.thi); };
    const int cx = lane & 15, cy = warp * 2 + (lane >> 4);
    unsigned long long npairs = 0;
    float acc[kTileZ], sum[kTileZ], cmp[kTileZ];
#pragma unroll
    for (int k = 0; k < kTileZ; ++k) acc[k] = sum[k] = cmp[k] = 0.f;

    if (warp == 0) {
        int spv;
        int n0 = warp_walk_start(a.e.tv, test, S.stack, spv, S.leaves);
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
            int n = warp_walk(a.e.tv, test, S.stack, spv, S.leaves, kBatch);
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
            grid_chunk<KER, BW, CLIP, CNT>(a, S, g, S.leaves + cb, min(kStage / kLeaf, nl - cb), acc,
                                           npairs);
            fold(acc, sum, cmp);
        }
        if (!more) break;
    }
    if (CNT) count_pairs_out(a, (cx < g.nv[0] && cy < g.nv[1]) ? npairs : 0ull);
    // ---- write the tile and its mass
    double msum = 0.0;
    const double inv_neff = S.inv_neff;
    if (cx < g.nv[0] && cy < g.nv[1]) {
        float *o = a.out + ((int64_t)g.gz0 * a.ny + (g.gy0 + cy)) * a.nx + (g.gx0 + cx);
        const int64_t zs = (int64_t)a.nx * a.ny;
#pragma unroll
        for (int k = 0; k < kTileZ; ++k) {
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
        a.mass_part[tile] = t;
    }
}

// ---------------------------------------------------------------------------
// Split pipeline: tiles over dense regions hold far more candidates than
// others, so each tile's candidate leaves are listed first and cut into
// balanced work items; persistent CTAs sum the items into per-item partial
// grids, and a per-tile reduction adds the partials in item order.
// ---------------------------------------------------------------------------
constexpr int kWalkWarps = 8;

struct WalkWarpSmem {
    int stack[kStack];
    int leaves[kBatch];
};

// One warp per tile: count (EMIT = false) or list (EMIT = true) its candidate leaves.
template <int KER, int BW, bool CLIP, bool EMIT>
__global__ void __launch_bounds__(kWalkWarps * 32) k_grid_walk(GridArgs a, int ntiles,
                                                               uint32_t *cnt, const uint32_t *off,
                                                               int *list) {
    __shared__ WalkWarpSmem W[kWalkWarps];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int tile = blockIdx.x * kWalkWarps + warp;
    if (tile >= ntiles) return;
    WalkWarpSmem &S = W[warp];
    int gx0, gy0, gz0, nv[3];
    tile_origin(a, tile, gx0, gy0, gz0, nv);
    float tlo[3], thi[3];
    tlo[0] = a.axis[gx0].x;
    thi[0] = a.axis[gx0 + nv[0] - 1].x;
    tlo[1] = a.axis[a.nx + gy0].x;
    thi[1] = a.axis[a.nx + gy0 + nv[1] - 1].x;
    tlo[2] = a.axis[a.nx + a.ny + gz0].x;
    thi[2] = a.axis[a.nx + a.ny + gz0 + nv[2] - 1].x;
    float uni[3];
    {
        const DensityParams *dp = a.e.dp;
        uni[0] = dp->ell_uniform[0];
        uni[1] = dp->ell_uniform[1];
        uni[2] = dp->ell_uniform[2];
    }
    auto test = [&](int64_t node) { return node_reaches<KER, BW, CLIP>(a.e, uni, node, tlo, thi); };
    int spv;
    int nl = warp_walk_start(a.e.tv, test, S.stack, spv, S.leaves);
    uint32_t total = 0;
    const uint32_t base = EMIT ? off[tile] : 0u;
    while (true) {
        if (nl == 0) {
            if (spv == 0) break;
            nl = warp_walk(a.e.tv, test, S.stack, spv, S.leaves, kBatch);
            if (nl == 0) break;
        }
        if (EMIT)
            for (int i = lane; i < nl; i += 32) list[base + total + i] = S.leaves[i];
        total += nl;
        __syncwarp();
        nl = 0;
    }
    if (!EMIT && lane == 0) cnt[tile] = total;
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

template <int KER, int BW, bool CLIP, bool CNT>
__global__ void __launch_bounds__(kGridThreads, 3)
    k_grid_work(GridArgs a, const int4 *__restrict__ items, const uint32_t *__restrict__ n_items,
                const int *__restrict__ list, double *__restrict__ part, unsigned int *next) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    GridSmem &S = *reinterpret_cast<GridSmem *>(smem_raw);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int cx = lane & 15, cy = warp * 2 + (lane >> 4);
    const uint32_t nitems = *n_items;
    unsigned long long npairs = 0;
    while (true) {
        if (tid == 0) S.item = (int)atomicAdd(next, 1u);
        __syncthreads();
        const int item = S.item;
        if ((uint32_t)item >= nitems) break;
        const int4 it = items[item];
        const TileGeom g = tile_setup(a, S, it.x);
        float acc[kTileZ], sum[kTileZ], cmp[kTileZ];
#pragma unroll
        for (int k = 0; k < kTileZ; ++k) acc[k] = sum[k] = cmp[k] = 0.f;
        unsigned long long np = 0;
        for (int lb = it.y; lb < it.z; lb += kStage / kLeaf) {
            grid_chunk<KER, BW, CLIP, CNT>(a, S, g, list + lb, min(kStage / kLeaf, it.z - lb), acc, np);
            fold(acc, sum, cmp);
        }
        if (CNT && cx < g.nv[0] && cy < g.nv[1]) npairs += np;
        double *o = part + ((int64_t)item * kGridThreads + tid) * kTileZ;
#pragma unroll
        for (int k = 0; k < kTileZ; ++k) o[k] = (double)sum[k] + (double)cmp[k];
    }
    if (CNT) count_pairs_out(a, npairs);
}

// Per tile: sum the items' partial grids in item order, scale, write, and the tile's mass.
__global__ void __launch_bounds__(kGridThreads) k_grid_reduce(GridArgs a,
                                                              const uint32_t *__restrict__ ic,
                                                              const uint32_t *__restrict__ ioff,
                                                              const double *__restrict__ part) {
    __shared__ double red[kGridThreads / 32];
    const int tile = blockIdx.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int cx = lane & 15, cy = warp * 2 + (lane >> 4);
    int gx0, gy0, gz0, nv[3];
    tile_origin(a, tile, gx0, gy0, gz0, nv);
    const double inv_neff = a.e.dp->inv_neff;
    double v[kTileZ];
#pragma unroll
    for (int k = 0; k < kTileZ; ++k) v[k] = 0.0;
    const uint32_t i0 = ioff[tile], ni = ic[tile];
    for (uint32_t i = 0; i < ni; ++i) {
        const double *pp = part + ((int64_t)(i0 + i) * kGridThreads + tid) * kTileZ;
#pragma unroll
        for (int k = 0; k < kTileZ; ++k) v[k] += pp[k];
    }
    double msum = 0.0;
    if (cx < nv[0] && cy < nv[1]) {
        float *o = a.out + ((int64_t)gz0 * a.ny + (gy0 + cy)) * a.nx + (gx0 + cx);
        const int64_t zs = (int64_t)a.nx * a.ny;
#pragma unroll
        for (int k = 0; k < kTileZ; ++k) {
            if (k < nv[2]) {
                const float fv = (float)(v[k] * inv_neff);
                o[k * zs] = fv;
                msum += (double)fv;
            }
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) msum += __shfl_xor_sync(0xffffffffu, msum, o);
    if (lane == 0) red[warp] = msum;
    __syncthreads();
    if (tid == 0) {
        double t = 0.0;
        for (int w = 0; w < kGridThreads / 32; ++w) t += red[w];
        a.mass_part[tile] = t;
    }
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

template <int KER, int BW, bool CLIP, bool CNT>
static cudaError_t launch_grid_t(const GridArgs &a, unsigned tiles, cudaStream_t s) {
    const size_t smem = sizeof(GridSmem);
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(k_grid<KER, BW, CLIP, CNT>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        attr = true;
    }
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

// The split pipeline for one (kernel, bandwidth mode, clip) combination.
template <int KER, int BW, bool CLIP>
static sf_status split_grid(const GridArgs &a0, int ntiles, cudaStream_t s) {
    GridArgs a = a0;
    Scratch sc(s);
    uint32_t *cnt = sc.get<uint32_t>(ntiles);
    uint32_t *off = sc.get<uint32_t>(ntiles);
    uint32_t *tot = sc.get<uint32_t>(2);
    SF_TRY_SCRATCH(sc);
    const unsigned wb = blocks_for(ntiles, kWalkWarps);
    SF_TRY_CUDA(launch(k_grid_walk<KER, BW, CLIP, false>, dim3(wb), dim3(kWalkWarps * 32), 0, s, a,
                       ntiles, cnt, (const uint32_t *)nullptr, (int *)nullptr));
    SF_TRY(scan_u32(cnt, off, ntiles, tot, s));
    uint32_t total = 0;
    SF_TRY_CUDA(cudaMemcpyAsync(&total, tot, sizeof total, cudaMemcpyDeviceToHost, s));
    SF_TRY_CUDA(cudaStreamSynchronize(s));
    int dev = 0, sms = 0, per_sm = 0;
    SF_TRY_CUDA(cudaGetDevice(&dev));
    SF_TRY_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const size_t smem = sizeof(GridSmem);
    static bool attr = false;
    if (!attr) {
        SF_TRY_CUDA(cudaFuncSetAttribute(k_grid_work<KER, BW, CLIP, false>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        SF_TRY_CUDA(cudaFuncSetAttribute(k_grid_work<KER, BW, CLIP, true>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        attr = true;
    }
    SF_TRY_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_grid_work<KER, BW, CLIP, false>,
                                                              kGridThreads, smem));
    if (per_sm < 1) per_sm = 1;
    const int64_t slots = (int64_t)sms * per_sm;
    // leaves per item: about four items per resident CTA, a multiple of the chunk
    uint32_t lpw = (uint32_t)std::max<int64_t>(16, (total + 4 * slots - 1) / (4 * slots));
    lpw = (lpw + 3) & ~3u;
    const int64_t max_items = ntiles + total / lpw + 1;
    int *list = sc.get<int>(std::max<int64_t>(1, total));
    uint32_t *ic = sc.get<uint32_t>(ntiles);
    uint32_t *ioff = sc.get<uint32_t>(ntiles);
    int4 *items = sc.get<int4>(max_items);
    double *part = sc.get<double>(max_items * kGridThreads * kTileZ);
    unsigned int *next = sc.get<unsigned int>(1);
    SF_TRY_SCRATCH(sc);
    SF_TRY_CUDA(launch(k_grid_walk<KER, BW, CLIP, true>, dim3(wb), dim3(kWalkWarps * 32), 0, s, a,
                       ntiles, (uint32_t *)nullptr, (const uint32_t *)off, list));
    SF_TRY_CUDA(launch(k_grid_item_counts, dim3(blocks_for(ntiles, 256)), dim3(256), 0, s,
                       (const uint32_t *)cnt, ntiles, lpw, ic));
    SF_TRY(scan_u32(ic, ioff, ntiles, tot + 1, s));
    SF_TRY_CUDA(launch(k_grid_items, dim3(blocks_for(ntiles, 256)), dim3(256), 0, s,
                       (const uint32_t *)cnt, (const uint32_t *)off, (const uint32_t *)ic,
                       (const uint32_t *)ioff, ntiles, lpw, items));
    SF_TRY_CUDA(cudaMemsetAsync(next, 0, sizeof(unsigned int), s));
    {
        KTimer t(a.pairs ? "k_grid_work_count" : "k_grid_work", s);
        if (a.pairs)
            SF_TRY_CUDA(launch(k_grid_work<KER, BW, CLIP, true>, dim3((unsigned)slots), dim3(kGridThreads),
                               smem, s, a, (const int4 *)items, (const uint32_t *)(tot + 1),
                               (const int *)list, part, next));
        else
            SF_TRY_CUDA(launch(k_grid_work<KER, BW, CLIP, false>, dim3((unsigned)slots), dim3(kGridThreads),
                               smem, s, a, (const int4 *)items, (const uint32_t *)(tot + 1),
                               (const int *)list, part, next));
    }
    SF_TRY_CUDA(launch(k_grid_reduce, dim3(ntiles), dim3(kGridThreads), 0, s, a, (const uint32_t *)ic,
                       (const uint32_t *)ioff, (const double *)part));
    return SF_OK;
}

template <int KER>
static sf_status dispatch_split(int bw, bool clip, const GridArgs &a, int ntiles, cudaStream_t s) {
    switch (bw * 2 + (clip ? 1 : 0)) {
        case BW_ISO * 2 + 0: return split_grid<KER, BW_ISO, false>(a, ntiles, s);
        case BW_ISO * 2 + 1: return split_grid<KER, BW_ISO, true>(a, ntiles, s);
        case BW_UNIFORM * 2 + 0: return split_grid<KER, BW_UNIFORM, false>(a, ntiles, s);
        case BW_UNIFORM * 2 + 1: return split_grid<KER, BW_UNIFORM, true>(a, ntiles, s);
        case BW_ANISO * 2 + 0: return split_grid<KER, BW_ANISO, false>(a, ntiles, s);
        default: return split_grid<KER, BW_ANISO, true>(a, ntiles, s);
    }
}

static float kernel_cnorm(int kernel) {
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

sf_status density_grid(sf_index *idx, const sf_box &roi, const GridSpec &g,
                       const DensityCall &call, float *d_out, double *d_mass, cudaStream_t s,
                       unsigned long long *d_pairs) {
    // node coordinates r_k(i) = lo_k + i s_k in double, split into float (hi, lo)
    std::vector<float2> ax((size_t)g.nx + g.ny + g.nz);
    const int nd[3] = {g.nx, g.ny, g.nz};
    size_t o = 0;
    for (int k = 0; k < 3; ++k)
        for (int i = 0; i < nd[k]; ++i) {
            const double r = g.lo[k] + (double)i * g.s[k];
            const float h = (float)r;
            ax[o++] = make_float2(h, (float)(r - (double)h));
        }
    GridArgs a;
    a.e = engine_args(idx, roi, call);
    a.nx = g.nx;
    a.ny = g.ny;
    a.nz = g.nz;
    a.tiles_x = (g.nx + kTileX - 1) / kTileX;
    a.tiles_y = (g.ny + kTileY - 1) / kTileY;
    a.tiles_z = (g.nz + kTileZ - 1) / kTileZ;
    const int64_t tiles = (int64_t)a.tiles_x * a.tiles_y * a.tiles_z;
    if (tiles >= (int64_t(1) << 31)) return fail(SF_ERR_INVALID_ARG, "grid too large");
    Scratch sc(s);
    float2 *d_axis = sc.get<float2>((int64_t)ax.size());
    double *mass_part = sc.get<double>(tiles);
    SF_TRY_SCRATCH(sc);
    SF_TRY_CUDA(cudaMemcpyAsync(d_axis, ax.data(), ax.size() * sizeof(float2),
                                cudaMemcpyHostToDevice, s));
    a.axis = d_axis;
    a.out = d_out;
    a.mass_part = mass_part;
    a.pairs = d_pairs;
    {
        KTimer t(d_pairs ? "k_grid_count" : "k_grid", s);
        if (call.kernel == SF_K_EPAN)
            SF_TRY(dispatch_split<SF_K_EPAN>(call.bw, call.clip != 0, a, (int)tiles, s));
        else
            SF_TRY(dispatch_split<SF_K_GAUSS3>(call.bw, call.clip != 0, a, (int)tiles, s));
    }
    if (d_mass) {
        const double cell = g.s[0] * g.s[1] * g.s[2];
        SF_TRY_CUDA(launch(k_mass_final, dim3(1), dim3(1024), 0, s, (const double *)mass_part,
                           tiles, cell, d_mass));
    }
    return SF_OK;
}

// Same result as density_grid with the monolithic kernel, on node coordinates
// and per-tile partial sums that the caller has already placed in device
// memory (no allocation here).
sf_status density_grid_prealloc(sf_index *idx, const sf_box &roi, const GridSpec &g,
                                const DensityCall &call, const float2 *d_axis,
                                double *d_mass_part, float *d_out, double *d_mass, cudaStream_t s) {
    GridArgs a;
    a.e = engine_args(idx, roi, call);
    a.nx = g.nx;
    a.ny = g.ny;
    a.nz = g.nz;
    a.tiles_x = (g.nx + kTileX - 1) / kTileX;
    a.tiles_y = (g.ny + kTileY - 1) / kTileY;
    a.tiles_z = (g.nz + kTileZ - 1) / kTileZ;
    const int64_t tiles = (int64_t)a.tiles_x * a.tiles_y * a.tiles_z;
    a.axis = d_axis;
    a.out = d_out;
    a.mass_part = d_mass_part;
    a.pairs = nullptr;
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
// Points (DIRECT)
// ===========================================================================
constexpr int kPtWarps = 4;

struct PointsArgs {
    EngineArgs e;
    float *rho_sorted;
    uint8_t *inroi;
    unsigned long long *pairs;  // counting variant
};

struct PtWarpSmem {
    int stack[kStack];
    int leaves[kBatch];
    float4 sp[kLeaf];
    float4 su[kLeaf];
};

template <int KER, int BW, bool CLIP, bool CNT>
__global__ void __launch_bounds__(kPtWarps * 32) k_points(PointsArgs a) {
    __shared__ PtWarpSmem W[kPtWarps];
    __shared__ float s_uni[3];
    __shared__ double s_inv;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (threadIdx.x == 0) {
        const DensityParams dp = *a.e.dp;
        s_uni[0] = dp.ell_uniform[0];
        s_uni[1] = dp.ell_uniform[1];
        s_uni[2] = dp.ell_uniform[2];
        s_inv = dp.inv_neff;
    }
    __syncthreads();
    PtWarpSmem &S = W[warp];
    const int64_t leaf = (int64_t)blockIdx.x * kPtWarps + warp;
    if (leaf >= a.e.tv.cnt[0]) return;
    const int64_t qi = leaf * kLeaf + lane;
    const bool valid = qi < a.e.tv.n;
    float4 q = make_float4(0.f, 0.f, 0.f, 0.f);
    if (valid) q = __ldg(&a.e.tv.pos[qi]);
    // query points: those inside the ROI box (closed)
    const bool active = valid && q.x >= a.e.blo[0] && q.x <= a.e.bhi[0] && q.y >= a.e.blo[1] &&
                        q.y <= a.e.bhi[1] && q.z >= a.e.blo[2] && q.z <= a.e.bhi[2];
    if (valid) a.inroi[qi] = active ? 1 : 0;
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
    auto test = [&](int64_t node) { return node_reaches<KER, BW, CLIP>(a.e, s_uni, node, tlo, thi); };

    float sum = 0.f, cmp = 0.f;
    unsigned long long npairs = 0;
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
            float l[3] = {0.f, 0.f, 0.f};
            if (j < a.e.tv.n) {
                if (BW == BW_ISO) {
                    l[0] = l[1] = l[2] = p.w;
                } else if (BW == BW_UNIFORM) {
                    l[0] = s_uni[0]; l[1] = s_uni[1]; l[2] = s_uni[2];
                } else {
                    l[0] = pe.x; l[1] = pe.y; l[2] = pe.z;
                }
                ok = l[0] > 0.f && l[1] > 0.f && l[2] > 0.f;
                if (CLIP)
                    ok = ok && p.x >= a.e.blo[0] && p.x <= a.e.bhi[0] && p.y >= a.e.blo[1] &&
                         p.y <= a.e.bhi[1] && p.z >= a.e.blo[2] && p.z <= a.e.bhi[2];
                const float pc[3] = {p.x, p.y, p.z};
                float qlb = 0.f;
#pragma unroll
                for (int k = 0; k < 3; ++k) {
                    float gap = fmaxf(fmaxf(tlo[k] - pc[k], pc[k] - thi[k]), 0.f);
                    gap = fmaxf(gap - 1.0e-6f * (fabsf(tlo[k]) + fabsf(thi[k])), 0.f);
                    const float t = gap / (l[k] * KDef<KER>::rmul);
                    qlb += t * t;
                }
                ok = ok && qlb < 1.0f + 1.0e-5f;
            }
            const unsigned m = __ballot_sync(0xffffffffu, ok);
            if (ok) {
                const int s = __popc(m & ((1u << lane) - 1u));
                S.sp[s] = make_float4(p.x, p.y, p.z, a.e.cnorm / ((l[0] * l[1]) * l[2]));
                const float u0 = KDef<KER>::uscale / l[0];
                if (BW == BW_ISO) {
                    S.su[s] = make_float4(u0 * u0, 0.f, 0.f, 0.f);
                } else {
                    S.su[s] = make_float4(u0, KDef<KER>::uscale / l[1], KDef<KER>::uscale / l[2], 0.f);
                }
            }
            __syncwarp();
            const int ns = __popc(m);
            float acc0 = 0.f, acc1 = 0.f;
            auto pair = [&](int s, float &acc) {
                const float4 P = S.sp[s];
                float qq;
                if (BW == BW_ISO) {
                    const float u2 = S.su[s].x;
                    const float dx = q.x - P.x, dy = q.y - P.y, dz = q.z - P.z;
                    qq = fmaf(dz, dz, fmaf(dy, dy, dx * dx)) * u2;
                } else {
                    const float4 U = S.su[s];
                    const float tx = (q.x - P.x) * U.x;
                    const float ty = (q.y - P.y) * U.y;
                    const float tz = (q.z - P.z) * U.z;
                    qq = fmaf(tz, tz, fmaf(ty, ty, tx * tx));
                }
                if (qq < KDef<KER>::qmax) {
                    if (KER == SF_K_GAUSS3) acc = fmaf(P.w, ex2_approx(-qq), acc);
                    else acc = fmaf(P.w, 1.0f - qq, acc);
                    if (CNT) ++npairs;
                }
            };
            int s = 0;
            for (; s + 2 <= ns; s += 2) {
                pair(s, acc0);
                pair(s + 1, acc1);
            }
            if (s < ns) pair(s, acc0);
            __syncwarp();
            const float acc = acc0 + acc1;
            const float t = sum + acc;
            const float bp = t - sum;
            cmp += (sum - (t - bp)) + (acc - bp);
            sum = t;
        }
        nl = 0;
    }
    if (active) a.rho_sorted[qi] = (float)(((double)sum + (double)cmp) * s_inv);
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

sf_status density_points(sf_index *idx, const sf_box &roi, const DensityCall &call,
                         float *d_rho_sorted, uint8_t *d_inroi, cudaStream_t s,
                         unsigned long long *d_pairs) {
    PointsArgs a;
    a.e = engine_args(idx, roi, call);
    a.rho_sorted = d_rho_sorted;
    a.inroi = d_inroi;
    a.pairs = d_pairs;
    cudaError_t e = (call.kernel == SF_K_EPAN)
                        ? dispatch_points<SF_K_EPAN>(call.bw, call.clip != 0, a, idx->cnt[0], s)
                        : dispatch_points<SF_K_GAUSS3>(call.bw, call.clip != 0, a, idx->cnt[0], s);
    SF_TRY_CUDA(e);
    return SF_OK;
}

}  // namespace sf
