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
    double *mass_part;   // per tile, sum of rho (before the cell volume)
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
    int stack[kStack];
    int leaves[kBatch];
    int wcnt[kGridThreads / 32];
    int nleaves, sp_top, nstage;
    float uni[3];
    double inv_neff;
    double red[kGridThreads / 32];
};

template <int KER, int BW, bool CLIP, bool CNT>
__global__ void __launch_bounds__(kGridThreads, 2) k_grid(GridArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    GridSmem &S = *reinterpret_cast<GridSmem *>(smem_raw);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int tile = blockIdx.x;
    const int tix = tile % a.tiles_x, tiy = (tile / a.tiles_x) % a.tiles_y,
              tiz = tile / (a.tiles_x * a.tiles_y);
    const int gx0 = tix * kTileX, gy0 = tiy * kTileY, gz0 = tiz * kTileZ;
    const int nvx = min(kTileX, a.nx - gx0), nvy = min(kTileY, a.ny - gy0),
              nvz = min(kTileZ, a.nz - gz0);

    if (tid < kTileX + kTileY + kTileZ) {
        float2 v = make_float2(0.f, 0.f);
        if (tid < kTileX) {
            if (tid < nvx) v = a.axis[gx0 + tid];
        } else if (tid < kTileX + kTileY) {
            const int j = tid - kTileX;
            if (j < nvy) v = a.axis[a.nx + gy0 + j];
        } else {
            const int j = tid - kTileX - kTileY;
            if (j < nvz) v = a.axis[a.nx + a.ny + gz0 + j];
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

    // tile box (float; node_reaches adds a rounding margin)
    float tlo[3], thi[3], sp3[3];
    tlo[0] = S.axt[0].x;
    thi[0] = S.axt[nvx - 1].x;
    tlo[1] = S.axt[kTileX].x;
    thi[1] = S.axt[kTileX + nvy - 1].x;
    tlo[2] = S.axt[kTileX + kTileY].x;
    thi[2] = S.axt[kTileX + kTileY + nvz - 1].x;
    // node spacing along each axis, for footprints (approximate; footprints are widened by 1)
    sp3[0] = nvx > 1 ? (S.axt[1].x - S.axt[0].x) : 1.f;
    sp3[1] = nvy > 1 ? (S.axt[kTileX + 1].x - S.axt[kTileX].x) : 1.f;
    sp3[2] = nvz > 1 ? (S.axt[kTileX + kTileY + 1].x - S.axt[kTileX + kTileY].x) : 1.f;
    const int nv[3] = {nvx, nvy, nvz};

    auto test = [&](int64_t node) { return node_reaches<KER, BW, CLIP>(a.e, S.uni, node, tlo, thi); };

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
            // ---- load and refine up to 128 candidate points (threads 0..127)
            bool acc_pt = false;
            float4 p = make_float4(0.f, 0.f, 0.f, 0.f);
            float l[3] = {0.f, 0.f, 0.f};
            int2 fp = make_int2(0, 0);
            if (tid < kStage) {
                const int li = cb + (tid >> 5);
                if (li < nl) {
                    const int64_t i = (int64_t)S.leaves[li] * kLeaf + lane;
                    if (i < a.e.tv.n) {
                        p = __ldg(&a.e.tv.pos[i]);
                        point_ell<BW>(a.e, S.uni, i, p, l);
                        acc_pt = l[0] > 0.f && l[1] > 0.f && l[2] > 0.f;
                        if (CLIP)
                            acc_pt = acc_pt && p.x >= a.e.blo[0] && p.x <= a.e.bhi[0] &&
                                     p.y >= a.e.blo[1] && p.y <= a.e.bhi[1] &&
                                     p.z >= a.e.blo[2] && p.z <= a.e.bhi[2];
                        const float pc[3] = {p.x, p.y, p.z};
                        int f0[3], f1[3];
                        float qlb = 0.f;
#pragma unroll
                        for (int k = 0; k < 3; ++k) {
                            const float R = l[k] * KDef<KER>::rmul;
                            if (sp3[k] > 0.f) {
                                const float a0 = fminf(fmaxf(ceilf((pc[k] - R - tlo[k]) / sp3[k]) - 1.f, -1.f), 64.f);
                                const float a1 = fminf(fmaxf(floorf((pc[k] + R - tlo[k]) / sp3[k]) + 1.f, -1.f), 64.f);
                                f0[k] = max(0, (int)a0);
                                f1[k] = min(nv[k] - 1, (int)a1);
                            } else {
                                f0[k] = 0;
                                f1[k] = nv[k] - 1;
                            }
                            if (f0[k] > f1[k]) acc_pt = false;
                            float gap = fmaxf(fmaxf(tlo[k] - pc[k], pc[k] - thi[k]), 0.f);
                            gap = fmaxf(gap - 1.0e-6f * (fabsf(tlo[k]) + fabsf(thi[k])), 0.f);
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
            int base = 0, tot = 0;
#pragma unroll
            for (int w = 0; w < kStage / 32; ++w) {
                const int c = S.wcnt[w];
                if (w < warp) base += c;
                tot += c;
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
            const int ns = tot;
            // ---- per-axis tables: 40 entries per staged point
            for (int e = tid; e < ns * (kTileX + kTileY + kTileZ); e += kGridThreads) {
                const int s = e / (kTileX + kTileY + kTileZ);
                const int j = e - s * (kTileX + kTileY + kTileZ);
                const float4 P = S.sp[s];
                const float4 U = S.su[s];
                const int2 F = S.sf[s];
                int axis, i, lo_i, hi_i;
                float pc, u;
                if (j < kTileX) {
                    axis = 0; i = j; lo_i = F.x & 255; hi_i = (F.x >> 8) & 255; pc = P.x; u = U.x;
                } else if (j < kTileX + kTileY) {
                    axis = 1; i = j - kTileX; lo_i = (F.x >> 16) & 255; hi_i = (F.x >> 24) & 255; pc = P.y; u = U.y;
                } else {
                    axis = 2; i = j - kTileX - kTileY; lo_i = F.y & 255; hi_i = (F.y >> 8) & 255; pc = P.z; u = U.z;
                }
                const bool in = i >= lo_i && i <= hi_i;
                const float2 nc = S.axt[j];
                const float d = (nc.x - pc) + nc.y;
                const float t = d * u;
                const float q = t * t;
                const bool sup = in && q < KDef<KER>::qmax;
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
            for (int s = 0; s < ns; ++s) {
                const int2 F = S.sf[s];
                const int y0 = (F.x >> 16) & 255, y1 = (F.x >> 24) & 255;
                if (warp * 2 + 1 < y0 || warp * 2 > y1) continue;
                const int z0 = F.y & 255, z1 = (F.y >> 8) & 255;
                const float2 ex = S.tx[s][cx];
                const float2 ey = S.ty[s][cy];
                if (KER == SF_K_GAUSS3) {
                    const float base = ex.x * ey.x;
                    const float qij = ex.y + ey.y;
#pragma unroll
                    for (int k = 0; k < kTileZ; ++k) {
                        if (k >= z0 && k <= z1) {
                            const float2 ez = S.tz[s][k];
                            if (qij < ez.y) {
                                acc[k] = fmaf(base, ez.x, acc[k]);
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
            // ---- fold the chunk into the compensated sums (TwoSum)
#pragma unroll
            for (int k = 0; k < kTileZ; ++k) {
                const float t = sum[k] + acc[k];
                const float bp = t - sum[k];
                cmp[k] += (sum[k] - (t - bp)) + (acc[k] - bp);
                sum[k] = t;
                acc[k] = 0.f;
            }
            __syncthreads();
        }
        if (!more) break;
    }

    if (CNT) {
        if (cx >= nvx || cy >= nvy) npairs = 0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) npairs += __shfl_xor_sync(0xffffffffu, npairs, o);
        if (lane == 0 && npairs) atomicAdd(a.pairs, npairs);
    }
    // ---- write the tile and its mass
    double msum = 0.0;
    const double inv_neff = S.inv_neff;
    if (cx < nvx && cy < nvy) {
        float *o = a.out + ((int64_t)gz0 * a.ny + (gy0 + cy)) * a.nx + (gx0 + cx);
        const int64_t zs = (int64_t)a.nx * a.ny;
#pragma unroll
        for (int k = 0; k < kTileZ; ++k) {
            if (k < nvz) {
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
    cudaError_t e = (call.kernel == SF_K_EPAN)
                        ? dispatch_grid<SF_K_EPAN>(call.bw, call.clip != 0, a, (unsigned)tiles, s)
                        : dispatch_grid<SF_K_GAUSS3>(call.bw, call.clip != 0, a, (unsigned)tiles, s);
    SF_TRY_CUDA(e);
    if (d_mass) {
        const double cell = g.s[0] * g.s[1] * g.s[2];
        SF_TRY_CUDA(launch(k_mass_final, dim3(1), dim3(1024), 0, s, (const double *)mass_part,
                           tiles, cell, d_mass));
    }
    return SF_OK;
}

// Same launch as density_grid, on node coordinates and per-tile partial sums
// that the caller has already placed in device memory (no allocation here).
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
        for (int li = 0; li < nl; ++li) {
            const int64_t j = (int64_t)S.leaves[li] * kLeaf + lane;
            bool ok = false;
            float4 p = make_float4(0.f, 0.f, 0.f, 0.f);
            float l[3] = {0.f, 0.f, 0.f};
            if (j < a.e.tv.n) {
                p = __ldg(&a.e.tv.pos[j]);
                point_ell<BW>(a.e, s_uni, j, p, l);
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
                S.su[s] = make_float4(KDef<KER>::uscale / l[0], KDef<KER>::uscale / l[1],
                                      KDef<KER>::uscale / l[2], 0.f);
            }
            __syncwarp();
            const int ns = __popc(m);
            float acc = 0.f;
            for (int s = 0; s < ns; ++s) {
                const float4 P = S.sp[s];
                const float4 U = S.su[s];
                const float tx = (q.x - P.x) * U.x;
                const float ty = (q.y - P.y) * U.y;
                const float tz = (q.z - P.z) * U.z;
                const float qq = fmaf(tz, tz, fmaf(ty, ty, tx * tx));
                if (qq < KDef<KER>::qmax) {
                    if (KER == SF_K_GAUSS3) acc = fmaf(P.w, ex2_approx(-qq), acc);
                    else acc = fmaf(P.w, 1.0f - qq, acc);
                    if (CNT) ++npairs;
                }
            }
            __syncwarp();
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
