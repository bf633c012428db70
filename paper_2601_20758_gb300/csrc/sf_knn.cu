// sf_knn.cu -- exact k-nearest-neighbour bandwidths h_j (the kNN bandwidth
// rule: h_j = distance from point j to its k-th nearest other point).
//
// Exactness contract: the neighbour set equals the one a brute-force FP64
// evaluation gives with d2 = ((dx*dx)+(dy*dy))+(dz*dz), dx = (double)x_i -
// (double)x_j, ties broken by the smaller original index; h = (float)sqrt(d2_k).
//
// One warp per leaf of 32 Morton-consecutive query points:
//  1. radius bound: the k-th smallest FP32 d2 among the points of the nearby
//     leaves in sorted order (a per-lane histogram over [0, max]) bounds the
//     true k-th distance from above;
//  2. histogram pass: every point the index returns within that bound is
//     binned by its FP32 d2 (32 bins, per lane, in shared memory); the bin
//     holding the k-th is found;
//  3. band pass: points clearly below the bin are in; the few whose FP32 d2
//     lies within a relative 2e-6 of the bin are re-evaluated in FP64 (no FMA
//     contraction) and ranked by (d2, original index). If a band overflows its
//     buffer the bin is split again; at FP32 resolution (exact duplicates) the
//     remaining members are extracted one by one.
// FP32 d2 carries a relative error below 5 * 2^-24, so the 2e-6 margins make
// every in/out decision outside the band exact.
#include "sf_internal.cuh"

namespace sf {

constexpr int kKnnWarps = 4;
constexpr int kNB = 32;        // histogram bins per lane
constexpr int kBand = 16;      // band buffer per lane
constexpr int kKBatch = 64;    // leaves per traversal batch
constexpr int kKStack = 32 * kMaxLevels;
constexpr float kDelta = 2.0e-6f;

struct KnnWarpSmem {
    int stack[kKStack];
    int leaves[kKBatch];
    float4 pts[kLeaf];
    uint32_t ids[kLeaf];
    uint32_t hist[kNB][32];
    double bd[kBand][32];
    uint32_t bi[kBand][32];
};

struct KnnArgs {
    TreeView tv;
    const uint32_t *perm;
    int k;
    float *h_sorted;        // out: h per sorted point
    uint32_t *nbr_orig;     // out (nullable): [n][k] by original index
};

__device__ __forceinline__ float d2_f32(float4 a, float4 b) {
    const float dx = a.x - b.x, dy = a.y - b.y, dz = a.z - b.z;
    return fmaf(dz, dz, fmaf(dy, dy, dx * dx));
}

__device__ __forceinline__ double d2_f64(float4 a, float4 b) {
    const double dx = __dsub_rn((double)a.x, (double)b.x);
    const double dy = __dsub_rn((double)a.y, (double)b.y);
    const double dz = __dsub_rn((double)a.z, (double)b.z);
    return __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
}

__device__ __forceinline__ bool key_less(double da, uint32_t ia, double db, uint32_t ib) {
    return da < db || (da == db && ia < ib);
}

// Is any point of node i within sqrt(r2) of the box [qlo, qhi]? (conservative)
__device__ __forceinline__ bool node_near(const TreeView &tv, int64_t i, const float qlo[3],
                                          const float qhi[3], float r2) {
    const float4 lo = __ldg(&tv.nlo[i]);
    const float4 hi = __ldg(&tv.nhi[i]);
    const float nl[3] = {lo.x, lo.y, lo.z}, nh[3] = {hi.x, hi.y, hi.z};
    float d2 = 0.f;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        float gap = fmaxf(fmaxf(nl[k] - qhi[k], qlo[k] - nh[k]), 0.f);
        gap = fmaxf(gap - 1.0e-6f * (fabsf(qlo[k]) + fabsf(qhi[k])), 0.f);
        d2 = fmaf(gap, gap, d2);
    }
    return d2 <= r2 * (1.0f + 1.0e-5f);
}

// Same resumable walk as the density engine (duplicated here to keep the
// translation units independent).
template <typename Test>
__device__ int knn_walk(const TreeView &tv, const Test &test, int *stack, int &sp, int *out,
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
        const int r = __popc(m & lt), kk = __popc(m);
        if (cl == 0) {
            if (ok) out[nout + r] = (int)c;
            nout += kk;
        } else {
            if (ok) stack[sp + (kk - 1 - r)] = (cl << 27) | (int)c;
            sp += kk;
        }
        __syncwarp();
    }
    return nout;
}

// Visit every point of every leaf the walk accepts, in traversal order:
// fn(point float4, original id, sorted index) is called by every lane for each
// of the (up to) 32 points of a leaf (the same point on all lanes).
template <typename Test, typename Fn>
__device__ void for_each_candidate(const KnnArgs &a, KnnWarpSmem &S, const Test &test, Fn fn) {
    const int lane = threadIdx.x & 31;
    const TreeView &tv = a.tv;
    const int top = tv.nlevels - 1;
    int sp = 0;
    int nl = 0;
    const bool root_ok = __shfl_sync(0xffffffffu, lane == 0 ? (int)test(tv.off[top]) : 0, 0) != 0;
    if (!root_ok) return;
    if (top == 0) {
        if (lane == 0) S.leaves[0] = 0;
        __syncwarp();
        nl = 1;
    } else {
        if (lane == 0) S.stack[0] = top << 27;
        __syncwarp();
        sp = 1;
    }
    while (true) {
        if (nl == 0) {
            if (sp == 0) break;
            nl = knn_walk(tv, test, S.stack, sp, S.leaves, kKBatch);
            if (nl == 0) break;
        }
        for (int li = 0; li < nl; ++li) {
            const int64_t base = (int64_t)S.leaves[li] * kLeaf;
            const int64_t j = base + lane;
            if (j < tv.n) {
                S.pts[lane] = __ldg(&tv.pos[j]);
                S.ids[lane] = __ldg(&a.perm[j]);
            }
            __syncwarp();
            const int cnt = (int)(tv.n - base < kLeaf ? tv.n - base : kLeaf);
            for (int t = 0; t < cnt; ++t) fn(S.pts[t], S.ids[t], base + t);
            __syncwarp();
        }
        nl = 0;
    }
}

__global__ void __launch_bounds__(kKnnWarps * 32) k_knn(KnnArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    KnnWarpSmem &S = reinterpret_cast<KnnWarpSmem *>(smem_raw)[threadIdx.x >> 5];
    const int lane = threadIdx.x & 31;
    const TreeView &tv = a.tv;
    const int64_t leaf = (int64_t)blockIdx.x * kKnnWarps + (threadIdx.x >> 5);
    if (leaf >= tv.cnt[0]) return;
    const int k = a.k;
    const int64_t qi = leaf * kLeaf + lane;
    const bool valid = qi < tv.n;
    const float4 q = valid ? __ldg(&tv.pos[qi]) : make_float4(0.f, 0.f, 0.f, 0.f);
    const uint32_t qid = valid ? __ldg(&a.perm[qi]) : 0u;

    auto clear_hist = [&]() {
        for (int b = 0; b < kNB; ++b) S.hist[b][lane] = 0;
        __syncwarp();
    };

    // ---- 1. radius bound from the neighbouring leaves in sorted order
    const int64_t nleaf = tv.cnt[0];
    const int64_t wl = (int64_t)((k + 1 + 31) / 32) + 2;
    int64_t w0 = leaf - wl / 2, w1;
    if (w0 < 0) w0 = 0;
    w1 = w0 + wl - 1;
    if (w1 >= nleaf) {
        w1 = nleaf - 1;
        w0 = w1 - wl + 1 < 0 ? 0 : w1 - wl + 1;
    }
    auto window_visit = [&](auto fn) {
        for (int64_t L = w0; L <= w1; ++L) {
            const int64_t base = L * kLeaf;
            if (base + lane < tv.n) S.pts[lane] = __ldg(&tv.pos[base + lane]);
            __syncwarp();
            const int cnt = (int)(tv.n - base < kLeaf ? tv.n - base : kLeaf);
            for (int t = 0; t < cnt; ++t) fn(S.pts[t], base + t);
            __syncwarp();
        }
    };
    float wmax = 0.f;
    window_visit([&](float4 p, int64_t j) {
        if (j != qi) wmax = fmaxf(wmax, d2_f32(q, p));
    });
    clear_hist();
    const float winv = wmax > 0.f ? (float)kNB / wmax : 0.f;
    window_visit([&](float4 p, int64_t j) {
        if (valid && j != qi) {
            const int b = min(kNB - 1, (int)(d2_f32(q, p) * winv));
            S.hist[b][lane] += 1;
        }
    });
    __syncwarp();
    float T = 0.f;  // squared radius holding at least k points
    {
        int cum = 0, b = 0;
        for (; b < kNB; ++b) {
            cum += S.hist[b][lane];
            if (cum >= k) break;
        }
        const float edge = (b >= kNB - 1) ? wmax : (float)(b + 1) * (wmax / (float)kNB);
        T = edge * (1.0f + 4.0e-6f) + 1.0e-37f;
    }
    if (!valid) T = 0.f;

    // query box and traversal radius (warp-wide)
    float qlo[3] = {valid ? q.x : INFINITY, valid ? q.y : INFINITY, valid ? q.z : INFINITY};
    float qhi[3] = {valid ? q.x : -INFINITY, valid ? q.y : -INFINITY, valid ? q.z : -INFINITY};
    float Tmax = T;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        Tmax = fmaxf(Tmax, __shfl_xor_sync(0xffffffffu, Tmax, o));
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            qlo[d] = fminf(qlo[d], __shfl_xor_sync(0xffffffffu, qlo[d], o));
            qhi[d] = fmaxf(qhi[d], __shfl_xor_sync(0xffffffffu, qhi[d], o));
        }
    }
    auto test = [&](int64_t node) { return node_near(tv, node, qlo, qhi, Tmax); };

    // ---- 2./3. histogram and band passes, refined until the band fits
    float lo_e = 0.f, hi_e = T;  // current bracket [lo_e, hi_e] in FP32 d2
    int below_base = 0;          // points with d2 < lo_e (exact side, see margins)
    bool done = !valid;
    int need = 0;
    double kth = 0.0;
    bool extract = false;        // fallback: extract band members one by one
    float band_lo = 0.f, band_hi = 0.f;
    int nb_below = 0;
    for (int round = 0; round < 8; ++round) {
        const bool any = __any_sync(0xffffffffu, !done && !extract);
        if (!any) break;
        // histogram of d2 within [lo_e, hi_e]
        clear_hist();
        const float width = hi_e - lo_e;
        const float inv = width > 0.f ? (float)kNB / width : 0.f;
        const bool act = !done && !extract;
        int below = 0;
        for_each_candidate(a, S, test, [&](float4 p, uint32_t, int64_t j) {
            if (act && j != qi) {
                const float d = d2_f32(q, p);
                if (d < lo_e) ++below;
                else if (d <= hi_e) {
                    const int b = min(kNB - 1, (int)((d - lo_e) * inv));
                    S.hist[b][lane] += 1;
                }
            }
        });
        __syncwarp();
        float e_lo = lo_e, e_hi = hi_e;
        if (act) {
            int cum = below, b = 0;
            for (; b < kNB; ++b) {
                const int c = S.hist[b][lane];
                if (cum + c >= k) break;
                cum += c;
            }
            if (b >= kNB) b = kNB - 1;  // cannot happen: T bounds the k-th
            e_lo = lo_e + (float)b * (width / (float)kNB);
            e_hi = (b == kNB - 1) ? hi_e : lo_e + (float)(b + 1) * (width / (float)kNB);
            below_base = below;
        }
        // band pass
        band_lo = e_lo * (1.0f - kDelta);
        band_hi = e_hi * (1.0f + kDelta);
        int nbelow = 0, nband = 0;
        for_each_candidate(a, S, test, [&](float4 p, uint32_t id, int64_t j) {
            if (act && j != qi) {
                const float d = d2_f32(q, p);
                if (d < band_lo) ++nbelow;
                else if (d <= band_hi) {
                    if (nband < kBand) {
                        S.bd[nband][lane] = d2_f64(q, p);
                        S.bi[nband][lane] = id;
                    }
                    ++nband;
                }
            }
        });
        __syncwarp();
        if (act) {
            need = k - nbelow;
            nb_below = nbelow;
            if (nband <= kBand) {
                // sort the band by (d2, id), take the need-th
                for (int x = 1; x < nband; ++x) {
                    const double dv = S.bd[x][lane];
                    const uint32_t iv = S.bi[x][lane];
                    int y = x - 1;
                    while (y >= 0 && key_less(dv, iv, S.bd[y][lane], S.bi[y][lane])) {
                        S.bd[y + 1][lane] = S.bd[y][lane];
                        S.bi[y + 1][lane] = S.bi[y][lane];
                        --y;
                    }
                    S.bd[y + 1][lane] = dv;
                    S.bi[y + 1][lane] = iv;
                }
                const int pick = min(max(need, 1), min(nband, kBand)) - 1;
                kth = S.bd[pick][lane];
                done = true;
            } else if (round == 7 || !(e_hi - e_lo > 4.0f * kDelta * e_hi)) {
                extract = true;  // bin cannot shrink further (or out of rounds)
            } else {
                lo_e = e_lo;
                hi_e = e_hi;
            }
        }
        __syncwarp();
    }
    // ---- fallback: extract the need smallest band members one by one
    {
        double last_d = -1.0;
        uint32_t last_i = 0;
        bool first = true;
        int got = 0;
        while (__any_sync(0xffffffffu, extract && got < need)) {
            const bool act = extract && got < need;
            double best_d = INFINITY;
            uint32_t best_i = 0xffffffffu;
            for_each_candidate(a, S, test, [&](float4 p, uint32_t id, int64_t j) {
                if (act && j != qi) {
                    const float d = d2_f32(q, p);
                    if (d >= band_lo && d <= band_hi) {
                        const double dd = d2_f64(q, p);
                        const bool after = first || key_less(last_d, last_i, dd, id);
                        if (after && key_less(dd, id, best_d, best_i)) {
                            best_d = dd;
                            best_i = id;
                        }
                    }
                }
            });
            if (act) {
                if (a.nbr_orig && nb_below + got < k) a.nbr_orig[(int64_t)qid * k + nb_below + got] = best_i;
                last_d = best_d;
                last_i = best_i;
                first = false;
                ++got;
                if (got == need) {
                    kth = best_d;
                    done = true;
                }
            }
        }
    }
    if (valid) a.h_sorted[qi] = (float)sqrt(kth);

    // ---- optional neighbour ids: the below set, then the band's first `need`
    if (a.nbr_orig) {
        int slot = 0;
        for_each_candidate(a, S, test, [&](float4 p, uint32_t id, int64_t j) {
            if (valid && j != qi) {
                const float d = d2_f32(q, p);
                if (d < band_lo && slot < k) a.nbr_orig[(int64_t)qid * k + slot++] = id;
            }
        });
        if (valid && !extract)
            for (int x = 0; x < need && x < kBand && slot + x < k; ++x)
                a.nbr_orig[(int64_t)qid * k + slot + x] = S.bi[x][lane];
    }
}

__global__ void k_store_h(const float *__restrict__ h, int64_t n, float4 *__restrict__ pos) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        pos[i].w = h[i];
}

__global__ void k_scatter_h(const float4 *__restrict__ pos, const uint32_t *__restrict__ perm,
                            int64_t n, float *__restrict__ h_orig) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        h_orig[perm[i]] = pos[i].w;
}

__global__ void k_scatter_f(const float *__restrict__ v, const uint32_t *__restrict__ perm,
                            int64_t n, float *__restrict__ out) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        out[perm[i]] = v[i];
}

sf_status knn_run(sf_index *idx, int k, uint32_t *d_nbr_orig, float *d_h_sorted, cudaStream_t s) {
    KnnArgs a;
    a.tv = idx->view();
    a.perm = idx->perm;
    a.k = k;
    a.h_sorted = d_h_sorted;
    a.nbr_orig = d_nbr_orig;
    const size_t smem = sizeof(KnnWarpSmem) * kKnnWarps;
    static bool attr = false;
    if (!attr) {
        SF_TRY_CUDA(cudaFuncSetAttribute(k_knn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        attr = true;
    }
    SF_TRY_CUDA(launch(k_knn, dim3(blocks_for(idx->cnt[0], kKnnWarps)), dim3(kKnnWarps * 32), smem,
                       s, a));
    return SF_OK;
}

// Bandwidths resident in the index: h into pos.w, node maxima rebuilt.
sf_status knn_bandwidths(sf_index *idx, int k, uint32_t *d_nbr_orig, float *d_h_sorted,
                         cudaStream_t s) {
    Scratch sc(s);
    float *h = d_h_sorted ? d_h_sorted : sc.get<float>(idx->n);
    SF_TRY_SCRATCH(sc);
    SF_TRY(knn_run(idx, k, d_nbr_orig, h, s));
    const unsigned g = std::min<unsigned>(blocks_for(idx->n, 256), 152 * 16);
    SF_TRY_CUDA(launch(k_store_h, dim3(g), dim3(256), 0, s, (const float *)h, idx->n, idx->pos));
    SF_TRY(build_node_ell(idx, BW_ISO, nullptr, nullptr, idx->nell, s));
    return SF_OK;
}

sf_status knn_neighbours(sf_index *idx, int k, uint32_t *d_nbr_orig, float *d_h_orig,
                         cudaStream_t s) {
    Scratch sc(s);
    float *h = sc.get<float>(idx->n);
    SF_TRY_SCRATCH(sc);
    SF_TRY(knn_run(idx, k, d_nbr_orig, h, s));
    if (d_h_orig) {
        const unsigned g = std::min<unsigned>(blocks_for(idx->n, 256), 152 * 16);
        SF_TRY_CUDA(launch(k_scatter_f, dim3(g), dim3(256), 0, s, (const float *)h,
                           (const uint32_t *)idx->perm, idx->n, d_h_orig));
    }
    return SF_OK;
}

sf_status scatter_bandwidths(const sf_index *idx, float *d_h_orig, cudaStream_t s) {
    const unsigned g = std::min<unsigned>(blocks_for(idx->n, 256), 152 * 16);
    SF_TRY_CUDA(launch(k_scatter_h, dim3(g), dim3(256), 0, s, (const float4 *)idx->pos,
                       (const uint32_t *)idx->perm, idx->n, d_h_orig));
    return SF_OK;
}

}  // namespace sf
