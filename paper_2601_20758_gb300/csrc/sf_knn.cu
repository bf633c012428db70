// sf_knn.cu -- exact k-nearest-neighbour bandwidths h_j (the kNN bandwidth
// rule: h_j = distance from point j to its k-th nearest other point).
//
// Exactness contract: the neighbour set equals the one a brute-force FP64
// evaluation gives with d2 = ((dx*dx)+(dy*dy))+(dz*dz), dx = (double)x_i -
// (double)x_j, ties broken by the smaller original index; h = (float)sqrt(d2_k).
//
// Persistent warps; each takes the next leaf of 32 Morton-consecutive query
// points from an atomic counter (no warp waits for another):
//  1. radius bound: per lane, the k-th smallest FP32 d2 among the points of
//     nearby leaves in sorted order (a bin edge above it, from 32-bin
//     histograms of 5 then 13 leaves at k = 64) -- an upper bound of the true
//     k-th distance;
//  2. candidates: the index walk keeps the leaves within that radius of at
//     least one lane's point, and records them in a per-warp leaf list in
//     global memory; their points inside the warp's envelope box are the
//     candidates (every pass reloads them leaf by leaf);
//  3. histogram while collecting: per lane, 32 bins of FP32 d2 over [0, T];
//     the bin holding the k-th is found;
//  4. band pass: points clearly below the bin are in; the ones whose FP32 d2
//     lies in the bin (widened by a relative 2e-6) are re-evaluated in FP64 (no
//     FMA contraction) into a per-lane buffer of 64 in global memory and ranked
//     by (d2, original index) -- one pass resolves almost every lane; recorded
//     leaves whose box lies wholly below or above every lane's band are counted
//     from their envelope masks instead of being reloaded. If a band
//     overflows its buffer the bin is split again (the band pass has already
//     binned the bracket for that round); at FP32 resolution (exact duplicates)
//     the remaining members are extracted one by one.
// FP32 d2 carries a relative error below 5 * 2^-24, so the 2e-6 margins make
// every in/out decision outside the band exact. If a warp's accepted leaves
// exceed its list, its passes walk the index again instead (same result).
#include "sf_internal.cuh"

namespace sf {

constexpr int kKnnWarps = 4;
constexpr int kNB = 32;        // histogram bins per lane
constexpr int kBand = 64;      // band buffer per lane (global memory, interleaved by lane)
constexpr int kCand = 64;      // candidate leaves per walk batch
constexpr int kLeafList = 4096;  // accepted leaves recorded per warp (global)
constexpr int kKStack = 32 * kMaxLevels;
constexpr float kDelta = 2.0e-6f;

struct KnnWarpSmem {
    int stack[kKStack];
    int cand[kCand];
    float4 blo[32], bhi[32];   // child boxes under test
    float4 pts[kLeaf];         // staged candidates (x, y, z, original id bits)
    uint32_t hist[kNB][32];
};

struct KnnArgs {
    TreeView tv;
    const uint32_t *perm;
    int k;
    float *h_sorted;          // out: h per sorted point
    uint32_t *nbr_orig;       // out (nullable): [n][k] by original index
    int *leaf_list;           // [slots][kLeafList] accepted leaves of the current query leaf
    uint32_t *leaf_mask;      // [slots][kLeafList] their points inside the warp envelope
    double *band_d;           // [slots][kBand][32] band members' FP64 d2
    uint32_t *band_i;         // [slots][kBand][32] band members' original ids
    unsigned int *next_leaf;  // work counter (zeroed before launch)
    unsigned long long *work; // nullable: [0] candidates staged (all passes), [1] query leaves
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

// Per-warp candidate search: every lane holds one query point and the squared
// radius r2 of its ball (negative: the lane takes no part). COUNT: the work
// accounting variant (sf_knn_work_counts).
template <bool COUNT>
struct KnnWarp {
    const TreeView &tv;
    const uint32_t *perm;
    KnnWarpSmem &S;
    int *leaf_list;        // this warp's recorded leaves
    uint32_t *leaf_mask;   // and, per leaf, its points inside the envelope
    float4 q;
    float r2;
    float env_lo[3], env_hi[3];  // warp envelope of all balls
    int nlist;
    bool overflow;
    unsigned long long ncand = 0;  // COUNT only: candidates staged over all passes

    __device__ KnnWarp(const TreeView &t, const uint32_t *p, KnnWarpSmem &s, int *c, uint32_t *cm)
        : tv(t), perm(p), S(s), leaf_list(c), leaf_mask(cm) {}

    // Mask of the children (lane c holds child c at level cl) within the ball
    // of at least one lane. Conservative: relative slack 1e-5.
    __device__ unsigned accept(int cl, int64_t c, bool valid) {
        const int lane = threadIdx.x & 31;
        bool pre = false;
        float4 lo = make_float4(0.f, 0.f, 0.f, 0.f), hi = lo;
        if (valid) {
            lo = __ldg(&tv.nlo[tv.off[cl] + c]);
            hi = __ldg(&tv.nhi[tv.off[cl] + c]);
            pre = lo.x <= env_hi[0] && hi.x >= env_lo[0] && lo.y <= env_hi[1] && hi.y >= env_lo[1] &&
                  lo.z <= env_hi[2] && hi.z >= env_lo[2];
        }
        unsigned m = __ballot_sync(0xffffffffu, pre);
        if (pre) {
            S.blo[lane] = lo;
            S.bhi[lane] = hi;
        }
        __syncwarp();
        unsigned acc = 0;
        const float lim = r2 * (1.0f + 1.0e-5f);
        while (m) {
            const int j = __ffs(m) - 1;
            m &= m - 1;
            const float4 bl = S.blo[j], bh = S.bhi[j];
            const float gx = fmaxf(fmaxf(bl.x - q.x, q.x - bh.x), 0.f);
            const float gy = fmaxf(fmaxf(bl.y - q.y, q.y - bh.y), 0.f);
            const float gz = fmaxf(fmaxf(bl.z - q.z, q.z - bh.z), 0.f);
            const float d2 = fmaf(gz, gz, fmaf(gy, gy, gx * gx));
            if (__any_sync(0xffffffffu, r2 >= 0.f && d2 <= lim)) acc |= 1u << j;
        }
        __syncwarp();
        return acc;
    }

    // Resumable walk: appends accepted leaves to S.cand until fewer than 32
    // slots remain or the stack is empty.
    __device__ int walk(int &sp) {
        const int lane = threadIdx.x & 31;
        const unsigned lt = (1u << lane) - 1u;
        int nout = 0;
        while (sp > 0 && nout <= kCand - 32) {
            const int e = S.stack[sp - 1];
            __syncwarp();
            sp -= 1;
            const int cl = (e >> 27) - 1;
            const int64_t c = (int64_t)(e & ((1 << 27) - 1)) * kFanout + lane;
            const unsigned m = accept(cl, c, c < tv.cnt[cl]);
            const bool ok = (m >> lane) & 1u;
            const int r = __popc(m & lt), kk = __popc(m);
            if (cl == 0) {
                if (ok) S.cand[nout + r] = (int)c;
                nout += kk;
            } else {
                if (ok) S.stack[sp + (kk - 1 - r)] = (cl << 27) | (int)c;
                sp += kk;
            }
            __syncwarp();
        }
        return nout;
    }

    __device__ int start(int &sp) {
        const int top = tv.nlevels - 1;
        if (top == 0) {
            sp = 0;
            if ((threadIdx.x & 31) == 0) S.cand[0] = 0;
            __syncwarp();
            return 1;
        }
        if ((threadIdx.x & 31) == 0) S.stack[0] = top << 27;
        __syncwarp();
        sp = 1;
        return 0;
    }

    // Stage the envelope-filtered points of the leaves S.cand[0..nl), one leaf
    // at a time (the next leaf's points load while the current one is used):
    // chunk(n) is called with S.pts[0..n) staged (x, y, z, original id bits).
    template <typename Chunk>
    __device__ __forceinline__ void visit(int nl, Chunk chunk, int record = -1) {
        const int lane = threadIdx.x & 31;
        float4 pn = make_float4(0.f, 0.f, 0.f, 0.f);
        uint32_t idn = 0;
        auto load = [&](int li) {
            const int64_t j = (int64_t)S.cand[li] * kLeaf + lane;
            if (j < tv.n) {
                pn = __ldg(&tv.pos[j]);
                idn = __ldg(&perm[j]);
            }
        };
        if (nl > 0) load(0);
        for (int li = 0; li < nl; ++li) {
            const int64_t j = (int64_t)S.cand[li] * kLeaf + lane;
            float4 p = pn;
            p.w = __uint_as_float(idn);
            if (li + 1 < nl) load(li + 1);
            const bool in = j < tv.n && p.x >= env_lo[0] && p.x <= env_hi[0] && p.y >= env_lo[1] &&
                            p.y <= env_hi[1] && p.z >= env_lo[2] && p.z <= env_hi[2];
            const unsigned m = __ballot_sync(0xffffffffu, in);
            if (COUNT) ncand += __popc(m);
            if (in) S.pts[__popc(m & ((1u << lane) - 1u))] = p;
            if (record >= 0 && lane == 0 && record + li < kLeafList) leaf_mask[record + li] = m;
            __syncwarp();
            chunk(__popc(m));
            __syncwarp();
        }
    }

    // Every accepted leaf by walking the index.
    template <typename Chunk>
    __device__ __forceinline__ void walk_points(Chunk chunk) {
        int sp;
        int nl = start(sp);
        while (true) {
            if (nl == 0) {
                if (sp == 0) break;
                nl = walk(sp);
                if (nl == 0) break;
            }
            visit(nl, chunk);
            nl = 0;
        }
    }

    // Walk once, recording the accepted leaves in the warp's global leaf list;
    // fn(n) sees each staged chunk S.pts[0..n) on the way (all lanes together).
    template <typename Fn>
    __device__ __forceinline__ void collect(Fn fn) {
        const int lane = threadIdx.x & 31;
        nlist = 0;
        overflow = false;
        int sp;
        int nl = start(sp);
        while (true) {
            if (nl == 0) {
                if (sp == 0) break;
                nl = walk(sp);
                if (nl == 0) break;
            }
            for (int i = lane; i < nl; i += 32)
                if (nlist + i < kLeafList) leaf_list[nlist + i] = S.cand[i];
            if (nlist + nl > kLeafList) overflow = true;
            visit(nl, fn, nlist);
            nlist += nl;
            nl = 0;
        }
        __syncwarp();
    }

    // fn(point with id bits in w) for every candidate, all lanes together: the
    // recorded leaves again (or a fresh walk if the list overflowed).
    template <typename Fn>
    __device__ __forceinline__ void each(Fn fn) {
        const int lane = threadIdx.x & 31;
        auto per_chunk = [&](int n) {
            int t = 0;
            for (; t + 2 <= n; t += 2) {
                const float4 a = S.pts[t], b = S.pts[t + 1];
                fn(a);
                fn(b);
            }
            if (t < n) fn(S.pts[t]);
        };
        if (!overflow) {
            for (int base = 0; base < nlist; base += kCand) {
                const int nb = min(kCand, nlist - base);
                __syncwarp();
                for (int i = lane; i < nb; i += 32) S.cand[i] = leaf_list[base + i];
                __syncwarp();
                visit(nb, per_chunk);
            }
            return;
        }
        walk_points(per_chunk);
    }

    // As each(), but a recorded leaf is loaded only if some lane needs its points:
    // cls(lo, hi) classifies the leaf box for this lane (0: visit, 1: every point
    // counts as below, 2: nothing to do) and below(n) adds the n envelope points of
    // a leaf classified 1 (the lane's own point excluded).
    template <typename Fn, typename Cls, typename Below>
    __device__ __forceinline__ void each_pruned(Fn fn, Cls cls, Below below, int64_t self_leaf) {
        const int lane = threadIdx.x & 31;
        if (overflow) {
            each(fn);
            return;
        }
        auto per_chunk = [&](int n) {
            for (int t = 0; t < n; ++t) fn(S.pts[t]);
        };
        for (int base = 0; base < nlist; base += 32) {
            const int nb = min(32, nlist - base);
            const int lidx = lane < nb ? leaf_list[base + lane] : 0;
            const uint32_t lmask = lane < nb ? leaf_mask[base + lane] : 0u;
            for (int t = 0; t < nb; ++t) {
                const int L = __shfl_sync(0xffffffffu, lidx, t);
                const uint32_t m = __shfl_sync(0xffffffffu, lmask, t);
                const float4 lo = __ldg(&tv.nlo[tv.off[0] + L]), hi = __ldg(&tv.nhi[tv.off[0] + L]);
                const int c = cls(lo, hi);
                if (!__any_sync(0xffffffffu, c == 0)) {
                    if (c == 1) below(__popc(m) - ((L == self_leaf && ((m >> lane) & 1u)) ? 1 : 0));
                    continue;
                }
                __syncwarp();
                if (lane == 0) S.cand[0] = L;
                __syncwarp();
                visit(1, per_chunk);
            }
        }
    }
};

template <bool COUNT>
__device__ void knn_leaf(const KnnArgs &a, KnnWarpSmem &S, int *leaf_list, uint32_t *leaf_mask, double *bd, uint32_t *bi,
                         int64_t leaf) {
    const int lane = threadIdx.x & 31;
    const TreeView &tv = a.tv;
    const int k = a.k;
    const int64_t qi = leaf * kLeaf + lane;
    const bool valid = qi < tv.n;
    KnnWarp<COUNT> W(tv, a.perm, S, leaf_list, leaf_mask);
    W.q = valid ? __ldg(&tv.pos[qi]) : make_float4(0.f, 0.f, 0.f, 0.f);
    const float4 q = W.q;
    const uint32_t qid = valid ? __ldg(&a.perm[qi]) : 0u;

    auto clear_hist = [&]() {
        for (int b = 0; b < kNB; ++b) S.hist[b][lane] = 0;
        __syncwarp();
    };

    // ---- 1. radius bound from the neighbouring leaves in sorted order
    const int64_t nleaf = tv.cnt[0];
    // a central window of (k + 1)/32 + 2 leaves brackets the bound, the full
    // window of (k + 1)/32 + 10 leaves (13 at k = 64) tightens it: any subset of
    // the other points gives an upper bound, more nearby points a tighter one
    auto window = [&](int64_t wl, int64_t &w0, int64_t &w1) {
        w0 = leaf - wl / 2;
        if (w0 < 0) w0 = 0;
        w1 = w0 + wl - 1;
        if (w1 >= nleaf) {
            w1 = nleaf - 1;
            w0 = w1 - wl + 1 < 0 ? 0 : w1 - wl + 1;
        }
    };
    int64_t c0, c1, w0, w1;
    window((int64_t)((k + 1 + 31) / 32) + 2, c0, c1);
    window((int64_t)((k + 1 + 31) / 32) + 10, w0, w1);
    // first bracket: the farthest corner of the central leaves' joint box
    float whi = 0.f;
    {
        float blo[3] = {INFINITY, INFINITY, INFINITY}, bhi[3] = {-INFINITY, -INFINITY, -INFINITY};
        for (int64_t L = c0; L <= c1; ++L) {
            const float4 lo = __ldg(&tv.nlo[L]), hi = __ldg(&tv.nhi[L]);
            blo[0] = fminf(blo[0], lo.x); blo[1] = fminf(blo[1], lo.y); blo[2] = fminf(blo[2], lo.z);
            bhi[0] = fmaxf(bhi[0], hi.x); bhi[1] = fmaxf(bhi[1], hi.y); bhi[2] = fmaxf(bhi[2], hi.z);
        }
        const float dx = fmaxf(q.x - blo[0], bhi[0] - q.x), dy = fmaxf(q.y - blo[1], bhi[1] - q.y),
                    dz = fmaxf(q.z - blo[2], bhi[2] - q.z);
        whi = fmaf(dz, dz, fmaf(dy, dy, dx * dx)) * (1.0f + 1.0e-5f);
    }
    auto window_visit = [&](int64_t L0, int64_t L1, auto fn) {
        for (int64_t L = L0; L <= L1; ++L) {
            const int64_t base = L * kLeaf;
            if (base + lane < tv.n) S.pts[lane] = __ldg(&tv.pos[base + lane]);
            __syncwarp();
            const int cnt = (int)(tv.n - base < kLeaf ? tv.n - base : kLeaf);
            for (int t = 0; t < cnt; ++t) fn(S.pts[t], base + t);
            __syncwarp();
        }
    };
    // round 0: the central leaves over [0, whi]; round 1: all window leaves over
    // [0, the central k-th's bin] (their k-th is no larger)
    for (int round = 0; round < 2; ++round) {
        float wlo = 0.f;
        clear_hist();
        const float width = whi - wlo;
        const float inv = width > 0.f ? (float)kNB / width : 0.f;
        int below = 0;
        window_visit(round == 0 ? c0 : w0, round == 0 ? c1 : w1, [&](float4 p, int64_t j) {
            if (j != qi) {
                const float d = d2_f32(q, p);
                if (d < wlo) ++below;
                else if (d <= whi) S.hist[min(kNB - 1, (int)((d - wlo) * inv))][lane] += 1;
            }
        });
        __syncwarp();
        int cum = below, b = 0;
        for (; b < kNB; ++b) {
            const int c = S.hist[b][lane];
            if (cum + c >= k) break;
            cum += c;
        }
        // keep the current bracket if rounding left the k-th outside it
        if (b < kNB && width > 0.f) {
            const float nhi = (b == kNB - 1 ? whi : wlo + (float)(b + 1) * (width / (float)kNB)) *
                              (1.0f + 1.0e-6f);
            whi = fminf(nhi, whi);
        }
    }
    const float T = valid ? whi * (1.0f + 4.0e-6f) + 1.0e-37f : -1.f;

    // ---- 2. candidates within sqrt(T) of at least one lane's point
    W.r2 = T;
    {
        const float r = valid ? sqrtf(T) * (1.0f + 1.0e-5f) : 0.f;
        float lo3[3] = {valid ? q.x - r : INFINITY, valid ? q.y - r : INFINITY, valid ? q.z - r : INFINITY};
        float hi3[3] = {valid ? q.x + r : -INFINITY, valid ? q.y + r : -INFINITY, valid ? q.z + r : -INFINITY};
#pragma unroll
        for (int d = 0; d < 3; ++d)
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                lo3[d] = fminf(lo3[d], __shfl_xor_sync(0xffffffffu, lo3[d], o));
                hi3[d] = fmaxf(hi3[d], __shfl_xor_sync(0xffffffffu, hi3[d], o));
            }
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            W.env_lo[d] = lo3[d];
            W.env_hi[d] = hi3[d];
        }
    }
    // first histogram (32 bins over [0, T]) while the candidates are collected
    clear_hist();
    {
        const float inv0 = (valid && T > 0.f) ? (float)kNB / T : 0.f;
        const float t_a = valid ? T : -INFINITY;
        W.collect([&](int n) {
            for (int t = 0; t < n; ++t) {
                const float4 p = S.pts[t];
                const float d = d2_f32(q, p);
                if (d <= t_a && __float_as_uint(p.w) != qid)
                    S.hist[min(kNB - 1, (int)(d * inv0))][lane] += 1;
            }
            __syncwarp();
        });
    }

    // ---- 3./4. band passes; each also bins the band's bracket for a further round
    float lo_e = 0.f, hi_e = valid ? T : 0.f;
    int below = 0;               // candidates with d2 < lo_e
    bool done = !valid;
    int need = 0;
    double kth = 0.0;
    bool extract = false;
    float band_lo = 0.f, band_hi = 0.f;
    int nb_below = 0;
    for (int round = 0; round < 8; ++round) {
        if (!__any_sync(0xffffffffu, !done && !extract)) break;
        const bool act = !done && !extract;
        const float width = hi_e - lo_e;
        float e_lo = lo_e, e_hi = hi_e;
        if (act) {
            int cum = below, b = 0;
            for (; b < kNB - 1; ++b) {
                const int c = S.hist[b][lane];
                if (cum + c >= k) break;
                cum += c;
            }
            e_lo = lo_e + (float)b * (width / (float)kNB);
            e_hi = (b == kNB - 1) ? hi_e : lo_e + (float)(b + 1) * (width / (float)kNB);
            band_lo = e_lo * (1.0f - kDelta);
            band_hi = e_hi * (1.0f + kDelta);
        }
        clear_hist();
        const float bhi_a = act ? band_hi : -INFINITY;
        const float sub_w = e_hi - e_lo;
        const float sub_inv = sub_w > 0.f ? (float)kNB / sub_w : 0.f;
        int nbelow = 0, nband = 0, below_next = 0;
        // leaves wholly below this lane's band (by the far corner of their box) or
        // wholly above it (by the near corner) need no point loads; the margins
        // cover the rounding of the FP32 distances
        auto cls = [&](float4 lo, float4 hi) -> int {
            if (!act) return 2;
            const float gx = fmaxf(fmaxf(lo.x - q.x, q.x - hi.x), 0.f);
            const float gy = fmaxf(fmaxf(lo.y - q.y, q.y - hi.y), 0.f);
            const float gz = fmaxf(fmaxf(lo.z - q.z, q.z - hi.z), 0.f);
            const float fx = fmaxf(fabsf(q.x - lo.x), fabsf(q.x - hi.x));
            const float fy = fmaxf(fabsf(q.y - lo.y), fabsf(q.y - hi.y));
            const float fz = fmaxf(fabsf(q.z - lo.z), fabsf(q.z - hi.z));
            const float dmin = fmaf(gz, gz, fmaf(gy, gy, gx * gx));
            const float dmax = fmaf(fz, fz, fmaf(fy, fy, fx * fx));
            if (dmax * (1.0f + 1.0e-5f) < band_lo) return 1;
            if (dmin * (1.0f - 1.0e-5f) > band_hi) return 2;
            return 0;
        };
        auto below_all = [&](int n) {
            nbelow += n;
            below_next += n;
        };
        W.each_pruned([&](float4 p) {
            const float d = d2_f32(q, p);
            if (d <= bhi_a) {
                const uint32_t id = __float_as_uint(p.w);
                if (id != qid) {
                    if (d < band_lo) {
                        ++nbelow;
                    } else {
                        if (nband < kBand) {
                            bd[nband * 32 + lane] = d2_f64(q, p);
                            bi[nband * 32 + lane] = id;
                        }
                        ++nband;
                    }
                    if (d < e_lo) ++below_next;
                    else if (d <= e_hi) S.hist[min(kNB - 1, (int)((d - e_lo) * sub_inv))][lane] += 1;
                }
            }
        }, cls, below_all, leaf);
        __syncwarp();
        if (act) {
            need = k - nbelow;
            nb_below = nbelow;
            if (nband <= kBand) {
                for (int x = 1; x < nband; ++x) {
                    const double dv = bd[x * 32 + lane];
                    const uint32_t iv = bi[x * 32 + lane];
                    int y = x - 1;
                    while (y >= 0 && key_less(dv, iv, bd[y * 32 + lane], bi[y * 32 + lane])) {
                        bd[(y + 1) * 32 + lane] = bd[y * 32 + lane];
                        bi[(y + 1) * 32 + lane] = bi[y * 32 + lane];
                        --y;
                    }
                    bd[(y + 1) * 32 + lane] = dv;
                    bi[(y + 1) * 32 + lane] = iv;
                }
                const int pick = min(max(need, 1), min(nband, kBand)) - 1;
                kth = bd[pick * 32 + lane];
                done = true;
            } else if (round == 7 || !(e_hi - e_lo > 4.0f * kDelta * e_hi)) {
                extract = true;  // bin cannot shrink further (or out of rounds)
            } else {
                lo_e = e_lo;     // the band pass already binned [e_lo, e_hi]
                hi_e = e_hi;
                below = below_next;
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
            W.each([&](float4 p) {
                const uint32_t id = __float_as_uint(p.w);
                if (act && id != qid) {
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
        const float blo_a = valid ? band_lo : -INFINITY;
        W.each([&](float4 p) {
            const float d = d2_f32(q, p);
            const uint32_t id = __float_as_uint(p.w);
            if (d < blo_a && id != qid && slot < k) a.nbr_orig[(int64_t)qid * k + slot++] = id;
        });
        if (valid && !extract)
            for (int x = 0; x < need && x < kBand && slot + x < k; ++x)
                a.nbr_orig[(int64_t)qid * k + slot + x] = bi[x * 32 + lane];
    }
    if (COUNT && lane == 0) {
        atomicAdd(&a.work[0], W.ncand);
        atomicAdd(&a.work[1], 1ull);
    }
}

template <bool COUNT>
__global__ void __launch_bounds__(kKnnWarps * 32, 7) k_knn(KnnArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int warp = threadIdx.x >> 5;
    KnnWarpSmem &S = reinterpret_cast<KnnWarpSmem *>(smem_raw)[warp];
    const int64_t slot = (int64_t)blockIdx.x * kKnnWarps + warp;
    int *leaf_list = a.leaf_list + slot * kLeafList;
    uint32_t *leaf_mask = a.leaf_mask + slot * kLeafList;
    double *bd = a.band_d + slot * (kBand * 32);
    uint32_t *bi = a.band_i + slot * (kBand * 32);
    const int64_t nleaf = a.tv.cnt[0];
    while (true) {
        unsigned int leaf = 0;
        if ((threadIdx.x & 31) == 0) leaf = atomicAdd(a.next_leaf, 1u);
        leaf = __shfl_sync(0xffffffffu, leaf, 0);
        if ((int64_t)leaf >= nleaf) break;
        knn_leaf<COUNT>(a, S, leaf_list, leaf_mask, bd, bi, (int64_t)leaf);
    }
}

// The kNN's work accounting: after a launch with a.work set.
__global__ void k_knn_work_out(const unsigned long long *work, int64_t *out) {
    if (threadIdx.x == 0) {
        out[0] = (int64_t)work[0] * 32;  // (lane, candidate) distance evaluations
        out[1] = (int64_t)work[0];
        out[2] = (int64_t)work[1];
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

sf_status knn_run(sf_index *idx, int k, uint32_t *d_nbr_orig, float *d_h_sorted, cudaStream_t s,
                  unsigned long long *d_work = nullptr) {
    KnnArgs a;
    a.tv = idx->view();
    a.perm = idx->perm;
    a.k = k;
    a.h_sorted = d_h_sorted;
    a.nbr_orig = d_nbr_orig;
    a.work = d_work;
    const size_t smem = sizeof(KnnWarpSmem) * kKnnWarps;
    auto kern = d_work ? k_knn<true> : k_knn<false>;
    static std::atomic<uint64_t> attr_plain{0}, attr_count{0};
    SF_TRY_CUDA(smem_attr_once(kern, smem, d_work ? attr_count : attr_plain));
    int dev = 0, sms = 0, per_sm = 0;
    SF_TRY_CUDA(cudaGetDevice(&dev));
    SF_TRY_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    SF_TRY_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kKnnWarps * 32, smem));
    if (per_sm < 1) per_sm = 1;
    // persistent: one resident wave, never more blocks than leaves need
    const int64_t need_blocks = (idx->cnt[0] + kKnnWarps - 1) / kKnnWarps;
    const int64_t blocks = std::max<int64_t>(1, std::min<int64_t>((int64_t)sms * per_sm, need_blocks));
    Scratch sc(s);
    a.leaf_list = sc.get<int>(blocks * kKnnWarps * (int64_t)kLeafList);
    a.leaf_mask = sc.get<uint32_t>(blocks * kKnnWarps * (int64_t)kLeafList);
    a.band_d = sc.get<double>(blocks * kKnnWarps * (int64_t)kBand * 32);
    a.band_i = sc.get<uint32_t>(blocks * kKnnWarps * (int64_t)kBand * 32);
    a.next_leaf = sc.get<unsigned int>(1);
    SF_TRY_SCRATCH(sc);
    SF_TRY_CUDA(cudaMemsetAsync(a.next_leaf, 0, sizeof(unsigned int), s));
    KTimer timer(d_work ? "k_knn_count" : "k_knn", s);
    SF_TRY_CUDA(launch(kern, dim3((unsigned)blocks), dim3(kKnnWarps * 32), smem, s, a));
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

// The work of one kNN run (the index's resident bandwidths are left as they are):
// h_counts[0] (lane, candidate) distance evaluations, [1] candidates staged per
// query leaf, summed over all passes, [2] query leaves. Synchronises the stream.
sf_status knn_work_counts(sf_index *idx, int k, int64_t *h_counts, cudaStream_t s) {
    Scratch sc(s);
    float *h = sc.get<float>(idx->n);
    unsigned long long *work = sc.get<unsigned long long>(2);
    int64_t *out = sc.get<int64_t>(3);
    SF_TRY_SCRATCH(sc);
    SF_TRY_CUDA(cudaMemsetAsync(work, 0, 2 * sizeof(unsigned long long), s));
    SF_TRY(knn_run(idx, k, nullptr, h, s, work));
    SF_TRY_CUDA(launch(k_knn_work_out, dim3(1), dim3(32), 0, s, (const unsigned long long *)work, out));
    SF_TRY_CUDA(cudaMemcpyAsync(h_counts, out, 3 * sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    SF_TRY_CUDA(cudaStreamSynchronize(s));
    return SF_OK;
}

sf_status scatter_bandwidths(const sf_index *idx, float *d_h_orig, cudaStream_t s) {
    const unsigned g = std::min<unsigned>(blocks_for(idx->n, 256), 152 * 16);
    SF_TRY_CUDA(launch(k_scatter_h, dim3(g), dim3(256), 0, s, (const float4 *)idx->pos,
                       (const uint32_t *)idx->perm, idx->n, d_h_orig));
    return SF_OK;
}

}  // namespace sf
