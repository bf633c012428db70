// sf_prims.cu -- device-wide primitives: exclusive scan, stable LSD radix sort
// of (64-bit key, 32-bit value) pairs, and radix selection of an order
// statistic. Integer-only, hence exact and deterministic.
#include <cstdarg>
#include <cstdio>
#include <string>

#include "sf_internal.cuh"

namespace sf {

std::atomic<uint64_t> g_launches{0};

static thread_local std::string t_last_error;

sf_status fail(sf_status st, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    t_last_error = buf;
    return st;
}

static thread_local ScratchStats t_scratch;

ScratchStats &scratch_stats() { return t_scratch; }

const char *last_error_cstr() { return t_last_error.c_str(); }

// Every entry point starts here: the error message and the scratch high-water
// mark of the previous call are closed.
void clear_error() {
    t_last_error.clear();
    t_scratch.peak = t_scratch.live;
}

int64_t last_call_scratch_peak() { return t_scratch.peak; }

// ---------------------------------------------------------------------------
// Kernel timing registry: event pairs recorded on the launching stream.
// ---------------------------------------------------------------------------
static std::atomic<int> g_timing{0};
static std::mutex g_timing_mu;
struct TimedPair {
    std::string name;
    cudaEvent_t a, b;
};
static std::vector<TimedPair> g_timed;

KTimer::KTimer(const char *n, cudaStream_t st) : name(n), s(st) {
    if (!g_timing.load(std::memory_order_relaxed)) return;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) return;
    if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess) {
        a = b = nullptr;
        return;
    }
    cudaEventRecord(a, s);
}

KTimer::~KTimer() {
    if (!a) return;
    cudaEventRecord(b, s);
    std::lock_guard<std::mutex> lk(g_timing_mu);
    g_timed.push_back({name, a, b});
}

// ---------------------------------------------------------------------------
// Block-level helpers
// ---------------------------------------------------------------------------
// Exclusive scan of one uint32 per thread across a block of blockDim.x (multiple
// of 32, <= 1024) threads. *total receives the block sum. Contains barriers.
__device__ uint32_t block_exclusive_scan(uint32_t v, uint32_t *total) {
    __shared__ uint32_t wsum[32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    uint32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) wsum[w] = x;
    __syncthreads();
    if (w == 0) {
        uint32_t t = lane < nw ? wsum[lane] : 0u;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(0xffffffffu, t, o);
            if (lane >= o) t += y;
        }
        wsum[lane] = t;  // inclusive
    }
    __syncthreads();
    uint32_t before = (w > 0) ? wsum[w - 1] : 0u;
    *total = wsum[nw - 1];
    __syncthreads();
    return before + x - v;
}

// ---------------------------------------------------------------------------
// Exclusive scan
// ---------------------------------------------------------------------------
constexpr int kScanThreads = 256;
constexpr int kScanItems = 8;
constexpr int kScanTile = kScanThreads * kScanItems;

__global__ void k_scan_reduce(const uint32_t *__restrict__ in, int64_t n,
                              uint32_t *__restrict__ parts) {
    int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
    uint32_t s = 0;
#pragma unroll
    for (int i = 0; i < kScanItems; ++i)
        if (base + i < n) s += in[base + i];
    uint32_t total;
    block_exclusive_scan(s, &total);
    if (threadIdx.x == 0) parts[blockIdx.x] = total;
}

__global__ void k_scan_parts(uint32_t *parts, int64_t nb, uint32_t *total_out) {
    // one block of 1024 threads; thread t owns a contiguous run of parts
    const int64_t per = (nb + blockDim.x - 1) / blockDim.x;
    const int64_t b0 = (int64_t)threadIdx.x * per;
    uint32_t s = 0;
    for (int64_t i = 0; i < per; ++i)
        if (b0 + i < nb) s += parts[b0 + i];
    uint32_t total;
    uint32_t run = block_exclusive_scan(s, &total);
    for (int64_t i = 0; i < per; ++i)
        if (b0 + i < nb) {
            uint32_t v = parts[b0 + i];
            parts[b0 + i] = run;
            run += v;
        }
    if (threadIdx.x == 0 && total_out) *total_out = total;
}

__global__ void k_scan_down(const uint32_t *__restrict__ in, uint32_t *__restrict__ out,
                            int64_t n, const uint32_t *__restrict__ parts) {
    int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
    uint32_t v[kScanItems];
    uint32_t s = 0;
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        v[i] = (base + i < n) ? in[base + i] : 0u;
        s += v[i];
    }
    uint32_t total;
    uint32_t run = block_exclusive_scan(s, &total) + parts[blockIdx.x];
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        if (base + i < n) out[base + i] = run;
        run += v[i];
    }
}

sf_status scan_u32(const uint32_t *d_in, uint32_t *d_out, int64_t n, uint32_t *d_total,
                   cudaStream_t s) {
    if (n <= 0) {
        if (d_total) SF_TRY_CUDA(cudaMemsetAsync(d_total, 0, sizeof(uint32_t), s));
        return SF_OK;
    }
    const int64_t nb = (n + kScanTile - 1) / kScanTile;
    Scratch sc(s);
    uint32_t *parts = sc.get<uint32_t>(nb);
    SF_TRY_SCRATCH(sc);
    SF_TRY_CUDA(launch(k_scan_reduce, dim3((unsigned)nb), dim3(kScanThreads), 0, s, d_in, n, parts));
    SF_TRY_CUDA(launch(k_scan_parts, dim3(1), dim3(1024), 0, s, parts, nb, d_total));
    SF_TRY_CUDA(launch(k_scan_down, dim3((unsigned)nb), dim3(kScanThreads), 0, s, d_in, d_out, n,
                       (const uint32_t *)parts));
    return SF_OK;
}

// ---------------------------------------------------------------------------
// Stable LSD radix sort, 8-bit digits, tiles of 4096 keys per block.
// Pass = histogram -> scan of the digit-major count table -> stable scatter.
// ---------------------------------------------------------------------------
constexpr int kRsThreads = 256;
constexpr int kRsWarps = kRsThreads / 32;
constexpr int kRsPerWarp = 512;
constexpr int kRsTile = kRsWarps * kRsPerWarp;  // 4096
constexpr int kRsIter = kRsPerWarp / 32;        // 16

__global__ void __launch_bounds__(kRsThreads)
    k_rs_hist(const uint64_t *__restrict__ keys, int64_t n, int shift,
              uint32_t *__restrict__ counts, int64_t nb) {
    __shared__ uint32_t h[kRsWarps][256];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int i = threadIdx.x; i < kRsWarps * 256; i += kRsThreads) (&h[0][0])[i] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * kRsTile + (int64_t)w * kRsPerWarp;
#pragma unroll 4
    for (int it = 0; it < kRsIter; ++it) {
        const int64_t g = base + it * 32 + lane;
        const bool valid = g < n;
        const unsigned active = __ballot_sync(0xffffffffu, valid);
        if (valid) {
            const unsigned d = (unsigned)(keys[g] >> shift) & 255u;
            const unsigned peers = __match_any_sync(active, d);
            if (lane == __ffs(peers) - 1) h[w][d] += __popc(peers);
        }
        __syncwarp();
    }
    __syncthreads();
    uint32_t c = 0;
#pragma unroll
    for (int ww = 0; ww < kRsWarps; ++ww) c += h[ww][threadIdx.x];
    counts[(int64_t)threadIdx.x * nb + blockIdx.x] = c;
}

__global__ void __launch_bounds__(kRsThreads)
    k_rs_scatter(const uint64_t *__restrict__ kin, const uint32_t *__restrict__ vin,
                 uint64_t *__restrict__ kout, uint32_t *__restrict__ vout, int64_t n, int shift,
                 const uint32_t *__restrict__ offs, int64_t nb) {
    __shared__ uint32_t wc[kRsWarps][256];
    __shared__ uint32_t goff[256];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int i = threadIdx.x; i < kRsWarps * 256; i += kRsThreads) (&wc[0][0])[i] = 0;
    goff[threadIdx.x] = offs[(int64_t)threadIdx.x * nb + blockIdx.x];
    __syncthreads();
    const unsigned lt = (1u << lane) - 1u;
    const int64_t base = (int64_t)blockIdx.x * kRsTile + (int64_t)w * kRsPerWarp;
    uint64_t kk[kRsIter];
    uint32_t vv[kRsIter];
    uint32_t rk[kRsIter];
#pragma unroll
    for (int it = 0; it < kRsIter; ++it) {
        const int64_t g = base + it * 32 + lane;
        const bool valid = g < n;
        const unsigned active = __ballot_sync(0xffffffffu, valid);
        unsigned d = 0, peers = 0, before = 0;
        if (valid) {
            kk[it] = kin[g];
            vv[it] = vin[g];
            d = (unsigned)(kk[it] >> shift) & 255u;
            peers = __match_any_sync(active, d);
            before = wc[w][d];
        }
        __syncwarp();
        if (valid && lane == __ffs(peers) - 1) wc[w][d] = before + __popc(peers);
        __syncwarp();
        rk[it] = before + __popc(peers & lt);
    }
    __syncthreads();
    {
        uint32_t run = 0;
#pragma unroll
        for (int ww = 0; ww < kRsWarps; ++ww) {
            uint32_t c = wc[ww][threadIdx.x];
            wc[ww][threadIdx.x] = run;
            run += c;
        }
    }
    __syncthreads();
#pragma unroll
    for (int it = 0; it < kRsIter; ++it) {
        const int64_t g = base + it * 32 + lane;
        if (g < n) {
            const unsigned d = (unsigned)(kk[it] >> shift) & 255u;
            const uint32_t p = goff[d] + wc[w][d] + rk[it];
            kout[p] = kk[it];
            vout[p] = vv[it];
        }
    }
}

sf_status radix_sort_pairs(uint64_t *keys, uint32_t *vals, uint64_t *keys_tmp,
                           uint32_t *vals_tmp, int64_t n, int bits, cudaStream_t s) {
    if (n <= 1) return SF_OK;
    const int64_t nb = (n + kRsTile - 1) / kRsTile;
    Scratch sc(s);
    uint32_t *counts = sc.get<uint32_t>(256 * nb);
    SF_TRY_SCRATCH(sc);
    KTimer timer("k_radix_sort", s);
    int passes = (bits + 7) / 8;
    if (passes & 1) ++passes;  // even number of passes: result lands back in (keys, vals)
    uint64_t *ka = keys, *kb = keys_tmp;
    uint32_t *va = vals, *vb = vals_tmp;
    for (int p = 0; p < passes; ++p) {
        const int shift = 8 * p;
        if (shift < 64) {
            SF_TRY_CUDA(launch(k_rs_hist, dim3((unsigned)nb), dim3(kRsThreads), 0, s,
                               (const uint64_t *)ka, n, shift, counts, nb));
            SF_TRY(scan_u32(counts, counts, 256 * nb, nullptr, s));
            SF_TRY_CUDA(launch(k_rs_scatter, dim3((unsigned)nb), dim3(kRsThreads), 0, s,
                               (const uint64_t *)ka, (const uint32_t *)va, kb, vb, n, shift,
                               (const uint32_t *)counts, nb));
        } else {
            SF_TRY_CUDA(cudaMemcpyAsync(kb, ka, n * sizeof(uint64_t), cudaMemcpyDeviceToDevice, s));
            SF_TRY_CUDA(cudaMemcpyAsync(vb, va, n * sizeof(uint32_t), cudaMemcpyDeviceToDevice, s));
        }
        std::swap(ka, kb);
        std::swap(va, vb);
    }
    return SF_OK;
}

// ---------------------------------------------------------------------------
// Radix select: the element of 0-based rank r among n ordered-uint32 keys.
// Four MSB-first passes of 8 bits; each keeps only keys matching the prefix.
// ---------------------------------------------------------------------------
struct SelState {
    uint32_t prefix, mask;
    int64_t rank;
    uint32_t hist[256];
};

__global__ void k_sel_init(SelState *st, const int64_t *d_rank) {
    if (threadIdx.x == 0) {
        st->prefix = 0;
        st->mask = 0;
        st->rank = *d_rank;
    }
    st->hist[threadIdx.x] = 0;
}

__global__ void k_sel_hist(const uint32_t *__restrict__ keys, int64_t n, int shift,
                           SelState *st) {
    __shared__ uint32_t h[256];
    h[threadIdx.x] = 0;
    __syncthreads();
    const uint32_t prefix = st->prefix, mask = st->mask;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t k = keys[i];
        if ((k & mask) == prefix) atomicAdd(&h[(k >> shift) & 255u], 1u);
    }
    __syncthreads();
    if (h[threadIdx.x]) atomicAdd(&st->hist[threadIdx.x], h[threadIdx.x]);
}

__global__ void k_sel_pick(SelState *st, int shift) {
    // 256 threads: exclusive scan of the histogram, find the digit holding rank
    const uint32_t c = st->hist[threadIdx.x];
    uint32_t total;
    const uint32_t ex = block_exclusive_scan(c, &total);
    const int64_t r = st->rank;
    if ((int64_t)ex <= r && r < (int64_t)(ex + c)) {
        st->prefix |= (uint32_t)threadIdx.x << shift;
        st->mask |= 255u << shift;
        st->rank = r - ex;
    }
    __syncthreads();
    st->hist[threadIdx.x] = 0;
}

__global__ void k_sel_out(const SelState *st, uint32_t *out) { *out = st->prefix; }

sf_status radix_select_u32(const uint32_t *d_keys, int64_t n, const int64_t *d_rank,
                           uint32_t *d_result, cudaStream_t s) {
    Scratch sc(s);
    SelState *st = sc.get<SelState>(1);
    SF_TRY_SCRATCH(sc);
    SF_TRY_CUDA(launch(k_sel_init, dim3(1), dim3(256), 0, s, st, d_rank));
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const unsigned grid = (unsigned)std::min<int64_t>(blocks_for(n, 256), (int64_t)sms * 8);
    for (int shift = 24; shift >= 0; shift -= 8) {
        SF_TRY_CUDA(launch(k_sel_hist, dim3(std::max(1u, grid)), dim3(256), 0, s, d_keys, n, shift, st));
        SF_TRY_CUDA(launch(k_sel_pick, dim3(1), dim3(256), 0, s, st, shift));
    }
    SF_TRY_CUDA(launch(k_sel_out, dim3(1), dim3(1), 0, s, (const SelState *)st, d_result));
    return SF_OK;
}

}  // namespace sf

using namespace sf;

extern "C" void sf_kernel_timing_enable(int enable) { g_timing.store(enable ? 1 : 0); }

extern "C" void sf_kernel_timing_reset(void) {
    std::lock_guard<std::mutex> lk(g_timing_mu);
    for (auto &t : g_timed) {
        cudaEventDestroy(t.a);
        cudaEventDestroy(t.b);
    }
    g_timed.clear();
}

extern "C" sf_status sf_kernel_timing_list(const char *name, double *h_ms, int64_t cap,
                                           int64_t *h_count) {
    if (!name || !h_count || (cap > 0 && !h_ms))
        return fail(SF_ERR_INVALID_ARG, "sf_kernel_timing_list: NULL argument");
    std::lock_guard<std::mutex> lk(g_timing_mu);
    int64_t cnt = 0;
    for (auto &t : g_timed) {
        if (t.name != name) continue;
        cudaError_t e = cudaEventSynchronize(t.b);
        if (e != cudaSuccess) return fail(SF_ERR_CUDA, "sf_kernel_timing_list: %s", cudaGetErrorString(e));
        float ms = 0.f;
        cudaEventElapsedTime(&ms, t.a, t.b);
        if (cnt < cap) h_ms[cnt] = ms;
        ++cnt;
    }
    *h_count = cnt;
    return SF_OK;
}

extern "C" sf_status sf_kernel_timing(const char *name, double *h_ms_total, int64_t *h_launches) {
    if (!name || !h_ms_total || !h_launches) return fail(SF_ERR_INVALID_ARG, "sf_kernel_timing: NULL argument");
    std::lock_guard<std::mutex> lk(g_timing_mu);
    double tot = 0.0;
    int64_t cnt = 0;
    for (auto &t : g_timed) {
        if (t.name != name) continue;
        cudaError_t e = cudaEventSynchronize(t.b);
        if (e != cudaSuccess) return fail(SF_ERR_CUDA, "sf_kernel_timing: %s", cudaGetErrorString(e));
        float ms = 0.f;
        cudaEventElapsedTime(&ms, t.a, t.b);
        tot += ms;
        ++cnt;
    }
    *h_ms_total = tot;
    *h_launches = cnt;
    return SF_OK;
}
