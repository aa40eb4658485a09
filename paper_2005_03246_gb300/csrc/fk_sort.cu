// fk_sort.cu -- device-wide exclusive scan and a stable LSD radix sort of
// (key, value) pairs, written for the rank transform of the sample-point path
// (Sec. 2.2, Algorithm 2: the per-axis sort permutations phi^j).
#include <algorithm>
#include <mutex>

#include "fk_internal.cuh"

namespace fk {

// ============================================================== exclusive scan (u32)
namespace {
constexpr int kScanThreads = 512;
constexpr int kScanItems = 8;
constexpr int kScanTile = kScanThreads * kScanItems;   // 4096

__device__ __forceinline__ uint32_t block_excl_scan_u32(uint32_t v, uint32_t* total) {
    __shared__ uint32_t warp_sums[kScanThreads / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_sums[warp] = x;
    __syncthreads();
    if (warp == 0) {
        uint32_t s = (lane < kScanThreads / 32) ? warp_sums[lane] : 0u;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += y;
        }
        if (lane < kScanThreads / 32) warp_sums[lane] = s;
    }
    __syncthreads();
    uint32_t warp_off = warp ? warp_sums[warp - 1] : 0u;
    if (total) *total = warp_sums[kScanThreads / 32 - 1];
    uint32_t r = warp_off + x - v;
    __syncthreads();
    return r;
}

__global__ void __launch_bounds__(kScanThreads) k_scan_reduce(const uint32_t* __restrict__ in,
                                                              int64_t n, uint32_t* __restrict__ sums) {
    int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
    uint32_t s = 0;
#pragma unroll
    for (int j = 0; j < kScanItems; ++j)
        if (base + j < n) s += in[base + j];
    uint32_t tot;
    block_excl_scan_u32(s, &tot);
    if (threadIdx.x == 0) sums[blockIdx.x] = tot;
}

__global__ void __launch_bounds__(kScanThreads) k_scan_apply(const uint32_t* in, int64_t n,
                                                             const uint32_t* __restrict__ offs,
                                                             uint32_t* out) {
    int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
    uint32_t v[kScanItems];
    uint32_t s = 0;
#pragma unroll
    for (int j = 0; j < kScanItems; ++j) {
        v[j] = (base + j < n) ? in[base + j] : 0u;
        s += v[j];
    }
    uint32_t run = block_excl_scan_u32(s, nullptr) + (offs ? offs[blockIdx.x] : 0u);
#pragma unroll
    for (int j = 0; j < kScanItems; ++j) {
        if (base + j < n) out[base + j] = run;
        run += v[j];
    }
}
}  // namespace

size_t scan_u32_tmp_words(int64_t n) {
    size_t w = 0;
    while (n > kScanTile) {
        n = (n + kScanTile - 1) / kScanTile;
        w += (size_t)n + 64;
    }
    return w + 64;
}

fk_status scan_u32_exclusive(const uint32_t* in, uint32_t* out, int64_t n, uint32_t* tmp,
                             cudaStream_t st) {
    if (n <= 0) return FK_OK;
    int64_t tiles = (n + kScanTile - 1) / kScanTile;
    if (tiles == 1) {
        k_scan_apply<<<1, kScanThreads, 0, st>>>(in, n, nullptr, out);
        FK_LAUNCH_CHECK();
        return FK_OK;
    }
    uint32_t* sums = tmp;
    uint32_t* rest = tmp + tiles + 64;
    k_scan_reduce<<<(unsigned)tiles, kScanThreads, 0, st>>>(in, n, sums);
    FK_LAUNCH_CHECK();
    FK_TRY(scan_u32_exclusive(sums, sums, tiles, rest, st));
    k_scan_apply<<<(unsigned)tiles, kScanThreads, 0, st>>>(in, n, sums, out);
    FK_LAUNCH_CHECK();
    return FK_OK;
}

// ============================================================== LSD radix sort
// One sweep per digit: a single pass over the keys histograms every digit
// position at once; each digit pass is then one launch whose CTAs take tiles
// in launch order (an atomic tile counter) and find the global start of each
// of their digit runs by a decoupled look-back over the tiles before them
// (each tile publishes its per-digit count, then its inclusive prefix).
namespace {
constexpr int kRadixBits = 8;
constexpr int kRadixBins = 1 << kRadixBits;
constexpr int kMaxPasses = 8;
constexpr int kSortThreads = 256;
constexpr int kSortWarps = kSortThreads / 32;
constexpr int kSortChunks = 16;                                  // 32-key chunks per warp
constexpr int kSortTile = kSortThreads * kSortChunks;             // 4096 keys per CTA
constexpr int kHistCtasPerSm = 4;

// Look-back status word of (tile, digit): bits 63..56 the pass it belongs to
// (pass + 1; any other value, e.g. the zero of the reset, means "not yet
// published"), bit 55 set once the value is the inclusive prefix over tiles
// 0..tile (clear: the tile's own count only), bits 54..0 the value.
constexpr uint64_t kStatInc = 1ull << 55;
constexpr uint64_t kStatVal = kStatInc - 1;
// Bound of every look-back wait, in polls of one status word (each an L2
// round trip plus a short sleep): a fraction of a second per thread in total,
// far beyond the microseconds a running predecessor tile needs to publish.
// On expiry the wait records DEV_TIMEOUT in the error word and continues, so
// the kernel always ends.
constexpr int kLookbackPolls = 1 << 18;

__device__ __forceinline__ uint64_t ld_relaxed_u64(const uint64_t* p) {
    uint64_t v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_relaxed_u64(uint64_t* p, uint64_t v) {
    asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// Scratch layout at the start of `tmp`: status [tiles][256] u64, the digit
// histograms [kMaxPasses][256] u32 and the tile counters [kMaxPasses] u32;
// all of it is zeroed once per sort.
struct SortScratch {
    uint64_t* status;
    uint32_t* ghist;
    uint32_t* ctr;
    size_t bytes;
    static size_t size(int64_t tiles) {
        return (size_t)tiles * kRadixBins * 8 + (size_t)kMaxPasses * kRadixBins * 4 + 256;
    }
    static SortScratch at(void* tmp, int64_t tiles) {
        SortScratch s;
        s.status = (uint64_t*)tmp;
        s.ghist = (uint32_t*)(s.status + (size_t)tiles * kRadixBins);
        s.ctr = s.ghist + kMaxPasses * kRadixBins;
        s.bytes = size(tiles);
        return s;
    }
};

// Histograms of all `passes` digit positions in one read of the keys.
template <class K>
__global__ void __launch_bounds__(kSortThreads) k_radix_hist_all(const K* __restrict__ keys, int64_t n, int passes,
                                                                 uint32_t* __restrict__ ghist) {
    __shared__ uint32_t cnt[kMaxPasses][kRadixBins];
    for (int b = threadIdx.x; b < kMaxPasses * kRadixBins; b += kSortThreads) (&cnt[0][0])[b] = 0;
    __syncthreads();
    const int64_t stride = (int64_t)gridDim.x * kSortThreads;
    for (int64_t i = (int64_t)blockIdx.x * kSortThreads + threadIdx.x; i < n; i += stride) {
        const K k = keys[i];
#pragma unroll
        for (int p = 0; p < kMaxPasses; ++p)
            if (p < passes) atomicAdd(&cnt[p][(uint32_t)(k >> (p * kRadixBits)) & (kRadixBins - 1)], 1u);
    }
    __syncthreads();
    for (int b = threadIdx.x; b < passes * kRadixBins; b += kSortThreads) {
        const uint32_t c = (&cnt[0][0])[b];
        if (c) atomicAdd(&ghist[b], c);
    }
}

// Stable scatter of one digit pass in three steps: the tile's keys are ranked
// and placed in shared memory in (digit, original position) order, the
// global start of each digit run comes from the digit histogram and the
// look-back, and the runs are written so that consecutive threads store
// consecutive elements of a digit's run.  Warp w owns keys
// [base + w*512, base + (w+1)*512) in chunk order, which is the tile's
// original order, so the ranking is stable.
template <class K>
struct ScatterSmem {
    static constexpr size_t o_key = 0;
    static constexpr size_t o_val = o_key + sizeof(K) * kSortTile;
    static constexpr size_t o_wcnt = o_val + 4 * kSortTile;
    static constexpr size_t o_dstart = o_wcnt + 4 * kSortWarps * kRadixBins;
    static constexpr size_t o_gofs = o_dstart + 4 * kRadixBins;
    static constexpr size_t o_wsum = o_gofs + 4 * kRadixBins;
    static constexpr size_t o_misc = o_wsum + 4 * 2 * kSortWarps;
    static constexpr size_t bytes = o_misc + 16;
};

// Block-wide exclusive scan over one value per thread (256 threads); wsum
// holds kSortWarps words.  Ends with a barrier.
__device__ __forceinline__ uint32_t sort_block_excl(uint32_t v, uint32_t* wsum) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) wsum[warp] = x;
    __syncthreads();
    uint32_t before = 0;
    for (int w = 0; w < warp; ++w) before += wsum[w];
    __syncthreads();
    return before + x - v;
}

template <class K>
__global__ void __launch_bounds__(kSortThreads) k_radix_onesweep(const K* __restrict__ keys,
                                                                 const uint32_t* __restrict__ vals,
                                                                 K* __restrict__ keys_out,
                                                                 uint32_t* __restrict__ vals_out, int64_t n, int pass,
                                                                 SortScratch sc, int* err) {
    static_assert(kSortThreads == kRadixBins, "one thread per digit");
    typedef ScatterSmem<K> L;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    K* s_key = reinterpret_cast<K*>(smem_raw + L::o_key);
    uint32_t* s_val = reinterpret_cast<uint32_t*>(smem_raw + L::o_val);
    uint32_t (*wcnt)[kRadixBins] = reinterpret_cast<uint32_t (*)[kRadixBins]>(smem_raw + L::o_wcnt);
    uint32_t* dstart = reinterpret_cast<uint32_t*>(smem_raw + L::o_dstart);
    uint32_t* gofs = reinterpret_cast<uint32_t*>(smem_raw + L::o_gofs);
    uint32_t* wsum = reinterpret_cast<uint32_t*>(smem_raw + L::o_wsum);
    uint32_t* s_tile = reinterpret_cast<uint32_t*>(smem_raw + L::o_misc);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int shift = pass * kRadixBits;
    if (threadIdx.x == 0) *s_tile = atomicAdd(&sc.ctr[pass], 1u);
    for (int b = threadIdx.x; b < kSortWarps * kRadixBins; b += kSortThreads) (&wcnt[0][0])[b] = 0;
    __syncthreads();
    const int64_t tile = *s_tile;
    const int64_t tbase = tile * kSortTile;
    const int64_t wbase = tbase + (int64_t)warp * (32 * kSortChunks);
    // keys into registers, per-warp digit counts
    K kr[kSortChunks];
    uint32_t vr[kSortChunks];
#pragma unroll
    for (int c = 0; c < kSortChunks; ++c) {
        const int64_t i = wbase + c * 32 + lane;
        kr[c] = 0;
        vr[c] = 0;
        if (i < n) {
            kr[c] = keys[i];
            vr[c] = vals[i];
            atomicAdd(&wcnt[warp][(uint32_t)(kr[c] >> shift) & (kRadixBins - 1)], 1u);
        }
    }
    __syncthreads();
    // thread b owns digit b: the tile's count, published at once; the global
    // start of digit b (exclusive scan of the pass histogram) and the count
    // of digit b in the tiles before this one (look-back)
    const int b = threadIdx.x;
    uint32_t tot = 0;
#pragma unroll
    for (int w = 0; w < kSortWarps; ++w) tot += wcnt[w][b];
    const uint64_t tag = (uint64_t)(pass + 1) << 56;
    uint64_t* my = sc.status + tile * kRadixBins + b;
    if (tile == 0) st_relaxed_u64(my, tag | kStatInc | tot);
    else st_relaxed_u64(my, tag | tot);
    const uint32_t ex = sort_block_excl(tot, wsum);
    const uint32_t dg = sort_block_excl(sc.ghist[pass * kRadixBins + b], wsum + kSortWarps);
    uint64_t before = 0;
    if (tile > 0) {
        int polls = 0;
        for (int64_t t = tile - 1; t >= 0; --t) {
            const uint64_t* q = sc.status + t * kRadixBins + b;
            uint64_t w = ld_relaxed_u64(q);
            while ((w & ~(kStatInc | kStatVal)) != tag && polls < kLookbackPolls) {
                ++polls;
                __nanosleep(64);
                w = ld_relaxed_u64(q);
            }
            if ((w & ~(kStatInc | kStatVal)) != tag) {
                if (err && *(volatile int*)err == 0) atomicCAS(err, 0, (int)DEV_TIMEOUT);
                break;
            }
            before += w & kStatVal;
            if (w & kStatInc) break;
        }
        st_relaxed_u64(my, tag | kStatInc | (before + tot));
    }
    dstart[b] = ex;
    gofs[b] = dg + (uint32_t)before;
    uint32_t run = ex;
#pragma unroll
    for (int w = 0; w < kSortWarps; ++w) {
        const uint32_t c = wcnt[w][b];
        wcnt[w][b] = run;
        run += c;
    }
    __syncthreads();
    // tile-local positions, keys and values into shared memory
    const unsigned lt = (1u << lane) - 1u;
#pragma unroll
    for (int c = 0; c < kSortChunks; ++c) {
        const int64_t i = wbase + c * 32 + lane;
        const bool valid = i < n;
        const unsigned active = __ballot_sync(0xffffffffu, valid);
        if (valid) {
            const uint32_t d = (uint32_t)(kr[c] >> shift) & (kRadixBins - 1);
            const unsigned peers = __match_any_sync(active, d);
            const uint32_t pos = wcnt[warp][d] + __popc(peers & lt);
            s_key[pos] = kr[c];
            s_val[pos] = vr[c];
            __syncwarp(active);
            if ((peers & lt) == 0) wcnt[warp][d] += __popc(peers);
        }
        __syncwarp();
    }
    __syncthreads();
    // runs of equal digits to consecutive global positions
    const int ln = (int)min((int64_t)kSortTile, n - tbase);
    for (int j = threadIdx.x; j < ln; j += kSortThreads) {
        const K k = s_key[j];
        const uint32_t d = (uint32_t)(k >> shift) & (kRadixBins - 1);
        const uint32_t g = gofs[d] + ((uint32_t)j - dstart[d]);
        keys_out[g] = k;
        vals_out[g] = s_val[j];
    }
}

// The scatter's shared memory exceeds the default 48 KB for 64-bit keys:
// raise the limit once per device.
template <class K>
fk_status scatter_smem_attr() {
    static std::mutex mu;
    static bool done[64] = {};
    int dev = 0;
    FK_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return set_error(FK_ERR_UNSUPPORTED, "device ordinal %d out of range", dev);
    std::lock_guard<std::mutex> lk(mu);
    if (!done[dev]) {
        FK_CUDA(cudaFuncSetAttribute(k_radix_onesweep<K>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)ScatterSmem<K>::bytes));
        done[dev] = true;
    }
    return FK_OK;
}

template <class K>
fk_status radix_sort_impl(K* keys, uint32_t* vals, K* keys_alt, uint32_t* vals_alt, int64_t n,
                          int key_bits, void* tmp, size_t tmp_bytes, cudaStream_t st,
                          bool* in_alt) {
    *in_alt = false;
    if (n <= 1) return FK_OK;
    if (n >= ((int64_t)1 << 32)) return set_error(FK_ERR_UNSUPPORTED, "radix sort of 2^32 or more keys");
    const int64_t tiles = (n + kSortTile - 1) / kSortTile;
    if (radix_sort_tmp_bytes(n, key_bits) > tmp_bytes)
        return set_error(FK_ERR_WORKSPACE, "radix sort scratch too small");
    const int passes = std::min(kMaxPasses, (std::max(key_bits, 1) + kRadixBits - 1) / kRadixBits);
    const SortScratch sc = SortScratch::at(tmp, tiles);
    FK_TRY(scatter_smem_attr<K>());
    int* errw = nullptr;
    FK_TRY(device_error_word(&errw));
    int dev = 0, sms = 0;
    FK_CUDA(cudaGetDevice(&dev));
    FK_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    FK_CUDA(cudaMemsetAsync(tmp, 0, sc.bytes, st));
    {
        ProfScope ps(PF_RADIX, (double)n * sizeof(K), st);
        const int64_t g = std::min<int64_t>((n + kSortThreads - 1) / kSortThreads, (int64_t)sms * kHistCtasPerSm);
        k_radix_hist_all<K><<<(unsigned)g, kSortThreads, 0, st>>>(keys, n, passes, sc.ghist);
        FK_LAUNCH_CHECK();
    }
    K* src_k = keys; uint32_t* src_v = vals;
    K* dst_k = keys_alt; uint32_t* dst_v = vals_alt;
    for (int p = 0; p < passes; ++p) {
        ProfScope ps(PF_RADIX, 2.0 * n * (sizeof(K) + 4), st);
        k_radix_onesweep<K><<<(unsigned)tiles, kSortThreads, ScatterSmem<K>::bytes, st>>>(
            src_k, src_v, dst_k, dst_v, n, p, sc, errw);
        FK_LAUNCH_CHECK();
        K* tk = src_k; src_k = dst_k; dst_k = tk;
        uint32_t* tv = src_v; src_v = dst_v; dst_v = tv;
        *in_alt = !*in_alt;
    }
    return FK_OK;
}
}  // namespace

// One digit pass whose first tile is never processed: the tile counter starts
// at 1 and only tiles - 1 CTAs run, so tile 1's look-back waits on a status
// word that nothing publishes, and every later tile reaches that word too.
// Each wait runs out after kLookbackPolls polls and records DEV_TIMEOUT.  The
// output is incomplete but every store stays inside it (a look-back that gave
// up sums fewer counts than the true prefix).  Buffers are allocated and freed
// here; the stream is synchronised before returning.
fk_status radix_lookback_timeout_probe(int64_t n, cudaStream_t st) {
    if (n < 2 * (int64_t)kSortTile || n > ((int64_t)1 << 24))
        return set_error(FK_ERR_INVALID_ARG, "probe size must be in [2 * 4096, 2^24]");
    const int64_t tiles = (n + kSortTile - 1) / kSortTile;
    const size_t tb = SortScratch::size(tiles);
    void* buf = nullptr;
    FK_CUDA(cudaMalloc(&buf, (size_t)n * 16 + tb));
    uint32_t* k0 = (uint32_t*)buf;
    uint32_t* v0 = k0 + n;
    uint32_t* k1 = v0 + n;
    uint32_t* v1 = k1 + n;
    void* tmp = (void*)(v1 + n);
    const SortScratch sc = SortScratch::at(tmp, tiles);
    fk_status rc = FK_OK;
    int* errw = nullptr;
    const uint32_t one = 1;
    if ((rc = scatter_smem_attr<uint32_t>()) != FK_OK || (rc = device_error_word(&errw)) != FK_OK) goto done;
    if (cudaMemsetAsync(buf, 0, (size_t)n * 16 + tb, st) != cudaSuccess ||
        cudaMemcpyAsync(&sc.ctr[0], &one, sizeof(one), cudaMemcpyHostToDevice, st) != cudaSuccess) {
        rc = set_error(FK_ERR_CUDA, "probe set-up failed");
        goto done;
    }
    k_radix_onesweep<uint32_t><<<(unsigned)(tiles - 1), kSortThreads, ScatterSmem<uint32_t>::bytes, st>>>(
        k0, v0, k1, v1, n, 0, sc, errw);
    if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(st) != cudaSuccess)
        rc = set_error(FK_ERR_CUDA, "probe launch failed");
done:
    cudaFree(buf);
    return rc;
}

size_t radix_sort_tmp_bytes(int64_t n, int key_bits) {
    (void)key_bits;
    const int64_t tiles = (std::max<int64_t>(n, 1) + kSortTile - 1) / kSortTile;
    return SortScratch::size(tiles);
}

fk_status radix_sort_pairs_u32(uint32_t* keys, uint32_t* vals, uint32_t* keys_alt,
                               uint32_t* vals_alt, int64_t n, int key_bits, void* tmp,
                               size_t tmp_bytes, cudaStream_t st, bool* in_alt) {
    return radix_sort_impl<uint32_t>(keys, vals, keys_alt, vals_alt, n, key_bits, tmp, tmp_bytes,
                                     st, in_alt);
}
fk_status radix_sort_pairs_u64(uint64_t* keys, uint32_t* vals, uint64_t* keys_alt,
                               uint32_t* vals_alt, int64_t n, int key_bits, void* tmp,
                               size_t tmp_bytes, cudaStream_t st, bool* in_alt) {
    return radix_sort_impl<uint64_t>(keys, vals, keys_alt, vals_alt, n, key_bits, tmp, tmp_bytes,
                                     st, in_alt);
}

}  // namespace fk
