// fk_sort.cu -- device-wide exclusive scan and a stable LSD radix sort of
// (key, value) pairs, written for the rank transform of the sample-point path
// (Sec. 2.2, Algorithm 2: the per-axis sort permutations phi^j).
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
namespace {
constexpr int kRadixBits = 8;
constexpr int kRadixBins = 1 << kRadixBits;
constexpr int kSortThreads = 256;
constexpr int kSortWarps = kSortThreads / 32;
constexpr int kSortChunks = 16;                                  // 32-key chunks per warp
constexpr int kSortTile = kSortThreads * kSortChunks;             // 4096 keys per CTA

template <class K>
__global__ void __launch_bounds__(kSortThreads) k_radix_hist(const K* __restrict__ keys, int64_t n,
                                                             int shift, uint32_t* __restrict__ hist,
                                                             int64_t tiles) {
    __shared__ uint32_t cnt[kRadixBins];
    for (int b = threadIdx.x; b < kRadixBins; b += kSortThreads) cnt[b] = 0;
    __syncthreads();
    int64_t base = (int64_t)blockIdx.x * kSortTile;
    for (int j = threadIdx.x; j < kSortTile; j += kSortThreads) {
        int64_t i = base + j;
        if (i < n) atomicAdd(&cnt[(uint32_t)(keys[i] >> shift) & (kRadixBins - 1)], 1u);
    }
    __syncthreads();
    for (int b = threadIdx.x; b < kRadixBins; b += kSortThreads)
        hist[(int64_t)b * tiles + blockIdx.x] = cnt[b];
}

// Stable scatter in two steps: the tile's keys are first ranked and placed
// in shared memory in (digit, original position) order, then written out so
// that consecutive threads store consecutive elements of each digit's run
// (runs of ~16 keys per digit and tile instead of one 4-byte store per key).
// Warp w owns keys [base + w*512, base + (w+1)*512) in chunk order, which is
// the tile's original order, so the ranking is stable.
template <class K>
struct ScatterSmem {
    static constexpr size_t o_key = 0;
    static constexpr size_t o_val = o_key + sizeof(K) * kSortTile;
    static constexpr size_t o_wcnt = o_val + 4 * kSortTile;
    static constexpr size_t o_dstart = o_wcnt + 4 * kSortWarps * kRadixBins;
    static constexpr size_t o_gofs = o_dstart + 4 * kRadixBins;
    static constexpr size_t o_wsum = o_gofs + 4 * kRadixBins;
    static constexpr size_t bytes = o_wsum + 4 * kSortWarps;
};

template <class K>
__global__ void __launch_bounds__(kSortThreads) k_radix_scatter(const K* __restrict__ keys,
                                                                const uint32_t* __restrict__ vals,
                                                                K* __restrict__ keys_out,
                                                                uint32_t* __restrict__ vals_out,
                                                                int64_t n, int shift,
                                                                const uint32_t* __restrict__ offs,
                                                                int64_t tiles) {
    static_assert(kSortThreads == kRadixBins, "one thread per digit in the tile-local scan");
    typedef ScatterSmem<K> L;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    K* s_key = reinterpret_cast<K*>(smem_raw + L::o_key);
    uint32_t* s_val = reinterpret_cast<uint32_t*>(smem_raw + L::o_val);
    uint32_t (*wcnt)[kRadixBins] = reinterpret_cast<uint32_t (*)[kRadixBins]>(smem_raw + L::o_wcnt);
    uint32_t* dstart = reinterpret_cast<uint32_t*>(smem_raw + L::o_dstart);
    uint32_t* gofs = reinterpret_cast<uint32_t*>(smem_raw + L::o_gofs);
    uint32_t* wsum = reinterpret_cast<uint32_t*>(smem_raw + L::o_wsum);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int b = threadIdx.x; b < kSortWarps * kRadixBins; b += kSortThreads) (&wcnt[0][0])[b] = 0;
    __syncthreads();
    const int64_t tbase = (int64_t)blockIdx.x * kSortTile;
    const int64_t wbase = tbase + (int64_t)warp * (32 * kSortChunks);
    // pass 1: keys into registers, per-warp digit counts
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
    // thread b: the tile-local start of digit b (exclusive scan over digits of
    // the tile's counts), the start of each warp's share of it, and the
    // global start of this tile's digit-b run
    {
        const int b = threadIdx.x;
        uint32_t tot = 0;
#pragma unroll
        for (int w = 0; w < kSortWarps; ++w) tot += wcnt[w][b];
        uint32_t x = tot;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) wsum[warp] = x;
        __syncthreads();
        uint32_t before = 0;
        for (int w = 0; w < warp; ++w) before += wsum[w];
        const uint32_t ex = before + x - tot;
        dstart[b] = ex;
        gofs[b] = offs[(int64_t)b * tiles + blockIdx.x];
        uint32_t run = ex;
#pragma unroll
        for (int w = 0; w < kSortWarps; ++w) {
            const uint32_t c = wcnt[w][b];
            wcnt[w][b] = run;
            run += c;
        }
    }
    __syncthreads();
    // pass 2: tile-local positions, keys and values into shared memory
    const unsigned lt = (1u << lane) - 1u;
#pragma unroll
    for (int c = 0; c < kSortChunks; ++c) {
        const int64_t i = wbase + c * 32 + lane;
        const bool valid = i < n;
        const unsigned active = __ballot_sync(0xffffffffu, valid);
        if (valid) {
            const uint32_t b = (uint32_t)(kr[c] >> shift) & (kRadixBins - 1);
            const unsigned peers = __match_any_sync(active, b);
            const uint32_t pos = wcnt[warp][b] + __popc(peers & lt);
            s_key[pos] = kr[c];
            s_val[pos] = vr[c];
            __syncwarp(active);
            if ((peers & lt) == 0) wcnt[warp][b] += __popc(peers);
        }
        __syncwarp();
    }
    __syncthreads();
    // pass 3: runs of equal digits to consecutive global positions
    const int ln = (int)min((int64_t)kSortTile, n - tbase);
    for (int j = threadIdx.x; j < ln; j += kSortThreads) {
        const K k = s_key[j];
        const uint32_t b = (uint32_t)(k >> shift) & (kRadixBins - 1);
        const uint32_t g = gofs[b] + ((uint32_t)j - dstart[b]);
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
        FK_CUDA(cudaFuncSetAttribute(k_radix_scatter<K>, cudaFuncAttributeMaxDynamicSharedMemorySize,
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
    int64_t tiles = (n + kSortTile - 1) / kSortTile;
    int64_t hn = tiles * kRadixBins;
    if (radix_sort_tmp_bytes(n, key_bits) > tmp_bytes)
        return set_error(FK_ERR_WORKSPACE, "radix sort scratch too small");
    uint32_t* hist = (uint32_t*)tmp;
    uint32_t* stmp = hist + ((hn + 63) & ~int64_t(63));
    FK_TRY(scatter_smem_attr<K>());
    K* src_k = keys; uint32_t* src_v = vals;
    K* dst_k = keys_alt; uint32_t* dst_v = vals_alt;
    for (int shift = 0; shift < key_bits; shift += kRadixBits) {
        ProfScope ps(PF_RADIX, 3.0 * n * (sizeof(K) + 4), st);
        k_radix_hist<K><<<(unsigned)tiles, kSortThreads, 0, st>>>(src_k, n, shift, hist, tiles);
        FK_LAUNCH_CHECK();
        FK_TRY(scan_u32_exclusive(hist, hist, hn, stmp, st));
        k_radix_scatter<K><<<(unsigned)tiles, kSortThreads, ScatterSmem<K>::bytes, st>>>(
            src_k, src_v, dst_k, dst_v, n, shift, hist, tiles);
        FK_LAUNCH_CHECK();
        K* tk = src_k; src_k = dst_k; dst_k = tk;
        uint32_t* tv = src_v; src_v = dst_v; dst_v = tv;
        *in_alt = !*in_alt;
    }
    return FK_OK;
}
}  // namespace

size_t radix_sort_tmp_bytes(int64_t n, int key_bits) {
    (void)key_bits;
    int64_t tiles = (n + kSortTile - 1) / kSortTile;
    int64_t hn = tiles * kRadixBins;
    return (size_t)(((hn + 63) & ~int64_t(63)) + scan_u32_tmp_words(hn)) * sizeof(uint32_t);
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
