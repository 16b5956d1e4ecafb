// Stable LSD radix sort of 64-bit keys with optional 32-bit payloads.
//
// Three kernels per 8-bit digit: a per-tile histogram, one exclusive scan of
// the digit-major histogram table, and a scatter that ranks each key among
// the earlier keys of its tile with the same digit (warp match + per-warp
// digit counters), so equal keys keep their order.
#include "gbfmm_internal.cuh"

namespace gbfmm {

namespace {
constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int kItems = 16;                   // keys per thread
constexpr int kTile = kThreads * kItems;     // 4096 keys per block
constexpr int kWarpItems = kTile / kWarps;   // 512 contiguous keys per warp
template <typename K, bool VAL>
constexpr size_t scatter_smem() {
    return (size_t)kTile * (sizeof(K) + (VAL ? 4 : 0)) + (size_t)(kWarps + 2) * 256 * 4;
}
// blocks per SM the scatter's registers are cut for: three for 32-bit keys
// without payload (80 registers, no spills), two otherwise
template <typename K, bool VAL>
constexpr int scatter_min_blocks() { return (sizeof(K) == 4 && !VAL) ? 3 : 2; }

template <typename K>
__global__ void __launch_bounds__(kThreads) k_hist(const K* __restrict__ keys, int64_t n,
                                                   const unsigned long long* __restrict__ dn, int shift,
                                                   uint32_t* __restrict__ hist, int nblocks) {
    __shared__ uint32_t h[256];
    if (dn && (int64_t)*dn < n) n = (int64_t)*dn;  // tiles past the count give empty histograms
    for (int i = threadIdx.x; i < 256; i += kThreads) h[i] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * kTile;
#pragma unroll 4
    for (int k = 0; k < kItems; ++k) {
        int64_t i = base + (int64_t)k * kThreads + threadIdx.x;
        if (i < n) atomicAdd(&h[(unsigned)(keys[i] >> shift) & 255u], 1u);
    }
    __syncthreads();
    for (int d = threadIdx.x; d < 256; d += kThreads) hist[(int64_t)d * nblocks + blockIdx.x] = h[d];
}

// Scatter: rank every key among the earlier keys of its tile with the same
// digit (warp match + per-warp digit counters), reorder the tile by digit in
// shared memory, then write each digit's run to its global position with
// consecutive threads writing consecutive addresses.
template <typename K, bool VAL>
__global__ void __launch_bounds__(kThreads, scatter_min_blocks<K, VAL>()) k_scatter(const K* __restrict__ kin,
                                                      const uint32_t* __restrict__ vin,
                                                      K* __restrict__ kout,
                                                      uint32_t* __restrict__ vout, int64_t n,
                                                      const unsigned long long* __restrict__ dn,
                                                      int shift, const uint32_t* __restrict__ offs,
                                                      int nblocks) {
    extern __shared__ __align__(16) unsigned char sh_scatter[];
    K* skey = reinterpret_cast<K*>(sh_scatter);                                  // kTile
    uint32_t* sval = reinterpret_cast<uint32_t*>(skey + kTile);                  // kTile (VAL only)
    uint32_t (*wcount)[256] = reinterpret_cast<uint32_t (*)[256]>(sval + (VAL ? kTile : 0));  // kWarps x 256
    uint32_t* boff = &wcount[kWarps][0];    // global start of each digit for this tile
    uint32_t* lstart = boff + 256;          // start of each digit inside the tile
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int i = threadIdx.x; i < kWarps * 256; i += kThreads) (&wcount[0][0])[i] = 0;
    for (int d = threadIdx.x; d < 256; d += kThreads) boff[d] = offs[(int64_t)d * nblocks + blockIdx.x];
    __syncthreads();
    const int64_t tile0 = (int64_t)blockIdx.x * kTile;
    if (dn && (int64_t)*dn < n) n = (int64_t)*dn;
    if (tile0 >= n) return;  // the whole block: nothing of this tile is present
    const int64_t base = tile0 + (int64_t)warp * kWarpItems;
    K key[kItems];
    uint32_t val[VAL ? kItems : 1], rank[kItems];
    // all loads first, so that they are in flight together
#pragma unroll
    for (int r = 0; r < kItems; ++r) {
        const int64_t i = base + r * 32 + lane;
        key[r] = i < n ? kin[i] : K(0);
        if (VAL) val[VAL ? r : 0] = i < n ? vin[i] : 0u;
    }
#pragma unroll
    for (int r = 0; r < kItems; ++r) {
        const int64_t i = base + r * 32 + lane;
        const bool valid = i < n;
        const uint32_t d = valid ? (uint32_t)(key[r] >> shift) & 255u : 0xFFFFFFFFu;
        const unsigned peers = __match_any_sync(0xffffffffu, d);
        const uint32_t before = valid ? wcount[warp][d] : 0u;
        rank[r] = before + __popc(peers & ((1u << lane) - 1u));
        __syncwarp();
        if (valid && lane == 31 - __clz(peers)) wcount[warp][d] = before + __popc(peers);
        __syncwarp();
    }
    __syncthreads();
    {
        const int d = threadIdx.x;  // kThreads == 256 digits
        uint32_t run = 0;
#pragma unroll
        for (int w = 0; w < kWarps; ++w) {
            const uint32_t t = wcount[w][d];
            wcount[w][d] = run;
            run += t;
        }
        lstart[d] = run;  // this digit's count in the tile, scanned below
    }
    __syncthreads();
    if (threadIdx.x < 32) {  // exclusive scan of the 256 digit counts
        uint32_t c[8], s = 0;
#pragma unroll
        for (int k = 0; k < 8; ++k) { c[k] = lstart[threadIdx.x * 8 + k]; s += c[k]; }
        uint32_t incl = s;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t v = __shfl_up_sync(0xffffffffu, incl, o);
            if ((int)threadIdx.x >= o) incl += v;
        }
        uint32_t run = incl - s;
#pragma unroll
        for (int k = 0; k < 8; ++k) { lstart[threadIdx.x * 8 + k] = run; run += c[k]; }
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < kItems; ++r) {
        const int64_t i = base + r * 32 + lane;
        if (i < n) {
            const uint32_t d = (uint32_t)(key[r] >> shift) & 255u;
            const uint32_t pos = lstart[d] + wcount[warp][d] + rank[r];
            skey[pos] = key[r];
            if (VAL) sval[pos] = val[VAL ? r : 0];
        }
    }
    __syncthreads();
    const int cnt = (int)((n - tile0) < kTile ? (n - tile0) : kTile);
    for (int j = threadIdx.x; j < cnt; j += kThreads) {
        const K k = skey[j];
        const uint32_t d = (uint32_t)(k >> shift) & 255u;
        const uint32_t pos = boff[d] + (uint32_t)j - lstart[d];
        kout[pos] = k;
        if (VAL) vout[pos] = sval[j];
    }
}

// Single-block exclusive scan in tiles of 4096 words: a coalesced load into
// shared memory, four consecutive words per thread, a block scan of the
// thread sums, a coalesced store, and a carry into the next tile.
__global__ void __launch_bounds__(1024) k_scan(uint32_t* data, int64_t count, uint32_t* total) {
    __shared__ __align__(16) uint32_t tile[4096];
    __shared__ uint32_t warp_sums[32];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    uint32_t carry = 0;
    for (int64_t base = 0; base < count; base += 4096) {
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int64_t i = base + k * 1024 + tid;
            tile[k * 1024 + tid] = i < count ? data[i] : 0u;
        }
        __syncthreads();
        const uint4 v = reinterpret_cast<const uint4*>(tile)[tid];
        const uint32_t s = v.x + v.y + v.z + v.w;
        uint32_t incl = s;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t t = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += t;
        }
        if (lane == 31) warp_sums[warp] = incl;
        __syncthreads();
        if (warp == 0) {
            const uint32_t ws = warp_sums[lane];
            uint32_t wi = ws;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t t = __shfl_up_sync(0xffffffffu, wi, o);
                if (lane >= o) wi += t;
            }
            warp_sums[lane] = wi - ws;  // exclusive offsets of the warps; the tile total is wi at lane 31
            if (lane == 31) tile[0] = wi;  // tile[0] was consumed above; reused to pass the total
        }
        __syncthreads();
        const uint32_t tile_total = tile[0];
        uint32_t run = carry + warp_sums[warp] + incl - s;
        __syncthreads();
        uint4 o;
        o.x = run; run += v.x;
        o.y = run; run += v.y;
        o.z = run; run += v.z;
        o.w = run;
        reinterpret_cast<uint4*>(tile)[tid] = o;
        __syncthreads();
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int64_t i = base + k * 1024 + tid;
            if (i < count) data[i] = tile[k * 1024 + tid];
        }
        carry += tile_total;
        __syncthreads();
    }
    if (tid == 0 && total) *total = carry;
}
// Large scans in three passes: segment sums, a scan of the sums, and a
// rescan of each segment from its offset.
constexpr int kSegment = 4096;
__global__ void __launch_bounds__(256) k_seg_sum(const uint32_t* __restrict__ data, int64_t count,
                                                 uint32_t* __restrict__ sums) {
    __shared__ uint32_t red[256];
    const int64_t base = (int64_t)blockIdx.x * kSegment;
    uint32_t s = 0;
    for (int k = threadIdx.x; k < kSegment; k += 256) {
        const int64_t i = base + k;
        if (i < count) s += data[i];
    }
    red[threadIdx.x] = s;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) sums[blockIdx.x] = red[0];
}

__global__ void __launch_bounds__(256) k_seg_scan(uint32_t* __restrict__ data, int64_t count,
                                                  const uint32_t* __restrict__ offs) {
    __shared__ uint32_t warp_sums[8];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t base = (int64_t)blockIdx.x * kSegment + (int64_t)threadIdx.x * (kSegment / 256);
    uint32_t v[kSegment / 256];
    uint32_t s = 0;
#pragma unroll
    for (int k = 0; k < kSegment / 256; ++k) {
        const int64_t i = base + k;
        v[k] = i < count ? data[i] : 0u;
        s += v[k];
    }
    uint32_t incl = s;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
    }
    if (lane == 31) warp_sums[warp] = incl;
    __syncthreads();
    uint32_t wo = 0;
    for (int w = 0; w < warp; ++w) wo += warp_sums[w];
    uint32_t run = offs[blockIdx.x] + wo + incl - s;
#pragma unroll
    for (int k = 0; k < kSegment / 256; ++k) {
        const int64_t i = base + k;
        if (i < count) data[i] = run;
        run += v[k];
    }
}
}  // namespace

size_t scan_scratch_words(int64_t count) { return (size_t)((count + kSegment - 1) / kSegment + 2); }

void scan_exclusive_u32_large(uint32_t* data, int64_t count, uint32_t* total, uint32_t* scratch,
                              cudaStream_t st) {
    // one block scans 4096 values at a time, one tile after another: beyond a
    // few tiles the three parallel passes finish sooner
    if (count <= 4 * 4096) {
        (k_scan<<<1, 1024, 0, st>>>(data, count, total), note_launch());
        return;
    }
    const int nseg = (int)((count + kSegment - 1) / kSegment);
    (k_seg_sum<<<nseg, 256, 0, st>>>(data, count, scratch), note_launch());
    (k_scan<<<1, 1024, 0, st>>>(scratch, nseg, total), note_launch());
    (k_seg_scan<<<nseg, 256, 0, st>>>(data, count, scratch), note_launch());
}

size_t radix_hist_words(int64_t n) {
    const int64_t nb = (n + kTile - 1) / kTile;
    const int64_t cells = 256 * (nb > 0 ? nb : 1);
    return (size_t)(cells + 1) + scan_scratch_words(cells);
}

void scan_exclusive_u32(uint32_t* data, int64_t count, uint32_t* total, cudaStream_t st) {
    (k_scan<<<1, 1024, 0, st>>>(data, count, total), note_launch());
}

namespace {
template <typename K, bool VAL>
int radix_sort_impl(K* k0, uint32_t* v0, K* k1, uint32_t* v1, int64_t n, int lo_bit, int bits, uint32_t* hist,
                    cudaStream_t st, const unsigned long long* dn) {
    if (n <= 1 || bits <= lo_bit) return 0;
    ensure_dyn_smem((const void*)k_scatter<K, VAL>, (int)scatter_smem<K, VAL>());
    const int nblocks = (int)((n + kTile - 1) / kTile);
    int cur = 0;
    for (int shift = lo_bit; shift < bits; shift += 8) {
        K* ki = cur ? k1 : k0;
        uint32_t* vi = cur ? v1 : v0;
        K* ko = cur ? k0 : k1;
        uint32_t* vo = cur ? v0 : v1;
        (k_hist<K><<<nblocks, kThreads, 0, st>>>(ki, n, dn, shift, hist, nblocks), note_launch());
        scan_exclusive_u32_large(hist, (int64_t)256 * nblocks, nullptr, hist + (size_t)256 * nblocks + 1, st);
        (k_scatter<K, VAL><<<nblocks, kThreads, scatter_smem<K, VAL>(), st>>>(ki, vi, ko, vo, n, dn, shift,
                                                                              hist, nblocks), note_launch());
        cur ^= 1;
    }
    return cur;
}
}  // namespace

int radix_sort(uint64_t* k0, uint32_t* v0, uint64_t* k1, uint32_t* v1, int64_t n, int bits,
               uint32_t* hist, cudaStream_t st, const unsigned long long* dn, int lo_bit) {
    return v0 ? radix_sort_impl<uint64_t, true>(k0, v0, k1, v1, n, lo_bit, bits, hist, st, dn)
              : radix_sort_impl<uint64_t, false>(k0, nullptr, k1, nullptr, n, lo_bit, bits, hist, st, dn);
}

int radix_sort32(uint32_t* k0, uint32_t* k1, int64_t n, int bits, uint32_t* hist, cudaStream_t st,
                 const unsigned long long* dn, int lo_bit) {
    return radix_sort_impl<uint32_t, false>(k0, nullptr, k1, nullptr, n, lo_bit, bits, hist, st, dn);
}

}  // namespace gbfmm
