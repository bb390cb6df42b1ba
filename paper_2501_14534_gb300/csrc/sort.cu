// Binning: visibility compaction, depth sort, key emission, tile sort and tile ranges.
//
// The keys are (global tile id, float32 bits of depth) with the Gaussian record index as
// value, stably sorted. Instead of one 64-bit sort over all keys, the visible (view,
// Gaussian) records are first sorted by depth bits (a 32-bit sort over V*N items), the keys
// are emitted in that order, and a stable sort on the tile id alone follows. A stable sort
// by tile of a sequence already ordered by (depth bits, record index) yields exactly the
// order of a stable sort of the full keys emitted in record order: equal tiles keep depth
// order, equal depths keep record order.
//
// Every primitive here is a reduce-then-scan design: no kernel waits on another block, so
// there is no spin loop anywhere in the binning.
#include "tgs_internal.cuh"

namespace tgs {
namespace {

constexpr int kScanThreads = 256;
constexpr int kScanItems = 8;
constexpr int kScanTile = kScanThreads * kScanItems;   // 2048
constexpr int kRadixThreads = 256;
constexpr int kRadixRounds = 16;
constexpr int kRadixTile = kRadixThreads * kRadixRounds;  // 4096
constexpr int kRadixBins = 256;

__device__ __forceinline__ int64_t count_of(const uint32_t *n_dev, int64_t n_cap) {
    if (!n_dev) return n_cap;
    int64_t n = (int64_t)*n_dev;
    return n < n_cap ? n : n_cap;
}

struct LoadPlain {
    const uint32_t *p;
    __device__ __forceinline__ uint32_t operator()(int64_t i) const { return p[i]; }
};
struct LoadVisible {
    const uint32_t *tt;
    __device__ __forceinline__ uint32_t operator()(int64_t i) const { return tt[i] > 0u ? 1u : 0u; }
};
struct LoadGathered {
    const uint32_t *ids, *tt;
    __device__ __forceinline__ uint32_t operator()(int64_t i) const { return tt[ids[i]]; }
};

__device__ __forceinline__ uint32_t warp_incl_scan(uint32_t x, int lane) {
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    return x;
}

// Exclusive scan of one value per thread over the block; returns the block total in *tot.
__device__ __forceinline__ uint32_t block_excl_scan(uint32_t x, uint32_t *s_warp, uint32_t *tot) {
    const int t = threadIdx.x, lane = t & 31, w = t >> 5;
    const int nw = blockDim.x >> 5;
    uint32_t inc = warp_incl_scan(x, lane);
    if (lane == 31) s_warp[w] = inc;
    __syncthreads();
    if (w == 0) {
        uint32_t s = lane < nw ? s_warp[lane] : 0u;
        uint32_t si = warp_incl_scan(s, lane);
        if (lane < nw) s_warp[lane] = si - s;
        if (lane == nw - 1) s_warp[32] = si;
    }
    __syncthreads();
    uint32_t r = inc - x + s_warp[w];
    *tot = s_warp[32];
    __syncthreads();
    return r;
}

template <class Load>
__global__ void __launch_bounds__(kScanThreads)
k_scan_reduce(Load ld, const uint32_t *n_dev, int64_t n_cap, uint32_t *partials) {
    __shared__ uint32_t s_warp[33];
    const int64_t n = count_of(n_dev, n_cap);
    const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
    uint32_t s = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; k++)
        if (base + k < n) s += ld(base + k);
    uint32_t tot;
    block_excl_scan(s, s_warp, &tot);
    if (threadIdx.x == 0) partials[blockIdx.x] = tot;
}

__global__ void __launch_bounds__(1024) k_scan_partials(uint32_t *partials, int64_t nb, uint32_t *total) {
    __shared__ uint32_t s_warp[33];
    uint32_t carry = 0;
    for (int64_t b0 = 0; b0 < nb; b0 += 1024) {
        const int64_t i = b0 + threadIdx.x;
        uint32_t x = i < nb ? partials[i] : 0u;
        uint32_t tot;
        uint32_t e = block_excl_scan(x, s_warp, &tot);
        if (i < nb) partials[i] = e + carry;
        carry += tot;
    }
    if (threadIdx.x == 0 && total) *total = carry;
}

template <class Load>
__global__ void __launch_bounds__(kScanThreads)
k_scan_down(Load ld, const uint32_t *n_dev, int64_t n_cap, const uint32_t *partials, uint32_t *out) {
    __shared__ uint32_t s_warp[33];
    const int64_t n = count_of(n_dev, n_cap);
    const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
    uint32_t v[kScanItems];
    uint32_t s = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; k++) {
        v[k] = (base + k < n) ? ld(base + k) : 0u;
        s += v[k];
    }
    uint32_t tot;
    uint32_t e = block_excl_scan(s, s_warp, &tot) + partials[blockIdx.x];
#pragma unroll
    for (int k = 0; k < kScanItems; k++) {
        if (base + k < n) out[base + k] = e;
        e += v[k];
    }
}

template <class Load>
void scan_generic(Load ld, const uint32_t *n_dev, int64_t n_cap, uint32_t *out, uint32_t *total,
                  uint32_t *partials, cudaStream_t st) {
    const int64_t nb = (n_cap + kScanTile - 1) / kScanTile;
    if (nb == 0) {
        if (total) cudaMemsetAsync(total, 0, sizeof(uint32_t), st);
        return;
    }
    count_launch();
    k_scan_reduce<<<(unsigned)nb, kScanThreads, 0, st>>>(ld, n_dev, n_cap, partials);
    count_launch();
    k_scan_partials<<<1, 1024, 0, st>>>(partials, nb, total);
    if (out) {
        count_launch();
        k_scan_down<<<(unsigned)nb, kScanThreads, 0, st>>>(ld, n_dev, n_cap, partials, out);
    }
}

// Compacts the visible records for the depth sort and replaces each visibility flag by the
// record's number of keys: the tiles of its rect that pass the cull test.
__global__ void k_compact(uint32_t *__restrict__ tt, const uint32_t *__restrict__ db,
                          const uint32_t *__restrict__ pos, int64_t n, const float4 *__restrict__ splats,
                          int B, uint32_t *__restrict__ keys, uint32_t *__restrict__ vals) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n || tt[i] == 0u) return;
    const uint32_t p = pos[i];
    keys[p] = db[i];
    vals[p] = (uint32_t)i;
    const float4 *rp = splats + (size_t)kSplatWords / 4 * i;
    tt[i] = (uint32_t)for_kept_tiles(rp[0], rp[1], rp[2], rp[3], B, [](int, int) {});
}

// ---- radix sort -------------------------------------------------------------------------

__global__ void __launch_bounds__(kRadixThreads)
k_radix_hist(const uint32_t *__restrict__ keys, const uint32_t *n_dev, int64_t n_cap, int shift,
             uint32_t mask, uint32_t *__restrict__ hist, int64_t nblocks) {
    __shared__ uint32_t s_h[kRadixBins];
    s_h[threadIdx.x] = 0u;
    __syncthreads();
    const int64_t n = count_of(n_dev, n_cap);
    const int64_t base = (int64_t)blockIdx.x * kRadixTile;
#pragma unroll 4
    for (int r = 0; r < kRadixRounds; r++) {
        const int64_t i = base + (int64_t)r * kRadixThreads + threadIdx.x;
        if (i < n) atomicAdd(&s_h[(keys[i] >> shift) & mask], 1u);
    }
    __syncthreads();
    hist[(int64_t)threadIdx.x * nblocks + blockIdx.x] = s_h[threadIdx.x];
}

// Stable scatter: items are ranked in index order. Within a round of 256 consecutive items
// the rank of an item among equal digits is (equal digits in earlier rounds of this block)
// + (equal digits in earlier warps of this round) + (equal digits in earlier lanes).
__global__ void __launch_bounds__(kRadixThreads)
k_radix_scatter(const uint32_t *__restrict__ keys_in, const uint32_t *__restrict__ vals_in,
                const uint32_t *n_dev, int64_t n_cap, int shift, uint32_t mask,
                const uint32_t *__restrict__ offsets, int64_t nblocks,
                uint32_t *__restrict__ keys_out, uint32_t *__restrict__ vals_out) {
    constexpr int NW = kRadixThreads / 32;
    __shared__ uint32_t s_cnt[NW][kRadixBins];
    __shared__ uint32_t s_base[kRadixBins];
    const int t = threadIdx.x, lane = t & 31, w = t >> 5;
    s_base[t] = offsets[(int64_t)t * nblocks + blockIdx.x];
#pragma unroll
    for (int k = 0; k < NW; k++) s_cnt[k][t] = 0u;
    __syncthreads();
    const int64_t n = count_of(n_dev, n_cap);
    const int64_t base = (int64_t)blockIdx.x * kRadixTile;
    if (base >= n) return;
    const uint32_t lt_mask = (1u << lane) - 1u;
    for (int r = 0; r < kRadixRounds; r++) {
        const int64_t i = base + (int64_t)r * kRadixThreads + t;
        if (base + (int64_t)r * kRadixThreads >= n) break;  // uniform across the block
        const bool valid = i < n;
        const uint32_t k = valid ? keys_in[i] : 0xffffffffu;
        const uint32_t d = valid ? ((k >> shift) & mask) : mask;
        const uint32_t peers = __match_any_sync(0xffffffffu, d);
        const uint32_t wr = __popc(peers & lt_mask);
        if (wr == 0u) s_cnt[w][d] = __popc(peers);
        __syncthreads();
        {
            // exclusive prefix over warps for digit t, and advance the block base
            uint32_t acc = s_base[t];
#pragma unroll
            for (int q = 0; q < NW; q++) {
                uint32_t c = s_cnt[q][t];
                s_cnt[q][t] = acc;
                acc += c;
            }
            s_base[t] = acc;
        }
        __syncthreads();
        if (valid) {
            const uint32_t p = s_cnt[w][d] + wr;
            keys_out[p] = k;
            vals_out[p] = vals_in[i];
        }
        __syncthreads();
#pragma unroll
        for (int q = 0; q < NW; q++) s_cnt[q][t] = 0u;
        __syncthreads();
    }
}

// ---- keys, ranges -------------------------------------------------------------------------

__global__ void k_emit(const uint32_t *__restrict__ sorted_ids, const uint32_t *__restrict__ offsets,
                       const uint32_t *n_dev, int64_t n_cap, const float4 *__restrict__ splats,
                       uint32_t n_gauss, const __grid_constant__ CamBatch cb,
                       uint32_t *__restrict__ tile_keys, uint32_t *__restrict__ tile_vals,
                       const uint32_t *K_dev, int64_t key_cap, uint32_t *status) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i == 0 && (int64_t)*K_dev > key_cap) atomicOr(status, kStatusCapacity);
    const int64_t n = count_of(n_dev, n_cap);
    if (i >= n) return;
    const uint32_t rec = sorted_ids[i];
    const int v = (int)(rec / n_gauss);
    const DevCam &c = cb.c[v];
    const float4 *rp = splats + (size_t)kSplatWords / 4 * rec;
    int64_t k = offsets[i];
    for_kept_tiles(rp[0], rp[1], rp[2], rp[3], cb.tile, [&](int tx, int ty) {
        if (k < key_cap) {
            const bool ok = tx < c.gx && ty < c.gy;   // records from outside may carry any rect
            tile_keys[k] = ok ? (uint32_t)(c.tile_offset + ty * c.gx + tx) : 0xffffffffu;
            tile_vals[k] = rec;
        }
        k++;
    });
}

__global__ void k_ranges(const uint32_t *__restrict__ keys, const uint32_t *K_dev, int64_t cap,
                         uint2 *__restrict__ ranges, uint32_t total_tiles) {
    const int64_t K = count_of(K_dev, cap);
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= K) return;
    const uint32_t t = keys[i];
    if (t >= total_tiles) return;
    if (i == 0 || keys[i - 1] != t) ranges[t].x = (uint32_t)i;
    if (i == K - 1 || keys[i + 1] != t) ranges[t].y = (uint32_t)(i + 1);
}

__global__ void k_full_keys(const uint32_t *__restrict__ tk, const uint32_t *__restrict__ tv,
                            const float4 *__restrict__ splats, const uint32_t *K_dev, int64_t cap,
                            uint64_t *__restrict__ out) {
    const int64_t K = count_of(K_dev, cap);
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= K) return;
    const float depth = splats[(size_t)kSplatWords / 4 * tv[i] + 2].w;
    out[i] = ((uint64_t)tk[i] << 32) | (uint64_t)__float_as_uint(depth);
}

__global__ void k_derive_touched(const float4 *__restrict__ splats, const int32_t *__restrict__ radii,
                                 int64_t n, int B, uint32_t *__restrict__ tt, uint32_t *__restrict__ db) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    if (radii[i] <= 0) {
        tt[i] = 0u;
        return;
    }
    // visibility flag; k_compact replaces it by the number of kept tiles
    tt[i] = 1u;
    db[i] = __float_as_uint(splats[(size_t)kSplatWords / 4 * i + 2].w);
}

inline unsigned blocks_for(int64_t n, int bs) { return (unsigned)((n + bs - 1) / bs); }

}  // namespace

size_t scan_partials_needed(int64_t n_items) {
    return (size_t)((n_items + kScanTile - 1) / kScanTile) + 1;
}

size_t radix_hist_needed(int64_t n_items) {
    return (size_t)kRadixBins * (size_t)((n_items + kRadixTile - 1) / kRadixTile) + 1;
}

void scan_flags(const uint32_t *tiles_touched, int64_t n_cap, uint32_t *out, uint32_t *total,
                uint32_t *partials, cudaStream_t st) {
    scan_generic(LoadVisible{tiles_touched}, nullptr, n_cap, out, total, partials, st);
}

void compact_visible(uint32_t *tiles_touched, const uint32_t *depth_bits, const uint32_t *pos,
                     int64_t n_cap, const float4 *splats, int tile, uint32_t *keys, uint32_t *vals,
                     cudaStream_t st) {
    if (n_cap <= 0) return;
    count_launch();
    k_compact<<<blocks_for(n_cap, 256), 256, 0, st>>>(tiles_touched, depth_bits, pos, n_cap, splats, tile,
                                                      keys, vals);
}

void radix_sort_pairs(uint32_t *&keys, uint32_t *&vals, uint32_t *keys_alt, uint32_t *vals_alt,
                      const uint32_t *n_dev, int64_t n_cap, int begin_bit, int end_bit,
                      uint32_t *hist, uint32_t *partials, cudaStream_t st) {
    const int64_t nb = (n_cap + kRadixTile - 1) / kRadixTile;
    if (nb == 0) return;
    for (int bit = begin_bit; bit < end_bit; bit += 8) {
        const int bits = (end_bit - bit) < 8 ? (end_bit - bit) : 8;
        const uint32_t mask = (1u << bits) - 1u;
        count_launch();
        k_radix_hist<<<(unsigned)nb, kRadixThreads, 0, st>>>(keys, n_dev, n_cap, bit, mask, hist, nb);
        scan_generic(LoadPlain{hist}, nullptr, (int64_t)kRadixBins * nb, hist, nullptr, partials, st);
        count_launch();
        k_radix_scatter<<<(unsigned)nb, kRadixThreads, 0, st>>>(keys, vals, n_dev, n_cap, bit, mask, hist,
                                                                nb, keys_alt, vals_alt);
        uint32_t *tk = keys, *tv = vals;
        keys = keys_alt;
        vals = vals_alt;
        keys_alt = tk;
        vals_alt = tv;
    }
}

void gather_tiles_scan(const uint32_t *sorted_ids, const uint32_t *tiles_touched, const uint32_t *n_dev,
                       int64_t n_cap, uint32_t *offsets, uint32_t *total, uint32_t *partials,
                       uint32_t *tmp, cudaStream_t st) {
    (void)tmp;
    scan_generic(LoadGathered{sorted_ids, tiles_touched}, n_dev, n_cap, offsets, total, partials, st);
}

void emit_keys(const uint32_t *sorted_ids, const uint32_t *offsets, const uint32_t *n_dev, int64_t n_cap,
               const float4 *splats, int64_t n_gauss, const CamBatch &cb, uint32_t *tile_keys,
               uint32_t *tile_vals, const uint32_t *K_dev, int64_t key_capacity, uint32_t *status,
               cudaStream_t st) {
    if (n_cap <= 0) return;
    count_launch();
    k_emit<<<blocks_for(n_cap, 256), 256, 0, st>>>(sorted_ids, offsets, n_dev, n_cap, splats,
                                                   (uint32_t)n_gauss, cb, tile_keys, tile_vals, K_dev,
                                                   key_capacity, status);
}

void find_ranges(const uint32_t *tile_keys, const uint32_t *K_dev, int64_t key_capacity, uint2 *ranges,
                 int total_tiles, cudaStream_t st) {
    cudaMemsetAsync(ranges, 0, sizeof(uint2) * (size_t)total_tiles, st);
    if (key_capacity <= 0) return;
    count_launch();
    k_ranges<<<blocks_for(key_capacity, 256), 256, 0, st>>>(tile_keys, K_dev, key_capacity, ranges,
                                                             (uint32_t)total_tiles);
}

void derive_touched(const float4 *splats, const int32_t *radii, int64_t n_rec, int tile,
                    uint32_t *tiles_touched, uint32_t *depth_bits, cudaStream_t st) {
    if (n_rec <= 0) return;
    count_launch();
    k_derive_touched<<<blocks_for(n_rec, 256), 256, 0, st>>>(splats, radii, n_rec, tile, tiles_touched,
                                                             depth_bits);
}

void make_full_keys(const uint32_t *tile_keys, const uint32_t *tile_vals, const float4 *splats,
                    const uint32_t *K_dev, int64_t cap, uint64_t *out, cudaStream_t st) {
    if (cap <= 0) return;
    count_launch();
    k_full_keys<<<blocks_for(cap, 256), 256, 0, st>>>(tile_keys, tile_vals, splats, K_dev, cap, out);
}

}  // namespace tgs
