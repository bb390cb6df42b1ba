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
constexpr int kRadixRounds = 8;
constexpr int kRadixTile = kRadixThreads * kRadixRounds;  // 2048
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
// For rects of at most 64 tiles it also stores which tiles (row-major within the rect) passed,
// so that the emission does not repeat the test.
__global__ void k_compact(uint32_t *__restrict__ tt, const uint32_t *__restrict__ db,
                          const uint32_t *__restrict__ pos, int64_t n, const float4 *__restrict__ splats,
                          int B, uint32_t *__restrict__ keys, uint32_t *__restrict__ vals,
                          uint2 *__restrict__ kmask) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n || tt[i] == 0u) return;
    const uint32_t p = pos[i];
    keys[p] = db[i];
    vals[p] = (uint32_t)i;
    const float4 *rp = splats + (size_t)kSplatWords / 4 * i;
    const uint32_t rx = __float_as_uint(rp[2].y);
    const int x0 = (int)(rx & 0xFFFFu) / B, nx = (int)(rx >> 16) / B - x0 + 1;
    uint64_t m = 0;
    tt[i] = (uint32_t)for_kept_tiles(rp[0], rp[1], rp[2], rp[3], B, [&](int tx, int ty) {
        const int b = (ty - ((int)(__float_as_uint(rp[2].z) & 0xFFFFu) / B)) * nx + (tx - x0);
        if (b < 64) m |= (uint64_t)1 << b;
    });
    if (kmask) kmask[i] = make_uint2((uint32_t)m, (uint32_t)(m >> 32));
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

// Stable scatter of one block of 2048 items. The block's items are first ranked into shared
// memory in (digit, index) order -- rank = start of the digit in the block + equal digits in
// earlier rounds + earlier warps of this round + earlier lanes -- and then written out in
// that order, so that each digit's run of this block goes to consecutive global addresses.
__global__ void __launch_bounds__(kRadixThreads)
k_radix_scatter(const uint32_t *__restrict__ keys_in, const uint32_t *__restrict__ vals_in,
                const uint32_t *n_dev, int64_t n_cap, int shift, uint32_t mask,
                const uint32_t *__restrict__ offsets, int64_t nblocks,
                uint32_t *__restrict__ keys_out, uint32_t *__restrict__ vals_out) {
    constexpr int NW = kRadixThreads / 32;
    __shared__ uint32_t s_cnt[NW][kRadixBins];
    __shared__ uint32_t s_run[kRadixBins];     // items of each digit placed so far
    __shared__ uint32_t s_start[kRadixBins];   // start of each digit in the block's order
    __shared__ uint32_t s_goff[kRadixBins];    // global position of the block's digit run
    __shared__ uint32_t s_warp[33];
    __shared__ uint32_t s_k[kRadixTile], s_v[kRadixTile];
    const int t = threadIdx.x, lane = t & 31, w = t >> 5;
    const int64_t n = count_of(n_dev, n_cap);
    const int64_t base = (int64_t)blockIdx.x * kRadixTile;
    if (base >= n) return;  // uniform across the block
    const int cnt = (int)((n - base) < kRadixTile ? (n - base) : kRadixTile);
    uint32_t kr[kRadixRounds], vr[kRadixRounds];
    s_run[t] = 0u;
#pragma unroll
    for (int q = 0; q < NW; q++) s_cnt[q][t] = 0u;
    __syncthreads();
#pragma unroll
    for (int r = 0; r < kRadixRounds; r++) {
        const int j = r * kRadixThreads + t;
        const bool valid = j < cnt;
        kr[r] = valid ? keys_in[base + j] : 0xffffffffu;
        vr[r] = valid ? vals_in[base + j] : 0u;
        if (valid) atomicAdd(&s_run[(kr[r] >> shift) & mask], 1u);
    }
    __syncthreads();
    uint32_t tot;
    const uint32_t start = block_excl_scan(s_run[t], s_warp, &tot);
    s_start[t] = start;
    s_goff[t] = offsets[(int64_t)t * nblocks + blockIdx.x];
    s_run[t] = 0u;
    __syncthreads();
    const uint32_t lt_mask = (1u << lane) - 1u;
#pragma unroll
    for (int r = 0; r < kRadixRounds; r++) {
        if (r * kRadixThreads >= cnt) continue;  // uniform: the block's tail rounds are empty
        const bool valid = r * kRadixThreads + t < cnt;
        const uint32_t d = valid ? ((kr[r] >> shift) & mask) : mask;
        // lanes holding the same digit: one ballot per digit bit (warp multisplit)
        uint32_t peers = 0xffffffffu;
#pragma unroll
        for (int b = 0; b < 8; b++) {
            const uint32_t bal = __ballot_sync(0xffffffffu, (d >> b) & 1u);
            peers &= ((d >> b) & 1u) ? bal : ~bal;
        }
        const uint32_t wr = __popc(peers & lt_mask);
        if (wr == 0u) s_cnt[w][d] = __popc(peers);
        __syncthreads();
        {
            uint32_t acc = s_run[t];
#pragma unroll
            for (int q = 0; q < NW; q++) {
                const uint32_t c = s_cnt[q][t];
                s_cnt[q][t] = acc;
                acc += c;
            }
            s_run[t] = acc;
        }
        __syncthreads();
        if (valid) {
            const uint32_t lp = s_start[d] + s_cnt[w][d] + wr;
            s_k[lp] = kr[r];
            s_v[lp] = vr[r];
        }
        __syncthreads();
#pragma unroll
        for (int q = 0; q < NW; q++) s_cnt[q][t] = 0u;
        __syncthreads();
    }
    for (int i = t; i < cnt; i += kRadixThreads) {
        const uint32_t k = s_k[i];
        const uint32_t d = (k >> shift) & mask;
        const uint32_t gp = s_goff[d] + ((uint32_t)i - s_start[d]);
        keys_out[gp] = k;
        vals_out[gp] = s_v[i];
    }
}

// ---- keys, ranges -------------------------------------------------------------------------

// Key emission. A warp takes 32 consecutive records of the depth order; their keys form one
// contiguous segment of the key array, which the warp assembles in shared memory and writes
// out with coalesced stores (segments longer than the buffer are written directly).
constexpr int kEmitThreads = 256;
constexpr int kEmitBuf = 512;  // keys staged per warp

__global__ void __launch_bounds__(kEmitThreads)
k_emit(const uint32_t *__restrict__ sorted_ids, const uint32_t *__restrict__ offsets,
       const uint32_t *n_dev, int64_t n_cap, const float4 *__restrict__ splats, uint32_t n_gauss,
       const __grid_constant__ CamBatch cb, const uint2 *__restrict__ kmask,
       uint32_t *__restrict__ tile_keys, uint32_t *__restrict__ tile_vals, const uint32_t *K_dev,
       int64_t key_cap, uint32_t *status) {
    __shared__ uint32_t s_k[kEmitThreads / 32][kEmitBuf], s_v[kEmitThreads / 32][kEmitBuf];
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t K = (int64_t)*K_dev;
    if (i == 0 && K > key_cap) atomicOr(status, kStatusCapacity);
    const int64_t n = count_of(n_dev, n_cap);
    if (i - lane >= n) return;  // the whole warp is past the end
    const bool valid = i < n;
    const uint32_t off = valid ? offsets[i] : 0u;
    const uint32_t end = valid ? (i + 1 < n ? offsets[i + 1] : (uint32_t)K) : 0u;
    const uint32_t seg0 = __shfl_sync(0xffffffffu, off, 0);
    const uint32_t seg_end = __reduce_max_sync(0xffffffffu, end);
    const uint32_t seg_len = seg_end - seg0;
    const bool staged = seg_len <= (uint32_t)kEmitBuf;
    if (valid && end > off) {
        const uint32_t rec = sorted_ids[i];
        const int v = (int)(rec / n_gauss);
        const DevCam &c = cb.c[v];
        const float4 *rp = splats + (size_t)kSplatWords / 4 * rec;
        const int B = cb.tile;
        const uint32_t rx = __float_as_uint(rp[2].y), ry = __float_as_uint(rp[2].z);
        const int x0 = (int)(rx & 0xFFFFu) / B, x1 = (int)(rx >> 16) / B;
        const int y0 = (int)(ry & 0xFFFFu) / B, y1 = (int)(ry >> 16) / B;
        const int nx = x1 - x0 + 1;
        int64_t k = off;
        auto put = [&](int tx, int ty) {
            const bool ok = tx < c.gx && ty < c.gy;   // records from outside may carry any rect
            const uint32_t key = ok ? (uint32_t)(c.tile_offset + ty * c.gx + tx) : 0xffffffffu;
            if (staged) {
                s_k[w][k - seg0] = key;
                s_v[w][k - seg0] = rec;
            } else if (k < key_cap) {
                tile_keys[k] = key;
                tile_vals[k] = rec;
            }
            k++;
        };
        if (nx * (y1 - y0 + 1) <= 64) {
            const uint2 mm = kmask[rec];
            uint64_t m = ((uint64_t)mm.y << 32) | mm.x;
            while (m) {
                const int b = __ffsll((long long)m) - 1;
                m &= m - 1;
                put(x0 + b % nx, y0 + b / nx);
            }
        } else {
            for_kept_tiles(rp[0], rp[1], rp[2], rp[3], B, put);
        }
    }
    __syncwarp();
    if (staged)
        for (uint32_t j = lane; j < seg_len; j += 32) {
            const int64_t gp = (int64_t)seg0 + j;
            if (gp < key_cap) {
                tile_keys[gp] = s_k[w][j];
                tile_vals[gp] = s_v[w][j];
            }
        }
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
                     uint2 *kmask, cudaStream_t st) {
    if (n_cap <= 0) return;
    count_launch();
    k_compact<<<blocks_for(n_cap, 256), 256, 0, st>>>(tiles_touched, depth_bits, pos, n_cap, splats, tile,
                                                      keys, vals, kmask);
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
               const float4 *splats, int64_t n_gauss, const CamBatch &cb, const uint2 *kmask,
               uint32_t *tile_keys, uint32_t *tile_vals, const uint32_t *K_dev, int64_t key_capacity,
               uint32_t *status, cudaStream_t st) {
    if (n_cap <= 0) return;
    count_launch();
    k_emit<<<blocks_for(n_cap, kEmitThreads), kEmitThreads, 0, st>>>(sorted_ids, offsets, n_dev, n_cap, splats,
                                                                     (uint32_t)n_gauss, cb, kmask, tile_keys,
                                                                     tile_vals, K_dev, key_capacity, status);
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
