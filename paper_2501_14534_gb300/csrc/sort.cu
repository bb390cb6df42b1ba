// Binning: depth sort, key count, key emission, tile sort and tile ranges.
//
// The keys are (global tile id, float32 bits of depth) with the Gaussian record index as
// value, stably sorted. Instead of one 64-bit sort over all keys, the (view, Gaussian)
// records are first sorted by depth bits (a 32-bit sort over V*N items; records not visible
// carry the key 0xffffffff and sort after every visible one), the keys are emitted in that
// order, and a stable sort on the tile id alone follows. A stable sort
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
// 16 items per thread (4096 per block): longer runs per digit in the scatter's writes and half
// the histogram rows of 2048 (binning 2.41 -> 2.28 ms per step on the 1M x 16-view step; 24
// items per thread: 2.37 ms)
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

// a = q d + r for a < 2^22, d < 2^22, with one float multiply by rcp = 1/d (rounded): the
// product is then within 1/d of a/d from below, so the truncated quotient is q or q - 1
__device__ __forceinline__ void divmod_small(uint32_t a, uint32_t d, float rcp, uint32_t &q, uint32_t &r) {
    if ((a | d) < (1u << 22)) {
        q = __float2uint_rz(__uint2float_rn(a) * rcp);
        r = a - q * d;
        if (r >= d) {
            q++;
            r -= d;
        }
    } else {
        q = a / d;
        r = a - q * d;
    }
}

// Key counts of the depth-sorted records. For each record of the depth order: the tiles of its
// rect that pass the cull test (their number; for rects of at most 64 tiles also which ones,
// row-major within the rect) and the packed pixel rect, all stored in depth order for the
// emission; and per block of kScanTile records the number of keys (the scan's partials).
//
// Work balance: warp w of a block takes 256 records, 32 at a time, and spreads the (record,
// rect tile) pairs of the 32 over its lanes, so that one large rect does not keep the other 31
// lanes idle. A lane finds the record of pair p by binary search over the exclusive prefix
// sums of the rect sizes (held one per lane and read with shuffles).
__global__ void __launch_bounds__(kScanThreads)
k_count_keys(const uint32_t *__restrict__ sorted_ids, const uint32_t *__restrict__ sorted_keys,
             const uint32_t *n_dev, int64_t n_cap, const float4 *__restrict__ splats, int B, KeyInfo ki,
             uint32_t *__restrict__ partials) {
    constexpr int NW = kScanThreads / 32;
    __shared__ float4 s_g[NW][32];     // mean2d x, y; conic a, b
    __shared__ float4 s_h[NW][32];     // conic c; tau; b / c; b / a
    __shared__ int4 s_r[NW][32];       // pixel rect x0, x1, y0, y1 (inclusive)
    __shared__ uint32_t s_m[NW][32][2];  // kept-tile bits of rects of at most 64 tiles
    __shared__ uint32_t s_c[NW][32];     // kept-tile counts
    __shared__ uint4 s_k[NW][32];        // pair prefix, nx (bit 31: at most 64 tiles), rcp(nx), tx0 | ty0 << 16
    __shared__ uint32_t s_warp[33];
    const int lb = __ffs(B) - 1;  // B is 8, 16 or 32
    const unsigned full = 0xffffffffu;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t n = count_of(n_dev, n_cap);
    const int64_t base = (int64_t)blockIdx.x * kScanTile;
    if (base >= n) {  // uniform across the block
        if (threadIdx.x == 0) partials[blockIdx.x] = 0u;
        return;
    }
    uint32_t wsum = 0u;
#pragma unroll 1
    for (int q = 0; q < kScanItems; q++) {
        const int64_t j = base + (int64_t)(w * kScanItems + q) * 32 + lane;
        // records not visible carry the key 0xffffffff and sort last
        const bool valid = j < n && sorted_keys[j] != kNoDepth;
        uint32_t ntiles = 0u, rx = 0u, ry = 0u;
        int tx0 = 0, ty0 = 0, nx = 1;
        if (valid) {
            const float4 *rp = splats + (size_t)kSplatWords / 4 * sorted_ids[j];
            const float4 s0 = rp[0], s1 = rp[1], s2 = rp[2], s3 = rp[3];
            rx = __float_as_uint(s2.y);
            ry = __float_as_uint(s2.z);
            const int ix0 = (int)(rx & 0xFFFFu), ix1 = (int)(rx >> 16);
            const int iy0 = (int)(ry & 0xFFFFu), iy1 = (int)(ry >> 16);
            tx0 = ix0 >> lb;
            ty0 = iy0 >> lb;
            nx = (ix1 >> lb) - tx0 + 1;
            const int ny = (iy1 >> lb) - ty0 + 1;
            ntiles = (nx > 0 && ny > 0) ? (uint32_t)nx * (uint32_t)ny : 0u;
            s_g[w][lane] = s0;
            s_h[w][lane] = make_float4(s1.x, s3.x, s3.y, s3.z);
            s_r[w][lane] = make_int4(ix0, ix1, iy0, iy1);
        }
        if (nx < 1) nx = 1;
        const float rcp = __frcp_rn((float)nx);
        s_m[w][lane][0] = 0u;
        s_m[w][lane][1] = 0u;
        s_c[w][lane] = 0u;
        const uint32_t inc = warp_incl_scan(ntiles, lane);
        const uint32_t excl = inc - ntiles;
        const uint32_t total = __shfl_sync(full, inc, 31);
        s_k[w][lane] = make_uint4(excl, (uint32_t)nx | (ntiles <= 64u ? 0x80000000u : 0u), __float_as_uint(rcp),
                                  (uint32_t)tx0 | ((uint32_t)ty0 << 16));
        __syncwarp();
        for (uint32_t p0 = 0; p0 < total; p0 += 32) {
            const uint32_t p = p0 + (uint32_t)lane;
            // owner: the last lane whose exclusive prefix is <= p (it has ntiles > 0)
            int r = 0;
#pragma unroll
            for (int step = 16; step >= 1; step >>= 1)
                if (__shfl_sync(full, excl, r + step) <= p) r += step;
            if (p < total) {
                const uint4 kr = s_k[w][r];
                const uint32_t local = p - kr.x;
                const uint32_t nxr = kr.y & 0x7FFFFFFFu;
                uint32_t row, col;
                divmod_small(local, nxr, __uint_as_float(kr.z), row, col);
                const int tx = (int)(kr.w & 0xFFFFu) + (int)col, ty = (int)(kr.w >> 16) + (int)row;
                const float4 g = s_g[w][r], h = s_h[w][r];
                const int4 rc = s_r[w][r];
                if (tile_keep(g.x, g.y, g.z, g.w, h.x, h.y, h.z, h.w, max(tx * B, rc.x),
                              min(tx * B + B - 1, rc.y), max(ty * B, rc.z), min(ty * B + B - 1, rc.w))) {
                    atomicAdd(&s_c[w][r], 1u);
                    if (kr.y & 0x80000000u) atomicOr(&s_m[w][r][local >> 5], 1u << (local & 31u));
                }
            }
        }
        __syncwarp();
        // every record's count is written, 0 for one not visible: the emission reads the counts
        // of all records, and this buffer may hold anything from an earlier use
        if (j < n) ki.cnt[j] = s_c[w][lane];
        if (valid) {
            const uint32_t c = s_c[w][lane];
            ki.km[j] = make_uint2(s_m[w][lane][0], s_m[w][lane][1]);
            ki.rx[j] = rx;
            ki.ry[j] = ry;
            wsum += c;
        }
        __syncwarp();
    }
    uint32_t tot;
    block_excl_scan(wsum, s_warp, &tot);
    if (threadIdx.x == 0) partials[blockIdx.x] = tot;
}

// ---- radix sort -------------------------------------------------------------------------
//
// LSD passes of 8 bits over blocks of kRadixTile items: a histogram pass (per block and
// digit), an exclusive scan of the histograms in digit-major order (the global start of each
// block's run of each digit), and a stable scatter.

__global__ void __launch_bounds__(kRadixThreads)
k_radix_hist(const uint32_t *__restrict__ keys, const uint32_t *n_dev, int64_t n_cap, int shift,
             uint32_t mask, uint32_t *__restrict__ hist, int64_t nblocks) {
    __shared__ uint32_t s_h[kRadixBins];
    s_h[threadIdx.x] = 0u;
    __syncthreads();
    const int64_t n = count_of(n_dev, n_cap);
    const int64_t base = (int64_t)blockIdx.x * kRadixTile;
    if (base + kRadixTile <= n && (reinterpret_cast<uintptr_t>(keys) & 15u) == 0u) {
        // full block of a 16-byte aligned array: 16-byte loads (kRadixTile % 4 == 0)
        const uint4 *k4 = reinterpret_cast<const uint4 *>(keys + base);
#pragma unroll
        for (int r = 0; r < kRadixRounds / 4; r++) {
            const uint4 q = k4[r * kRadixThreads + threadIdx.x];
            atomicAdd(&s_h[(q.x >> shift) & mask], 1u);
            atomicAdd(&s_h[(q.y >> shift) & mask], 1u);
            atomicAdd(&s_h[(q.z >> shift) & mask], 1u);
            atomicAdd(&s_h[(q.w >> shift) & mask], 1u);
        }
    } else {
        for (int r = 0; r < kRadixRounds; r++) {
            const int64_t i = base + (int64_t)r * kRadixThreads + threadIdx.x;
            if (i < n) atomicAdd(&s_h[(keys[i] >> shift) & mask], 1u);
        }
    }
    __syncthreads();
    hist[(int64_t)threadIdx.x * nblocks + blockIdx.x] = s_h[threadIdx.x];
}

// Exclusive scan, in place, of each digit's row of per-block counts (the histogram is
// digit-major: hist[d * nblocks + b]); row d's total goes to hist[256 * nblocks + d], which
// k_digit_starts then turns into the digit's start. One CTA per digit.
__global__ void __launch_bounds__(1024) k_hist_rows(uint32_t *__restrict__ hist, int64_t nblocks) {
    __shared__ uint32_t s_warp[33];
    const int d = blockIdx.x;
    uint32_t *row = hist + (int64_t)d * nblocks;
    uint32_t carry = 0u;
    for (int64_t b0 = 0; b0 < nblocks; b0 += 4 * 1024) {
        const int64_t i = b0 + 4 * (int64_t)threadIdx.x;
        uint32_t v[4], sum = 0u;
#pragma unroll
        for (int k = 0; k < 4; k++) {
            v[k] = i + k < nblocks ? row[i + k] : 0u;
            sum += v[k];
        }
        uint32_t tot;
        uint32_t e = block_excl_scan(sum, s_warp, &tot) + carry;
#pragma unroll
        for (int k = 0; k < 4; k++) {
            if (i + k < nblocks) row[i + k] = e;
            e += v[k];
        }
        carry += tot;
    }
    if (threadIdx.x == 0) hist[(int64_t)kRadixBins * nblocks + d] = carry;
}

__global__ void __launch_bounds__(kRadixBins) k_digit_starts(uint32_t *__restrict__ hist, int64_t nblocks) {
    __shared__ uint32_t s_warp[33];
    uint32_t *tot = hist + (int64_t)kRadixBins * nblocks;
    uint32_t all;
    const uint32_t e = block_excl_scan(tot[threadIdx.x], s_warp, &all);
    tot[threadIdx.x] = e;
}

// Stable scatter of one block of kRadixTile items. Warp w owns the items
// [w * 32 * R, (w + 1) * 32 * R) of the block and ranks them on its own, R rounds of 32 lanes,
// with per-warp digit counters (a warp multisplit: one ballot per digit bit finds the lanes
// holding the same digit). Then one pass over the digits turns the per-warp counts into each
// warp's start within each digit, the items are placed in shared memory in (digit, index)
// order, and written out so that each digit's run of the block goes to consecutive addresses.
// The values are read from global memory only when placed (registers only for keys and ranks,
// no shared-memory copy of the input values: 43 KB of shared memory and at most 64 registers,
// 4 CTAs per SM instead of 3 -- binning 2.28 -> 2.15 ms per step on the 1M x 16-view step).
template <int BITS>
__global__ void __launch_bounds__(kRadixThreads, 4)
k_radix_scatter(const uint32_t *__restrict__ keys_in, const uint32_t *__restrict__ vals_in,
                const uint32_t *n_dev, int64_t n_cap, int shift, uint32_t mask,
                const uint32_t *__restrict__ offsets, int64_t nblocks,
                uint32_t *__restrict__ keys_out, uint32_t *__restrict__ vals_out) {
    constexpr int NW = kRadixThreads / 32, R = kRadixRounds;
    __shared__ uint32_t s_cnt[NW][kRadixBins];  // per-warp digit counts, then per-warp starts
    __shared__ uint32_t s_start[kRadixBins];    // start of each digit in the block's order
    __shared__ uint32_t s_goff[kRadixBins];     // global position of the block's digit run
    __shared__ uint32_t s_warp[33];
    __shared__ uint32_t s_k[kRadixTile], s_v[kRadixTile];
    const int t = threadIdx.x, lane = t & 31, w = t >> 5;
    const unsigned full = 0xffffffffu;
    const int64_t n = count_of(n_dev, n_cap);
    const int64_t base = (int64_t)blockIdx.x * kRadixTile;
    if (base >= n) return;  // uniform across the block
    const int cnt = (int)((n - base) < kRadixTile ? (n - base) : kRadixTile);
#pragma unroll
    for (int q = 0; q < NW; q++) s_cnt[q][t] = 0u;
    // global start of this block's run of digit t: the digit's start + earlier blocks' counts
    s_goff[t] = offsets[(int64_t)kRadixBins * nblocks + t] + offsets[(int64_t)t * nblocks + blockIdx.x];
    __syncthreads();
    uint32_t kr[R], rk[R];
    const uint32_t lt_mask = (1u << lane) - 1u;
    const int wbase = w * 32 * R;
#pragma unroll
    for (int r = 0; r < R; r++) {
        const int j = wbase + r * 32 + lane;
        const bool valid = j < cnt;
        kr[r] = valid ? keys_in[base + j] : 0u;
    }
#pragma unroll
    for (int r = 0; r < R; r++) {
        const int j = wbase + r * 32 + lane;
        const bool valid = j < cnt;
        const uint32_t d = (kr[r] >> shift) & mask;
        uint32_t peers = __ballot_sync(full, valid);
#pragma unroll
        for (int b = 0; b < BITS; b++) {  // one ballot per bit of the digit
            const uint32_t bal = __ballot_sync(full, (d >> b) & 1u);
            peers &= bal ^ (((d >> b) & 1u) - 1u);   // bal where the bit is set, ~bal where not
        }
        const uint32_t before = s_cnt[w][d];
        rk[r] = before + __popc(peers & lt_mask);
        __syncwarp();
        if (valid && (peers & lt_mask) == 0u) s_cnt[w][d] = before + __popc(peers);
        __syncwarp();
    }
    __syncthreads();
    // thread t = digit t: per-warp starts within the digit, and the digit's start in the block
    uint32_t acc = 0u;
#pragma unroll
    for (int q = 0; q < NW; q++) {
        const uint32_t c = s_cnt[q][t];
        s_cnt[q][t] = acc;
        acc += c;
    }
    uint32_t tot;
    s_start[t] = block_excl_scan(acc, s_warp, &tot);
    __syncthreads();
#pragma unroll
    for (int r = 0; r < R; r++) {
        const int j = wbase + r * 32 + lane;
        if (j < cnt) {
            const uint32_t d = (kr[r] >> shift) & mask;
            const uint32_t lp = s_start[d] + s_cnt[w][d] + rk[r];
            s_k[lp] = kr[r];
            // no input values: the items' own positions (the first pass of a sort of indices)
            s_v[lp] = vals_in ? vals_in[base + j] : (uint32_t)(base + j);
        }
    }
    __syncthreads();
    for (int i = t; i < cnt; i += kRadixThreads) {
        const uint32_t k = s_k[i];
        const uint32_t d = (k >> shift) & mask;
        const uint32_t gp = s_goff[d] + ((uint32_t)i - s_start[d]);
        keys_out[gp] = k;
        vals_out[gp] = s_v[i];
    }
}

// ---- keys, ranges -------------------------------------------------------------------------

// Position of the k-th set bit (k from 0) of the 64-bit mask hi:lo; k < popc(mask).
__device__ __forceinline__ int select_bit(uint32_t lo, uint32_t hi, uint32_t k) {
    const uint32_t pl = __popc(lo);
    uint32_t x = lo;
    int b = 0;
    if (k >= pl) {
        x = hi;
        k -= pl;
        b = 32;
    }
    uint32_t c = __popc(x & 0xFFFFu);
    if (k >= c) { k -= c; x >>= 16; b += 16; }
    c = __popc(x & 0xFFu);
    if (k >= c) { k -= c; x >>= 8; b += 8; }
    c = __popc(x & 0xFu);
    if (k >= c) { k -= c; x >>= 4; b += 4; }
    c = __popc(x & 0x3u);
    if (k >= c) { k -= c; x >>= 2; b += 2; }
    if (k >= (x & 1u)) b += 1;
    return b;
}

// Key emission. Block b takes the same kScanTile depth-sorted records as block b of the key
// count, whose keys start at block_off[b]; warp w takes 256 of them, 32 at a time. The keys of
// 32 records form one contiguous segment, which the warp's lanes fill position by position
// (coalesced stores, balanced work): the lane of position p finds its record by binary search
// over the prefix sums, and its tile as the k-th set bit of the record's kept-tile mask.
// Records of more than 64 rect tiles (no mask) are done by the whole warp, 32 tiles at a time.
//
// The work is bounded by the data the count pass scanned, whatever the count buffer holds: a
// block first checks that its records' counts add up to the keys the count pass scanned for
// it (block_off[b + 1] - block_off[b]) and that no record claims more tiles than the batch
// has; otherwise it sets kStatusInconsistent and emits nothing. A warp also stops at the key
// capacity, so a count beyond the capacity costs no more than the capacity.
__global__ void __launch_bounds__(kScanThreads)
k_emit(const uint32_t *__restrict__ sorted_ids, const uint32_t *__restrict__ block_off,
       const uint32_t *n_dev, int64_t n_cap, const KeyInfo ki, const float4 *__restrict__ splats,
       uint32_t n_gauss, uint32_t n_magic, const __grid_constant__ CamBatch cb, uint32_t *__restrict__ tile_keys,
       uint32_t *__restrict__ tile_vals, const uint32_t *K_dev, int64_t key_cap, uint32_t *status) {
    constexpr int NW = kScanThreads / 32;
    __shared__ uint64_t s_wtot[NW];
    __shared__ int s_bad;
    const unsigned full = 0xffffffffu;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (blockIdx.x == 0 && threadIdx.x == 0 && (int64_t)*K_dev > key_cap) atomicOr(status, kStatusCapacity);
    const int64_t n = count_of(n_dev, n_cap);
    const int64_t base = (int64_t)blockIdx.x * kScanTile;
    if (base >= n) return;  // uniform across the block
    const int64_t wbase = base + (int64_t)w * 32 * kScanItems;
    uint64_t wsum = 0u;
    bool bad = false;
#pragma unroll
    for (int q = 0; q < kScanItems; q++) {
        const int64_t j = wbase + q * 32 + lane;
        const uint32_t c = j < n ? ki.cnt[j] : 0u;
        bad = bad || c > (uint32_t)cb.total_tiles;
        wsum += c;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) wsum += __shfl_xor_sync(full, wsum, o);
    bad = __any_sync(full, bad);
    if (lane == 0) s_wtot[w] = bad ? ~(uint64_t)0 : wsum;
    __syncthreads();
    if (threadIdx.x == 0) {
        // the counts must add up to the keys the count pass scanned for this block
        uint64_t sum = 0u;
        bool b = false;
        for (int q = 0; q < NW; q++) {
            b = b || s_wtot[q] == ~(uint64_t)0;
            sum += s_wtot[q];
        }
        const uint64_t end = blockIdx.x + 1 < gridDim.x ? block_off[blockIdx.x + 1] : *K_dev;
        b = b || end < block_off[blockIdx.x] || sum != end - block_off[blockIdx.x];
        if (b) atomicOr(status, kStatusInconsistent);
        s_bad = b ? 1 : 0;
    }
    __syncthreads();
    if (s_bad) return;  // uniform across the block
    int64_t off = (int64_t)block_off[blockIdx.x];
    for (int q = 0; q < w; q++) off += (int64_t)s_wtot[q];
    const int B = cb.tile, lb = __ffs(cb.tile) - 1;
#pragma unroll 1
    for (int q = 0; q < kScanItems; q++) {
        if (off >= key_cap) break;  // uniform across the warp: every later key is beyond capacity
        const int64_t j = wbase + q * 32 + lane;
        const bool valid = j < n;
        const uint32_t cnt = valid ? ki.cnt[j] : 0u;
        const uint32_t inc = warp_incl_scan(cnt, lane);
        const uint32_t excl = inc - cnt;
        const uint32_t total = __shfl_sync(full, inc, 31);
        if (total == 0u) continue;  // uniform
        // the lane's record: view, tile rect and mask
        uint32_t rec = 0u;
        int tx0 = 0, ty0 = 0, nx = 1, gx = 0, gy = 0, toff = 0;
        uint2 m = make_uint2(0u, 0u);
        bool big = false;
        if (cnt > 0u) {
            rec = sorted_ids[j];
            uint32_t v = rec;  // view = rec / n_gauss, by multiplying with ceil(2^32 / n_gauss)
            if (n_magic) {
                v = __umulhi(rec, n_magic);
                if ((uint64_t)v * n_gauss > rec) v--;
            }
            const DevCam &c = cb.c[v];
            gx = c.gx;
            gy = c.gy;
            toff = c.tile_offset;
            const uint32_t rx = ki.rx[j], ry = ki.ry[j];
            tx0 = (int)(rx & 0xFFFFu) >> lb;
            ty0 = (int)(ry & 0xFFFFu) >> lb;
            nx = ((int)(rx >> 16) >> lb) - tx0 + 1;
            const int ny = ((int)(ry >> 16) >> lb) - ty0 + 1;
            big = (int64_t)nx * ny > 64;
            if (!big) m = ki.km[j];
        }
        const float rcp = __frcp_rn((float)nx);
        // records of more than 64 rect tiles: the cull test again, on 32 rect tiles at a time
        uint32_t bigs = __ballot_sync(full, big);
        while (bigs) {
            const int o = __ffs(bigs) - 1;
            bigs &= bigs - 1u;
            const uint32_t r = __shfl_sync(full, rec, o);
            const int txo = __shfl_sync(full, tx0, o), tyo = __shfl_sync(full, ty0, o), nxo = __shfl_sync(full, nx, o);
            const int gxo = __shfl_sync(full, gx, o), gyo = __shfl_sync(full, gy, o), toffo = __shfl_sync(full, toff, o);
            const int64_t k0 = off + __shfl_sync(full, excl, o);
            const float4 *rp = splats + (size_t)kSplatWords / 4 * r;
            const float4 s0 = rp[0], s1 = rp[1], s2 = rp[2], s3 = rp[3];
            const uint32_t rx = __float_as_uint(s2.y), ry = __float_as_uint(s2.z);
            const int ix0 = (int)(rx & 0xFFFFu), ix1 = (int)(rx >> 16);
            const int iy0 = (int)(ry & 0xFFFFu), iy1 = (int)(ry >> 16);
            const int64_t nt = (int64_t)nxo * ((iy1 >> lb) - tyo + 1);
            int64_t kept = 0;
            for (int64_t t0 = 0; t0 < nt; t0 += 32) {
                const int64_t tl = t0 + lane;
                bool keep = false;
                int tx = 0, ty = 0;
                if (tl < nt) {
                    tx = txo + (int)(tl % nxo);
                    ty = tyo + (int)(tl / nxo);
                    keep = tile_keep(s0.x, s0.y, s0.z, s0.w, s1.x, s3.x, s3.y, s3.z, max(tx * B, ix0),
                                     min(tx * B + B - 1, ix1), max(ty * B, iy0), min(ty * B + B - 1, iy1));
                }
                const uint32_t kb = __ballot_sync(full, keep);
                const int64_t k = k0 + kept + __popc(kb & ((1u << lane) - 1u));
                if (keep && k < key_cap) {
                    const bool ok = tx < gxo && ty < gyo;   // records from outside may carry any rect
                    tile_keys[k] = ok ? (uint32_t)(toffo + ty * gxo + tx) : 0xffffffffu;
                    tile_vals[k] = r;
                }
                kept += __popc(kb);
            }
        }
        const uint32_t lim = (int64_t)total < key_cap - off ? total : (uint32_t)(key_cap - off);
        for (uint32_t p0 = 0; p0 < lim; p0 += 32) {
            const uint32_t p = p0 + (uint32_t)lane;
            int o = 0;
#pragma unroll
            for (int step = 16; step >= 1; step >>= 1)
                if (__shfl_sync(full, excl, o + step) <= p) o += step;
            const uint32_t eo = __shfl_sync(full, excl, o);
            const uint32_t mlo = __shfl_sync(full, m.x, o), mhi = __shfl_sync(full, m.y, o);
            const uint32_t nxo = (uint32_t)__shfl_sync(full, nx, o);
            const float rcpo = __shfl_sync(full, rcp, o);
            const int txo = __shfl_sync(full, tx0, o), tyo = __shfl_sync(full, ty0, o);
            const int gxo = __shfl_sync(full, gx, o), gyo = __shfl_sync(full, gy, o);
            const int toffo = __shfl_sync(full, toff, o);
            const uint32_t reco = __shfl_sync(full, rec, o);
            const bool bigo = __shfl_sync(full, big ? 1 : 0, o) != 0;
            const int64_t gp = off + p;
            if (p < total && !bigo && gp < key_cap) {
                uint32_t row, col;
                divmod_small((uint32_t)select_bit(mlo, mhi, p - eo), nxo, rcpo, row, col);
                const int tx = txo + (int)col, ty = tyo + (int)row;
                const bool ok = tx < gxo && ty < gyo;
                tile_keys[gp] = ok ? (uint32_t)(toffo + ty * gxo + tx) : 0xffffffffu;
                tile_vals[gp] = reco;
            }
        }
        off += total;
    }
}
// Ranges of the sorted tile keys: ranges[t] = [first, last + 1) of tile t (untouched tiles
// keep the zeros set before). Each thread looks at 4 consecutive keys and their neighbours.
__global__ void k_ranges(const uint32_t *__restrict__ keys, const uint32_t *K_dev, int64_t cap,
                         uint2 *__restrict__ ranges, uint32_t total_tiles) {
    const int64_t K = count_of(K_dev, cap);
    const int64_t i0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) * 4;
    if (i0 >= K) return;
    uint32_t k[6];
    k[0] = i0 > 0 ? keys[i0 - 1] : 0xffffffffu;
    if (i0 + 4 <= K && (reinterpret_cast<uintptr_t>(keys) & 15u) == 0u) {
        const uint4 q = *reinterpret_cast<const uint4 *>(keys + i0);  // aligned: i0 % 4 == 0
        k[1] = q.x;
        k[2] = q.y;
        k[3] = q.z;
        k[4] = q.w;
    } else {
#pragma unroll
        for (int j = 0; j < 4; j++) k[1 + j] = i0 + j < K ? keys[i0 + j] : 0xffffffffu;
    }
    k[5] = i0 + 4 < K ? keys[i0 + 4] : 0xffffffffu;
#pragma unroll
    for (int j = 0; j < 4; j++) {
        const int64_t i = i0 + j;
        const uint32_t t = k[1 + j];
        if (i >= K || t >= total_tiles) continue;
        if (i == 0 || k[j] != t) ranges[t].x = (uint32_t)i;
        if (i == K - 1 || k[2 + j] != t) ranges[t].y = (uint32_t)(i + 1);
    }
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
    const bool vis = radii[i] > 0;
    if (tt) tt[i] = vis ? 1u : 0u;
    // depth key of every record; the ones not visible sort last
    db[i] = vis ? __float_as_uint(splats[(size_t)kSplatWords / 4 * i + 2].w) : kNoDepth;
}

inline unsigned blocks_for(int64_t n, int bs) { return (unsigned)((n + bs - 1) / bs); }

}  // namespace

size_t scan_partials_needed(int64_t n_items) {
    return (size_t)((n_items + kScanTile - 1) / kScanTile) + 1;
}

size_t radix_hist_needed(int64_t n_items) {  // per-block counts and the 256 digit totals
    return (size_t)kRadixBins * (size_t)((n_items + kRadixTile - 1) / kRadixTile) + kRadixBins;
}

void radix_sort_pairs(uint32_t *&keys, uint32_t *&vals, uint32_t *keys_alt, uint32_t *vals_alt,
                      const uint32_t *n_dev, int64_t n_cap, int begin_bit, int end_bit,
                      uint32_t *hist, uint32_t *partials, cudaStream_t st, bool index_vals) {
    (void)partials;
    const int64_t nb = (n_cap + kRadixTile - 1) / kRadixTile;
    if (nb == 0) return;
    bool first = true;
    for (int bit = begin_bit; bit < end_bit; bit += 8) {
        const int bits = (end_bit - bit) < 8 ? (end_bit - bit) : 8;
        const uint32_t mask = (1u << bits) - 1u;
        count_launch();
        k_radix_hist<<<(unsigned)nb, kRadixThreads, 0, st>>>(keys, n_dev, n_cap, bit, mask, hist, nb);
        count_launch();
        k_hist_rows<<<kRadixBins, 1024, 0, st>>>(hist, nb);
        count_launch();
        k_digit_starts<<<1, kRadixBins, 0, st>>>(hist, nb);
        count_launch();
        const uint32_t *vin = (first && index_vals) ? nullptr : vals;
        if (bits == 8)
            k_radix_scatter<8><<<(unsigned)nb, kRadixThreads, 0, st>>>(keys, vin, n_dev, n_cap, bit, mask, hist, nb,
                                                                       keys_alt, vals_alt);
        else if (bits == 7)
            k_radix_scatter<7><<<(unsigned)nb, kRadixThreads, 0, st>>>(keys, vin, n_dev, n_cap, bit, mask, hist, nb,
                                                                       keys_alt, vals_alt);
        else
            k_radix_scatter<6><<<(unsigned)nb, kRadixThreads, 0, st>>>(keys, vin, n_dev, n_cap, bit, mask, hist, nb,
                                                                       keys_alt, vals_alt);
        first = false;
        uint32_t *tk = keys, *tv = vals;
        keys = keys_alt;
        vals = vals_alt;
        keys_alt = tk;
        vals_alt = tv;
    }
}

void count_keys(const uint32_t *sorted_ids, const uint32_t *sorted_keys, const uint32_t *n_dev, int64_t n_cap,
                const float4 *splats, int tile, const KeyInfo &ki, uint32_t *block_offsets, uint32_t *total,
                cudaStream_t st) {
    const int64_t nb = (n_cap + kScanTile - 1) / kScanTile;
    if (nb == 0) {
        if (total) cudaMemsetAsync(total, 0, sizeof(uint32_t), st);
        return;
    }
    count_launch();
    k_count_keys<<<(unsigned)nb, kScanThreads, 0, st>>>(sorted_ids, sorted_keys, n_dev, n_cap, splats, tile, ki,
                                                        block_offsets);
    count_launch();
    k_scan_partials<<<1, 1024, 0, st>>>(block_offsets, nb, total);
}

void emit_keys(const uint32_t *sorted_ids, const uint32_t *block_offsets, const uint32_t *n_dev, int64_t n_cap,
               const KeyInfo &ki, const float4 *splats, int64_t n_gauss, const CamBatch &cb,
               uint32_t *tile_keys, uint32_t *tile_vals, const uint32_t *K_dev, int64_t key_capacity,
               uint32_t *status, cudaStream_t st) {
    if (n_cap <= 0) return;
    count_launch();
    // ceil(2^32 / n_gauss), 0 for n_gauss = 1 (the view of record r is r / n_gauss)
    const uint32_t n_magic = n_gauss > 1 ? (uint32_t)(0xFFFFFFFFull / (uint64_t)n_gauss + 1ull) : 0u;
    k_emit<<<blocks_for(n_cap, kScanTile), kScanThreads, 0, st>>>(sorted_ids, block_offsets, n_dev, n_cap, ki,
                                                                  splats, (uint32_t)n_gauss, n_magic, cb, tile_keys,
                                                                  tile_vals, K_dev, key_capacity, status);
}

void find_ranges(const uint32_t *tile_keys, const uint32_t *K_dev, int64_t key_capacity, uint2 *ranges,
                 int total_tiles, cudaStream_t st) {
    cudaMemsetAsync(ranges, 0, sizeof(uint2) * (size_t)total_tiles, st);
    if (key_capacity <= 0) return;
    count_launch();
    k_ranges<<<blocks_for((key_capacity + 3) / 4, 256), 256, 0, st>>>(tile_keys, K_dev, key_capacity, ranges,
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
