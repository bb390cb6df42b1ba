// Compaction of the Gaussian arrays: removes the Gaussians a pruning step names -- those whose
// volume mask is 0 (Sec. "Pruning with Volume Masking": masked Gaussians are removed at
// densification steps and every 500 iterations afterwards) and those a significance round
// selects (Eq. significance-score) -- keeping the others in their order.
//
// Three launches: per block of 1024 Gaussians the number kept; one block turns those counts
// into block offsets (and the total); then each warp takes its chunks of 32 Gaussians, ranks
// the kept ones with a ballot and copies their rows. A warp's kept Gaussians land in
// consecutive output rows, so for each array the warp writes one contiguous run, lane e of a
// round taking element e of the run (row e / width via the ballot's (e / width)-th set bit).
#include "tgs_internal.cuh"

namespace tgs {
namespace {

constexpr int kCompactThreads = 256;
constexpr int kCompactItems = 1024;   // Gaussians per block: 8 warps x 4 chunks of 32

__device__ __forceinline__ bool kept(const GaussPtrs &g, const uint8_t *remove, bool masked, int64_t i) {
    if (remove && remove[i]) return false;
    if (masked && g.mask && !(g.mask[i] > g.tau_m)) return false;   // M = 0, the preprocess's test
    return true;
}

__global__ void __launch_bounds__(kCompactThreads)
k_compact_count(GaussPtrs g, const uint8_t *__restrict__ remove, bool masked, uint32_t *__restrict__ block_counts) {
    __shared__ uint32_t s[kCompactThreads / 32];
    const int64_t base = (int64_t)blockIdx.x * kCompactItems;
    uint32_t c = 0;
#pragma unroll
    for (int k = 0; k < kCompactItems / kCompactThreads; k++) {
        const int64_t i = base + k * kCompactThreads + threadIdx.x;
        c += (i < g.n && kept(g, remove, masked, i)) ? 1u : 0u;
    }
    c = __reduce_add_sync(0xffffffffu, c);
    if ((threadIdx.x & 31) == 0) s[threadIdx.x >> 5] = c;
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t t = 0;
        for (int w = 0; w < kCompactThreads / 32; w++) t += s[w];
        block_counts[blockIdx.x] = t;
    }
}

// Exclusive scan of the block counts in place (one block); total -> *total.
__global__ void __launch_bounds__(1024) k_compact_scan(uint32_t *__restrict__ counts, int nb, uint32_t *__restrict__ total) {
    __shared__ uint32_t s[32];
    __shared__ uint32_t carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int b0 = 0; b0 < nb; b0 += 1024) {
        const int i = b0 + threadIdx.x;
        const uint32_t x = i < nb ? counts[i] : 0u;
        uint32_t incl = x;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        if (lane == 31) s[w] = incl;
        __syncthreads();
        if (w == 0) {
            uint32_t v = s[lane], vi = v;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t y = __shfl_up_sync(0xffffffffu, vi, o);
                if (lane >= o) vi += y;
            }
            s[lane] = vi - v;   // exclusive prefix of the warp totals
        }
        __syncthreads();
        const uint32_t c0 = carry;
        if (i < nb) counts[i] = c0 + s[w] + incl - x;
        __syncthreads();
        if (threadIdx.x == 1023) carry = c0 + s[w] + incl;
        __syncthreads();
    }
    if (threadIdx.x == 0) *total = carry;
}

// Position of the r-th (0-based) set bit of m, r < popc(m): binary search on bit counts.
__device__ __forceinline__ int nth_set_bit(uint32_t m, int r) {
    int pos = 0;
#pragma unroll
    for (int s = 16; s > 0; s >>= 1) {
        const int c = __popc(m & ((1u << s) - 1u));
        if (r >= c) {
            r -= c;
            m >>= s;
            pos += s;
        }
    }
    return pos;
}

// Copies the rows of the kept Gaussians of one chunk (kept mask km over items base + lane) of
// an array of `width` values per Gaussian to the contiguous output rows starting at out_row.
template <typename T>
__device__ __forceinline__ void copy_rows(const T *__restrict__ src, T *__restrict__ dst, int width, int64_t base,
                                          uint32_t km, int64_t out_row, int lane) {
    if (!src || !dst) return;
    const int total = __popc(km) * width;
    for (int e = lane; e < total; e += 32) {
        const int r = e / width, c = e - r * width;
        const int src_lane = nth_set_bit(km, r);   // lane of the r-th kept Gaussian
        dst[(out_row + r) * width + c] = src[(base + src_lane) * width + c];
    }
}

__global__ void __launch_bounds__(kCompactThreads)
k_compact_copy(GaussPtrs g, const uint8_t *__restrict__ remove, bool masked, const uint32_t *__restrict__ block_off,
               GradPtrs out, uint8_t *__restrict__ deg_out, uint32_t *__restrict__ kept_index) {
    constexpr int kChunks = kCompactItems / 32;
    __shared__ uint32_t s_mask[kChunks];
    __shared__ uint32_t s_off[kChunks];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t base = (int64_t)blockIdx.x * kCompactItems;
    for (int q = w; q < kChunks; q += kCompactThreads / 32) {
        const int64_t i = base + q * 32 + lane;
        s_mask[q] = __ballot_sync(0xffffffffu, i < g.n && kept(g, remove, masked, i));
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t o = block_off[blockIdx.x];
        for (int q = 0; q < kChunks; q++) {
            s_off[q] = o;
            o += __popc(s_mask[q]);
        }
    }
    __syncthreads();
    for (int q = w; q < kChunks; q += kCompactThreads / 32) {
        const uint32_t km = s_mask[q];
        if (!km) continue;
        const int64_t cb = base + q * 32, row = s_off[q];
        if (kept_index && ((km >> lane) & 1u))
            kept_index[row + __popc(km & ((1u << lane) - 1u))] = (uint32_t)(cb + lane);
        copy_rows(g.means, out.means, 3, cb, km, row, lane);
        copy_rows(g.log_scales, out.log_scales, 3, cb, km, row, lane);
        copy_rows(g.quats, out.quats, 4, cb, km, row, lane);
        copy_rows(g.opac, out.opac, 1, cb, km, row, lane);
        copy_rows(g.sh_dc, out.sh_dc, 3, cb, km, row, lane);
        copy_rows(g.sh_rest, out.sh_rest, 45, cb, km, row, lane);
        copy_rows(g.mask, out.mask, 1, cb, km, row, lane);
        copy_rows(g.shmask, out.shmask, 3, cb, km, row, lane);
        copy_rows(g.sh_degree, deg_out, 1, cb, km, row, lane);
    }
}

// ---- densification: clone and split (3DGS's rule, driven by the 2D-mean gradient statistics) ----
//
// Class of Gaussian i: 0 stays as it is, 1 stays and gets an identical clone, 2 is replaced by two
// children. Decided in float32 exactly as stated: avg = accum / count (IEEE division; count 0 is
// never chosen), chosen = avg >= tau_g, large = max log-scale > tau_ls.
__device__ __forceinline__ int densify_class(const DensifyArgs &d, const float *__restrict__ ls, int64_t i) {
    const int c = d.count[i];
    if (c <= 0) return 0;
    if (!(__fdiv_rn(d.accum[i], (float)c) >= d.tau_g)) return 0;
    const float m = fmaxf(fmaxf(ls[3 * i], ls[3 * i + 1]), ls[3 * i + 2]);
    return m > d.tau_ls ? 2 : 1;
}

__global__ void __launch_bounds__(kCompactThreads)
k_densify_count(GaussPtrs g, DensifyArgs d, uint32_t *__restrict__ block_counts, int64_t nb) {
    __shared__ uint32_t s[3][kCompactThreads / 32];
    const int64_t base = (int64_t)blockIdx.x * kCompactItems;
    uint32_t c[3] = {0u, 0u, 0u};   // not split, clones, splits
#pragma unroll
    for (int k = 0; k < kCompactItems / kCompactThreads; k++) {
        const int64_t i = base + k * kCompactThreads + threadIdx.x;
        if (i >= g.n) continue;
        const int cl = densify_class(d, g.log_scales, i);
        c[0] += cl != 2;
        c[1] += cl == 1;
        c[2] += cl == 2;
    }
#pragma unroll
    for (int r = 0; r < 3; r++) {
        c[r] = __reduce_add_sync(0xffffffffu, c[r]);
        if ((threadIdx.x & 31) == 0) s[r][threadIdx.x >> 5] = c[r];
    }
    __syncthreads();
    if (threadIdx.x < 3) {
        uint32_t t = 0;
        for (int w = 0; w < kCompactThreads / 32; w++) t += s[threadIdx.x][w];
        block_counts[threadIdx.x * (nb + 1) + blockIdx.x] = t;
    }
}

// Rows of the Gaussians of one chunk that a mask names, copied to the contiguous rows starting at
// out_row; every array except means and log-scales when `rest_only`.
__device__ __forceinline__ void copy_all(const GaussPtrs &g, const GradPtrs &out, uint8_t *deg_out, int64_t cb,
                                         uint32_t m, int64_t row, int lane, bool rest_only) {
    if (!rest_only) {
        copy_rows(g.means, out.means, 3, cb, m, row, lane);
        copy_rows(g.log_scales, out.log_scales, 3, cb, m, row, lane);
    }
    copy_rows(g.quats, out.quats, 4, cb, m, row, lane);
    copy_rows(g.opac, out.opac, 1, cb, m, row, lane);
    copy_rows(g.sh_dc, out.sh_dc, 3, cb, m, row, lane);
    copy_rows(g.sh_rest, out.sh_rest, 45, cb, m, row, lane);
    copy_rows(g.mask, out.mask, 1, cb, m, row, lane);
    copy_rows(g.shmask, out.shmask, 3, cb, m, row, lane);
    copy_rows(g.sh_degree, deg_out, 1, cb, m, row, lane);
}

// block_off: the three exclusive scans (rows of nb + 1 words); totals[0..2]: Gaussians not split,
// clones, splits. Regions of the output: [0, n_keep) kept, then the clones, then the first and
// the second children of the split Gaussians.
__global__ void __launch_bounds__(kCompactThreads)
k_densify_copy(GaussPtrs g, DensifyArgs d, const uint32_t *__restrict__ block_off, int64_t nb,
               const uint32_t *__restrict__ totals, GradPtrs out, uint8_t *__restrict__ deg_out,
               uint32_t *__restrict__ src_index) {
    constexpr int kChunks = kCompactItems / 32;
    __shared__ uint32_t s_mask[3][kChunks];
    __shared__ uint32_t s_off[3][kChunks];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t base = (int64_t)blockIdx.x * kCompactItems;
    for (int q = w; q < kChunks; q += kCompactThreads / 32) {
        const int64_t i = base + q * 32 + lane;
        const int cl = i < g.n ? densify_class(d, g.log_scales, i) : -1;
        s_mask[0][q] = __ballot_sync(0xffffffffu, cl == 0 || cl == 1);
        s_mask[1][q] = __ballot_sync(0xffffffffu, cl == 1);
        s_mask[2][q] = __ballot_sync(0xffffffffu, cl == 2);
    }
    __syncthreads();
    if (threadIdx.x < 3) {
        uint32_t o = block_off[threadIdx.x * (nb + 1) + blockIdx.x];
        for (int q = 0; q < kChunks; q++) {
            s_off[threadIdx.x][q] = o;
            o += __popc(s_mask[threadIdx.x][q]);
        }
    }
    __syncthreads();
    const int64_t n_keep = totals[0], n_clone = totals[1], n_split = totals[2];
    const uint32_t below = (1u << lane) - 1u;
    for (int q = w; q < kChunks; q += kCompactThreads / 32) {
        const int64_t cb = base + q * 32;
        const uint32_t mk = s_mask[0][q], mc = s_mask[1][q], ms = s_mask[2][q];
        const int64_t rk = s_off[0][q], rc = n_keep + s_off[1][q];
        const int64_t r1 = n_keep + n_clone + s_off[2][q], r2 = r1 + n_split;
        if (mk) copy_all(g, out, deg_out, cb, mk, rk, lane, false);
        if (mc) copy_all(g, out, deg_out, cb, mc, rc, lane, false);
        if (ms) {
            copy_all(g, out, deg_out, cb, ms, r1, lane, true);
            copy_all(g, out, deg_out, cb, ms, r2, lane, true);
        }
        const uint32_t me = 1u << lane;
        const int64_t i = cb + lane;
        if (src_index) {
            if (mk & me) src_index[rk + __popc(mk & below)] = (uint32_t)i;
            if (mc & me) src_index[rc + __popc(mc & below)] = (uint32_t)i;
            if (ms & me) {
                src_index[r1 + __popc(ms & below)] = (uint32_t)i;
                src_index[r2 + __popc(ms & below)] = (uint32_t)i;
            }
        }
        if (ms & me) {
            // children: mu + R(q / |q|) (exp(l) * z_c), log-scales l - log(1.6)
            const float qw = g.quats[4 * i], qx = g.quats[4 * i + 1], qy = g.quats[4 * i + 2], qz = g.quats[4 * i + 3];
            const float inv = rsqrtf(qw * qw + qx * qx + qy * qy + qz * qz);
            const float w0 = qw * inv, x = qx * inv, y = qy * inv, z = qz * inv;
            const float R[9] = {1.f - 2.f * (y * y + z * z), 2.f * (x * y - w0 * z), 2.f * (x * z + w0 * y),
                                2.f * (x * y + w0 * z), 1.f - 2.f * (x * x + z * z), 2.f * (y * z - w0 * x),
                                2.f * (x * z - w0 * y), 2.f * (y * z + w0 * x), 1.f - 2.f * (x * x + y * y)};
            float sc[3], l[3];
#pragma unroll
            for (int k = 0; k < 3; k++) {
                l[k] = g.log_scales[3 * i + k];
                sc[k] = expf(l[k]);
            }
            const int64_t rows[2] = {r1 + __popc(ms & below), r2 + __popc(ms & below)};
#pragma unroll
            for (int c = 0; c < 2; c++) {
                const float *zc = d.normals + 6 * i + 3 * c;
                const float v[3] = {sc[0] * zc[0], sc[1] * zc[1], sc[2] * zc[2]};
#pragma unroll
                for (int k = 0; k < 3; k++) {
                    if (out.means)
                        out.means[3 * rows[c] + k] = g.means[3 * i + k] + (R[3 * k] * v[0] + R[3 * k + 1] * v[1] + R[3 * k + 2] * v[2]);
                    if (out.log_scales) out.log_scales[3 * rows[c] + k] = l[k] - kLogSplitDivisor;
                }
            }
        }
    }
}

}  // namespace

void launch_densify(const GaussPtrs &g, const DensifyArgs &d, const GradPtrs &out, uint8_t *deg_out,
                    uint32_t *src_index, uint32_t *scratch, uint32_t *totals, bool copy, cudaStream_t st) {
    const int64_t nb = compact_blocks(g.n);
    if (nb <= 0) return;
    if (!copy) {
        count_launch(4);
        k_densify_count<<<(unsigned)nb, kCompactThreads, 0, st>>>(g, d, scratch, nb);
        for (int r = 0; r < 3; r++) k_compact_scan<<<1, 1024, 0, st>>>(scratch + r * (nb + 1), (int)nb, totals + r);
        return;
    }
    count_launch();
    k_densify_copy<<<(unsigned)nb, kCompactThreads, 0, st>>>(g, d, scratch, nb, totals, out, deg_out, src_index);
}

int64_t compact_blocks(int64_t n) { return (n + kCompactItems - 1) / kCompactItems; }

void launch_compact(const GaussPtrs &g, const uint8_t *remove, bool masked, const GradPtrs &out, uint8_t *deg_out,
                    uint32_t *kept_index, uint32_t *block_counts, uint32_t *total, cudaStream_t st) {
    const int64_t nb = compact_blocks(g.n);
    if (nb <= 0) return;
    count_launch(3);
    k_compact_count<<<(unsigned)nb, kCompactThreads, 0, st>>>(g, remove, masked, block_counts);
    k_compact_scan<<<1, 1024, 0, st>>>(block_counts, (int)nb, total);
    k_compact_copy<<<(unsigned)nb, kCompactThreads, 0, st>>>(g, remove, masked, block_counts, out, deg_out,
                                                             kept_index);
}

}  // namespace tgs
