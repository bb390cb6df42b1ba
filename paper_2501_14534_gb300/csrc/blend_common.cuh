// Per-tile forward and backward blending (Eq. 2 of the paper), as device functions shared by
// the one-CTA-per-tile kernels (blend.cu) and the persistent fused kernel (fused.cu).
//
// Pixel layout: each warp owns a compact block of BW x BH pixels of the tile (PPT pixels per
// lane), so that a splat whose pixel rect misses a warp's block is skipped by that warp with
// one warp-uniform test (sub-tile skipping), and a splat that covers the whole block needs no
// per-pixel rect test.
//
// The forward and the backward evaluate each fragment with the same function on the same
// staged values, so their skip decisions (alpha < 1/255, the rect) agree bit for bit.
#pragma once

#include <type_traits>

#include "tgs_internal.cuh"

namespace tgs {

template <int TILE, int PPT>
struct BlendLayout {
    static constexpr int NT = TILE * TILE / PPT;  // threads per CTA
    static constexpr int NW = NT / 32;            // warps per CTA
    static constexpr int BW = (PPT == 4) ? 16 : 8;  // warp block width
    static constexpr int BH = 32 * PPT / BW;        // warp block height
    static constexpr int WX = TILE / BW;            // warp blocks per tile row
    static constexpr int RS = 32 / BW;              // rows covered by one pass of 32 lanes
    static_assert(NT % 32 == 0, "at least one warp");
    static_assert((TILE / BW) * (TILE / BH) == NW, "warp blocks tile the tile");
};

template <int NT>
struct BlendSmem {
    float4 a[NT];     // mean2d x, y; scaled conic A, B
    float4 b[NT];     // scaled conic C; opacity; r, g
    int4 rect[NT];    // inclusive pixel rect x_lo, x_hi, y_lo, y_hi
    uint32_t hit[NT]; // bit w: the rect meets warp w's pixel block
    uint32_t vis[NT]; // bit w: in addition some point of (block x rect) may reach alpha >= 1/255
    float4 d[NT];     // b; qmin = -log2(255 o') (q below it gives alpha < 1/255); cover bits
                      // (bit w: the rect covers warp w's pixel block); splat record index
    int maxlast;
};

// Stage one splat record: conic pre-scaled so that alpha = o * 2^q with
// q = log2(e) * power, power = -1/2 (a dx^2 + c dy^2) - b dx dy.
// Bits of the warp blocks (WX x WY of BW x BH pixels, row-major) of the tile at (tx0, ty0)
// that the inclusive rect [xl, xh] x [yl, yh] meets, and those it covers entirely.
template <int TILE, int PPT>
__device__ __forceinline__ void block_masks(int xl, int xh, int yl, int yh, int tx0, int ty0,
                                            uint32_t &hit, uint32_t &cov) {
    using L = BlendLayout<TILE, PPT>;
    constexpr int WX = L::WX, WY = TILE / L::BH;
    hit = cov = 0u;
    const int x0 = xl - tx0, x1 = xh - tx0, y0 = yl - ty0, y1 = yh - ty0;  // tile-local
    if (x1 < 0 || y1 < 0 || x0 > TILE - 1 || y0 > TILE - 1) return;
    const int cl = max(x0, 0) / L::BW, ch = min(x1, TILE - 1) / L::BW;
    const int rl = max(y0, 0) / L::BH, rh = min(y1, TILE - 1) / L::BH;
    const uint32_t cols = ((1u << (ch - cl + 1)) - 1u) << cl;
    // fully covered columns / rows: block start >= x0 and block end <= x1
    const int ccl = x0 <= 0 ? 0 : (x0 + L::BW - 1) / L::BW;
    const int cch = (x1 + 1) / L::BW - 1;
    const int crl = y0 <= 0 ? 0 : (y0 + L::BH - 1) / L::BH;
    const int crh = (y1 + 1) / L::BH - 1;
    const uint32_t ccols = (cch >= ccl) ? (((1u << (min(cch, WX - 1) - ccl + 1)) - 1u) << ccl) : 0u;
#pragma unroll
    for (int r = 0; r < WY; r++) {
        if (r >= rl && r <= rh) hit |= cols << (r * WX);
        if (r >= crl && r <= crh) cov |= ccols << (r * WX);
    }
}

// With VIS the warps that may see alpha >= 1/255 are found by the cull test below; without,
// the caller stores sm.vis itself.
template <int TILE, int PPT, int NT, bool VIS = true>
__device__ __forceinline__ void stage_splat(BlendSmem<NT> &sm, int slot,
                                            const float4 *__restrict__ splats, uint32_t id,
                                            int tx0, int ty0) {
    const float4 *rp = splats + (size_t)kSplatWords / 4 * id;
    const float4 s0 = __ldg(rp), s1 = __ldg(rp + 1), s2 = __ldg(rp + 2);
    sm.a[slot] = make_float4(s0.x, s0.y, __fmul_rn(-0.5f * kLog2e, s0.z), __fmul_rn(-kLog2e, s0.w));
    sm.b[slot] = make_float4(__fmul_rn(-0.5f * kLog2e, s1.x), s1.y, s1.z, s1.w);
    // o' 2^q < 1/255  <=>  q < -log2(255 o'): the skip test before any exponential
    const float qmin = -log2f(__fmul_rn(255.f, s1.y));
    const uint32_t rx = __float_as_uint(s2.y), ry = __float_as_uint(s2.z);
    const int4 r = make_int4((int)(rx & 0xFFFFu), (int)(rx >> 16), (int)(ry & 0xFFFFu), (int)(ry >> 16));
    sm.rect[slot] = r;
    uint32_t hit, cov;
    block_masks<TILE, PPT>(r.x, r.y, r.z, r.w, tx0, ty0, hit, cov);
    sm.hit[slot] = hit;
    sm.d[slot] = make_float4(s2.x, qmin, __uint_as_float(cov), __uint_as_float(id));
    // warp blocks whose part of the rect stays below alpha = 1/255 everywhere (the cull test of
    // the keys, on the block): those warps skip the splat, whose fragments they would skip
    if (!VIS) return;
    using L = BlendLayout<TILE, PPT>;
    const float4 s3 = __ldg(rp + 3);
    uint32_t vis = hit, bits = hit;
    while (bits) {
        const int w = __ffs(bits) - 1;
        bits &= bits - 1u;
        const int bx0 = tx0 + (w % L::WX) * L::BW, by0 = ty0 + (w / L::WX) * L::BH;
        if (!tile_keep(s0.x, s0.y, s0.z, s0.w, s1.x, s3.x, s3.y, s3.z, max(bx0, r.x),
                       min(bx0 + L::BW - 1, r.y), max(by0, r.z), min(by0 + L::BH - 1, r.w)))
            vis &= ~(1u << w);
    }
    sm.vis[slot] = vis;
}

// Exponent of one fragment, with explicit roundings (no contraction choices left to the
// compiler) so that every kernel computes the same bits.
// A thread's pixels share their column, so dx and A dx are computed once per splat (Adx).
__device__ __forceinline__ float frag_q(float Adx, float Bq, float Cq, float dx, float dy) {
    const float u = __fmaf_rn(Bq, dy, Adx);
    const float w = __fmul_rn(__fmul_rn(Cq, dy), dy);
    return __fmaf_rn(dx, u, w);
}

// Pixels of this thread in tile (tx, ty).
template <int TILE, int PPT>
struct TilePixels {
    int x[PPT], y[PPT];
    float fx[PPT], fy[PPT];
    bool inside[PPT];
    int bx0, bx1, by0, by1;  // the warp's pixel block
    int tx0, ty0;            // the tile's first pixel
    uint32_t wbit;           // this warp's bit in the hit / cover masks

    __device__ __forceinline__ void init(int tx, int ty, int W, int H) {
        using L = BlendLayout<TILE, PPT>;
        const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
        tx0 = tx * TILE;
        ty0 = ty * TILE;
        wbit = 1u << w;
        bx0 = tx * TILE + (w % L::WX) * L::BW;
        by0 = ty * TILE + (w / L::WX) * L::BH;
        bx1 = bx0 + L::BW - 1;
        by1 = by0 + L::BH - 1;
#pragma unroll
        for (int k = 0; k < PPT; k++) {
            x[k] = bx0 + lane % L::BW;
            y[k] = by0 + lane / L::BW + k * L::RS;
            fx[k] = (float)x[k];
            fy[k] = (float)y[k];
            inside[k] = x[k] < W && y[k] < H;
        }
    }
};

// Forward state of this thread's pixels.
template <int PPT>
struct FwdState {
    float T[PPT], Cr[PPT], Cg[PPT], Cb[PPT];
    int last[PPT], exam[PPT];
    int eval[PPT], contrib[PPT];  // with COUNT: fragments evaluated (pixel in rect), contributing
    bool done[PPT];
};

// Front-to-back blend of one tile's list [rg.x, rg.y). On return every pixel holds its
// colour sum, transmittance, last contributor (1-based list position, 0 if none) and the
// number of list entries it examined.
// With HITS every blended fragment counts one ray hit of its Gaussian (Eq.
// significance-score): hits[record - rec_off] += the pixels of the warp that blended it.
template <int TILE, int PPT, bool COUNT = false, bool KEEPVIS = false, bool HITS = false, int SB = 1>
__device__ __forceinline__ void tile_forward(BlendSmem<SB * TILE * TILE / PPT> &sm,
                                             const float4 *__restrict__ splats,
                                             const uint32_t *__restrict__ ids, uint2 rg,
                                             const TilePixels<TILE, PPT> &P, FwdState<PPT> &S,
                                             uint16_t *__restrict__ vis_out = nullptr,
                                             uint32_t *__restrict__ hits = nullptr, uint32_t rec_off = 0) {
    constexpr int NT = TILE * TILE / PPT;
    constexpr int BS = SB * NT;  // splats per shared-memory batch
    const unsigned full = 0xffffffffu;
    const int t = threadIdx.x;
#pragma unroll
    for (int k = 0; k < PPT; k++) {
        S.T[k] = 1.f;
        S.Cr[k] = S.Cg[k] = S.Cb[k] = 0.f;
        S.last[k] = 0;
        S.exam[k] = 0;
        S.eval[k] = S.contrib[k] = 0;
        S.done[k] = !P.inside[k];
    }
    for (uint32_t base = rg.x; base < rg.y; base += BS) {
        bool mine = true;
#pragma unroll
        for (int k = 0; k < PPT; k++) mine = mine && S.done[k];
        if (__syncthreads_count(mine) == NT) break;
#pragma unroll
        for (int sl = t; sl < BS; sl += NT) {
            const uint32_t j = base + sl;
            if (j < rg.y) {
                stage_splat<TILE, PPT>(sm, sl, splats, __ldg(ids + j), P.tx0, P.ty0);
                if (KEEPVIS) vis_out[j] = (uint16_t)sm.vis[sl];  // read back by the backward's staging
            }
        }
        __syncthreads();
        if (__all_sync(full, mine)) continue;  // this warp is finished
        const int cnt = min((uint32_t)BS, rg.y - base);
        const int pos0 = (int)(base - rg.x);
        bool warp_done = false;
        for (int c0 = 0; c0 < cnt && !warp_done; c0 += 32) {
          // the splats of this chunk of 32 that meet this warp's pixel block, in list order
          // with COUNT every fragment in the rect is evaluated (the counters' definition)
          uint32_t bits = __ballot_sync(full, (c0 + (t & 31) < cnt) &&
                                                  ((COUNT ? sm.hit : sm.vis)[c0 + (t & 31)] & P.wbit));
          while (bits) {
            const int m = c0 + __ffs(bits) - 1;
            bits &= bits - 1u;
            const int4 r = sm.rect[m];
            const float4 a = sm.a[m], b = sm.b[m], dd = sm.d[m];
            const bool cover = (__float_as_uint(dd.z) & P.wbit) != 0u;
            const float cbl = dd.x, qmin = dd.y;
            const float dx = a.x - P.fx[0], Adx = __fmul_rn(a.z, dx);  // same column for all PPT
            const bool xin = cover || (unsigned)(P.x[0] - r.x) <= (unsigned)(r.y - r.x);
            uint32_t nb = 0;  // pixels of this thread that blend the splat (HITS)
#pragma unroll
            for (int k = 0; k < PPT; k++) {
                if (S.done[k]) continue;
                if (!cover && !(xin && (unsigned)(P.y[k] - r.z) <= (unsigned)(r.w - r.z))) continue;
                if (COUNT) S.eval[k]++;
                const float dy = a.y - P.fy[k];
                const float q = frag_q(Adx, a.w, b.x, dx, dy);
                if (q > 0.f || q < qmin) continue;   // alpha < 1/255: skipped
                const float alpha = fminf(kAlphaMax, __fmul_rn(b.y, ex2_approx(q)));
                const float tT = __fmul_rn(S.T[k], __fsub_rn(1.f, alpha));
                if (tT < kTMin) {
                    S.done[k] = true;
                    S.exam[k] = pos0 + m + 1;
                    continue;
                }
                if (COUNT) S.contrib[k]++;
                const float w = __fmul_rn(alpha, S.T[k]);
                S.Cr[k] = __fmaf_rn(b.z, w, S.Cr[k]);
                S.Cg[k] = __fmaf_rn(b.w, w, S.Cg[k]);
                S.Cb[k] = __fmaf_rn(cbl, w, S.Cb[k]);
                S.T[k] = tT;
                S.last[k] = pos0 + m + 1;
                if (HITS) nb++;
            }
            if (HITS) {
                const uint32_t tot = __reduce_add_sync(full, nb);
                if ((t & 31) == 0 && tot) atomicAdd(hits + (__float_as_uint(dd.w) - rec_off), tot);
            }
          }
          // checked once per chunk: a warp whose pixels all stopped leaves the list
          bool all = true;
#pragma unroll
          for (int k = 0; k < PPT; k++) all = all && S.done[k];
          warp_done = __all_sync(full, all);
        }
    }
    const int len = (int)(rg.y - rg.x);
#pragma unroll
    for (int k = 0; k < PPT; k++)
        if (P.inside[k] && S.exam[k] == 0) S.exam[k] = len;   // never stopped: saw the whole list
}

// Sums v[0..7] over the warp; afterwards lanes with (lane & 3) == 0 hold the total of
// value (lane >> 2). Four levels of halving exchange instead of eight full butterflies.
__device__ __forceinline__ void warp_transpose_reduce8(float v[8], int lane) {
    const unsigned full = 0xffffffffu;
    {
        const bool up = lane & 16;
#pragma unroll
        for (int i = 0; i < 4; i++) {
            const float send = up ? v[i] : v[i + 4];
            const float keep = up ? v[i + 4] : v[i];
            v[i] = keep + __shfl_xor_sync(full, send, 16);
        }
    }
    {
        const bool up = lane & 8;
#pragma unroll
        for (int i = 0; i < 2; i++) {
            const float send = up ? v[i] : v[i + 2];
            const float keep = up ? v[i + 2] : v[i];
            v[i] = keep + __shfl_xor_sync(full, send, 8);
        }
    }
    {
        const bool up = lane & 4;
        const float send = up ? v[0] : v[1];
        const float keep = up ? v[1] : v[0];
        v[0] = keep + __shfl_xor_sync(full, send, 4);
    }
    v[0] += __shfl_xor_sync(full, v[0], 2);
    v[0] += __shfl_xor_sync(full, v[0], 1);
}

__device__ __forceinline__ float warp_sum(float x) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    return x;
}

// What the backward needs per pixel.
template <int PPT>
struct BwdInput {
    int last[PPT];   // 1-based list position of the last contributor, 0 = none
    float Tfin[PPT]; // final transmittance
    float dR[PPT], dG[PPT], dB[PPT];  // dL/d pixel colour
};

// Reverse walk of one tile's list from each pixel's last contributor. The transmittance in
// front of fragment i is recovered as T_i = T_{i+1} / (1 - a_i) from T_final; of the colour
// behind fragment i only its dot product with dL/dC is needed, and it is accumulated from the
// back. Per fragment the gradients of the pixels of a warp are summed (transposed reduction)
// and added with atomics into the splat gradient record: dL/d mean2d (2), dL/d conic a, b, c,
// dL/d opacity, dL/d rgb (3). With MOMENTS the record receives instead the pixel sums that
// these are linear in -- sum u dx, sum u dy, sum u dx^2, sum u dx dy, sum u dy^2 (u = dL/dG'
// for the unclamped fragments, dx, dy = mean2d - pixel) -- then dL/d opacity = sum u and
// dL/d rgb, and the consumer applies the splat's conic and opacity (see splat_grads in
// preprocess.cu): that takes the per-fragment conversion out of the loop.
// At most this many contributing lanes: each adds its own sums with vector atomics instead of
// a warp reduction. The atomics are fire-and-forget work for the L2; the reduction costs
// ~45 issue slots of a kernel bound by issue. Swept on the benchmark step (fused kernel, ms):
// never 6.70, 8 lanes 6.60, 16 6.48, 24 6.39, 28 6.37, 31 6.36, always 9.39 (same-address
// contention of full warps).
constexpr int kDirectLanes = 28;

template <int TILE, int PPT, bool MOMENTS = false, bool KEEPVIS = false, int SB = 1>
__device__ __forceinline__ void tile_backward(BlendSmem<SB * TILE * TILE / PPT> &sm,
                                              const float4 *__restrict__ splats,
                                              const uint32_t *__restrict__ ids, uint2 rg,
                                              const TilePixels<TILE, PPT> &P, const BwdInput<PPT> &in,
                                              float bg0, float bg1, float bg2,
                                              float *__restrict__ sgrads,
                                              const uint16_t *__restrict__ vis_in = nullptr) {
    constexpr int NT = TILE * TILE / PPT;
    constexpr int BS = SB * NT;  // splats per shared-memory batch
    const unsigned full = 0xffffffffu;
    const int t = threadIdx.x, lane = t & 31;
    // acd = (colour of the fragments behind the current one, blended among themselves) . dL/dC
    float T[PPT], acd[PPT], tbg[PPT];
    int mymax = 0;
#pragma unroll
    for (int k = 0; k < PPT; k++) {
        T[k] = in.Tfin[k];
        acd[k] = 0.f;
        tbg[k] = in.Tfin[k] * (bg0 * in.dR[k] + bg1 * in.dG[k] + bg2 * in.dB[k]);
        mymax = max(mymax, in.last[k]);
    }
    const int wmax = __reduce_max_sync(full, mymax);
    __syncthreads();  // smem of a previous use is free
    if (t == 0) sm.maxlast = 0;
    __syncthreads();
    if (lane == 0) atomicMax(&sm.maxlast, wmax);
    __syncthreads();
    const uint32_t end = min(rg.y, rg.x + (uint32_t)sm.maxlast);

    for (uint32_t bend = end; bend > rg.x;) {
        const uint32_t bstart = (bend - rg.x > (uint32_t)BS) ? bend - BS : rg.x;
        const int cnt = (int)(bend - bstart);
        __syncthreads();
#pragma unroll
        for (int sl = t; sl < BS; sl += NT) {
            if (sl < cnt) {  // slot sl holds list position bend-1-sl
                stage_splat<TILE, PPT, BS, !KEEPVIS>(sm, sl, splats, __ldg(ids + bend - 1 - sl), P.tx0, P.ty0);
                if (KEEPVIS) sm.vis[sl] = vis_in[bend - 1 - sl];  // as the forward's staging found it
            }
        }
        __syncthreads();
        const int top = (int)(bend - rg.x);   // 1-based position of slot 0
        const int m0 = max(0, top - wmax);    // positions beyond this warp's last contributors
        for (int c0 = (m0 / 32) * 32; c0 < cnt; c0 += 32) {
          const int mi = c0 + lane;
          uint32_t bits = __ballot_sync(full, mi >= m0 && mi < cnt && (sm.vis[mi] & P.wbit));
          while (bits) {
            const int m = c0 + __ffs(bits) - 1;
            bits &= bits - 1u;
            const int pos = top - m;
            const int4 r = sm.rect[m];
            const float4 a = sm.a[m], b = sm.b[m], dd = sm.d[m];
            const bool cover = (__float_as_uint(dd.z) & P.wbit) != 0u;
            const float cbl = dd.x, qmin = dd.y;
            const float dx = a.x - P.fx[0], Adx = __fmul_rn(a.z, dx);  // same column for all PPT
            const bool xin = cover || (unsigned)(P.x[0] - r.x) <= (unsigned)(r.y - r.x);
            // per-warp sums over the pixels of u = dL/da G (for the unclamped fragments):
            // g[0] = sum u dx, g[1] = sum u dy, g[2] = sum u dx^2, g[3] = sum u dx dy,
            // g[4] = sum u dy^2, g[5] = sum u, g[6..8] = dL/d rgb; turned into the gradients
            // of mean2d, conic and opacity after the reduction
            float g[9];
#pragma unroll
            for (int e = 0; e < 9; e++) g[e] = 0.f;
            bool contrib = false;
#pragma unroll
            for (int k = 0; k < PPT; k++) {
                if (pos > in.last[k]) continue;
                if (!cover && !(xin && (unsigned)(P.y[k] - r.z) <= (unsigned)(r.w - r.z))) continue;
                const float dy = a.y - P.fy[k];
                const float q = frag_q(Adx, a.w, b.x, dx, dy);
                if (q > 0.f || q < qmin) continue;   // skipped in the forward too
                const float G = ex2_approx(q);
                const float x = __fmul_rn(b.y, G);
                const float alpha = fminf(kAlphaMax, x);
                contrib = true;
                const float inv = __fdividef(1.f, 1.f - alpha);
                T[k] *= inv;                         // transmittance in front of this fragment
                const float w = alpha * T[k];
                g[6] = fmaf(w, in.dR[k], g[6]);
                g[7] = fmaf(w, in.dG[k], g[7]);
                g[8] = fmaf(w, in.dB[k], g[8]);
                // dC/da = T (c - acc) - T_final / (1 - a) bg, acc = colour behind this fragment
                const float cd = fmaf(cbl, in.dB[k], fmaf(b.w, in.dG[k], b.z * in.dR[k]));
                const float diff = cd - acd[k];
                const float dLda = fmaf(diff, T[k], -tbg[k] * inv);
                acd[k] = fmaf(alpha, diff, acd[k]);   // now includes this fragment
                if (x <= kAlphaMax) {
                    // the pixels of a thread share dx: sum u, u dy, u dy^2 here and apply dx
                    // once below (g[0] = dx sum u, g[2] = dx^2 sum u, g[3] = dx sum u dy)
                    const float u = dLda * G;
                    const float uy = u * dy;
                    g[5] += u;
                    g[1] += uy;
                    g[4] = fmaf(uy, dy, g[4]);
                }
            }
            const uint32_t cmask = __ballot_sync(full, contrib);
            if (cmask == 0u) continue;
            g[0] = g[5] * dx;
            g[2] = g[0] * dx;
            g[3] = g[1] * dx;
            float *dst = sgrads + 12 * (size_t)__float_as_uint(dd.w);
            if (__popc(cmask) <= kDirectLanes) {
                // not nearly the whole warp: each contributing lane adds its own sums (converted
                // to the splat gradients first unless MOMENTS), no warp reduction
                if (contrib) {
                    if (!MOMENTS) {
                        const float o = b.y, on = o * kLn2;
                        const float gmx = on * fmaf(2.f * a.z, g[0], a.w * g[1]);
                        const float gmy = on * fmaf(2.f * b.x, g[1], a.w * g[0]);
                        g[0] = gmx;
                        g[1] = gmy;
                        g[2] *= -0.5f * o;
                        g[3] *= -o;
                        g[4] *= -0.5f * o;
                    }
                    atomicAdd(reinterpret_cast<float4 *>(dst), make_float4(g[0], g[1], g[2], g[3]));
                    atomicAdd(reinterpret_cast<float4 *>(dst + 4), make_float4(g[4], g[5], g[6], g[7]));
                    atomicAdd(dst + 8, g[8]);
                }
                continue;
            }
            warp_transpose_reduce8(g, lane);
            const float gb = warp_sum(g[8]);
            if (MOMENTS) {
                // lane 4j holds the total of value j: one reduction of 8 lanes, one of 1
                if ((lane & 3) == 0) atomicAdd(dst + (lane >> 2), g[0]);
                if (lane == 0) atomicAdd(dst + 8, gb);
                continue;
            }
            // lane 4j holds the total of value j. dL/dpower = o' u; with the scaled conic
            // -a dx - b dy = ln2 (2A dx + B dy), -c dy - b dx = ln2 (2C dy + B dx)
            const int j = lane >> 2;
            const float Sx = __shfl_sync(full, g[0], 0), Sy = __shfl_sync(full, g[0], 4);
            const float o = b.y;
            // branch-free per lane: j = 0, 1 mean2d; 2, 3, 4 conic; 5 opacity; 6, 7 rgb
            const float lin = (j == 0) ? fmaf(2.f * a.z, Sx, a.w * Sy) : fmaf(2.f * b.x, Sy, a.w * Sx);
            const float sc = (j < 2) ? o * kLn2 : ((j == 3) ? -o : ((j == 2 || j == 4) ? -0.5f * o : 1.f));
            const float val = sc * ((j < 2) ? lin : g[0]);
            // lanes 0 and 16 collect values 0..3 and 4..7; three 16-byte atomics per splat
            const float v1 = __shfl_down_sync(full, val, 4), v2 = __shfl_down_sync(full, val, 8),
                        v3 = __shfl_down_sync(full, val, 12);
            if ((lane & 15) == 0)
                atomicAdd(reinterpret_cast<float4 *>(dst + (lane >> 2)), make_float4(val, v1, v2, v3));
            if (lane == 0) atomicAdd(dst + 8, gb);
          }
        }
        bend = bstart;
    }
}

// ---- packed pairs (2 pixels per thread) ----------------------------------------------------
//
// A thread's two pixels share their column (rows y and y + RS), so every splat operand is the
// same for both: their arithmetic runs as fma/mul/add/sub.rn.f32x2 on (pixel 0, pixel 1) pairs.
// Each half of a packed instruction is the IEEE operation the scalar code applies to that pixel,
// in the same order, so images, transmittances and every blend decision are bit-identical to
// the scalar path; the floating-point instructions issued halve. The staged splat scalars are
// stored pre-duplicated as pairs, so one 16-byte shared load yields two ready pair operands.

typedef unsigned long long f2_t;  // two floats (pixel 0, pixel 1) in one 64-bit register pair

__device__ __forceinline__ f2_t f2(float lo, float hi) {
    f2_t r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}
__device__ __forceinline__ void f2get(f2_t a, float &lo, float &hi) {
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(a));
}
__device__ __forceinline__ f2_t add2(f2_t a, f2_t b) {
    f2_t r;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ f2_t sub2(f2_t a, f2_t b) {
    f2_t r;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ f2_t mul2(f2_t a, f2_t b) {
    f2_t r;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ f2_t fma2(f2_t a, f2_t b, f2_t c) {  // a * b + c
    f2_t r;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
    return r;
}
__device__ __forceinline__ float sum2(f2_t a) {
    float lo, hi;
    f2get(a, lo, hi);
    return lo + hi;
}

template <int NT>
struct BlendSmem2 {
    ulonglong2 p0[NT];  // (mx, mx), (my, my)
    ulonglong2 p1[NT];  // (A, A), (B, B): the conic scaled as in stage_splat
    ulonglong2 p2[NT];  // (C, C), (o, o)
    ulonglong2 p3[NT];  // (r, r), (g, g)
    float4 p4[NT];      // b, b, qmin, cover bits
    int4 rect[NT];      // inclusive pixel rect x_lo, x_hi, y_lo, y_hi
    uint32_t hit[NT], vis[NT], id[NT];
    int maxlast;
};

// The values of stage_splat, stored as pairs.
template <int TILE, int NT, bool VIS = true>
__device__ __forceinline__ void stage_splat2(BlendSmem2<NT> &sm, int slot, const float4 *__restrict__ splats,
                                             uint32_t id, int tx0, int ty0) {
    constexpr int PPT = 2;
    const float4 *rp = splats + (size_t)kSplatWords / 4 * id;
    const float4 s0 = __ldg(rp), s1 = __ldg(rp + 1), s2 = __ldg(rp + 2);
    const float A = __fmul_rn(-0.5f * kLog2e, s0.z), B = __fmul_rn(-kLog2e, s0.w);
    const float Cq = __fmul_rn(-0.5f * kLog2e, s1.x);
    sm.p0[slot] = make_ulonglong2(f2(s0.x, s0.x), f2(s0.y, s0.y));
    sm.p1[slot] = make_ulonglong2(f2(A, A), f2(B, B));
    sm.p2[slot] = make_ulonglong2(f2(Cq, Cq), f2(s1.y, s1.y));
    sm.p3[slot] = make_ulonglong2(f2(s1.z, s1.z), f2(s1.w, s1.w));
    const float qmin = -log2f(__fmul_rn(255.f, s1.y));
    const uint32_t rx = __float_as_uint(s2.y), ry = __float_as_uint(s2.z);
    const int4 r = make_int4((int)(rx & 0xFFFFu), (int)(rx >> 16), (int)(ry & 0xFFFFu), (int)(ry >> 16));
    sm.rect[slot] = r;
    uint32_t hit, cov;
    block_masks<TILE, PPT>(r.x, r.y, r.z, r.w, tx0, ty0, hit, cov);
    sm.hit[slot] = hit;
    sm.p4[slot] = make_float4(s2.x, s2.x, qmin, __uint_as_float(cov));
    sm.id[slot] = id;
    if (!VIS) return;
    using L = BlendLayout<TILE, PPT>;
    const float4 s3 = __ldg(rp + 3);
    uint32_t vis = hit, bits = hit;
    while (bits) {
        const int w = __ffs(bits) - 1;
        bits &= bits - 1u;
        const int bx0 = tx0 + (w % L::WX) * L::BW, by0 = ty0 + (w / L::WX) * L::BH;
        if (!tile_keep(s0.x, s0.y, s0.z, s0.w, s1.x, s3.x, s3.y, s3.z, max(bx0, r.x),
                       min(bx0 + L::BW - 1, r.y), max(by0, r.z), min(by0 + L::BH - 1, r.w)))
            vis &= ~(1u << w);
    }
    sm.vis[slot] = vis;
}

// tile_forward for 2 pixels per thread with packed pairs (no per-pixel counters).
template <int TILE, bool KEEPVIS = false, bool HITS = false, int SB = 1>
__device__ __forceinline__ void tile_forward2(BlendSmem2<SB * TILE * TILE / 2> &sm, const float4 *__restrict__ splats,
                                              const uint32_t *__restrict__ ids, uint2 rg,
                                              const TilePixels<TILE, 2> &P, FwdState<2> &S,
                                              uint16_t *__restrict__ vis_out = nullptr,
                                              uint32_t *__restrict__ hits = nullptr, uint32_t rec_off = 0) {
    constexpr int NT = TILE * TILE / 2;
    constexpr int BS = SB * NT;  // splats per shared-memory batch
    const unsigned full = 0xffffffffu;
    const int t = threadIdx.x;
    const f2_t one2 = f2(1.f, 1.f);
    const f2_t fx2 = f2(P.fx[0], P.fx[0]);  // same column
    const f2_t fy2 = f2(P.fy[0], P.fy[1]);
    f2_t T2 = one2, Cr2 = f2(0.f, 0.f), Cg2 = Cr2, Cb2 = Cr2;
    int last0 = 0, last1 = 0, exam0 = 0, exam1 = 0;
    bool done0 = !P.inside[0], done1 = !P.inside[1];
    for (uint32_t base = rg.x; base < rg.y; base += BS) {
        const bool mine = done0 && done1;
        if (__syncthreads_count(mine) == NT) break;
#pragma unroll
        for (int sl = t; sl < BS; sl += NT) {
            const uint32_t j = base + sl;
            if (j < rg.y) {
                stage_splat2<TILE, BS>(sm, sl, splats, __ldg(ids + j), P.tx0, P.ty0);
                if (KEEPVIS) vis_out[j] = (uint16_t)sm.vis[sl];  // read back by the backward's staging
            }
        }
        __syncthreads();
        if (__all_sync(full, mine)) continue;  // this warp is finished
        const int cnt = min((uint32_t)BS, rg.y - base);
        const int pos0 = (int)(base - rg.x);
        bool warp_done = false;
        for (int c0 = 0; c0 < cnt && !warp_done; c0 += 32) {
            uint32_t bits = __ballot_sync(full, (c0 + (t & 31) < cnt) && (sm.vis[c0 + (t & 31)] & P.wbit));
            while (bits) {
                const int m = c0 + __ffs(bits) - 1;
                bits &= bits - 1u;
                const int4 r = sm.rect[m];
                const float4 p4 = sm.p4[m];
                const bool cover = (__float_as_uint(p4.w) & P.wbit) != 0u;
                const bool xin = cover || (unsigned)(P.x[0] - r.x) <= (unsigned)(r.y - r.x);
                const bool in0 = !done0 && (cover || (xin && (unsigned)(P.y[0] - r.z) <= (unsigned)(r.w - r.z)));
                const bool in1 = !done1 && (cover || (xin && (unsigned)(P.y[1] - r.z) <= (unsigned)(r.w - r.z)));
                bool b0 = false, b1 = false;  // the pixels that blend this fragment
                if (in0 || in1) {
                    const ulonglong2 a = sm.p0[m], b = sm.p1[m], c = sm.p2[m];
                    const f2_t dx2 = sub2(a.x, fx2);
                    const f2_t dy2 = sub2(a.y, fy2);
                    const f2_t q2 = fma2(dx2, fma2(b.y, dy2, mul2(b.x, dx2)), mul2(mul2(c.x, dy2), dy2));
                    float qa, qb;
                    f2get(q2, qa, qb);
                    const float qmin = p4.z;
                    const bool v0 = in0 && !(qa > 0.f || qa < qmin);  // alpha >= 1/255
                    const bool v1 = in1 && !(qb > 0.f || qb < qmin);
                    if (v0 || v1) {
                        float xa, xb;
                        f2get(mul2(c.y, f2(ex2_approx(qa), ex2_approx(qb))), xa, xb);
                        const f2_t al2 = f2(v0 ? fminf(kAlphaMax, xa) : 0.f, v1 ? fminf(kAlphaMax, xb) : 0.f);
                        const f2_t tT2 = mul2(T2, sub2(one2, al2));
                        float ta, tb;
                        f2get(tT2, ta, tb);
                        const bool s0 = v0 && ta < kTMin, s1 = v1 && tb < kTMin;  // stop before this fragment
                        b0 = v0 && !s0;
                        b1 = v1 && !s1;
                        const int pos = pos0 + m + 1;
                        if (s0) {
                            done0 = true;
                            exam0 = pos;
                        }
                        if (s1) {
                            done1 = true;
                            exam1 = pos;
                        }
                        if (b0 || b1) {
                            float wa, wb, Ta, Tb;
                            f2get(mul2(al2, T2), wa, wb);
                            const f2_t w2 = f2(b0 ? wa : 0.f, b1 ? wb : 0.f);
                            const ulonglong2 col = sm.p3[m];
                            Cr2 = fma2(col.x, w2, Cr2);
                            Cg2 = fma2(col.y, w2, Cg2);
                            Cb2 = fma2(f2(p4.x, p4.y), w2, Cb2);
                            f2get(T2, Ta, Tb);
                            T2 = f2(b0 ? ta : Ta, b1 ? tb : Tb);
                            if (b0) last0 = pos;
                            if (b1) last1 = pos;
                        }
                    }
                }
                if (HITS) {
                    const uint32_t tot = __reduce_add_sync(full, (uint32_t)b0 + (uint32_t)b1);
                    if ((t & 31) == 0 && tot) atomicAdd(hits + (sm.id[m] - rec_off), tot);
                }
            }
            warp_done = __all_sync(full, done0 && done1);
        }
    }
    const int len = (int)(rg.y - rg.x);
    f2get(T2, S.T[0], S.T[1]);
    f2get(Cr2, S.Cr[0], S.Cr[1]);
    f2get(Cg2, S.Cg[0], S.Cg[1]);
    f2get(Cb2, S.Cb[0], S.Cb[1]);
    S.last[0] = last0;
    S.last[1] = last1;
    S.exam[0] = (P.inside[0] && exam0 == 0) ? len : exam0;  // never stopped: saw the whole list
    S.exam[1] = (P.inside[1] && exam1 == 0) ? len : exam1;
    S.done[0] = done0;
    S.done[1] = done1;
    S.eval[0] = S.eval[1] = S.contrib[0] = S.contrib[1] = 0;
}

// Shared memory of a forward blend: the packed layout for 2 pixels per thread (without per-pixel
// counters), the scalar one otherwise. The backward always stages the scalar layout: with its
// chain of per-pixel decisions the pairs do not pay (measured: 4.98 ms scalar, 5.12 ms packed,
// 5.36 ms packed exponents only, per batched step at tile 32), while the packed forward does
// (2.98 -> 2.75 ms).
template <int TILE, int PPT, bool COUNT = false>
using BlendSmemFor = typename std::conditional<PPT == 2 && !COUNT, BlendSmem2<TILE * TILE / 2>,
                                               BlendSmem<TILE * TILE / PPT>>::type;

// The fused kernel's shared memory: the forward's layout, then the backward's in the same space.
template <int TILE, int PPT, int SB = 1>
union FusedSmem {
    typename std::conditional<PPT == 2, BlendSmem2<SB * TILE * TILE / 2>, BlendSmem<SB * TILE * TILE / PPT>>::type f;
    BlendSmem<SB * TILE * TILE / PPT> b;
};

}  // namespace tgs
