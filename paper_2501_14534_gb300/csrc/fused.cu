// Persistent fused forward + L1 loss + backward over (view, tile) work items.
//
// The batched training step renders many views of any sizes with one launch: a grid of
// (SM count x resident CTAs per SM) CTAs takes work items -- one (view, tile) each -- from an
// atomic counter, heaviest first, and for each item runs the forward blend, the L1 loss and
// its gradient (pixel-local, so it needs nothing from other tiles), and the backward blend,
// keeping every pixel's state in registers between the two passes.
//
// Heaviest first: items are ordered by a log-scale key of their list length (8 buckets per
// doubling), descending, with one stable 8-bit radix pass; ties keep tile order.
#include <mutex>

#include "blend_common.cuh"

namespace tgs {
namespace {

__global__ void k_item_keys(const uint2 *__restrict__ ranges, int n, uint32_t *__restrict__ keys,
                            uint32_t *__restrict__ vals) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const uint2 r = ranges[i];
    const uint32_t len = r.y - r.x;
    uint32_t key = 255u;  // empty tiles last
    if (len > 0u) {
        const int e = 31 - __clz(len);                      // floor(log2 len)
        const uint32_t frac = e >= 3 ? (len >> (e - 3)) & 7u : (len << (3 - e)) & 7u;
        const uint32_t lg8 = min(254u, (uint32_t)(e * 8) + frac);
        key = 254u - lg8;                                   // descending length
    }
    keys[i] = key;
    vals[i] = (uint32_t)i;
}

template <int TILE, int PPT, bool HITS, int SB>
__global__ void __launch_bounds__(TILE * TILE / PPT)
k_fused_l1(const float4 *__restrict__ splats, const uint32_t *__restrict__ ids,
           const uint2 *__restrict__ ranges, const uint32_t *__restrict__ order, int n_items,
           int *__restrict__ counter, const __grid_constant__ CamBatch cb,
           const __grid_constant__ PixPtrs px, float bg0, float bg1, float bg2,
           float *__restrict__ sgrads, float *__restrict__ loss, uint16_t *__restrict__ vis_keys,
           uint32_t *__restrict__ hits, uint32_t n_gauss) {
    constexpr int NT = TILE * TILE / PPT;
    constexpr int NW = NT / 32;
    static_assert(NW <= 16, "the per-key warp masks are 16 bits");
    extern __shared__ __align__(16) unsigned char s_dyn[];  // FusedSmem<TILE, PPT, SB>
    FusedSmem<TILE, PPT, SB> &sm = *reinterpret_cast<FusedSmem<TILE, PPT, SB> *>(s_dyn);
    __shared__ int s_item;
    __shared__ float s_loss[NW];
    const int t = threadIdx.x, lane = t & 31, w = t >> 5;
    for (;;) {
        __syncthreads();
        if (t == 0) s_item = atomicAdd(counter, 1);
        __syncthreads();
        const int it = s_item;
        if (it >= n_items) break;
        const int gt = (int)order[it];
        const int v = view_of_tile(cb, gt);
        const DevCam &cam = cb.c[v];
        const int lt = gt - cam.tile_offset;
        TilePixels<TILE, PPT> P;
        P.init(lt % cam.gx, lt / cam.gx, cam.W, cam.H);
        const uint2 rg = ranges[gt];
        FwdState<PPT> S;
        if constexpr (PPT == 2)
            tile_forward2<TILE, true, HITS, SB>(sm.f, splats, ids, rg, P, S, vis_keys, hits, (uint32_t)v * n_gauss);
        else
            tile_forward<TILE, PPT, false, true, HITS, SB>(sm.f, splats, ids, rg, P, S, vis_keys, hits,
                                                           (uint32_t)v * n_gauss);

        // L1 loss: L = mean over views of mean over 3HW |C - target|; dL/dC = sign / (3HWV)
        const int HW = cam.W * cam.H;
        const float scale = 1.f / (3.f * (float)HW * (float)cb.V);
        const float *tg = px.target[v];
        float *img = px.image[v];
        BwdInput<PPT> in;
        float lsum = 0.f;
#pragma unroll
        for (int k = 0; k < PPT; k++) {
            in.last[k] = S.last[k];
            in.Tfin[k] = S.T[k];
            in.dR[k] = in.dG[k] = in.dB[k] = 0.f;
            if (!P.inside[k]) continue;
            const int pix = P.y[k] * cam.W + P.x[k];
            const float cr = S.Cr[k] + S.T[k] * bg0;
            const float cg = S.Cg[k] + S.T[k] * bg1;
            const float cbv = S.Cb[k] + S.T[k] * bg2;
            if (img) {
                img[pix] = cr;
                img[HW + pix] = cg;
                img[2 * HW + pix] = cbv;
            }
            const float er = cr - tg[pix], eg = cg - tg[HW + pix], eb = cbv - tg[2 * HW + pix];
            lsum += fabsf(er) + fabsf(eg) + fabsf(eb);
            in.dR[k] = er > 0.f ? scale : (er < 0.f ? -scale : 0.f);
            in.dG[k] = eg > 0.f ? scale : (eg < 0.f ? -scale : 0.f);
            in.dB[k] = eb > 0.f ? scale : (eb < 0.f ? -scale : 0.f);
        }
        lsum = warp_sum(lsum);
        if (lane == 0) s_loss[w] = lsum;
        tile_backward<TILE, PPT, true, true, SB>(sm.b, splats, ids, rg, P, in, bg0, bg1, bg2, sgrads, vis_keys);
        // s_loss was written before the barriers inside tile_backward
        if (t == 0 && loss) {
            float x = 0.f;
#pragma unroll
            for (int q = 0; q < NW; q++) x += s_loss[q];
            atomicAdd(loss, x * scale);
        }
    }
}

// ---- warp items: one 8 x 8 pixel block of a 32 x 32 tile per warp ------------------------
//
// At 32 x 32 tiles and 2 pixels per thread the 16 warps of a tile share nothing but the tile's
// list, yet in k_fused_l1 they pass the forward, the loss and the backward in step: each phase
// lasts as long as the tile's busiest warp, and near its end a scheduler has too few warps left
// to issue every cycle. Here every warp takes one (view, tile, 8 x 8 block) item of its own from
// the counter and walks the tile's list on its own, 32 entries at a time: it loads the 32
// records, keeps those whose rect meets its block and that may reach alpha >= 1/255 there (the
// per-warp-block bits of block_masks and stage_splat, for this block alone), packs them in list
// order into its own shared-memory slots and blends them. No barrier but __syncwarp. The pixel
// layout, the blend decisions and every arithmetic step of a fragment are those of
// tile_forward2 and tile_backward (moments), so images and transmittances are bit-identical to
// k_fused_l1 at the same configuration and the gradients differ only in the order of the float
// atomics.

constexpr int kWarpItemThreads = 128;
constexpr int kWB = 8;  // block side: BlendLayout<32, 2> has BW = BH = 8 and RS = 4

struct WarpFwdSlots {
    ulonglong2 p0[32];  // (mx, mx), (my, my)
    ulonglong2 p1[32];  // (A, A), (B, B)
    ulonglong2 p2[32];  // (C, C), (o, o)
    ulonglong2 p3[32];  // (r, r), (g, g)
    float4 p4[32];      // b, b, qmin, cover (as bits: 1 if the rect covers the block)
    int4 rect[32];
    int pos[32];        // 1-based list position
    uint32_t id[32];
};

struct WarpBwdSlots {
    float4 a[32];       // mean2d x, y; scaled conic A, B
    float4 b[32];       // scaled conic C; opacity; r, g
    float4 d[32];       // b; qmin; cover (bits); record index (bits)
    int4 rect[32];
    int pos[32];
};

union WarpSlots {
    WarpFwdSlots f;
    WarpBwdSlots b;
};

// Whether the splat with record words s0, s1 (rp: its record) and rect r meets the block at
// (bx0, by0) and may reach alpha >= 1/255 on it; cover: the rect contains the block.
__device__ __forceinline__ bool block_vis(const float4 &s0, const float4 &s1, const float4 *__restrict__ rp,
                                          const int4 &r, int bx0, int by0, bool &cover) {
    const int bx1 = bx0 + kWB - 1, by1 = by0 + kWB - 1;
    cover = r.x <= bx0 && r.y >= bx1 && r.z <= by0 && r.w >= by1;
    if (!(r.y >= bx0 && r.x <= bx1 && r.w >= by0 && r.z <= by1)) return false;
    const float4 s3 = __ldg(rp + 3);
    return tile_keep(s0.x, s0.y, s0.z, s0.w, s1.x, s3.x, s3.y, s3.z, max(bx0, r.x), min(bx1, r.y), max(by0, r.z),
                     min(by1, r.w));
}

__device__ __forceinline__ int4 rect_of(const float4 &s2) {
    const uint32_t rx = __float_as_uint(s2.y), ry = __float_as_uint(s2.z);
    return make_int4((int)(rx & 0xFFFFu), (int)(rx >> 16), (int)(ry & 0xFFFFu), (int)(ry >> 16));
}

template <bool HITS>
__global__ void __launch_bounds__(kWarpItemThreads)
k_fused_warp(const float4 *__restrict__ splats, const uint32_t *__restrict__ ids,
             const uint2 *__restrict__ ranges, const uint32_t *__restrict__ order, int n_items,
             int *__restrict__ counter, const __grid_constant__ CamBatch cb,
             const __grid_constant__ PixPtrs px, float bg0, float bg1, float bg2,
             float *__restrict__ sgrads, float *__restrict__ loss, uint32_t *__restrict__ hits, uint32_t n_gauss) {
    constexpr int TILE = 32, RS = 4, BPT = (TILE / kWB) * (TILE / kWB);  // 16 blocks per tile
    __shared__ WarpSlots s_slots[kWarpItemThreads / 32];
    const unsigned full = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const uint32_t lt = (1u << lane) - 1u;
    WarpSlots &sm = s_slots[threadIdx.x >> 5];
    float loss_acc = 0.f;  // this warp's share of the loss over all its items
    for (;;) {
        int it = 0;
        if (lane == 0) it = atomicAdd(counter, 1);
        it = __shfl_sync(full, it, 0);
        if (it >= n_items * BPT) break;
        const int gt = (int)order[it / BPT], blk = it % BPT;
        const int v = view_of_tile(cb, gt);
        const DevCam &cam = cb.c[v];
        const int lt_ = gt - cam.tile_offset;
        const int bx0 = (lt_ % cam.gx) * TILE + (blk % (TILE / kWB)) * kWB;
        const int by0 = (lt_ / cam.gx) * TILE + (blk / (TILE / kWB)) * kWB;
        const int x = bx0 + lane % kWB, y0 = by0 + lane / kWB, y1 = y0 + RS;
        const bool inside0 = x < cam.W && y0 < cam.H, inside1 = x < cam.W && y1 < cam.H;
        const uint2 rg = ranges[gt];
        const uint32_t rec_off = (uint32_t)v * n_gauss;

        // ---- forward (tile_forward2's fragment steps) ----
        const f2_t one2 = f2(1.f, 1.f);
        const f2_t fx2 = f2((float)x, (float)x);
        const f2_t fy2 = f2((float)y0, (float)y1);
        f2_t T2 = one2, Cr2 = f2(0.f, 0.f), Cg2 = Cr2, Cb2 = Cr2;
        int last0 = 0, last1 = 0;
        bool done0 = !inside0, done1 = !inside1;
        for (uint32_t c0 = rg.x; c0 < rg.y; c0 += 32) {
            if (__all_sync(full, done0 && done1)) break;
            const uint32_t j = c0 + (uint32_t)lane;
            bool vis = false, cover = false;
            float4 s0 = make_float4(0.f, 0.f, 0.f, 0.f), s1 = s0, s2 = s0;
            int4 r = make_int4(0, 0, 0, 0);
            uint32_t id = 0u;
            if (j < rg.y) {
                id = __ldg(ids + j);
                const float4 *rp = splats + (size_t)kSplatWords / 4 * id;
                s0 = __ldg(rp);
                s1 = __ldg(rp + 1);
                s2 = __ldg(rp + 2);
                r = rect_of(s2);
                vis = block_vis(s0, s1, rp, r, bx0, by0, cover);
            }
            const uint32_t vb = __ballot_sync(full, vis);
            if (vis) {
                const int sl = __popc(vb & lt);
                const float A = __fmul_rn(-0.5f * kLog2e, s0.z), B = __fmul_rn(-kLog2e, s0.w);
                const float Cq = __fmul_rn(-0.5f * kLog2e, s1.x);
                sm.f.p0[sl] = make_ulonglong2(f2(s0.x, s0.x), f2(s0.y, s0.y));
                sm.f.p1[sl] = make_ulonglong2(f2(A, A), f2(B, B));
                sm.f.p2[sl] = make_ulonglong2(f2(Cq, Cq), f2(s1.y, s1.y));
                sm.f.p3[sl] = make_ulonglong2(f2(s1.z, s1.z), f2(s1.w, s1.w));
                const float qmin = -log2f(__fmul_rn(255.f, s1.y));
                sm.f.p4[sl] = make_float4(s2.x, s2.x, qmin, __uint_as_float(cover ? 1u : 0u));
                sm.f.rect[sl] = r;
                sm.f.pos[sl] = (int)(j - rg.x) + 1;
                sm.f.id[sl] = id;
            }
            __syncwarp();
            const int nv = __popc(vb);
            for (int m = 0; m < nv; m++) {
                const int4 rr = sm.f.rect[m];
                const float4 p4 = sm.f.p4[m];
                const bool cov = __float_as_uint(p4.w) != 0u;
                const bool xin = cov || (unsigned)(x - rr.x) <= (unsigned)(rr.y - rr.x);
                const bool in0 = !done0 && (cov || (xin && (unsigned)(y0 - rr.z) <= (unsigned)(rr.w - rr.z)));
                const bool in1 = !done1 && (cov || (xin && (unsigned)(y1 - rr.z) <= (unsigned)(rr.w - rr.z)));
                bool b0 = false, b1 = false;  // the pixels that blend this fragment
                if (in0 || in1) {
                    const ulonglong2 a = sm.f.p0[m], b = sm.f.p1[m], c = sm.f.p2[m];
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
                        const bool st0 = v0 && ta < kTMin, st1 = v1 && tb < kTMin;  // stop before it
                        b0 = v0 && !st0;
                        b1 = v1 && !st1;
                        if (st0) done0 = true;
                        if (st1) done1 = true;
                        if (b0 || b1) {
                            const int pos = sm.f.pos[m];
                            float wa, wb, Ta, Tb;
                            f2get(mul2(al2, T2), wa, wb);
                            const f2_t w2 = f2(b0 ? wa : 0.f, b1 ? wb : 0.f);
                            const ulonglong2 col = sm.f.p3[m];
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
                    if (lane == 0 && tot) atomicAdd(hits + (sm.f.id[m] - rec_off), tot);
                }
            }
            __syncwarp();
        }

        // ---- L1 loss and its gradient (as k_fused_l1) ----
        const int HW = cam.W * cam.H;
        const float scale = 1.f / (3.f * (float)HW * (float)cb.V);
        const float *tg = px.target[v];
        float *img = px.image[v];
        float Tf[2], Cr[2], Cg[2], Cb[2], dR[2] = {0.f, 0.f}, dG[2] = {0.f, 0.f}, dB[2] = {0.f, 0.f};
        f2get(T2, Tf[0], Tf[1]);
        f2get(Cr2, Cr[0], Cr[1]);
        f2get(Cg2, Cg[0], Cg[1]);
        f2get(Cb2, Cb[0], Cb[1]);
        const int last[2] = {last0, last1};
        float lsum = 0.f;
#pragma unroll
        for (int k = 0; k < 2; k++) {
            if (!(k == 0 ? inside0 : inside1)) continue;
            const int pix = (k == 0 ? y0 : y1) * cam.W + x;
            const float cr = Cr[k] + Tf[k] * bg0;
            const float cg = Cg[k] + Tf[k] * bg1;
            const float cbv = Cb[k] + Tf[k] * bg2;
            if (img) {
                img[pix] = cr;
                img[HW + pix] = cg;
                img[2 * HW + pix] = cbv;
            }
            const float er = cr - tg[pix], eg = cg - tg[HW + pix], eb = cbv - tg[2 * HW + pix];
            lsum += fabsf(er) + fabsf(eg) + fabsf(eb);
            dR[k] = er > 0.f ? scale : (er < 0.f ? -scale : 0.f);
            dG[k] = eg > 0.f ? scale : (eg < 0.f ? -scale : 0.f);
            dB[k] = eb > 0.f ? scale : (eb < 0.f ? -scale : 0.f);
        }
        loss_acc += warp_sum(lsum) * scale;

        // ---- backward (tile_backward's fragment steps, pixel sums) ----
        float T[2], acd[2], tbg[2];
#pragma unroll
        for (int k = 0; k < 2; k++) {
            T[k] = Tf[k];
            acd[k] = 0.f;
            tbg[k] = Tf[k] * (bg0 * dR[k] + bg1 * dG[k] + bg2 * dB[k]);
        }
        const int wmax = __reduce_max_sync(full, max(last0, last1));
        const uint32_t end = min(rg.y, rg.x + (uint32_t)wmax);
        const float fx = (float)x, fy[2] = {(float)y0, (float)y1};
        const int py[2] = {y0, y1};
        for (uint32_t e1 = end; e1 > rg.x;) {
            const uint32_t e0 = (e1 - rg.x > 32u) ? e1 - 32u : rg.x;
            // lane l takes entry e1 - 1 - l: the slots come out in descending list order
            const uint32_t j = e1 - 1u - (uint32_t)lane;
            bool vis = false, cover = false;
            float4 s0 = make_float4(0.f, 0.f, 0.f, 0.f), s1 = s0, s2 = s0;
            int4 r = make_int4(0, 0, 0, 0);
            uint32_t id = 0u;
            if ((uint32_t)lane < e1 - e0) {
                id = __ldg(ids + j);
                const float4 *rp = splats + (size_t)kSplatWords / 4 * id;
                s0 = __ldg(rp);
                s1 = __ldg(rp + 1);
                s2 = __ldg(rp + 2);
                r = rect_of(s2);
                vis = block_vis(s0, s1, rp, r, bx0, by0, cover);
            }
            const uint32_t vb = __ballot_sync(full, vis);
            if (vis) {
                const int sl = __popc(vb & lt);
                sm.b.a[sl] = make_float4(s0.x, s0.y, __fmul_rn(-0.5f * kLog2e, s0.z), __fmul_rn(-kLog2e, s0.w));
                sm.b.b[sl] = make_float4(__fmul_rn(-0.5f * kLog2e, s1.x), s1.y, s1.z, s1.w);
                const float qmin = -log2f(__fmul_rn(255.f, s1.y));
                sm.b.d[sl] = make_float4(s2.x, qmin, __uint_as_float(cover ? 1u : 0u), __uint_as_float(id));
                sm.b.rect[sl] = r;
                sm.b.pos[sl] = (int)(j - rg.x) + 1;
            }
            __syncwarp();
            const int nv = __popc(vb);
            for (int m = 0; m < nv; m++) {
                const int pos = sm.b.pos[m];
                const int4 rr = sm.b.rect[m];
                const float4 a = sm.b.a[m], b = sm.b.b[m], dd = sm.b.d[m];
                const bool cov = __float_as_uint(dd.z) != 0u;
                const float cbl = dd.x, qmin = dd.y;
                const float dx = a.x - fx, Adx = __fmul_rn(a.z, dx);
                const bool xin = cov || (unsigned)(x - rr.x) <= (unsigned)(rr.y - rr.x);
                float g[9];
#pragma unroll
                for (int e = 0; e < 9; e++) g[e] = 0.f;
                bool contrib = false;
#pragma unroll
                for (int k = 0; k < 2; k++) {
                    if (pos > last[k]) continue;
                    if (!cov && !(xin && (unsigned)(py[k] - rr.z) <= (unsigned)(rr.w - rr.z))) continue;
                    const float dy = a.y - fy[k];
                    const float q = frag_q(Adx, a.w, b.x, dx, dy);
                    if (q > 0.f || q < qmin) continue;   // skipped in the forward too
                    const float G = ex2_approx(q);
                    const float xg = __fmul_rn(b.y, G);
                    const float alpha = fminf(kAlphaMax, xg);
                    contrib = true;
                    const float inv = __fdividef(1.f, 1.f - alpha);
                    T[k] *= inv;                         // transmittance in front of this fragment
                    const float w = alpha * T[k];
                    g[6] = fmaf(w, dR[k], g[6]);
                    g[7] = fmaf(w, dG[k], g[7]);
                    g[8] = fmaf(w, dB[k], g[8]);
                    // dC/da = T (c - acc) - T_final / (1 - a) bg, acc = colour behind this fragment
                    const float cd = fmaf(cbl, dB[k], fmaf(b.w, dG[k], b.z * dR[k]));
                    const float diff = cd - acd[k];
                    const float dLda = fmaf(diff, T[k], -tbg[k] * inv);
                    acd[k] = fmaf(alpha, diff, acd[k]);
                    if (xg <= kAlphaMax) {
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
                    if (contrib) {
                        atomicAdd(reinterpret_cast<float4 *>(dst), make_float4(g[0], g[1], g[2], g[3]));
                        atomicAdd(reinterpret_cast<float4 *>(dst + 4), make_float4(g[4], g[5], g[6], g[7]));
                        atomicAdd(dst + 8, g[8]);
                    }
                    continue;
                }
                warp_transpose_reduce8(g, lane);
                const float gb = warp_sum(g[8]);
                if ((lane & 3) == 0) atomicAdd(dst + (lane >> 2), g[0]);
                if (lane == 0) atomicAdd(dst + 8, gb);
            }
            __syncwarp();
            e1 = e0;
        }
    }
    if (lane == 0 && loss) atomicAdd(loss, loss_acc);
}

template <bool HITS>
void warp_launch_t(const float4 *splats, const uint32_t *ids, const uint2 *ranges, const uint32_t *order,
                   int *counter, const CamBatch &cb, const PixPtrs &px, const float *bg, float *sgrads,
                   float *loss, uint32_t *hits, uint32_t n_gauss, cudaStream_t st) {
    // persistent grid: SMs x resident CTAs per SM, found once per device
    constexpr int kDevices = 64;
    static std::mutex mu;
    static int grid_of[kDevices] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        dev = 0;
    }
    int grid = 0;
    {
        std::lock_guard<std::mutex> lock(mu);
        if (dev >= 0 && dev < kDevices && grid_of[dev] > 0) {
            grid = grid_of[dev];
        } else {
            int sms = 1, b = 0;
            if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1) {
                cudaGetLastError();
                sms = 1;
            }
            if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_fused_warp<HITS>, kWarpItemThreads, 0) !=
                cudaSuccess) {
                cudaGetLastError();
                b = 1;
            }
            grid = sms * (b < 1 ? 1 : b);
            if (dev >= 0 && dev < kDevices) grid_of[dev] = grid;
        }
    }
    const int64_t warps = (int64_t)cb.total_tiles * 16;
    if ((int64_t)grid * (kWarpItemThreads / 32) > warps) grid = (int)((warps + 3) / 4);
    if (grid < 1) grid = 1;
    count_launch();
    k_fused_warp<HITS><<<grid, kWarpItemThreads, 0, st>>>(splats, ids, ranges, order, cb.total_tiles, counter, cb, px,
                                                        bg[0], bg[1], bg[2], sgrads, loss, hits, n_gauss);
}

template <int TILE, int PPT, bool HITS, int SB>
int fused_blocks_per_sm() {
    int b = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_fused_l1<TILE, PPT, HITS, SB>, TILE * TILE / PPT,
                                                      sizeof(FusedSmem<TILE, PPT, SB>)) != cudaSuccess) {
        cudaGetLastError();
        b = 1;
    }
    return b < 1 ? 1 : b;
}

template <int TILE, int PPT, bool HITS, int SB>
void fused_launch_t(const float4 *splats, const uint32_t *ids, const uint2 *ranges, const uint32_t *order,
                    int *counter, const CamBatch &cb, const PixPtrs &px, const float *bg, float *sgrads,
                    float *loss, uint16_t *vis_keys, uint32_t *hits, uint32_t n_gauss, cudaStream_t st) {
    constexpr size_t smem = sizeof(FusedSmem<TILE, PPT, SB>);
    // persistent grid: SMs x resident CTAs per SM, found once per device
    constexpr int kDevices = 64;
    static std::mutex mu;
    static int grid_of[kDevices] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        dev = 0;
    }
    int grid = 0;
    {
        std::lock_guard<std::mutex> lock(mu);
        const bool cached = dev >= 0 && dev < kDevices && grid_of[dev] > 0;
        if (cached) {
            grid = grid_of[dev];
        } else {
            int sms = 1;
            if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1) {
                cudaGetLastError();
                sms = 1;
            }
            // dynamic shared memory beyond the default 48 KB is opted into once per device
            if (cudaFuncSetAttribute(k_fused_l1<TILE, PPT, HITS, SB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)smem) != cudaSuccess)
                cudaGetLastError();
            grid = sms * fused_blocks_per_sm<TILE, PPT, HITS, SB>();
            if (dev >= 0 && dev < kDevices) grid_of[dev] = grid;
        }
    }
    if (grid > cb.total_tiles) grid = cb.total_tiles;
    if (grid < 1) grid = 1;
    count_launch();
    k_fused_l1<TILE, PPT, HITS, SB><<<grid, TILE * TILE / PPT, smem, st>>>(
        splats, ids, ranges, order, cb.total_tiles, counter, cb, px, bg[0], bg[1], bg[2], sgrads, loss, vis_keys,
        hits, n_gauss);
}

template <int TILE, int PPT>
void fused_launch(int batch, const float4 *splats, const uint32_t *ids, const uint2 *ranges, const uint32_t *order,
                  int *counter, const CamBatch &cb, const PixPtrs &px, const float *bg, float *sgrads,
                  float *loss, uint16_t *vis_keys, uint32_t *hits, uint32_t n_gauss, cudaStream_t st) {
#define TGS_FUSED(H, S)                                                                                     \
    fused_launch_t<TILE, PPT, H, S>(splats, ids, ranges, order, counter, cb, px, bg, sgrads, loss, vis_keys, \
                                    hits, n_gauss, st)
    if (batch == 2) {
        if (hits) TGS_FUSED(true, 2);
        else TGS_FUSED(false, 2);
    } else {
        if (hits) TGS_FUSED(true, 1);
        else TGS_FUSED(false, 1);
    }
#undef TGS_FUSED
}

}  // namespace

void build_item_order(const uint2 *ranges, int total_tiles, uint32_t *k0, uint32_t *v0, uint32_t *k1,
                      uint32_t *v1, uint32_t **order, uint32_t *hist, uint32_t *partials, cudaStream_t st) {
    if (total_tiles <= 0) return;
    count_launch();
    k_item_keys<<<(total_tiles + 255) / 256, 256, 0, st>>>(ranges, total_tiles, k0, v0);
    uint32_t *k = k0, *v = v0;
    radix_sort_pairs(k, v, k1, v1, nullptr, total_tiles, 0, 8, hist, partials, st);
    *order = v;
}

void launch_fused_l1(int tile, int ppt, int batch, const float4 *splats, const uint32_t *ids, const uint2 *ranges,
                     const uint32_t *order, int *counter, const CamBatch &cb, const PixPtrs &px,
                     const float *bg, float *sgrads, float *loss, uint16_t *vis_keys, cudaStream_t st,
                     uint32_t *hits, int64_t n_gauss) {
    if (cb.total_tiles <= 0) return;
    const uint32_t n = (uint32_t)n_gauss;
    if (tile == 8 && ppt == 1) fused_launch<8, 1>(batch, splats, ids, ranges, order, counter, cb, px, bg, sgrads, loss, vis_keys, hits, n, st);
    else if (tile == 8 && ppt == 2) fused_launch<8, 2>(batch, splats, ids, ranges, order, counter, cb, px, bg, sgrads, loss, vis_keys, hits, n, st);
    else if (tile == 16 && ppt == 1) fused_launch<16, 1>(batch, splats, ids, ranges, order, counter, cb, px, bg, sgrads, loss, vis_keys, hits, n, st);
    else if (tile == 16 && ppt == 2) fused_launch<16, 2>(batch, splats, ids, ranges, order, counter, cb, px, bg, sgrads, loss, vis_keys, hits, n, st);
    else if (tile == 16 && ppt == 4) fused_launch<16, 4>(batch, splats, ids, ranges, order, counter, cb, px, bg, sgrads, loss, vis_keys, hits, n, st);
    else if (tile == 32 && ppt == 2 && batch == 1) {
        if (hits) warp_launch_t<true>(splats, ids, ranges, order, counter, cb, px, bg, sgrads, loss, hits, n, st);
        else warp_launch_t<false>(splats, ids, ranges, order, counter, cb, px, bg, sgrads, loss, hits, n, st);
    }
    else if (tile == 32 && ppt == 2) fused_launch<32, 2>(batch, splats, ids, ranges, order, counter, cb, px, bg, sgrads, loss, vis_keys, hits, n, st);
    else if (tile == 32 && ppt == 4) fused_launch<32, 4>(batch, splats, ids, ranges, order, counter, cb, px, bg, sgrads, loss, vis_keys, hits, n, st);
}

}  // namespace tgs
