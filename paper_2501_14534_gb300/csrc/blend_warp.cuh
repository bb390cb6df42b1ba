// Warp items: one 8 x 8 pixel block of a 32 x 32 tile per warp, 2 pixels per thread.
//
// In the CTA kernels the 16 warps of a 32 x 32 tile share nothing but the tile's list, yet they
// pass each phase in step: a phase lasts as long as the tile's busiest warp, and near its end a
// scheduler has too few warps left to issue every cycle. Here a warp takes one (view, tile,
// block) item and walks the tile's list on its own, 32 entries at a time: it loads the 32
// records, keeps those whose rect meets its block and that may reach alpha >= 1/255 there (the
// per-warp-block bits of block_masks and stage_splat, for this block alone), packs them in list
// order into its own shared-memory slots and blends them. No barrier but __syncwarp. A slot
// carries the block's pixels inside the splat's rect as a 64-bit mask (block_pixels), so a
// fragment's rect test is one bit test per pixel.
//
// The pixel layout (BlendLayout<32, 2>: 8 columns x 4 rows of lanes, rows y and y + 4 per
// thread), the blend decisions and every arithmetic step of a fragment are those of
// tile_forward2 and tile_backward, so images, transmittances, last contributors and examined
// counts are bit-identical to the CTA kernels at the same configuration, and gradients differ
// only in the order of the float atomics.
#pragma once

#include "blend_common.cuh"

namespace tgs {

constexpr int kWB = 8;        // block side (BW = BH = 8 in BlendLayout<32, 2>)
constexpr int kWRS = 4;       // rows between a thread's two pixels
constexpr int kWTile = 32;    // tile side of the lists
constexpr int kWBlocks = 16;  // blocks per tile
// Up to this many contributing lanes a fragment's sums go out as per-lane atomics, above it
// through a warp reduction (measured on the 1M x 16-view step, fused blend per step: 16 -> 5.80,
// 20 -> 5.79, 24 -> 5.82, 28 -> 5.93 ms; with the 12-shuffle reduction of the moments
// 12 -> 5.18, 16 -> 5.15, 20 -> 5.17, 24 -> 5.28 ms).
constexpr int kWarpDirectLanes = 16;

struct WarpFwdSlots {
    ulonglong2 p0[32];  // (mx, mx), (my, my)
    ulonglong2 p1[32];  // (A, A), (B, B): the conic scaled as in stage_splat
    ulonglong2 p2[32];  // (C, C), (o, o)
    ulonglong2 p3[32];  // (r, r), (g, g)
    float4 p4[32];      // b, b, qmin, 1-based list position (int bits; in the same load as qmin)
    uint2 pm[32];       // the block's pixels inside the rect (block_pixels)
    uint32_t id[32];
};

struct WarpBwdSlots {
    float4 a[32];       // mean2d x, y; scaled conic A, B
    float4 b[32];       // scaled conic C; opacity; r, g
    float4 d[32];       // b; qmin; 1-based list position (int bits); record index (bits)
    uint2 pm[32];       // the block's pixels inside the rect (block_pixels)
};

union WarpSlots {
    WarpFwdSlots f;
    WarpBwdSlots b;
};

// The pixels of lane (threadIdx.x & 31) in block blk of local tile lt of camera cam.
struct WarpPixels {
    int bx0, by0, x, y0, y1;
    bool in0, in1;
    __device__ __forceinline__ void init(const DevCam &cam, int lt, int blk) {
        const int lane = threadIdx.x & 31;
        bx0 = (lt % cam.gx) * kWTile + (blk % (kWTile / kWB)) * kWB;
        by0 = (lt / cam.gx) * kWTile + (blk / (kWTile / kWB)) * kWB;
        x = bx0 + lane % kWB;
        y0 = by0 + lane / kWB;
        y1 = y0 + kWRS;
        in0 = x < cam.W && y0 < cam.H;
        in1 = x < cam.W && y1 < cam.H;
    }
};

// The pixels of the 8 x 8 block at (bx0, by0) that lie inside rect r (which meets the block):
// bit l of .x is pixel 0 of lane l (row l / 8, column l % 8), bit l of .y its pixel 1 (4 rows
// further down).
__device__ __forceinline__ uint2 block_pixels(const int4 &r, int bx0, int by0) {
    const int cx0 = max(r.x - bx0, 0), cx1 = min(r.y - bx0, kWB - 1);
    const int cy0 = max(r.z - by0, 0), cy1 = min(r.w - by0, kWB - 1);
    const uint32_t cols = ((0xFFu >> (kWB - 1 - cx1)) & (0xFFu << cx0)) * 0x01010101u;  // in every row
    const unsigned long long rows = (~0ull >> (8 * (kWB - 1 - cy1))) & (~0ull << (8 * cy0));
    return make_uint2(cols & (uint32_t)rows, cols & (uint32_t)(rows >> 32));
}

__device__ __forceinline__ int4 rect_of(const float4 &s2) {
    const uint32_t rx = __float_as_uint(s2.y), ry = __float_as_uint(s2.z);
    return make_int4((int)(rx & 0xFFFFu), (int)(rx >> 16), (int)(ry & 0xFFFFu), (int)(ry >> 16));
}

// Whether the splat with record words s0, s1 (rp: its record) and rect r meets the block at
// (bx0, by0) and may reach alpha >= 1/255 on it.
__device__ __forceinline__ bool block_vis(const float4 &s0, const float4 &s1, const float4 *__restrict__ rp,
                                          const int4 &r, int bx0, int by0) {
    const int bx1 = bx0 + kWB - 1, by1 = by0 + kWB - 1;
    if (!(r.y >= bx0 && r.x <= bx1 && r.w >= by0 && r.z <= by1)) return false;
    const float4 s3 = __ldg(rp + 3);
    return tile_keep_flat(s0.x, s0.y, s0.z, s0.w, s1.x, s3.x, s3.y, s3.z, max(bx0, r.x), min(bx1, r.y),
                          max(by0, r.z), min(by1, r.w));
}

// Loads entry j of the list (if take) and tests it against the block.
__device__ __forceinline__ bool warp_take(const float4 *__restrict__ splats, const uint32_t *__restrict__ ids,
                                          uint32_t j, bool take, int bx0, int by0, float4 &s0, float4 &s1,
                                          float4 &s2, int4 &r, uint32_t &id) {
    if (!take) return false;
    id = __ldg(ids + j);
    const float4 *rp = splats + (size_t)kSplatWords / 4 * id;
    s0 = __ldg(rp);
    s1 = __ldg(rp + 1);
    s2 = __ldg(rp + 2);
    r = rect_of(s2);
    return block_vis(s0, s1, rp, r, bx0, by0);
}

// Forward of the block over the list [rg.x, rg.y) (tile_forward2's steps). On return each
// pixel holds its colour sum, transmittance and last contributor (1-based position, 0 if none);
// with EXAM also the number of entries it examined (tile_forward2's exam).
template <bool HITS, bool EXAM>
__device__ __forceinline__ void warp_forward(WarpFwdSlots &sm, const float4 *__restrict__ splats,
                                             const uint32_t *__restrict__ ids, uint2 rg, const WarpPixels &P,
                                             float T[2], float Cr[2], float Cg[2], float Cb[2], int last[2],
                                             int exam[2], uint32_t *__restrict__ hits, uint32_t rec_off) {
    const unsigned full = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const uint32_t lt = (1u << lane) - 1u;
    const f2_t one2 = f2(1.f, 1.f);
    const f2_t fx2 = f2((float)P.x, (float)P.x);
    const f2_t fy2 = f2((float)P.y0, (float)P.y1);
    f2_t T2 = one2, Cr2 = f2(0.f, 0.f), Cg2 = Cr2, Cb2 = Cr2;
    int last0 = 0, last1 = 0, exam0 = 0, exam1 = 0;
    bool done0 = !P.in0, done1 = !P.in1;
    // this lane's bit while its pixel still blends, else 0
    uint32_t live0 = P.in0 ? (1u << lane) : 0u, live1 = P.in1 ? (1u << lane) : 0u;
    for (uint32_t c0 = rg.x; c0 < rg.y; c0 += 32) {
        if (__all_sync(full, done0 && done1)) break;
        const uint32_t j = c0 + (uint32_t)lane;
        float4 s0 = make_float4(0.f, 0.f, 0.f, 0.f), s1 = s0, s2 = s0;
        int4 r = make_int4(0, 0, 0, 0);
        uint32_t id = 0u;
        const bool vis = warp_take(splats, ids, j, j < rg.y, P.bx0, P.by0, s0, s1, s2, r, id);
        const uint32_t vb = __ballot_sync(full, vis);
        if (vis) {
            const int sl = __popc(vb & lt);
            const float A = __fmul_rn(-0.5f * kLog2e, s0.z), B = __fmul_rn(-kLog2e, s0.w);
            const float Cq = __fmul_rn(-0.5f * kLog2e, s1.x);
            sm.p0[sl] = make_ulonglong2(f2(s0.x, s0.x), f2(s0.y, s0.y));
            sm.p1[sl] = make_ulonglong2(f2(A, A), f2(B, B));
            sm.p2[sl] = make_ulonglong2(f2(Cq, Cq), f2(s1.y, s1.y));
            sm.p3[sl] = make_ulonglong2(f2(s1.z, s1.z), f2(s1.w, s1.w));
            const float qmin = -log2f(__fmul_rn(255.f, s1.y));
            sm.p4[sl] = make_float4(s2.x, s2.x, qmin, __int_as_float((int)(j - rg.x) + 1));
            sm.pm[sl] = block_pixels(r, P.bx0, P.by0);
            sm.id[sl] = id;
        }
        __syncwarp();
        const int nv = __popc(vb);
#pragma unroll 2
        for (int m = 0; m < nv; m++) {
            // every 8 fragments: a warp whose pixels all stopped leaves the chunk
            if ((m & 7) == 7 && __all_sync(full, done0 && done1)) break;
            const uint2 pm = sm.pm[m];
            const float4 p4 = sm.p4[m];
            const bool in0 = (pm.x & live0) != 0u;
            const bool in1 = (pm.y & live1) != 0u;
            bool b0 = false, b1 = false;  // the pixels that blend this fragment
            {  // no branch on in0 || in1: some lane of the warp nearly always has one
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
                    const bool st0 = v0 && ta < kTMin, st1 = v1 && tb < kTMin;  // stop before this fragment
                    b0 = v0 && !st0;
                    b1 = v1 && !st1;
                    if (st0) {
                        done0 = true;
                        live0 = 0u;
                        if (EXAM) exam0 = __float_as_int(p4.w);
                    }
                    if (st1) {
                        done1 = true;
                        live1 = 0u;
                        if (EXAM) exam1 = __float_as_int(p4.w);
                    }
                    if (b0 || b1) {
                        const int pos = __float_as_int(p4.w);
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
                if (lane == 0 && tot) atomicAdd(hits + (sm.id[m] - rec_off), tot);
            }
        }
        __syncwarp();
    }
    f2get(T2, T[0], T[1]);
    f2get(Cr2, Cr[0], Cr[1]);
    f2get(Cg2, Cg[0], Cg[1]);
    f2get(Cb2, Cb[0], Cb[1]);
    last[0] = last0;
    last[1] = last1;
    if (EXAM) {
        const int len = (int)(rg.y - rg.x);
        exam[0] = (P.in0 && exam0 == 0) ? len : exam0;  // never stopped: saw the whole list
        exam[1] = (P.in1 && exam1 == 0) ? len : exam1;
    }
}

// Backward of the block (tile_backward's steps): the reverse walk from the warp's last
// contributor with dL/d pixel colour dR, dG, dB and the forward's final transmittances Tf.
// MOMENTS: the pixel sums of each fragment are added to its gradient record (the preprocess
// backward applies the conic and opacity); else the splat gradients themselves. BG: the
// background colour is not zero (with a zero background its term of dL/dalpha is 0 and skipped).
template <bool MOMENTS, bool BG>
__device__ __forceinline__ void warp_backward(WarpBwdSlots &sm, const float4 *__restrict__ splats,
                                              const uint32_t *__restrict__ ids, uint2 rg, const WarpPixels &P,
                                              const int last[2], const float Tf[2], const float dR[2],
                                              const float dG[2], const float dB[2], float bg0, float bg1,
                                              float bg2, float *__restrict__ sgrads) {
    const unsigned full = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const uint32_t lt = (1u << lane) - 1u, lm = 1u << lane;
    float T[2], acd[2], tbg[2];
#pragma unroll
    for (int k = 0; k < 2; k++) {
        T[k] = Tf[k];
        acd[k] = 0.f;
        tbg[k] = Tf[k] * (bg0 * dR[k] + bg1 * dG[k] + bg2 * dB[k]);
    }
    const int wmax = __reduce_max_sync(full, max(last[0], last[1]));
    const uint32_t end = min(rg.y, rg.x + (uint32_t)wmax);
    const float fx = (float)P.x, fy[2] = {(float)P.y0, (float)P.y1};
    for (uint32_t e1 = end; e1 > rg.x;) {
        const uint32_t e0 = (e1 - rg.x > 32u) ? e1 - 32u : rg.x;
        // lane l takes entry e1 - 1 - l: the slots come out in descending list order
        const uint32_t j = e1 - 1u - (uint32_t)lane;
        float4 s0 = make_float4(0.f, 0.f, 0.f, 0.f), s1 = s0, s2 = s0;
        int4 r = make_int4(0, 0, 0, 0);
        uint32_t id = 0u;
        const bool vis = warp_take(splats, ids, j, (uint32_t)lane < e1 - e0, P.bx0, P.by0, s0, s1, s2, r, id);
        const uint32_t vb = __ballot_sync(full, vis);
        if (vis) {
            const int sl = __popc(vb & lt);
            sm.a[sl] = make_float4(s0.x, s0.y, __fmul_rn(-0.5f * kLog2e, s0.z), __fmul_rn(-kLog2e, s0.w));
            sm.b[sl] = make_float4(__fmul_rn(-0.5f * kLog2e, s1.x), s1.y, s1.z, s1.w);
            const float qmin = -log2f(__fmul_rn(255.f, s1.y));
            sm.d[sl] = make_float4(s2.x, qmin, __int_as_float((int)(j - rg.x) + 1), __uint_as_float(id));
            sm.pm[sl] = block_pixels(r, P.bx0, P.by0);
        }
        __syncwarp();
        const int nv = __popc(vb);
        for (int m = 0; m < nv; m++) {
            const uint2 pm = sm.pm[m];
            const float4 a = sm.a[m], b = sm.b[m], dd = sm.d[m];
            const int pos = __float_as_int(dd.z);
            const float cbl = dd.x, qmin = dd.y;
            const float dx = a.x - fx, Adx = __fmul_rn(a.z, dx);
            const uint32_t inr[2] = {pm.x & lm, pm.y & lm};
            // per-warp sums over the pixels of u = dL/da G (tile_backward's g[0..8])
            float g[9];
#pragma unroll
            for (int e = 0; e < 9; e++) g[e] = 0.f;
            bool contrib = false;
#pragma unroll
            for (int k = 0; k < 2; k++) {
                if (pos > last[k] || inr[k] == 0u) continue;
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
                const float dLda = BG ? fmaf(diff, T[k], -tbg[k] * inv) : diff * T[k];
                acd[k] = fmaf(alpha, diff, acd[k]);   // now includes this fragment
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
            if (__popc(cmask) <= kWarpDirectLanes) {
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
            if (MOMENTS) {
                // values 0..7 by halving exchange over lanes 16, 8, 4 with value 8 summed alongside,
                // then (value, value 8) by one more exchange over lane 2 and a butterfly over
                // lane 1: 12 shuffles instead of 14; lane 4j holds the total of value j, lane 2
                // that of value 8
                {
                    const bool up = lane & 16;
#pragma unroll
                    for (int e = 0; e < 4; e++) {
                        const float send = up ? g[e] : g[e + 4];
                        const float keep = up ? g[e + 4] : g[e];
                        g[e] = keep + __shfl_xor_sync(full, send, 16);
                    }
                    g[8] += __shfl_xor_sync(full, g[8], 16);
                }
                {
                    const bool up = lane & 8;
#pragma unroll
                    for (int e = 0; e < 2; e++) {
                        const float send = up ? g[e] : g[e + 2];
                        const float keep = up ? g[e + 2] : g[e];
                        g[e] = keep + __shfl_xor_sync(full, send, 8);
                    }
                    g[8] += __shfl_xor_sync(full, g[8], 8);
                }
                {
                    const bool up = lane & 4;
                    const float send = up ? g[0] : g[1];
                    const float keep = up ? g[1] : g[0];
                    g[0] = keep + __shfl_xor_sync(full, send, 4);
                    g[8] += __shfl_xor_sync(full, g[8], 4);
                }
                {
                    const bool up = lane & 2;
                    const float send = up ? g[0] : g[8];
                    const float keep = up ? g[8] : g[0];
                    g[0] = keep + __shfl_xor_sync(full, send, 2);
                }
                g[0] += __shfl_xor_sync(full, g[0], 1);
                if ((lane & 3) == 0) atomicAdd(dst + (lane >> 2), g[0]);
                if (lane == 2) atomicAdd(dst + 8, g[0]);
                continue;
            }
            warp_transpose_reduce8(g, lane);
            const float gb = warp_sum(g[8]);
            // as tile_backward: values 0, 1 mean2d; 2, 3, 4 conic; 5 opacity; 6, 7 rgb
            const int jj = lane >> 2;
            const float Sx = __shfl_sync(full, g[0], 0), Sy = __shfl_sync(full, g[0], 4);
            const float o = b.y;
            const float lin = (jj == 0) ? fmaf(2.f * a.z, Sx, a.w * Sy) : fmaf(2.f * b.x, Sy, a.w * Sx);
            const float sc = (jj < 2) ? o * kLn2 : ((jj == 3) ? -o : ((jj == 2 || jj == 4) ? -0.5f * o : 1.f));
            const float val = sc * ((jj < 2) ? lin : g[0]);
            const float v1 = __shfl_down_sync(full, val, 4), v2 = __shfl_down_sync(full, val, 8),
                        v3 = __shfl_down_sync(full, val, 12);
            if ((lane & 15) == 0)
                atomicAdd(reinterpret_cast<float4 *>(dst + (lane >> 2)), make_float4(val, v1, v2, v3));
            if (lane == 0) atomicAdd(dst + 8, gb);
        }
        __syncwarp();
        e1 = e0;
    }
}

}  // namespace tgs
