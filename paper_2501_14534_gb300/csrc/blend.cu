// Front-to-back alpha blending (Eq. 2 of the paper) and its backward.
//
// One CTA per (view, tile); TILE*TILE/PPT threads, each owning PPT pixels of the tile.
// The tile's depth-sorted list is streamed through shared memory in batches of one splat
// per thread. The forward stops a pixel before the fragment that would bring its
// transmittance below 1e-4 and leaves the CTA's loop once every pixel has stopped. The
// backward walks the list in reverse from each pixel's last contributor, recovering the
// transmittance in front of each fragment from T_final by division, and scatters the
// per-splat gradients with one warp-level transposed reduction and one atomic per value
// per warp.
#include "tgs_internal.cuh"

namespace tgs {
namespace {

// One staged splat: conic pre-scaled by -log2(e)/2 so that alpha = o * 2^q.
struct StagedSplat {
    float mx, my, A, Bq, Cq, op, r, g, b;
    uint32_t rx, ry;
};

__device__ __forceinline__ void stage_splat(const float4 *__restrict__ splats, uint32_t id,
                                            float4 &a, float4 &b, float4 &c, uint32_t &rx,
                                            uint32_t &ry) {
    float4 s0 = __ldg(splats + 3 * (size_t)id);
    float4 s1 = __ldg(splats + 3 * (size_t)id + 1);
    float4 s2 = __ldg(splats + 3 * (size_t)id + 2);
    // q = log2(e) * power, power = -1/2 (ca dx^2 + cc dy^2) - cb dx dy
    a = make_float4(s0.x, s0.y, __fmul_rn(-0.5f * kLog2e, s0.z), __fmul_rn(-kLog2e, s0.w));
    b = make_float4(__fmul_rn(-0.5f * kLog2e, s1.x), s1.y, s1.z, s1.w);
    c = make_float4(s2.x, 0.f, 0.f, 0.f);
    rx = __float_as_uint(s2.y);
    ry = __float_as_uint(s2.z);
}

// Exponent of one fragment, written with explicit roundings so that the forward and the
// backward kernels compute bit-identical values.
__device__ __forceinline__ float frag_q(float A, float Bq, float Cq, float dx, float dy) {
    float u = __fmaf_rn(A, dx, __fmul_rn(Bq, dy));
    float w = __fmul_rn(__fmul_rn(Cq, dy), dy);
    return __fmaf_rn(dx, u, w);
}

__device__ __forceinline__ bool in_rect(int px, int py, uint32_t rx, uint32_t ry) {
    return (unsigned)(px - (int)(rx & 0xFFFFu)) <= (unsigned)((int)(rx >> 16) - (int)(rx & 0xFFFFu)) &&
           (unsigned)(py - (int)(ry & 0xFFFFu)) <= (unsigned)((int)(ry >> 16) - (int)(ry & 0xFFFFu));
}

template <int TILE, int PPT>
__global__ void __launch_bounds__(TILE * TILE / PPT)
k_blend_fwd(const float4 *__restrict__ splats, const uint32_t *__restrict__ ids,
            const uint2 *__restrict__ ranges, const __grid_constant__ CamBatch cb,
            const __grid_constant__ PixPtrs px, float bg0, float bg1, float bg2) {
    constexpr int NT = TILE * TILE / PPT;
    __shared__ float4 s_a[NT], s_b[NT];
    __shared__ float s_c[NT];
    __shared__ uint32_t s_rx[NT], s_ry[NT];

    const int gt = blockIdx.x;
    const int v = view_of_tile(cb, gt);
    const DevCam &cam = cb.c[v];
    const int lt = gt - cam.tile_offset;
    const int tx = lt % cam.gx, ty = lt / cam.gx;
    const uint2 rg = ranges[gt];
    const int t = threadIdx.x;

    int pxs[PPT], pys[PPT], last[PPT], exam[PPT];
    bool done[PPT];
    float T[PPT], Cr[PPT], Cg[PPT], Cb[PPT];
#pragma unroll
    for (int k = 0; k < PPT; k++) {
        int p = t + k * NT;
        pxs[k] = tx * TILE + (p % TILE);
        pys[k] = ty * TILE + (p / TILE);
        done[k] = !(pxs[k] < cam.W && pys[k] < cam.H);
        T[k] = 1.f;
        Cr[k] = Cg[k] = Cb[k] = 0.f;
        last[k] = 0;
        exam[k] = 0;
    }

    for (uint32_t base = rg.x; base < rg.y; base += NT) {
        bool mine = true;
#pragma unroll
        for (int k = 0; k < PPT; k++) mine = mine && done[k];
        if (__syncthreads_count(mine) == NT) break;
        const uint32_t j = base + t;
        if (j < rg.y) {
            float4 a, b, c;
            uint32_t rx, ry;
            stage_splat(splats, __ldg(ids + j), a, b, c, rx, ry);
            s_a[t] = a;
            s_b[t] = b;
            s_c[t] = c.x;
            s_rx[t] = rx;
            s_ry[t] = ry;
        }
        __syncthreads();
        const int cnt = min((uint32_t)NT, rg.y - base);
        const int pos0 = (int)(base - rg.x);
        for (int m = 0; m < cnt; m++) {
            const float4 a = s_a[m], b = s_b[m];
            const float cbl = s_c[m];
            const uint32_t rx = s_rx[m], ry = s_ry[m];
#pragma unroll
            for (int k = 0; k < PPT; k++) {
                if (done[k]) continue;
                exam[k] = pos0 + m + 1;
                if (!in_rect(pxs[k], pys[k], rx, ry)) continue;
                const float dx = a.x - (float)pxs[k], dy = a.y - (float)pys[k];
                const float q = frag_q(a.z, a.w, b.x, dx, dy);
                if (q > 0.f) continue;
                const float alpha = fminf(kAlphaMax, __fmul_rn(b.y, ex2_approx(q)));
                if (alpha < kAlphaMin) continue;
                const float tT = __fmul_rn(T[k], __fsub_rn(1.f, alpha));
                if (tT < kTMin) {
                    done[k] = true;
                    continue;
                }
                const float w = __fmul_rn(alpha, T[k]);
                Cr[k] = __fmaf_rn(b.z, w, Cr[k]);
                Cg[k] = __fmaf_rn(b.w, w, Cg[k]);
                Cb[k] = __fmaf_rn(cbl, w, Cb[k]);
                T[k] = tT;
                last[k] = pos0 + m + 1;
            }
        }
    }
    const int HW = cam.W * cam.H;
    float *img = px.image[v];
    float *Tf = px.T_final[v];
    int32_t *ls = px.last[v];
    int32_t *ex = px.n_exam[v];
#pragma unroll
    for (int k = 0; k < PPT; k++) {
        if (!(pxs[k] < cam.W && pys[k] < cam.H)) continue;
        const int pix = pys[k] * cam.W + pxs[k];
        img[pix] = Cr[k] + T[k] * bg0;
        img[HW + pix] = Cg[k] + T[k] * bg1;
        img[2 * HW + pix] = Cb[k] + T[k] * bg2;
        if (Tf) Tf[pix] = T[k];
        if (ls) ls[pix] = last[k];
        if (ex) ex[pix] = exam[k];
    }
}

// Sums v[0..7] over the warp; afterwards lanes with (lane & 3) == 0 hold the total of
// value (lane >> 2). Four levels of halving exchange instead of eight full butterflies.
__device__ __forceinline__ void warp_transpose_reduce8(float v[8], int lane) {
    const unsigned full = 0xffffffffu;
    {
        const bool up = lane & 16;
#pragma unroll
        for (int i = 0; i < 4; i++) {
            float send = up ? v[i] : v[i + 4];
            float keep = up ? v[i + 4] : v[i];
            v[i] = keep + __shfl_xor_sync(full, send, 16);
        }
    }
    {
        const bool up = lane & 8;
#pragma unroll
        for (int i = 0; i < 2; i++) {
            float send = up ? v[i] : v[i + 2];
            float keep = up ? v[i + 2] : v[i];
            v[i] = keep + __shfl_xor_sync(full, send, 8);
        }
    }
    {
        const bool up = lane & 4;
        float send = up ? v[0] : v[1];
        float keep = up ? v[1] : v[0];
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

template <int TILE, int PPT>
__global__ void __launch_bounds__(TILE * TILE / PPT)
k_blend_bwd(const float4 *__restrict__ splats, const uint32_t *__restrict__ ids,
            const uint2 *__restrict__ ranges, const __grid_constant__ CamBatch cb,
            const __grid_constant__ PixPtrs px, float bg0, float bg1, float bg2,
            float *__restrict__ sgrads) {
    constexpr int NT = TILE * TILE / PPT;
    __shared__ float4 s_a[NT], s_b[NT];
    __shared__ float s_c[NT];
    __shared__ uint32_t s_rx[NT], s_ry[NT], s_id[NT];
    __shared__ int s_maxlast;

    const int gt = blockIdx.x;
    const int v = view_of_tile(cb, gt);
    const DevCam &cam = cb.c[v];
    const int lt = gt - cam.tile_offset;
    const int tx = lt % cam.gx, ty = lt / cam.gx;
    const uint2 rg = ranges[gt];
    const int t = threadIdx.x;
    const int lane = t & 31;
    const int HW = cam.W * cam.H;

    int pxs[PPT], pys[PPT], lastp[PPT];
    float T[PPT], Tfin[PPT], dR[PPT], dG[PPT], dB[PPT], acR[PPT], acG[PPT], acB[PPT];
    float la[PPT], lR[PPT], lG[PPT], lB[PPT], bgdot[PPT];
    int mymax = 0;
#pragma unroll
    for (int k = 0; k < PPT; k++) {
        int p = t + k * NT;
        pxs[k] = tx * TILE + (p % TILE);
        pys[k] = ty * TILE + (p / TILE);
        const bool inside = pxs[k] < cam.W && pys[k] < cam.H;
        const int pix = pys[k] * cam.W + pxs[k];
        lastp[k] = inside ? px.last[v][pix] : 0;
        T[k] = Tfin[k] = inside ? px.T_final[v][pix] : 1.f;
        const float *d = px.dL[v];
        dR[k] = inside ? d[pix] : 0.f;
        dG[k] = inside ? d[HW + pix] : 0.f;
        dB[k] = inside ? d[2 * HW + pix] : 0.f;
        bgdot[k] = bg0 * dR[k] + bg1 * dG[k] + bg2 * dB[k];
        acR[k] = acG[k] = acB[k] = 0.f;
        la[k] = 0.f;
        lR[k] = lG[k] = lB[k] = 0.f;
        mymax = max(mymax, lastp[k]);
    }
    if (t == 0) s_maxlast = 0;
    __syncthreads();
    atomicMax(&s_maxlast, mymax);
    __syncthreads();
    const uint32_t end = min(rg.y, rg.x + (uint32_t)s_maxlast);

    for (uint32_t bend = end; bend > rg.x;) {
        const uint32_t bstart = (bend - rg.x > (uint32_t)NT) ? bend - NT : rg.x;
        const int cnt = (int)(bend - bstart);
        __syncthreads();
        if (t < cnt) {
            const uint32_t j = bend - 1 - t;  // smem slot t holds list position j
            const uint32_t id = __ldg(ids + j);
            float4 a, b, c;
            uint32_t rx, ry;
            stage_splat(splats, id, a, b, c, rx, ry);
            s_a[t] = a;
            s_b[t] = b;
            s_c[t] = c.x;
            s_rx[t] = rx;
            s_ry[t] = ry;
            s_id[t] = id;
        }
        __syncthreads();
        for (int m = 0; m < cnt; m++) {
            const int pos = (int)(bend - rg.x) - m;  // 1-based position in the tile list
            const float4 a = s_a[m], b = s_b[m];
            const float cbl = s_c[m];
            const uint32_t rx = s_rx[m], ry = s_ry[m];
            float g[9];
#pragma unroll
            for (int e = 0; e < 9; e++) g[e] = 0.f;
            bool contrib = false;
#pragma unroll
            for (int k = 0; k < PPT; k++) {
                if (pos > lastp[k]) continue;
                if (!in_rect(pxs[k], pys[k], rx, ry)) continue;
                const float dx = a.x - (float)pxs[k], dy = a.y - (float)pys[k];
                const float q = frag_q(a.z, a.w, b.x, dx, dy);
                if (q > 0.f) continue;
                const float G = ex2_approx(q);
                const float x = __fmul_rn(b.y, G);
                const float alpha = fminf(kAlphaMax, x);
                if (alpha < kAlphaMin) continue;
                contrib = true;
                const float om = __fsub_rn(1.f, alpha);
                T[k] = T[k] / om;
                const float w = alpha * T[k];
                g[6] += w * dR[k];
                g[7] += w * dG[k];
                g[8] += w * dB[k];
                acR[k] = la[k] * lR[k] + (1.f - la[k]) * acR[k];
                acG[k] = la[k] * lG[k] + (1.f - la[k]) * acG[k];
                acB[k] = la[k] * lB[k] + (1.f - la[k]) * acB[k];
                float dLda = (b.z - acR[k]) * dR[k] + (b.w - acG[k]) * dG[k] + (cbl - acB[k]) * dB[k];
                dLda = dLda * T[k] - Tfin[k] / om * bgdot[k];
                la[k] = alpha;
                lR[k] = b.z;
                lG[k] = b.w;
                lB[k] = cbl;
                if (x <= kAlphaMax) {
                    // d power / d q = ln 2; with the scaled conic, -a dx - b dy = ln2 (2A dx + B dy)
                    const float dLdp = dLda * b.y * G;
                    g[5] += dLda * G;
                    g[0] += dLdp * kLn2 * (2.f * a.z * dx + a.w * dy);
                    g[1] += dLdp * kLn2 * (2.f * b.x * dy + a.w * dx);
                    g[2] += -0.5f * dLdp * dx * dx;
                    g[3] += -dLdp * dx * dy;
                    g[4] += -0.5f * dLdp * dy * dy;
                }
            }
            if (__ballot_sync(0xffffffffu, contrib) == 0u) continue;
            const uint32_t id = s_id[m];
            float *dst = sgrads + 12 * (size_t)id;
            warp_transpose_reduce8(g, lane);
            const float gb_ = warp_sum(g[8]);
            if ((lane & 3) == 0) atomicAdd(dst + (lane >> 2), g[0]);
            if (lane == 0) atomicAdd(dst + 8, gb_);
        }
        bend = bstart;
    }
}

__global__ void k_l1(const float *__restrict__ img, const float *__restrict__ tgt, int64_t count,
                     float scale, float *__restrict__ loss, float *__restrict__ grad) {
    float acc = 0.f;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count;
         i += (int64_t)gridDim.x * blockDim.x) {
        const float d = img[i] - tgt[i];
        acc += fabsf(d);
        if (grad) grad[i] = d > 0.f ? scale : (d < 0.f ? -scale : 0.f);
    }
    acc = warp_sum(acc);
    __shared__ float s[32];
    if ((threadIdx.x & 31) == 0) s[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x < 32) {
        float x = threadIdx.x < (blockDim.x >> 5) ? s[threadIdx.x] : 0.f;
        x = warp_sum(x);
        if (threadIdx.x == 0 && loss) atomicAdd(loss, x * scale);
    }
}

template <int TILE, int PPT>
void fwd_launch(const float4 *splats, const uint32_t *ids, const uint2 *ranges, const CamBatch &cb,
                const PixPtrs &px, const float *bg, cudaStream_t st) {
    count_launch();
    k_blend_fwd<TILE, PPT><<<cb.total_tiles, TILE * TILE / PPT, 0, st>>>(splats, ids, ranges, cb, px,
                                                                         bg[0], bg[1], bg[2]);
}

template <int TILE, int PPT>
void bwd_launch(const float4 *splats, const uint32_t *ids, const uint2 *ranges, const CamBatch &cb,
                const PixPtrs &px, const float *bg, float *sg, cudaStream_t st) {
    count_launch();
    k_blend_bwd<TILE, PPT><<<cb.total_tiles, TILE * TILE / PPT, 0, st>>>(splats, ids, ranges, cb, px,
                                                                         bg[0], bg[1], bg[2], sg);
}

}  // namespace

int blend_supported(int tile, int ppt) {
    if (tile != 8 && tile != 16 && tile != 32) return 0;
    if (ppt != 1 && ppt != 2 && ppt != 4) return 0;
    if (tile == 8 && ppt == 4) return 0;     // 16 threads: below one warp
    if (tile == 32 && ppt == 1) return 0;    // 1024 threads: too many registers
    return 1;
}

#define TGS_DISPATCH(FN, ...)                                               \
    do {                                                                    \
        if (tile == 8 && ppt == 1) FN<8, 1>(__VA_ARGS__);                   \
        else if (tile == 8 && ppt == 2) FN<8, 2>(__VA_ARGS__);              \
        else if (tile == 16 && ppt == 1) FN<16, 1>(__VA_ARGS__);            \
        else if (tile == 16 && ppt == 2) FN<16, 2>(__VA_ARGS__);            \
        else if (tile == 16 && ppt == 4) FN<16, 4>(__VA_ARGS__);            \
        else if (tile == 32 && ppt == 2) FN<32, 2>(__VA_ARGS__);            \
        else if (tile == 32 && ppt == 4) FN<32, 4>(__VA_ARGS__);            \
    } while (0)

void launch_blend_forward(int tile, int ppt, const float4 *splats, const uint32_t *ids,
                          const uint2 *ranges, const CamBatch &cb, const PixPtrs &px,
                          const float *bg, cudaStream_t st) {
    if (cb.total_tiles <= 0) return;
    TGS_DISPATCH(fwd_launch, splats, ids, ranges, cb, px, bg, st);
}

void launch_blend_backward(int tile, int ppt, const float4 *splats, const uint32_t *ids,
                           const uint2 *ranges, const CamBatch &cb, const PixPtrs &px,
                           const float *bg, float *sgrads, cudaStream_t st) {
    if (cb.total_tiles <= 0) return;
    TGS_DISPATCH(bwd_launch, splats, ids, ranges, cb, px, bg, sgrads, st);
}

void launch_l1(const float *img, const float *tgt, int64_t count, float scale, float *loss,
               float *grad, cudaStream_t st) {
    if (count <= 0) return;
    int64_t blocks = (count + 255) / 256;
    if (blocks > 152 * 8) blocks = 152 * 8;
    count_launch();
    k_l1<<<(unsigned)blocks, 256, 0, st>>>(img, tgt, count, scale, loss, grad);
}

}  // namespace tgs
