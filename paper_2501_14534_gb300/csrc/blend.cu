// Front-to-back alpha blending (Eq. 2 of the paper) and its backward, one CTA per (view,
// tile), or at 32 x 32 tiles and 2 pixels per thread one warp per 8 x 8 block (blend_warp.cuh). The per-tile work lives in blend_common.cuh (shared with the fused kernel): the
// tile's depth-sorted list is streamed through shared memory in batches of one splat per
// thread; the forward stops a pixel before the fragment that would bring its transmittance
// below 1e-4; the backward walks the list in reverse from each pixel's last contributor and
// scatters per-splat gradients with one transposed warp reduction and one atomic per value.
#include <algorithm>
#include <map>
#include <mutex>
#include <utility>

#include "blend_warp.cuh"

namespace tgs {
namespace {

template <int TILE, int PPT, bool COUNT, bool HITS>
__global__ void __launch_bounds__(TILE * TILE / PPT)
k_blend_fwd(const float4 *__restrict__ splats, const uint32_t *__restrict__ ids,
            const uint2 *__restrict__ ranges, const __grid_constant__ CamBatch cb,
            const __grid_constant__ PixPtrs px, float bg0, float bg1, float bg2,
            uint32_t *__restrict__ hits, uint32_t n_gauss) {
    __shared__ BlendSmemFor<TILE, PPT, COUNT> sm;
    const int gt = blockIdx.x;
    const int v = view_of_tile(cb, gt);
    const DevCam &cam = cb.c[v];
    const int lt = gt - cam.tile_offset;
    TilePixels<TILE, PPT> P;
    P.init(lt % cam.gx, lt / cam.gx, cam.W, cam.H);
    FwdState<PPT> S;
    if constexpr (PPT == 2 && !COUNT)
        tile_forward2<TILE, false, HITS>(sm, splats, ids, ranges[gt], P, S, nullptr, hits, (uint32_t)v * n_gauss);
    else
        tile_forward<TILE, PPT, COUNT, false, HITS>(sm, splats, ids, ranges[gt], P, S, nullptr, hits,
                                                    (uint32_t)v * n_gauss);
    const int HW = cam.W * cam.H;
    float *img = px.image[v];
    float *Tf = px.T_final[v];
    int32_t *ls = px.last[v];
    int32_t *ex = px.n_exam[v];
#pragma unroll
    for (int k = 0; k < PPT; k++) {
        if (!P.inside[k]) continue;
        const int pix = P.y[k] * cam.W + P.x[k];
        if (img) {
            img[pix] = S.Cr[k] + S.T[k] * bg0;
            img[HW + pix] = S.Cg[k] + S.T[k] * bg1;
            img[2 * HW + pix] = S.Cb[k] + S.T[k] * bg2;
        }
        if (Tf) Tf[pix] = S.T[k];
        if (ls) ls[pix] = S.last[k];
        if (ex) ex[pix] = S.exam[k];
        if (COUNT) {
            if (px.n_contrib[v]) px.n_contrib[v][pix] = S.contrib[k];
            if (px.n_eval[v]) px.n_eval[v][pix] = S.eval[k];
        }
    }
}

template <int TILE, int PPT, bool MOMENTS>
__global__ void __launch_bounds__(TILE * TILE / PPT)
k_blend_bwd(const float4 *__restrict__ splats, const uint32_t *__restrict__ ids,
            const uint2 *__restrict__ ranges, const __grid_constant__ CamBatch cb,
            const __grid_constant__ PixPtrs px, float bg0, float bg1, float bg2,
            float *__restrict__ sgrads) {
    __shared__ BlendSmem<TILE * TILE / PPT> sm;
    const int gt = blockIdx.x;
    const int v = view_of_tile(cb, gt);
    const DevCam &cam = cb.c[v];
    const int lt = gt - cam.tile_offset;
    TilePixels<TILE, PPT> P;
    P.init(lt % cam.gx, lt / cam.gx, cam.W, cam.H);
    const int HW = cam.W * cam.H;
    const float *d = px.dL[v];
    BwdInput<PPT> in;
#pragma unroll
    for (int k = 0; k < PPT; k++) {
        const int pix = P.y[k] * cam.W + P.x[k];
        const bool ok = P.inside[k];
        in.last[k] = ok ? px.last[v][pix] : 0;
        in.Tfin[k] = ok ? px.T_final[v][pix] : 1.f;
        in.dR[k] = ok ? d[pix] : 0.f;
        in.dG[k] = ok ? d[HW + pix] : 0.f;
        in.dB[k] = ok ? d[2 * HW + pix] : 0.f;
    }
    tile_backward<TILE, PPT, MOMENTS>(sm, splats, ids, ranges[gt], P, in, bg0, bg1, bg2, sgrads);
}

// Warp items at 32 x 32 tiles and 2 pixels per thread (blend_warp.cuh). Without an item
// order, CTA b takes 4 of the 16 blocks of tile b / 4, one per warp, so that the warps reading
// one tile's records share L1. With one (order: tiles heaviest first, counter: zero before the
// launch), a persistent grid takes (tile, block) items from the counter in that order.
constexpr int kWarpCta = 128;

// The next item of this warp: false when there is none.
__device__ __forceinline__ bool next_warp_item(const uint32_t *__restrict__ order, int *__restrict__ counter,
                                               int n_tiles, bool first, int &gt, int &blk) {
    if (!counter) {  // one item per warp
        if (!first) return false;
        gt = blockIdx.x / (kWBlocks / (kWarpCta / 32));
        blk = (blockIdx.x % (kWBlocks / (kWarpCta / 32))) * (kWarpCta / 32) + (threadIdx.x >> 5);
        return true;
    }
    int it = 0;
    if ((threadIdx.x & 31) == 0) it = atomicAdd(counter, 1);
    it = __shfl_sync(0xffffffffu, it, 0);
    if (it >= n_tiles * kWBlocks) return false;
    gt = (int)order[it / kWBlocks];
    blk = it % kWBlocks;
    return true;
}

template <bool HITS>
__global__ void __launch_bounds__(kWarpCta)
k_blend_fwd_warp(const float4 *__restrict__ splats, const uint32_t *__restrict__ ids,
                 const uint2 *__restrict__ ranges, const __grid_constant__ CamBatch cb,
                 const __grid_constant__ PixPtrs px, float bg0, float bg1, float bg2,
                 uint32_t *__restrict__ hits, uint32_t n_gauss, const uint32_t *__restrict__ order,
                 int *__restrict__ counter) {
    __shared__ WarpSlots s_slots[kWarpCta / 32];
    const int w = threadIdx.x >> 5;
    int gt = 0, blk = 0;
    for (bool first = true; next_warp_item(order, counter, cb.total_tiles, first, gt, blk); first = false) {
        const int v = view_of_tile(cb, gt);
        const DevCam &cam = cb.c[v];
        WarpPixels P;
        P.init(cam, gt - cam.tile_offset, blk);
        float T[2], Cr[2], Cg[2], Cb[2];
        int last[2], exam[2];
        warp_forward<HITS, true>(s_slots[w].f, splats, ids, ranges[gt], P, T, Cr, Cg, Cb, last, exam, hits,
                                 (uint32_t)v * n_gauss);
        const int HW = cam.W * cam.H;
        float *img = px.image[v];
        float *Tf = px.T_final[v];
        int32_t *ls = px.last[v];
        int32_t *ex = px.n_exam[v];
#pragma unroll
        for (int k = 0; k < 2; k++) {
            if (!(k == 0 ? P.in0 : P.in1)) continue;
            const int pix = (k == 0 ? P.y0 : P.y1) * cam.W + P.x;
            if (img) {
                img[pix] = Cr[k] + T[k] * bg0;
                img[HW + pix] = Cg[k] + T[k] * bg1;
                img[2 * HW + pix] = Cb[k] + T[k] * bg2;
            }
            if (Tf) Tf[pix] = T[k];
            if (ls) ls[pix] = last[k];
            if (ex) ex[pix] = exam[k];
        }
    }
}

template <bool MOMENTS, bool BG>
__global__ void __launch_bounds__(kWarpCta)
k_blend_bwd_warp(const float4 *__restrict__ splats, const uint32_t *__restrict__ ids,
                 const uint2 *__restrict__ ranges, const __grid_constant__ CamBatch cb,
                 const __grid_constant__ PixPtrs px, float bg0, float bg1, float bg2,
                 float *__restrict__ sgrads, const uint32_t *__restrict__ order, int *__restrict__ counter) {
    __shared__ WarpSlots s_slots[kWarpCta / 32];
    const int w = threadIdx.x >> 5;
    int gt = 0, blk = 0;
    for (bool first = true; next_warp_item(order, counter, cb.total_tiles, first, gt, blk); first = false) {
        const int v = view_of_tile(cb, gt);
        const DevCam &cam = cb.c[v];
        WarpPixels P;
        P.init(cam, gt - cam.tile_offset, blk);
        const int HW = cam.W * cam.H;
        const float *d = px.dL[v];
        int last[2];
        float Tf[2], dR[2], dG[2], dB[2];
#pragma unroll
        for (int k = 0; k < 2; k++) {
            const bool ok = k == 0 ? P.in0 : P.in1;
            const int pix = (k == 0 ? P.y0 : P.y1) * cam.W + P.x;
            last[k] = ok ? px.last[v][pix] : 0;
            Tf[k] = ok ? px.T_final[v][pix] : 1.f;
            dR[k] = ok ? d[pix] : 0.f;
            dG[k] = ok ? d[HW + pix] : 0.f;
            dB[k] = ok ? d[2 * HW + pix] : 0.f;
        }
        warp_backward<MOMENTS, BG>(s_slots[w].b, splats, ids, ranges[gt], P, last, Tf, dR, dG, dB, bg0, bg1, bg2, sgrads);
    }
}

// Grid of a warp-item launch: one CTA per 4 blocks without a counter, else a persistent grid of
// SMs x resident CTAs (found once per device and kernel), capped by the items.
template <class K>
unsigned warp_grid(K kernel, const CamBatch &cb, bool persistent) {
    const unsigned one = (unsigned)cb.total_tiles * (kWBlocks / (kWarpCta / 32));
    if (!persistent) return one;
    static std::mutex mu;
    static std::map<std::pair<int, const void *>, int> grid_of;  // (device, kernel) -> grid
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        dev = 0;
    }
    const auto key = std::make_pair(dev, reinterpret_cast<const void *>(kernel));
    std::lock_guard<std::mutex> lock(mu);
    auto it = grid_of.find(key);
    if (it == grid_of.end()) {
        int sms = 1, b = 0;
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1) {
            cudaGetLastError();
            sms = 1;
        }
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, kernel, kWarpCta, 0) != cudaSuccess) {
            cudaGetLastError();
            b = 1;
        }
        it = grid_of.emplace(key, sms * (b < 1 ? 1 : b)).first;
    }
    return std::min(one, (unsigned)it->second);
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
                const PixPtrs &px, const float *bg, uint32_t *hits, int64_t n_gauss, const uint32_t *order,
                int *counter, cudaStream_t st) {
    bool count = false;
    for (int v = 0; v < cb.V; v++) count = count || px.n_contrib[v] || px.n_eval[v];
    const uint32_t n = (uint32_t)n_gauss;
    count_launch();
    if (TILE == 32 && PPT == 2 && !count) {
        const bool pers = order && counter;
        if (!pers) order = nullptr, counter = nullptr;
        if (hits)
            k_blend_fwd_warp<true><<<warp_grid(k_blend_fwd_warp<true>, cb, pers), kWarpCta, 0, st>>>(
                splats, ids, ranges, cb, px, bg[0], bg[1], bg[2], hits, n, order, counter);
        else
            k_blend_fwd_warp<false><<<warp_grid(k_blend_fwd_warp<false>, cb, pers), kWarpCta, 0, st>>>(
                splats, ids, ranges, cb, px, bg[0], bg[1], bg[2], hits, n, order, counter);
        return;
    }
#define TGS_FWD(C, HT)                                                                                 \
    k_blend_fwd<TILE, PPT, C, HT><<<cb.total_tiles, TILE * TILE / PPT, 0, st>>>(splats, ids, ranges, cb, px, \
                                                                               bg[0], bg[1], bg[2], hits, n)
    if (count && hits) TGS_FWD(true, true);
    else if (count) TGS_FWD(true, false);
    else if (hits) TGS_FWD(false, true);
    else TGS_FWD(false, false);
#undef TGS_FWD
}

template <int TILE, int PPT, bool MOMENTS>
void bwd_launch_t(const float4 *splats, const uint32_t *ids, const uint2 *ranges, const CamBatch &cb,
                  const PixPtrs &px, const float *bg, float *sg, const uint32_t *order, int *counter,
                  cudaStream_t st) {
    count_launch();
    if (TILE == 32 && PPT == 2) {
        const bool pers = order && counter;
        if (!pers) order = nullptr, counter = nullptr;
        if (bg[0] != 0.f || bg[1] != 0.f || bg[2] != 0.f)
            k_blend_bwd_warp<MOMENTS, true><<<warp_grid(k_blend_bwd_warp<MOMENTS, true>, cb, pers), kWarpCta, 0, st>>>(
                splats, ids, ranges, cb, px, bg[0], bg[1], bg[2], sg, order, counter);
        else
            k_blend_bwd_warp<MOMENTS, false><<<warp_grid(k_blend_bwd_warp<MOMENTS, false>, cb, pers), kWarpCta, 0,
                                                st>>>(splats, ids, ranges, cb, px, bg[0], bg[1], bg[2], sg, order,
                                                      counter);
        return;
    }
    k_blend_bwd<TILE, PPT, MOMENTS><<<cb.total_tiles, TILE * TILE / PPT, 0, st>>>(splats, ids, ranges, cb, px,
                                                                                  bg[0], bg[1], bg[2], sg);
}

template <int TILE, int PPT>
void bwd_launch(const float4 *splats, const uint32_t *ids, const uint2 *ranges, const CamBatch &cb,
                const PixPtrs &px, const float *bg, float *sg, const uint32_t *order, int *counter, int moments,
                cudaStream_t st) {
    if (moments) bwd_launch_t<TILE, PPT, true>(splats, ids, ranges, cb, px, bg, sg, order, counter, st);
    else bwd_launch_t<TILE, PPT, false>(splats, ids, ranges, cb, px, bg, sg, order, counter, st);
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
                          const float *bg, cudaStream_t st, uint32_t *hits, int64_t n_gauss,
                          const uint32_t *order, int *counter) {
    if (cb.total_tiles <= 0) return;
    TGS_DISPATCH(fwd_launch, splats, ids, ranges, cb, px, bg, hits, n_gauss, order, counter, st);
}

void launch_blend_backward(int tile, int ppt, const float4 *splats, const uint32_t *ids,
                           const uint2 *ranges, const CamBatch &cb, const PixPtrs &px,
                           const float *bg, float *sgrads, cudaStream_t st, const uint32_t *order,
                           int *counter, int moments) {
    if (cb.total_tiles <= 0) return;
    TGS_DISPATCH(bwd_launch, splats, ids, ranges, cb, px, bg, sgrads, order, counter, moments, st);
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
