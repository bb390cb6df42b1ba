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

#include "blend_warp.cuh"

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

// ---- warp items (blend_warp.cuh): one 8 x 8 block of a 32 x 32 tile per warp --------------

constexpr int kWarpItemThreads = 128;

template <bool HITS, bool BG>
__global__ void __launch_bounds__(kWarpItemThreads)
k_fused_warp(const float4 *__restrict__ splats, const uint32_t *__restrict__ ids,
             const uint2 *__restrict__ ranges, const uint32_t *__restrict__ order, int n_items,
             int *__restrict__ counter, const __grid_constant__ CamBatch cb,
             const __grid_constant__ PixPtrs px, float bg0, float bg1, float bg2,
             float *__restrict__ sgrads, float *__restrict__ loss, uint32_t *__restrict__ hits, uint32_t n_gauss) {
    __shared__ WarpSlots s_slots[kWarpItemThreads / 32];
    const unsigned full = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    WarpSlots &sm = s_slots[threadIdx.x >> 5];
    float loss_acc = 0.f;  // this warp's share of the loss over all its items
    for (;;) {
        int it = 0;
        if (lane == 0) it = atomicAdd(counter, 1);
        it = __shfl_sync(full, it, 0);
        if (it >= n_items * kWBlocks) break;
        const int gt = (int)order[it / kWBlocks];
        const int v = view_of_tile(cb, gt);
        const DevCam &cam = cb.c[v];
        WarpPixels P;
        P.init(cam, gt - cam.tile_offset, it % kWBlocks);
        const uint2 rg = ranges[gt];
        float Tf[2], Cr[2], Cg[2], Cb[2];
        int last[2], exam[2];
        warp_forward<HITS, false>(sm.f, splats, ids, rg, P, Tf, Cr, Cg, Cb, last, exam, hits, (uint32_t)v * n_gauss);

        // L1 loss: L = mean over views of mean over 3HW |C - target|; dL/dC = sign / (3HWV)
        const int HW = cam.W * cam.H;
        const float scale = 1.f / (3.f * (float)HW * (float)cb.V);
        const float *tg = px.target[v];
        float *img = px.image[v];
        float dR[2] = {0.f, 0.f}, dG[2] = {0.f, 0.f}, dB[2] = {0.f, 0.f};
        float lsum = 0.f;
#pragma unroll
        for (int k = 0; k < 2; k++) {
            if (!(k == 0 ? P.in0 : P.in1)) continue;
            const int pix = (k == 0 ? P.y0 : P.y1) * cam.W + P.x;
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
        warp_backward<true, BG>(sm.b, splats, ids, rg, P, last, Tf, dR, dG, dB, bg0, bg1, bg2, sgrads);
    }
    if (lane == 0 && loss) atomicAdd(loss, loss_acc);
}

template <bool HITS, bool BG>
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
            if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_fused_warp<HITS, BG>, kWarpItemThreads, 0) !=
                cudaSuccess) {
                cudaGetLastError();
                b = 1;
            }
            grid = sms * (b < 1 ? 1 : b);
            if (dev >= 0 && dev < kDevices) grid_of[dev] = grid;
        }
    }
    const int64_t warps = (int64_t)cb.total_tiles * kWBlocks;
    if ((int64_t)grid * (kWarpItemThreads / 32) > warps) grid = (int)((warps + 3) / 4);
    if (grid < 1) grid = 1;
    count_launch();
    k_fused_warp<HITS, BG><<<grid, kWarpItemThreads, 0, st>>>(splats, ids, ranges, order, cb.total_tiles, counter, cb, px,
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
        const bool nzbg = bg[0] != 0.f || bg[1] != 0.f || bg[2] != 0.f;
        if (hits && nzbg) warp_launch_t<true, true>(splats, ids, ranges, order, counter, cb, px, bg, sgrads, loss, hits, n, st);
        else if (hits) warp_launch_t<true, false>(splats, ids, ranges, order, counter, cb, px, bg, sgrads, loss, hits, n, st);
        else if (nzbg) warp_launch_t<false, true>(splats, ids, ranges, order, counter, cb, px, bg, sgrads, loss, hits, n, st);
        else warp_launch_t<false, false>(splats, ids, ranges, order, counter, cb, px, bg, sgrads, loss, hits, n, st);
    }
    else if (tile == 32 && ppt == 2) fused_launch<32, 2>(batch, splats, ids, ranges, order, counter, cb, px, bg, sgrads, loss, vis_keys, hits, n, st);
    else if (tile == 32 && ppt == 4) fused_launch<32, 4>(batch, splats, ids, ranges, order, counter, cb, px, bg, sgrads, loss, vis_keys, hits, n, st);
}

}  // namespace tgs
