// Front-to-back alpha blending (Eq. 2 of the paper) and its backward, one CTA per (view,
// tile). The per-tile work lives in blend_common.cuh (shared with the fused kernel): the
// tile's depth-sorted list is streamed through shared memory in batches of one splat per
// thread; the forward stops a pixel before the fragment that would bring its transmittance
// below 1e-4; the backward walks the list in reverse from each pixel's last contributor and
// scatters per-splat gradients with one transposed warp reduction and one atomic per value.
#include "blend_common.cuh"

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

template <int TILE, int PPT>
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
    tile_backward<TILE, PPT>(sm, splats, ids, ranges[gt], P, in, bg0, bg1, bg2, sgrads);
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
                const PixPtrs &px, const float *bg, uint32_t *hits, int64_t n_gauss, cudaStream_t st) {
    bool count = false;
    for (int v = 0; v < cb.V; v++) count = count || px.n_contrib[v] || px.n_eval[v];
    const uint32_t n = (uint32_t)n_gauss;
    count_launch();
#define TGS_FWD(C, HT)                                                                                 \
    k_blend_fwd<TILE, PPT, C, HT><<<cb.total_tiles, TILE * TILE / PPT, 0, st>>>(splats, ids, ranges, cb, px, \
                                                                               bg[0], bg[1], bg[2], hits, n)
    if (count && hits) TGS_FWD(true, true);
    else if (count) TGS_FWD(true, false);
    else if (hits) TGS_FWD(false, true);
    else TGS_FWD(false, false);
#undef TGS_FWD
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
                          const float *bg, cudaStream_t st, uint32_t *hits, int64_t n_gauss) {
    if (cb.total_tiles <= 0) return;
    TGS_DISPATCH(fwd_launch, splats, ids, ranges, cb, px, bg, hits, n_gauss, st);
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
