// Internal declarations shared by the libtgs translation units (device structs, launch
// helpers). Not part of the public ABI (see include/tgs.h).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "tgs.h"

namespace tgs {

constexpr int kMaxViews = TGS_MAX_VIEWS;
constexpr float kLog2e = 1.4426950408889634f;
constexpr float kLn2 = 0.6931471805599453f;
constexpr float kAlphaMin = 1.0f / 255.0f;
constexpr float kAlphaMax = 0.99f;
constexpr float kTMin = 1e-4f;

// One view as the kernels see it (passed by value inside CamBatch).
struct DevCam {
    float R[9];       // world -> camera rotation, row-major
    float t[3];       // world -> camera translation
    float campos[3];  // camera centre
    float fx, fy, cx, cy;
    float limx, limy; // 1.3 * W / (2 fx), 1.3 * H / (2 fy)
    float s;          // low-pass term of Sigma' + sI
    int W, H;
    int gx, gy;       // tiles per row / column
    int tile_offset;  // first global tile id of this view
    int pix_offset;   // first global pixel of this view (batched loss reduction)
};

struct CamBatch {
    int V;
    int total_tiles;
    int tile;
    int n_over_v;     // unused padding
    DevCam c[kMaxViews];
};

struct GaussPtrs {
    const float *means, *log_scales, *quats, *opac, *sh_dc, *sh_rest;
    const uint8_t *sh_degree;
    const float *mask, *shmask;
    int64_t n;
    int deg_max;
    float tau_m, tau_sh;   // thresholds on the logits
    int support;
    float near_z;
    int half;              // parameters stored as IEEE half (render path only)
};

struct GradPtrs {
    float *means, *log_scales, *quats, *opac, *sh_dc, *sh_rest, *mask, *shmask;
    float *stat_accum;
    int32_t *stat_count, *stat_maxr;
    int accumulate;
    // mask losses of Eq. loss3dgs folded into the mask-logit gradients (0: none): lambda_m / N
    // and lambda_sh / N
    float lam_m_n, lam_sh_n;
};

struct PixPtrs {
    float *image[kMaxViews];
    float *T_final[kMaxViews];
    int32_t *last[kMaxViews];
    int32_t *n_exam[kMaxViews];
    const float *dL[kMaxViews];
    const float *target[kMaxViews];
    int32_t *n_contrib[kMaxViews];
    int32_t *n_eval[kMaxViews];
};

// Kernel launches issued by the library on this host thread (the batched step counts its own).
extern thread_local int64_t g_launches;
inline void count_launch(int k = 1) { g_launches += k; }

// Device status word bits.
constexpr uint32_t kNoDepth = 0xffffffffu;  // depth key of a record that is not visible
constexpr uint32_t kStatusCapacity = 1u;
constexpr uint32_t kStatusInconsistent = 2u;  // a consistency check of scratch data failed

__device__ __forceinline__ int view_of_tile(const CamBatch &cb, int gt) {
    int lo = 0, hi = cb.V - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (cb.c[mid].tile_offset <= gt) lo = mid; else hi = mid - 1;
    }
    return lo;
}

__device__ __forceinline__ float ex2_approx(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Words per splat record (see include/tgs.h): 12 used by the blend + the cull threshold.
constexpr int kSplatWords = 16;
// Margin of the tile cull test: a (Gaussian, tile) key is dropped only when every pixel of the
// tile stays below (1 - kCullMargin) / 255 in exact arithmetic.
constexpr float kCullMargin = 1e-3f;

// Minimum over the pixel-centre rectangle [x0, x1] x [y0, y1] of the quadratic form
// Q(p) = (p - m)^T [[a, b], [b, c]] (p - m) of a splat, compared with its threshold tau:
// true when some point of the rectangle has Q <= tau (the tile may hold a pixel with
// alpha >= 1/255), false when none has. Every operation is an explicitly rounded float32
// operation in a fixed order, so any IEEE binary32 implementation of the same steps agrees
// bit for bit.
__device__ __forceinline__ float cull_quad(float a, float b, float c, float dx, float dy) {
    const float q1 = __fmul_rn(__fmul_rn(a, dx), dx);
    const float q2 = __fmul_rn(__fmul_rn(__fmul_rn(2.f, b), dx), dy);
    const float q3 = __fmul_rn(__fmul_rn(c, dy), dy);
    return __fadd_rn(__fadd_rn(q1, q2), q3);
}
__device__ __forceinline__ bool tile_keep(float mx, float my, float a, float b, float c, float tau,
                                          float b_over_c, float b_over_a, int x0, int x1, int y0,
                                          int y1) {
    const float fx0 = (float)x0, fx1 = (float)x1, fy0 = (float)y0, fy1 = (float)y1;
    if (mx >= fx0 && mx <= fx1 && my >= fy0 && my <= fy1) return 0.f <= tau;
    float q = __int_as_float(0x7f800000);  // +inf
    // the minimum lies on an edge facing the centre; on a vertical edge x = xe it is at
    // y = my - (b / c) (xe - mx) clamped to the edge, on a horizontal edge symmetrically
    // (b / c and b / a are stored in the record)
    if (mx < fx0 || mx > fx1) {
        const float xe = mx < fx0 ? fx0 : fx1;
        const float dx = __fsub_rn(xe, mx);
        const float ys = __fsub_rn(my, __fmul_rn(b_over_c, dx));
        const float dy = __fsub_rn(fminf(fmaxf(ys, fy0), fy1), my);
        q = fminf(q, cull_quad(a, b, c, dx, dy));
    }
    if (my < fy0 || my > fy1) {
        const float ye = my < fy0 ? fy0 : fy1;
        const float dy = __fsub_rn(ye, my);
        const float xs = __fsub_rn(mx, __fmul_rn(b_over_a, dy));
        const float dx = __fsub_rn(fminf(fmaxf(xs, fx0), fx1), mx);
        q = fminf(q, cull_quad(a, b, c, dx, dy));
    }
    return q <= tau;
}

// tile_keep without branches: the same steps, both edge candidates always evaluated and
// selected, so the result is the same bit for bit. Cheaper where the lanes of a warp take
// different cases (the blend's per-block tests); the key count keeps the branches (measured
// faster there).
__device__ __forceinline__ bool tile_keep_flat(float mx, float my, float a, float b, float c, float tau,
                                               float b_over_c, float b_over_a, int x0, int x1, int y0,
                                               int y1) {
    const float fx0 = (float)x0, fx1 = (float)x1, fy0 = (float)y0, fy1 = (float)y1;
    const bool xin = mx >= fx0 && mx <= fx1, yin = my >= fy0 && my <= fy1;
    const float xe = mx < fx0 ? fx0 : fx1;
    const float dx1 = __fsub_rn(xe, mx);
    const float ys = __fsub_rn(my, __fmul_rn(b_over_c, dx1));
    const float dy1 = __fsub_rn(fminf(fmaxf(ys, fy0), fy1), my);
    const float q1 = cull_quad(a, b, c, dx1, dy1);
    const float ye = my < fy0 ? fy0 : fy1;
    const float dy2 = __fsub_rn(ye, my);
    const float xs = __fsub_rn(mx, __fmul_rn(b_over_a, dy2));
    const float dx2 = __fsub_rn(fminf(fmaxf(xs, fx0), fx1), mx);
    const float q2 = cull_quad(a, b, c, dx2, dy2);
    const float inf = __int_as_float(0x7f800000);
    float q = fminf(fminf(inf, xin ? inf : q1), yin ? inf : q2);
    if (xin && yin) q = 0.f;
    return q <= tau;
}

// ---- launchers implemented in the .cu files --------------------------------------------

// preprocess.cu: lambda_m L_m + lambda_sh L_sh (Eq. loss3dgs) over n Gaussians added to *loss
// (if not null) and their gradients added to gmask / gshmask (if not null)
void launch_mask_loss(const float *mask, const float *shmask, int64_t n, float lam_m, float lam_sh, float *loss,
                      float *gmask, float *gshmask, cudaStream_t st);
// preprocess.cu. depth_bits [n*V]: the depth key of every record (kNoDepth where not
// visible); tiles_touched (may be null): visibility flags.
void launch_preprocess(const GaussPtrs &g, const CamBatch &cb, float4 *splats, int32_t *radii,
                       uint32_t *tiles_touched, uint32_t *depth_bits, float *zero_grads,
                       cudaStream_t st);
// moments != 0: the gradient records hold the pixel sums of the fused blend backward
void launch_preprocess_backward(const GaussPtrs &g, const CamBatch &cb, const float4 *sgrads,
                                const int32_t *radii, const GradPtrs &out, int no_sh_rest,
                                int moments, cudaStream_t st);

// sort.cu
struct SortScratch {
    uint32_t *hist;       // 256 * max_blocks
    uint32_t *partials;   // scan partial sums
    int64_t max_items;
};
size_t scan_partials_needed(int64_t n_items);
size_t radix_hist_needed(int64_t n_items);
// Stable LSD sort of (keys, vals) on bits [begin_bit, end_bit); on return keys/vals point to
// the sorted arrays (one of the two buffer pairs). index_vals: the input values are the items'
// positions (vals is then only written).
void radix_sort_pairs(uint32_t *&keys, uint32_t *&vals, uint32_t *keys_alt, uint32_t *vals_alt,
                      const uint32_t *n_dev, int64_t n_cap, int begin_bit, int end_bit,
                      uint32_t *hist, uint32_t *partials, cudaStream_t st, bool index_vals = false);
// Per depth-sorted record (arrays of n_cap, in depth order): number of kept tiles, kept-tile
// mask (rects of at most 64 tiles), packed pixel rect x and y.
struct KeyInfo {
    uint32_t *cnt;
    uint2 *km;
    uint32_t *rx, *ry;
};
// Culls the rect tiles of each depth-sorted record and counts its keys (KeyInfo); per block of
// 2048 records the exclusive start of its keys (block_offsets, scan_partials_needed(n_cap)
// words) and the total in *total.
void count_keys(const uint32_t *sorted_ids, const uint32_t *sorted_keys, const uint32_t *n_dev, int64_t n_cap,
                const float4 *splats, int tile, const KeyInfo &ki, uint32_t *block_offsets, uint32_t *total,
                cudaStream_t st);
void emit_keys(const uint32_t *sorted_ids, const uint32_t *block_offsets, const uint32_t *n_dev,
               int64_t n_cap, const KeyInfo &ki, const float4 *splats, int64_t n_gauss, const CamBatch &cb,
               uint32_t *tile_keys, uint32_t *tile_vals, const uint32_t *K_dev, int64_t key_capacity,
               uint32_t *status, cudaStream_t st);
void find_ranges(const uint32_t *tile_keys, const uint32_t *K_dev, int64_t key_capacity,
                 uint2 *ranges, int total_tiles, cudaStream_t st);
// Depth keys (and, if tiles_touched is not null, visibility flags) of splat records given
// from outside, as the preprocess writes them.
void derive_touched(const float4 *splats, const int32_t *radii, int64_t n_rec, int tile,
                    uint32_t *tiles_touched, uint32_t *depth_bits, cudaStream_t st);
void make_full_keys(const uint32_t *tile_keys, const uint32_t *tile_vals, const float4 *splats,
                    const uint32_t *K_dev, int64_t cap, uint64_t *out, cudaStream_t st);

// blend.cu
int blend_supported(int tile, int ppt);
// hits (may be null): per-Gaussian ray hits added in (Eq. significance-score); record r of
// view v is Gaussian r - v n_gauss
// order / counter (both or neither): tiles heaviest first (build_item_order) and a zeroed item
// counter; at tile 32 / 2 px per thread the warp-item kernels then run a persistent grid in
// that order (other configurations ignore them)
void launch_blend_forward(int tile, int ppt, const float4 *splats, const uint32_t *ids,
                          const uint2 *ranges, const CamBatch &cb, const PixPtrs &px,
                          const float *bg, cudaStream_t st, uint32_t *hits = nullptr,
                          int64_t n_gauss = 0, const uint32_t *order = nullptr, int *counter = nullptr);
// moments != 0: the records receive the pixel sums of the fused step's backward (see
// tile_backward) instead of the splat gradients, for launch_preprocess_backward(moments = 1)
void launch_blend_backward(int tile, int ppt, const float4 *splats, const uint32_t *ids,
                           const uint2 *ranges, const CamBatch &cb, const PixPtrs &px,
                           const float *bg, float *sgrads, cudaStream_t st, const uint32_t *order = nullptr,
                           int *counter = nullptr, int moments = 0);
void launch_l1(const float *img, const float *tgt, int64_t count, float scale, float *loss,
               float *grad, cudaStream_t st);

// fused.cu
void build_item_order(const uint2 *ranges, int total_tiles, uint32_t *k0, uint32_t *v0, uint32_t *k1,
                      uint32_t *v1, uint32_t **order, uint32_t *hist, uint32_t *partials, cudaStream_t st);
// vis_keys: scratch of one uint16 per key (key capacity): the forward's per-warp visibility
// masks of each list entry, read back by the backward
void launch_fused_l1(int tile, int ppt, int batch, const float4 *splats, const uint32_t *ids, const uint2 *ranges,
                     const uint32_t *order, int *counter, const CamBatch &cb, const PixPtrs &px,
                     const float *bg, float *sgrads, float *loss, uint16_t *vis_keys, cudaStream_t st,
                     uint32_t *hits = nullptr, int64_t n_gauss = 0);

// ssim.cu (Eq. loss3dgs): loss += mean over views of (1 - lam) mean |x - y| + lam (1 - mean
// SSIM), grad[v] = dL/dx[v]; scratch: ssim_scratch_floats floats
int64_t ssim_scratch_floats(const int *W, const int *H, int V);
void launch_l1_dssim(int V, const int *W, const int *H, const float *const *x, const float *const *y,
                     float *const *grad, float lam, float *scratch, float *loss, cudaStream_t st);

// half.cu: float32 -> IEEE half, round to nearest even (n values)
void launch_to_half(const float *src, uint16_t *dst, int64_t n, cudaStream_t st);

// compact.cu: kept Gaussians (not removed, and M = 1 if masked) copied in order; block_counts:
// compact_blocks(n) + 1 words of scratch, the last one receiving the number kept
int64_t compact_blocks(int64_t n);
void launch_compact(const GaussPtrs &g, const uint8_t *remove, bool masked, const GradPtrs &out, uint8_t *deg_out,
                    uint32_t *kept_index, uint32_t *block_counts, uint32_t *total, cudaStream_t st);

// compact.cu: densification by clone and split (3DGS's rule as stated in include/tgs.h).
struct DensifyArgs {
    const float *accum;      // [n] summed per-view |dL/d mean2d| (pixels)
    const int32_t *count;    // [n] views where visible
    const float *normals;    // [n,2,3] standard normals of the caller
    float tau_g;             // threshold on accum / count
    float tau_ls;            // float32(log(scale threshold)) on the largest log-scale
};
constexpr float kLogSplitDivisor = 0.47000362924573558f;  // log(1.6): children's scales / (0.8 x 2)
// copy == false: per-block counts of (not split, clones, splits) and their scans into scratch
// (3 (compact_blocks(n) + 1) words) with the totals in totals[0..2]; copy == true: the rows.
void launch_densify(const GaussPtrs &g, const DensifyArgs &d, const GradPtrs &out, uint8_t *deg_out,
                    uint32_t *src_index, uint32_t *scratch, uint32_t *totals, bool copy, cudaStream_t st);

// significance.cu (Eq. significance-score)
void launch_volumes(const GaussPtrs &g, float *vol, uint32_t *keys, cudaStream_t st);
void launch_scores(const GaussPtrs &g, const uint32_t *hits, const float *vol, const uint32_t *sorted_vol_bits,
                   int64_t q_rank, float *scores, cudaStream_t st);
void launch_score_keys(const float *scores, int64_t n, uint32_t *keys, cudaStream_t st);
void launch_mark(const uint32_t *sorted_idx, int64_t k, uint8_t *prune, cudaStream_t st);

}  // namespace tgs
