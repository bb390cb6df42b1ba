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
};

struct GradPtrs {
    float *means, *log_scales, *quats, *opac, *sh_dc, *sh_rest, *mask, *shmask;
    float *stat_accum;
    int32_t *stat_count, *stat_maxr;
    int accumulate;
};

struct PixPtrs {
    float *image[kMaxViews];
    float *T_final[kMaxViews];
    int32_t *last[kMaxViews];
    int32_t *n_exam[kMaxViews];
    const float *dL[kMaxViews];
    const float *target[kMaxViews];
};

// Kernel launches issued by the library on this host thread (the batched step counts its own).
extern thread_local int64_t g_launches;
inline void count_launch(int k = 1) { g_launches += k; }

// Device status word bits.
constexpr uint32_t kStatusCapacity = 1u;
constexpr uint32_t kStatusTimeout = 2u;

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

// ---- launchers implemented in the .cu files --------------------------------------------

// preprocess.cu
void launch_preprocess(const GaussPtrs &g, const CamBatch &cb, float4 *splats, int32_t *radii,
                       uint32_t *tiles_touched, uint32_t *depth_bits, float *zero_grads,
                       cudaStream_t st);
void launch_preprocess_backward(const GaussPtrs &g, const CamBatch &cb, const float4 *sgrads,
                                const int32_t *radii, const GradPtrs &out, int no_sh_rest,
                                cudaStream_t st);

// sort.cu
struct SortScratch {
    uint32_t *hist;       // 256 * max_blocks
    uint32_t *partials;   // scan partial sums
    int64_t max_items;
};
size_t scan_partials_needed(int64_t n_items);
size_t radix_hist_needed(int64_t n_items);
// out[i] = exclusive prefix of in_fn(i) for i < *n_dev; *total = sum. n_cap bounds the grid.
void scan_flags(const uint32_t *tiles_touched, int64_t n_cap, uint32_t *out, uint32_t *total,
                uint32_t *partials, cudaStream_t st);
void compact_visible(const uint32_t *tiles_touched, const uint32_t *depth_bits,
                     const uint32_t *pos, int64_t n_cap, uint32_t *keys, uint32_t *vals,
                     cudaStream_t st);
void radix_sort_pairs(uint32_t *&keys, uint32_t *&vals, uint32_t *keys_alt, uint32_t *vals_alt,
                      const uint32_t *n_dev, int64_t n_cap, int begin_bit, int end_bit,
                      uint32_t *hist, uint32_t *partials, cudaStream_t st);
void gather_tiles_scan(const uint32_t *sorted_ids, const uint32_t *tiles_touched,
                       const uint32_t *n_dev, int64_t n_cap, uint32_t *offsets, uint32_t *total,
                       uint32_t *partials, uint32_t *tmp, cudaStream_t st);
void emit_keys(const uint32_t *sorted_ids, const uint32_t *offsets, const uint32_t *n_dev,
               int64_t n_cap, const float4 *splats, int64_t n_gauss, const CamBatch &cb,
               uint32_t *tile_keys, uint32_t *tile_vals, const uint32_t *K_dev,
               int64_t key_capacity, uint32_t *status, cudaStream_t st);
void find_ranges(const uint32_t *tile_keys, const uint32_t *K_dev, int64_t key_capacity,
                 uint2 *ranges, int total_tiles, cudaStream_t st);
void derive_touched(const float4 *splats, const int32_t *radii, int64_t n_rec, int tile,
                    uint32_t *tiles_touched, uint32_t *depth_bits, cudaStream_t st);
void make_full_keys(const uint32_t *tile_keys, const uint32_t *tile_vals, const float4 *splats,
                    const uint32_t *K_dev, int64_t cap, uint64_t *out, cudaStream_t st);

// blend.cu
int blend_supported(int tile, int ppt);
void launch_blend_forward(int tile, int ppt, const float4 *splats, const uint32_t *ids,
                          const uint2 *ranges, const CamBatch &cb, const PixPtrs &px,
                          const float *bg, cudaStream_t st);
void launch_blend_backward(int tile, int ppt, const float4 *splats, const uint32_t *ids,
                           const uint2 *ranges, const CamBatch &cb, const PixPtrs &px,
                           const float *bg, float *sgrads, cudaStream_t st);
void launch_l1(const float *img, const float *tgt, int64_t count, float scale, float *loss,
               float *grad, cudaStream_t st);

// fused.cu
void build_item_order(const uint2 *ranges, int total_tiles, uint32_t *k0, uint32_t *v0, uint32_t *k1,
                      uint32_t *v1, uint32_t **order, uint32_t *hist, uint32_t *partials, cudaStream_t st);
void launch_fused_l1(int tile, int ppt, const float4 *splats, const uint32_t *ids, const uint2 *ranges,
                     const uint32_t *order, int *counter, const CamBatch &cb, const PixPtrs &px,
                     const float *bg, float *sgrads, float *loss, cudaStream_t st);

}  // namespace tgs
