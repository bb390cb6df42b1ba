// Significance pruning (Eq. significance-score of the paper): the score of each Gaussian from
// its ray hits (counted in the forward blend, blend_common.cuh), opacity and volume, and the
// selection of the Gaussians a pruning round removes.
//
// GS_j = hits_j * alpha_j * gamma_j with alpha_j = M_j sigmoid(o_j) (the opacity the blend
// uses) and gamma_j = min(V_j / V_q, 1): V_j = s_x s_y s_z with the masked scales M exp(l),
// V_q the volume at rank floor(q (n - 1)) of all volumes sorted ascending (the paper's
// normalisation by the volume at the 90 % point of the sorted volumes, q = 0.9), gamma = 1
// where V_q = 0.
#include "tgs_internal.cuh"

namespace tgs {
namespace {

__device__ __forceinline__ float mask_of(const GaussPtrs &g, int64_t i) {
    return (g.mask && !(g.mask[i] > g.tau_m)) ? 0.f : 1.f;
}

// Volume of each Gaussian, and its float bits as sort key (volumes are >= 0, so the bits
// order like the values).
__global__ void k_volumes(GaussPtrs g, float *__restrict__ vol, uint32_t *__restrict__ keys) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= g.n) return;
    const float M = mask_of(g, i);
    const float v = (M * expf(g.log_scales[3 * i])) * (M * expf(g.log_scales[3 * i + 1])) *
                    (M * expf(g.log_scales[3 * i + 2]));
    vol[i] = v;
    keys[i] = __float_as_uint(v);
}

__global__ void k_scores(GaussPtrs g, const uint32_t *__restrict__ hits, const float *__restrict__ vol,
                         const uint32_t *__restrict__ sorted_vol_bits, int64_t q_rank,
                         float *__restrict__ scores) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= g.n) return;
    const float vq = __uint_as_float(sorted_vol_bits[q_rank]);
    const float opac = mask_of(g, i) * (1.f / (1.f + expf(-g.opac[i])));
    const float gamma = vq > 0.f ? fminf(vol[i] / vq, 1.f) : 1.f;
    scores[i] = (float)hits[i] * opac * gamma;
}

__global__ void k_score_keys(const float *__restrict__ scores, int64_t n, uint32_t *__restrict__ keys) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) keys[i] = __float_as_uint(scores[i]);   // scores >= 0: bits order like values
}

__global__ void k_mark(const uint32_t *__restrict__ sorted_idx, int64_t k, uint8_t *__restrict__ prune) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < k) prune[sorted_idx[i]] = 1u;
}

inline unsigned blocks(int64_t n) { return (unsigned)((n + 255) / 256); }

}  // namespace

void launch_volumes(const GaussPtrs &g, float *vol, uint32_t *keys, cudaStream_t st) {
    if (g.n <= 0) return;
    count_launch();
    k_volumes<<<blocks(g.n), 256, 0, st>>>(g, vol, keys);
}

void launch_scores(const GaussPtrs &g, const uint32_t *hits, const float *vol, const uint32_t *sorted_vol_bits,
                   int64_t q_rank, float *scores, cudaStream_t st) {
    if (g.n <= 0) return;
    count_launch();
    k_scores<<<blocks(g.n), 256, 0, st>>>(g, hits, vol, sorted_vol_bits, q_rank, scores);
}

void launch_score_keys(const float *scores, int64_t n, uint32_t *keys, cudaStream_t st) {
    if (n <= 0) return;
    count_launch();
    k_score_keys<<<blocks(n), 256, 0, st>>>(scores, n, keys);
}

void launch_mark(const uint32_t *sorted_idx, int64_t k, uint8_t *prune, cudaStream_t st) {
    if (k <= 0) return;
    count_launch();
    k_mark<<<blocks(k), 256, 0, st>>>(sorted_idx, k, prune);
}

}  // namespace tgs
