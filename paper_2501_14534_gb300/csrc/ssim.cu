// L1 + D-SSIM loss of Eq. loss3dgs (without the mask terms) and its gradient with respect to
// the rendered images, over a batch of views of any sizes.
//
// SSIM (Wang et al., with the settings 3DGS trains with): per channel, local means, variances
// and covariance under an 11 x 11 Gaussian window of sigma 1.5 (normalised, zero outside the
// image), S = (2 mu_x mu_y + C1)(2 sigma_xy + C2) / ((mu_x^2 + mu_y^2 + C1)(sigma_x^2 +
// sigma_y^2 + C2)), C1 = 0.01^2, C2 = 0.03^2; L = mean over views of
// (1 - lambda) mean |x - y| + lambda (1 - mean S).
//
// The 2D window is the outer product of two normalised 1D windows, so every window sum is two
// 1D passes (Sec. "Accelerated training": two 1D convolutions instead of the 11 x 11 one, the
// metric computed in one kernel from their outputs). Two kernels:
//   k_ssim_fwd: per 32 x 22 output tile, the five window sums of x, y, x^2, y^2, xy (a row pass
//     over the 32 x 42 haloed tile in shared memory, then a column pass), the SSIM map, the
//     loss, and the three maps of the gradient's chain rule through the raw moments:
//     d1 = dL/dS (dS/dmu_x - 2 mu_x dS/dvar_x - mu_y dS/dcov), d2 = dL/dS dS/dvar_x,
//     d3 = dL/dS dS/dcov;
//   k_ssim_bwd: the window sums of d1, d2, d3 (the window is symmetric, so the adjoint of a
//     window sum is a window sum) and dL/dx = W(d1) + 2 x W(d2) + y W(d3) + the L1 term.
// Each thread of the row pass produces 8 adjacent outputs from 18 inputs and each thread of
// the column pass 11 outputs from 21, so every shared-memory value loaded feeds up to 8 (11)
// outputs; pairs of sums with the same weight -- (x, y), (x^2, y^2), (d1, d2) -- share one
// packed f32x2 FMA. The haloed tiles arrive by asynchronous zero-filling copies. Map planes:
// (d1, d2) interleaved, then d3, then the per-block loss partials.
#include <cmath>

#include "tgs_internal.cuh"

namespace tgs {
namespace {

constexpr int kR = 5;                 // window radius
constexpr int kK = 2 * kR + 1;        // 11 taps
constexpr int kTX = 32;               // output tile width
constexpr int kTY = 22;               // output tile height (2 column groups of 11)
constexpr int kInW = kTX + 2 * kR;    // 42
constexpr int kInH = kTY + 2 * kR;    // 32
constexpr int kInP = 43;              // row pitch of the haloed tile (odd: no bank conflicts)
constexpr int kHP = kTX + 1;          // row pitch of the row-pass output
constexpr int kGX = 8;                // outputs per thread in the row pass
constexpr int kGY = 11;               // outputs per thread in the column pass
constexpr int kNT = 64;               // threads per block
constexpr float kC1 = 0.01f * 0.01f;
constexpr float kC2 = 0.03f * 0.03f;

static_assert(kInH == 32 && kTX / kGX * kInH == 2 * kNT, "row pass: 2 tasks per thread");
static_assert(kTX * (kTY / kGY) == kNT, "column pass: 1 task per thread");

struct SsimViews {
    int V, total_tiles;
    float lam;
    float w[kK];                      // normalised 1D window
    int tile_off[kMaxViews + 1];      // first tile of each view (tiles of one channel)
    int W[kMaxViews], H[kMaxViews], tx[kMaxViews];
    int64_t off[kMaxViews];           // element offset of view v in the map planes
    float inv_n[kMaxViews];           // 1 / (3 H W V)
    const float *x[kMaxViews];        // rendered images [3,H,W]
    const float *y[kMaxViews];        // targets [3,H,W]
    float *grad[kMaxViews];           // dL/dx [3,H,W]
};

__device__ __forceinline__ int view_of(const SsimViews &b, int tile) {
    int lo = 0, hi = b.V - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (b.tile_off[mid] <= tile) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

__device__ __forceinline__ float block_sum(float v, float *s) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) s[threadIdx.x >> 5] = v;
    __syncthreads();
    return s[0] + s[1];
}

// Packed pairs of float32 in one 64-bit register: fma.rn.f32x2 and mul.rn.f32x2 round each
// half exactly as fmaf and a * b do, with one instruction for the pair.
typedef unsigned long long f2;

__device__ __forceinline__ f2 pk(float a, float b) {
    f2 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
    return r;
}
__device__ __forceinline__ float2 upk(f2 v) {
    float2 r;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(r.x), "=f"(r.y) : "l"(v));
    return r;
}
__device__ __forceinline__ f2 fma2(f2 a, f2 b, f2 c) {
    f2 d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}
__device__ __forceinline__ f2 mul2(f2 a, f2 b) {
    f2 d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}

// Asynchronous copy of 4 or 8 bytes to shared memory; ok == false zero-fills (source size 0,
// the source address is then not read).
template <int BYTES>
__device__ __forceinline__ void cp_async(void *dst, const void *src, bool ok) {
    const uint32_t d = (uint32_t)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2, %3;\n" ::"r"(d), "l"(src), "n"(BYTES),
                 "r"(ok ? BYTES : 0)
                 : "memory");
}

__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// Calls f(r, cc, gy, gx, ok) for every element of the haloed tile: warp w takes rows w, w + 2,
// ..., lanes take columns.
template <class F>
__device__ __forceinline__ void for_halo(int W, int H, int x0, int y0, F f) {
    const int lane = threadIdx.x & 31;
    for (int r = threadIdx.x >> 5; r < kInH; r += kNT / 32) {
        const int gy = y0 - kR + r;
        const bool rok = gy >= 0 && gy < H;
#pragma unroll
        for (int cc = lane; cc < kInW; cc += 32) {
            const int gx = x0 - kR + cc;
            f(r, cc, gy, gx, rok && gx >= 0 && gx < W);
        }
    }
}

__global__ void __launch_bounds__(kNT)
k_ssim_fwd(const __grid_constant__ SsimViews b, float *__restrict__ maps, int64_t plane, float *__restrict__ part) {
    __shared__ f2 in[kInH][kInP];      // (x, y)
    __shared__ f2 h01[kInH][kHP];      // row sums of (x, y)
    __shared__ f2 h23[kInH][kHP];      // row sums of (x^2, y^2)
    __shared__ float h4[kInH][kHP];    // row sums of x y
    __shared__ float red[2];
    const int t = threadIdx.x, ch = blockIdx.y;
    const int v = view_of(b, blockIdx.x);
    const int W = b.W[v], H = b.H[v];
    const int lt = blockIdx.x - b.tile_off[v];
    const int x0 = (lt % b.tx[v]) * kTX, y0 = (lt / b.tx[v]) * kTY;
    const int64_t HW = (int64_t)W * H;
    const float *xs = b.x[v] + ch * HW, *ys = b.y[v] + ch * HW;
    for_halo(W, H, x0, y0, [&](int r, int cc, int gy, int gx, bool ok) {
        const int64_t p = ok ? (int64_t)gy * W + gx : 0;
        float *d = reinterpret_cast<float *>(&in[r][cc]);
        cp_async<4>(d, xs + p, ok);
        cp_async<4>(d + 1, ys + p, ok);
    });
    f2 w2[kK];
#pragma unroll
    for (int k = 0; k < kK; k++) w2[k] = pk(b.w[k], b.w[k]);
    cp_async_wait_all();
    __syncthreads();

    // row pass: 32 rows x 4 groups of 8 columns; lanes take consecutive rows
#pragma unroll
    for (int k = 0; k < 2; k++) {
        const int task = t + k * kNT;
        const int r = task & 31, c0 = (task >> 5) * kGX;
        f2 a01[kGX], a23[kGX];
        float a4[kGX];
#pragma unroll
        for (int o = 0; o < kGX; o++) {
            a01[o] = a23[o] = 0ull;
            a4[o] = 0.f;
        }
#pragma unroll
        for (int j = 0; j < kGX + 2 * kR; j++) {
            const f2 val = in[r][c0 + j];
            const f2 sq = mul2(val, val);
            const float2 xy = upk(val);
            const float pr = xy.x * xy.y;
#pragma unroll
            for (int o = 0; o < kGX; o++) {
                if (j - o < 0 || j - o >= kK) continue;
                a01[o] = fma2(w2[j - o], val, a01[o]);
                a23[o] = fma2(w2[j - o], sq, a23[o]);
                a4[o] = fmaf(b.w[j - o], pr, a4[o]);
            }
        }
#pragma unroll
        for (int o = 0; o < kGX; o++) {
            h01[r][c0 + o] = a01[o];
            h23[r][c0 + o] = a23[o];
            h4[r][c0 + o] = a4[o];
        }
    }
    __syncthreads();

    // column pass: lane = column, warp = group of 11 rows
    const int c = t & 31, r0 = (t >> 5) * kGY;
    f2 a01[kGY], a23[kGY];
    float a4[kGY];
#pragma unroll
    for (int o = 0; o < kGY; o++) {
        a01[o] = a23[o] = 0ull;
        a4[o] = 0.f;
    }
#pragma unroll
    for (int j = 0; j < kGY + 2 * kR; j++) {
        const f2 v01 = h01[r0 + j][c], v23 = h23[r0 + j][c];
        const float v4 = h4[r0 + j][c];
#pragma unroll
        for (int o = 0; o < kGY; o++) {
            if (j - o < 0 || j - o >= kK) continue;
            a01[o] = fma2(w2[j - o], v01, a01[o]);
            a23[o] = fma2(w2[j - o], v23, a23[o]);
            a4[o] = fmaf(b.w[j - o], v4, a4[o]);
        }
    }

    const float dLdS = -b.lam * b.inv_n[v];
    f2 *d12 = reinterpret_cast<f2 *>(maps) + b.off[v] + ch * HW;
    float *d3 = maps + 2 * plane + b.off[v] + ch * HW;
    const int gx = x0 + c;
    float ssum = 0.f, l1 = 0.f;
#pragma unroll
    for (int o = 0; o < kGY; o++) {
        const int gy = y0 + r0 + o;
        if (gx >= W || gy >= H) continue;
        const float2 m = upk(a01[o]), e2 = upk(a23[o]);
        const float mx = m.x, my = m.y;
        const float vx = e2.x - mx * mx, vy = e2.y - my * my, cov = a4[o] - mx * my;
        const float A1 = 2.f * mx * my + kC1, A2 = 2.f * cov + kC2;
        const float B1 = mx * mx + my * my + kC1, B2 = vx + vy + kC2;
        const float rB1 = __fdividef(1.f, B1), rB2 = __fdividef(1.f, B2);
        const float S = A1 * A2 * rB1 * rB2;
        const float dS_dmx = 2.f * rB1 * (my * A2 * rB2 - mx * S);   // 2 my A2 / (B1 B2) - 2 mx S / B1
        const float dS_dvx = -S * rB2;
        const float dS_dcov = 2.f * A1 * rB1 * rB2;
        const int64_t p = (int64_t)gy * W + gx;
        d12[p] = pk(dLdS * (dS_dmx - 2.f * mx * dS_dvx - my * dS_dcov), dLdS * dS_dvx);
        d3[p] = dLdS * dS_dcov;
        ssum += S;
        const float2 xy = upk(in[r0 + o + kR][c + kR]);
        l1 += fabsf(xy.x - xy.y);
    }
    if (part) {
        const float tot = block_sum(b.inv_n[v] * ((1.f - b.lam) * l1 - b.lam * ssum), red);
        if (t == 0) part[blockIdx.y * gridDim.x + blockIdx.x] = tot;
    }
}

// loss += lam + the sum of the per-block partials, in a fixed order (one block).
__global__ void __launch_bounds__(1024) k_loss_sum(const float *__restrict__ part, int n, float lam,
                                                   float *__restrict__ loss) {
    __shared__ float s[32];
    float x = 0.f;
    for (int i = threadIdx.x; i < n; i += blockDim.x) x += part[i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    if ((threadIdx.x & 31) == 0) s[threadIdx.x >> 5] = x;
    __syncthreads();
    if (threadIdx.x < 32) {
        x = s[threadIdx.x];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
        if (threadIdx.x == 0) *loss += x + lam;
    }
}

__global__ void __launch_bounds__(kNT)
k_ssim_bwd(const __grid_constant__ SsimViews b, const float *__restrict__ maps, int64_t plane) {
    __shared__ f2 in12[kInH][kInP];    // (d1, d2)
    __shared__ float in3[kInH][kInP];  // d3
    __shared__ f2 h12[kInH][kHP];
    __shared__ float h3[kInH][kHP];
    const int t = threadIdx.x, ch = blockIdx.y;
    const int v = view_of(b, blockIdx.x);
    const int W = b.W[v], H = b.H[v];
    const int lt = blockIdx.x - b.tile_off[v];
    const int x0 = (lt % b.tx[v]) * kTX, y0 = (lt / b.tx[v]) * kTY;
    const int64_t HW = (int64_t)W * H;
    const f2 *m12 = reinterpret_cast<const f2 *>(maps) + b.off[v] + ch * HW;
    const float *m3 = maps + 2 * plane + b.off[v] + ch * HW;
    for_halo(W, H, x0, y0, [&](int r, int cc, int gy, int gx, bool ok) {
        const int64_t p = ok ? (int64_t)gy * W + gx : 0;
        cp_async<8>(&in12[r][cc], m12 + p, ok);
        cp_async<4>(&in3[r][cc], m3 + p, ok);
    });
    // this thread's outputs: column c, rows r0 .. r0 + 10; their x and y load meanwhile
    const int c = t & 31, r0 = (t >> 5) * kGY, gx = x0 + c;
    const float *xs = b.x[v] + ch * HW, *ys = b.y[v] + ch * HW;
    float xv[kGY], yv[kGY];
#pragma unroll
    for (int o = 0; o < kGY; o++) {
        const int gy = y0 + r0 + o;
        const bool ok = gx < W && gy < H;
        const int64_t p = (int64_t)gy * W + gx;
        xv[o] = ok ? __ldg(xs + p) : 0.f;
        yv[o] = ok ? __ldg(ys + p) : 0.f;
    }
    f2 w2[kK];
#pragma unroll
    for (int k = 0; k < kK; k++) w2[k] = pk(b.w[k], b.w[k]);
    cp_async_wait_all();
    __syncthreads();

#pragma unroll
    for (int k = 0; k < 2; k++) {
        const int task = t + k * kNT;
        const int r = task & 31, c0 = (task >> 5) * kGX;
        f2 a12[kGX];
        float a3[kGX];
#pragma unroll
        for (int o = 0; o < kGX; o++) {
            a12[o] = 0ull;
            a3[o] = 0.f;
        }
#pragma unroll
        for (int j = 0; j < kGX + 2 * kR; j++) {
            const f2 v12 = in12[r][c0 + j];
            const float v3 = in3[r][c0 + j];
#pragma unroll
            for (int o = 0; o < kGX; o++) {
                if (j - o < 0 || j - o >= kK) continue;
                a12[o] = fma2(w2[j - o], v12, a12[o]);
                a3[o] = fmaf(b.w[j - o], v3, a3[o]);
            }
        }
#pragma unroll
        for (int o = 0; o < kGX; o++) {
            h12[r][c0 + o] = a12[o];
            h3[r][c0 + o] = a3[o];
        }
    }
    __syncthreads();

    f2 a12[kGY];
    float a3[kGY];
#pragma unroll
    for (int o = 0; o < kGY; o++) {
        a12[o] = 0ull;
        a3[o] = 0.f;
    }
#pragma unroll
    for (int j = 0; j < kGY + 2 * kR; j++) {
        const f2 v12 = h12[r0 + j][c];
        const float v3 = h3[r0 + j][c];
#pragma unroll
        for (int o = 0; o < kGY; o++) {
            if (j - o < 0 || j - o >= kK) continue;
            a12[o] = fma2(w2[j - o], v12, a12[o]);
            a3[o] = fmaf(b.w[j - o], v3, a3[o]);
        }
    }

    float *g = b.grad[v] + ch * HW;
    const float l1s = (1.f - b.lam) * b.inv_n[v];
#pragma unroll
    for (int o = 0; o < kGY; o++) {
        const int gy = y0 + r0 + o;
        if (gx >= W || gy >= H) continue;
        const float2 s12 = upk(a12[o]);
        const float d = xv[o] - yv[o];
        const float sg = d > 0.f ? l1s : (d < 0.f ? -l1s : 0.f);
        g[(int64_t)gy * W + gx] = s12.x + 2.f * xv[o] * s12.y + yv[o] * a3[o] + sg;
    }
}

}  // namespace

namespace {

int64_t elems_of(const int *W, const int *H, int V) {
    int64_t e = 0;
    for (int v = 0; v < V; v++) e += 3 * (int64_t)W[v] * H[v];
    return e;
}

int64_t tiles_of(const int *W, const int *H, int V) {
    int64_t t = 0;
    for (int v = 0; v < V; v++) t += (int64_t)((W[v] + kTX - 1) / kTX) * ((H[v] + kTY - 1) / kTY);
    return t;
}

}  // namespace

int64_t ssim_scratch_floats(const int *W, const int *H, int V) {
    return 3 * elems_of(W, H, V) + 3 * tiles_of(W, H, V);
}

void launch_l1_dssim(int V, const int *W, const int *H, const float *const *x, const float *const *y,
                     float *const *grad, float lam, float *scratch, float *loss, cudaStream_t st) {
    SsimViews b{};
    b.V = V;
    b.lam = lam;
    double w[kK], sum = 0.0;
    for (int k = 0; k < kK; k++) sum += (w[k] = std::exp(-(double)((k - kR) * (k - kR)) / (2.0 * 1.5 * 1.5)));
    for (int k = 0; k < kK; k++) b.w[k] = (float)(w[k] / sum);
    int tiles = 0;
    int64_t off = 0;
    for (int v = 0; v < V; v++) {
        b.tile_off[v] = tiles;
        b.W[v] = W[v];
        b.H[v] = H[v];
        b.tx[v] = (W[v] + kTX - 1) / kTX;
        tiles += b.tx[v] * ((H[v] + kTY - 1) / kTY);
        b.off[v] = off;
        off += 3 * (int64_t)W[v] * H[v];
        b.inv_n[v] = (float)(1.0 / (3.0 * (double)W[v] * H[v] * V));
        b.x[v] = x[v];
        b.y[v] = y[v];
        b.grad[v] = grad[v];
    }
    b.tile_off[V] = tiles;
    b.total_tiles = tiles;
    if (tiles <= 0) return;
    const int64_t plane = off;
    float *part = loss ? scratch + 3 * plane : nullptr;   // 3 * tiles partial sums
    const dim3 grid((unsigned)tiles, 3);
    count_launch(loss ? 3 : 2);
    k_ssim_fwd<<<grid, kNT, 0, st>>>(b, scratch, plane, part);
    if (loss) k_loss_sum<<<1, 1024, 0, st>>>(part, 3 * tiles, lam, loss);
    k_ssim_bwd<<<grid, kNT, 0, st>>>(b, scratch, plane);
}

}  // namespace tgs
