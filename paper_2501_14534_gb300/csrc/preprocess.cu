// Preprocess forward and backward: one thread per Gaussian, looping over the views of the
// launch so that each Gaussian's parameters are read once per launch.
//
// Forward (Eq. 1 of the paper plus the masks): straight-through volume mask M on opacity and
// scale, Sigma = R S S^T R^T, t = W mu + tau, Sigma' = J W Sigma W^T J^T + sI, conic =
// Sigma'^-1, radius, inclusive pixel rect, tiles touched, and the colour from SH with
// straight-through band masks (Eq. sh-masks). Backward: the chain rule from the splat
// gradient records to every input, plus the 2D-mean gradient-norm statistics.
#include <cuda_fp16.h>

#include <type_traits>

#include "tgs_internal.cuh"

namespace tgs {
namespace {

// Real SH normalisation constants: k0 = 1/(2 sqrt(pi)), k1 = sqrt(3/(4 pi)),
// k2a = sqrt(15/pi)/2, k2b = sqrt(5/pi)/4, k2c = sqrt(15/pi)/4, k3a = sqrt(35/(2 pi))/4,
// k3b = sqrt(105/pi)/2, k3c = sqrt(21/(2 pi))/4, k3d = sqrt(7/pi)/4, k3e = sqrt(105/pi)/4.
constexpr float k0 = 0.28209479177387814f;
constexpr float k1 = 0.4886025119029199f;
constexpr float k2a = 1.0925484305920792f;
constexpr float k2b = 0.31539156525252005f;
constexpr float k2c = 0.5462742152960396f;
constexpr float k3a = 0.5900435899266435f;
constexpr float k3b = 2.890611442640554f;
constexpr float k3c = 0.4570457994644658f;
constexpr float k3d = 0.3731763325901154f;
constexpr float k3e = 1.445305721320277f;

// Basis values for a unit direction (3DGS sign convention; index k = l*l + l + m).
__device__ __forceinline__ void sh_basis(float x, float y, float z, float Y[16]) {
    float xx = x * x, yy = y * y, zz = z * z;
    Y[0] = k0;
    Y[1] = -k1 * y;
    Y[2] = k1 * z;
    Y[3] = -k1 * x;
    Y[4] = k2a * x * y;
    Y[5] = -k2a * y * z;
    Y[6] = k2b * (2.f * zz - xx - yy);
    Y[7] = -k2a * x * z;
    Y[8] = k2c * (xx - yy);
    Y[9] = -k3a * y * (3.f * xx - yy);
    Y[10] = k3b * x * y * z;
    Y[11] = -k3c * y * (4.f * zz - xx - yy);
    Y[12] = k3d * z * (2.f * zz - 3.f * xx - 3.f * yy);
    Y[13] = -k3c * x * (4.f * zz - xx - yy);
    Y[14] = k3e * z * (xx - yy);
    Y[15] = -k3a * x * (xx - 3.f * yy);
}

// Adds s * grad Y_k(x, y, z) (gradient of the polynomial form above) to g.
__device__ __forceinline__ void sh_basis_grad_add(int k, float x, float y, float z, float s,
                                                  float3 &g) {
    float xx = x * x, yy = y * y, zz = z * z;
    float gx = 0.f, gy = 0.f, gz = 0.f;
    switch (k) {
        case 1: gy = -k1; break;
        case 2: gz = k1; break;
        case 3: gx = -k1; break;
        case 4: gx = k2a * y; gy = k2a * x; break;
        case 5: gy = -k2a * z; gz = -k2a * y; break;
        case 6: gx = -2.f * k2b * x; gy = -2.f * k2b * y; gz = 4.f * k2b * z; break;
        case 7: gx = -k2a * z; gz = -k2a * x; break;
        case 8: gx = 2.f * k2c * x; gy = -2.f * k2c * y; break;
        case 9: gx = -6.f * k3a * x * y; gy = -3.f * k3a * (xx - yy); break;
        case 10: gx = k3b * y * z; gy = k3b * x * z; gz = k3b * x * y; break;
        case 11: gx = 2.f * k3c * x * y; gy = -k3c * (4.f * zz - xx - 3.f * yy); gz = -8.f * k3c * y * z; break;
        case 12: gx = -6.f * k3d * x * z; gy = -6.f * k3d * y * z; gz = k3d * (6.f * zz - 3.f * xx - 3.f * yy); break;
        case 13: gx = -k3c * (4.f * zz - 3.f * xx - yy); gy = 2.f * k3c * x * y; gz = -8.f * k3c * x * z; break;
        case 14: gx = 2.f * k3e * x * z; gy = -2.f * k3e * y * z; gz = k3e * (xx - yy); break;
        case 15: gx = -3.f * k3a * (xx - yy); gy = 6.f * k3a * x * y; break;
        default: break;
    }
    g.x += s * gx;
    g.y += s * gy;
    g.z += s * gz;
}

__device__ __forceinline__ int band_of(int k) { return k < 4 ? 1 : (k < 9 ? 2 : 3); }

__device__ __forceinline__ float sigmoidf_(float x) { return 1.f / (1.f + expf(-x)); }

// Rotation matrix of a unit quaternion (w, x, y, z), row-major.
__device__ __forceinline__ void quat_rot(float w, float x, float y, float z, float R[9]) {
    R[0] = 1.f - 2.f * (y * y + z * z);
    R[1] = 2.f * (x * y - w * z);
    R[2] = 2.f * (x * z + w * y);
    R[3] = 2.f * (x * y + w * z);
    R[4] = 1.f - 2.f * (x * x + z * z);
    R[5] = 2.f * (y * z - w * x);
    R[6] = 2.f * (x * z - w * y);
    R[7] = 2.f * (y * z + w * x);
    R[8] = 1.f - 2.f * (x * x + y * y);
}

// Everything the forward and the backward share about one Gaussian (view independent).
struct GaussState {
    float M;            // hard volume mask
    bool band[4];       // effective band on/off (band[0] always on)
    int deg;            // active degree
    float3 mu;
    float scale[3];
    float sig_o, op;
    float qn[4], qnorm;
    float R[9];
    float S[6];         // Sigma: xx, xy, xz, yy, yz, zz
    bool ok;
};

// A parameter value: float32, or IEEE half widened to float32 (the FP16 storage of trained
// scenes, read by the render path only).
template <typename T>
__device__ __forceinline__ float ldp(const float *p, int64_t k) {
    if constexpr (std::is_same<T, __half>::value) return __half2float(reinterpret_cast<const __half *>(p)[k]);
    else return p[k];
}

template <typename T = float>
__device__ __forceinline__ GaussState load_state(const GaussPtrs &g, int64_t i) {
    GaussState s;
    s.M = 1.f;
    if (g.mask) s.M = (ldp<T>(g.mask, i) > g.tau_m) ? 1.f : 0.f;
    s.deg = g.deg_max;
    if (g.sh_degree) s.deg = min(s.deg, (int)g.sh_degree[i]);
    s.band[0] = true;
#pragma unroll
    for (int l = 1; l <= 3; l++) {
        bool on = l <= s.deg;
        if (g.shmask) on = on && (ldp<T>(g.shmask, 3 * i + l - 1) > g.tau_sh);
        s.band[l] = on;
    }
    s.mu = make_float3(ldp<T>(g.means, 3 * i), ldp<T>(g.means, 3 * i + 1), ldp<T>(g.means, 3 * i + 2));
    float ls0 = ldp<T>(g.log_scales, 3 * i), ls1 = ldp<T>(g.log_scales, 3 * i + 1),
          ls2 = ldp<T>(g.log_scales, 3 * i + 2);
    s.scale[0] = s.M * expf(ls0);
    s.scale[1] = s.M * expf(ls1);
    s.scale[2] = s.M * expf(ls2);
    s.sig_o = sigmoidf_(ldp<T>(g.opac, i));
    s.op = s.M * s.sig_o;
    float4 q = make_float4(ldp<T>(g.quats, 4 * i), ldp<T>(g.quats, 4 * i + 1), ldp<T>(g.quats, 4 * i + 2),
                            ldp<T>(g.quats, 4 * i + 3));
    float qq = q.x * q.x + q.y * q.y + q.z * q.z + q.w * q.w;
    s.qnorm = sqrtf(qq);
    float inv = 1.f / s.qnorm;
    s.qn[0] = q.x * inv;
    s.qn[1] = q.y * inv;
    s.qn[2] = q.z * inv;
    s.qn[3] = q.w * inv;
    quat_rot(s.qn[0], s.qn[1], s.qn[2], s.qn[3], s.R);
    // Sigma = sum_k s_k^2 r_k r_k^T with r_k the k-th column of R
    float a0 = s.scale[0] * s.scale[0], a1 = s.scale[1] * s.scale[1], a2 = s.scale[2] * s.scale[2];
    const float *R = s.R;
    s.S[0] = a0 * R[0] * R[0] + a1 * R[1] * R[1] + a2 * R[2] * R[2];
    s.S[1] = a0 * R[0] * R[3] + a1 * R[1] * R[4] + a2 * R[2] * R[5];
    s.S[2] = a0 * R[0] * R[6] + a1 * R[1] * R[7] + a2 * R[2] * R[8];
    s.S[3] = a0 * R[3] * R[3] + a1 * R[4] * R[4] + a2 * R[5] * R[5];
    s.S[4] = a0 * R[3] * R[6] + a1 * R[4] * R[7] + a2 * R[5] * R[8];
    s.S[5] = a0 * R[6] * R[6] + a1 * R[7] * R[7] + a2 * R[8] * R[8];
    s.ok = (s.M > 0.f) && qq > 0.f && isfinite(qq) && isfinite(s.mu.x) && isfinite(s.mu.y) &&
           isfinite(s.mu.z) && isfinite(s.S[0] + s.S[1] + s.S[2] + s.S[3] + s.S[4] + s.S[5]);
    return s;
}

// Everything about one Gaussian in one view.
struct ViewGeom {
    float tx, ty, tz, inv_tz;
    float u, w;          // clamped t_x/t_z, t_y/t_z
    bool cx_on, cy_on;   // clamp active
    float T0[3], T1[3];  // rows of J W
    float c00, c01, c11; // Sigma'
    float det;
    float ca, cb, cc;    // conic
    float mx, my;
};

__device__ __forceinline__ bool view_geom(const GaussState &s, const DevCam &c, float near_z,
                                          ViewGeom &v) {
    const float *W = c.R;
    v.tx = W[0] * s.mu.x + W[1] * s.mu.y + W[2] * s.mu.z + c.t[0];
    v.ty = W[3] * s.mu.x + W[4] * s.mu.y + W[5] * s.mu.z + c.t[1];
    v.tz = W[6] * s.mu.x + W[7] * s.mu.y + W[8] * s.mu.z + c.t[2];
    if (!(v.tz > near_z)) return false;
    v.inv_tz = 1.f / v.tz;
    float ux = v.tx * v.inv_tz, uy = v.ty * v.inv_tz;
    v.cx_on = (ux < -c.limx) || (ux > c.limx);
    v.cy_on = (uy < -c.limy) || (uy > c.limy);
    v.u = fminf(c.limx, fmaxf(-c.limx, ux));
    v.w = fminf(c.limy, fmaxf(-c.limy, uy));
    float jx = c.fx * v.inv_tz, jy = c.fy * v.inv_tz;
    // rows of T = J W: T0 = fx/tz (W0 - u W2), T1 = fy/tz (W1 - w W2)
#pragma unroll
    for (int k = 0; k < 3; k++) {
        v.T0[k] = jx * (W[k] - v.u * W[6 + k]);
        v.T1[k] = jy * (W[3 + k] - v.w * W[6 + k]);
    }
    const float *S = s.S;
    float s0x = S[0] * v.T0[0] + S[1] * v.T0[1] + S[2] * v.T0[2];
    float s0y = S[1] * v.T0[0] + S[3] * v.T0[1] + S[4] * v.T0[2];
    float s0z = S[2] * v.T0[0] + S[4] * v.T0[1] + S[5] * v.T0[2];
    float s1x = S[0] * v.T1[0] + S[1] * v.T1[1] + S[2] * v.T1[2];
    float s1y = S[1] * v.T1[0] + S[3] * v.T1[1] + S[4] * v.T1[2];
    float s1z = S[2] * v.T1[0] + S[4] * v.T1[1] + S[5] * v.T1[2];
    v.c00 = v.T0[0] * s0x + v.T0[1] * s0y + v.T0[2] * s0z + c.s;
    v.c01 = v.T0[0] * s1x + v.T0[1] * s1y + v.T0[2] * s1z;
    v.c11 = v.T1[0] * s1x + v.T1[1] * s1y + v.T1[2] * s1z + c.s;
    v.det = v.c00 * v.c11 - v.c01 * v.c01;
    if (!(v.det > 0.f) || !isfinite(v.det)) return false;
    float id = 1.f / v.det;
    v.ca = v.c11 * id;
    v.cb = -v.c01 * id;
    v.cc = v.c00 * id;
    v.mx = c.fx * ux + c.cx - 0.5f;
    v.my = c.fy * uy + c.cy - 0.5f;
    return isfinite(v.mx) && isfinite(v.my);
}

// SH coefficients of one Gaussian kept in registers (only bands that are on).
struct ShCoeffs {
    float3 f[16];
};

template <typename T = float>
__device__ __forceinline__ void load_sh(const GaussPtrs &g, int64_t i, const GaussState &s,
                                        ShCoeffs &sh) {
    sh.f[0] = make_float3(ldp<T>(g.sh_dc, 3 * i), ldp<T>(g.sh_dc, 3 * i + 1), ldp<T>(g.sh_dc, 3 * i + 2));
    const int64_t r = 45 * i;
#pragma unroll
    for (int k = 1; k < 16; k++) {
        if (g.sh_rest && s.deg >= band_of(k))
            sh.f[k] = make_float3(ldp<T>(g.sh_rest, r + 3 * (k - 1)), ldp<T>(g.sh_rest, r + 3 * (k - 1) + 1),
                                  ldp<T>(g.sh_rest, r + 3 * (k - 1) + 2));
        else
            sh.f[k] = make_float3(0.f, 0.f, 0.f);
    }
}

// Un-clamped colour 1/2 + sum over active bands.
__device__ __forceinline__ float3 sh_raw(const GaussState &s, const ShCoeffs &sh, const float Y[16]) {
    float3 c = make_float3(0.5f + Y[0] * sh.f[0].x, 0.5f + Y[0] * sh.f[0].y, 0.5f + Y[0] * sh.f[0].z);
#pragma unroll
    for (int k = 1; k < 16; k++) {
        if (!s.band[band_of(k)]) continue;
        c.x += Y[k] * sh.f[k].x;
        c.y += Y[k] * sh.f[k].y;
        c.z += Y[k] * sh.f[k].z;
    }
    return c;
}

// One thread per Gaussian, looping over the views. A warp's 32 Gaussians have consecutive
// records in every view, so the records (and the zeroed gradient records) go out through
// shared memory as one contiguous run per warp: full-sector stores instead of four 16-byte
// pieces per 64-byte record from each thread. Records of Gaussians not visible in a view
// hold zeros; nothing reads them.
template <typename T>
__global__ void __launch_bounds__(128) k_preprocess(GaussPtrs g, const __grid_constant__ CamBatch cb,
                                                    float4 *__restrict__ splats,
                                                    int32_t *__restrict__ radii,
                                                    uint32_t *__restrict__ tiles_touched,
                                                    uint32_t *__restrict__ depth_bits,
                                                    float4 *__restrict__ zero_grads) {
    constexpr int RW = kSplatWords / 4;  // float4 per record
    __shared__ float4 s_rec[4][32 * RW];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t n = g.n;
    const int64_t i0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t wfirst = i0 - lane;
    if (wfirst >= n) return;  // the whole warp is past the end
    const bool inb = i0 < n;
    const int64_t i = inb ? i0 : wfirst;
    const int wn = (int)min((int64_t)32, n - wfirst);  // Gaussians of this warp
    GaussState s = load_state<T>(g, i);
    if (!inb) s.ok = false;
    ShCoeffs sh;
    if (s.ok) load_sh<T>(g, i, s, sh);
    for (int v = 0; v < cb.V; v++) {
        const DevCam &c = cb.c[v];
        const int64_t r = (int64_t)v * n + i;
        int rad = 0;
        uint32_t touched = 0;
        float4 rec[RW];
#pragma unroll
        for (int k = 0; k < RW; k++) rec[k] = make_float4(0.f, 0.f, 0.f, 0.f);
        ViewGeom vg;
        if (s.ok && view_geom(s, c, g.near_z, vg)) {
            float mid = 0.5f * (vg.c00 + vg.c11);
            float lam = mid + sqrtf(fmaxf(0.1f, mid * mid - vg.det));
            float rf;
            bool alive = true;
            if (g.support == TGS_SUPPORT_ALPHA) {
                alive = s.op >= kAlphaMin;
                rf = ceilf(sqrtf(2.f * lam * logf(255.f * s.op)));
            } else {
                rf = ceilf(3.f * sqrtf(lam));
            }
            rf = fminf(rf, 1073741824.f);
            float xlo = ceilf(vg.mx - rf), xhi = floorf(vg.mx + rf);
            float ylo = ceilf(vg.my - rf), yhi = floorf(vg.my + rf);
            xlo = fmaxf(xlo, 0.f);
            ylo = fmaxf(ylo, 0.f);
            xhi = fminf(xhi, (float)(c.W - 1));
            yhi = fminf(yhi, (float)(c.H - 1));
            if (alive && rf >= 1.f && xlo <= xhi && ylo <= yhi) {
                float dx = s.mu.x - c.campos[0], dy = s.mu.y - c.campos[1], dz = s.mu.z - c.campos[2];
                float dn = sqrtf(dx * dx + dy * dy + dz * dz);
                float inv = 1.f / dn;
                float Y[16];
                sh_basis(dx * inv, dy * inv, dz * inv, Y);
                float3 raw = sh_raw(s, sh, Y);
                float3 rgb = make_float3(fmaxf(raw.x, 0.f), fmaxf(raw.y, 0.f), fmaxf(raw.z, 0.f));
                if (dn > 0.f && isfinite(rgb.x + rgb.y + rgb.z) &&
                    isfinite(vg.ca + vg.cb + vg.cc)) {
                    int ix0 = (int)xlo, ix1 = (int)xhi, iy0 = (int)ylo, iy1 = (int)yhi;
                    rad = (int)rf;
                    uint32_t rx = (uint32_t)ix0 | ((uint32_t)ix1 << 16);
                    uint32_t ry = (uint32_t)iy0 | ((uint32_t)iy1 << 16);
                    // cull threshold: a tile is kept when some point of it has
                    // Q <= tau = 2 ln(255 o' / (1 - margin)), i.e. alpha may reach 1/255
                    const float tau = 2.f * logf(255.f * s.op / (1.f - kCullMargin));
                    // visible; the binning counts the tiles that pass the cull test
                    touched = 1u;
                    rec[0] = make_float4(vg.mx, vg.my, vg.ca, vg.cb);
                    rec[1] = make_float4(vg.cc, s.op, rgb.x, rgb.y);
                    rec[2] = make_float4(rgb.z, __uint_as_float(rx), __uint_as_float(ry), vg.tz);
                    rec[3] = make_float4(tau, __fdiv_rn(vg.cb, vg.cc), __fdiv_rn(vg.cb, vg.ca), 0.f);
                }
            }
        }
        if (inb) {
            radii[r] = rad;
            if (tiles_touched) tiles_touched[r] = touched;
            // depth key of every record for the depth sort; the ones not visible sort last
            depth_bits[r] = touched ? __float_as_uint(rec[2].w) : kNoDepth;
        }
#pragma unroll
        for (int k = 0; k < RW; k++) s_rec[w][RW * lane + k] = rec[k];
        __syncwarp();
        const int64_t r0 = (int64_t)v * n + wfirst;  // the warp's first record in this view
#pragma unroll
        for (int k = 0; k < RW; k++) {
            const int u = lane + 32 * k;
            if (u < RW * wn) splats[RW * r0 + u] = s_rec[w][u];
        }
        if (zero_grads) {
            const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
            for (int k = 0; k < 3; k++) {
                const int u = lane + 32 * k;
                if (u < 3 * wn) zero_grads[3 * r0 + u] = z;
            }
        }
        __syncwarp();
    }
}

__device__ __forceinline__ void out_write(float *p, int64_t idx, float v, int acc) {
    if (!p) return;
    if (acc) p[idx] += v; else p[idx] = v;
}

// EWA backward of one view: dL/dSigma (full-matrix entries xx, xy, xz, yy, yz, zz) and dL/dmu
// from the view's dL/d mean2d and dL/d conic.
__device__ __forceinline__ void view_geom_backward(const GaussState &s, const DevCam &c, const ViewGeom &vg,
                                                   float gmx, float gmy, float gca, float gcb, float gcc,
                                                   float g_S[6], float3 &g_mu) {
    // ---- conic -> Sigma': G = -Q dL/dQ Q, dL/dQ = [[ga, gb/2], [gb/2, gc]] ----
    float a = vg.ca, b = vg.cb, cc = vg.cc;
    float G00 = -(a * a * gca + a * b * gcb + b * b * gcc);
    float G01 = -(a * b * gca + 0.5f * (b * b + a * cc) * gcb + b * cc * gcc);
    float G11 = -(b * b * gca + b * cc * gcb + cc * cc * gcc);
    // ---- Sigma' = T Sigma T^T: dL/dSigma = T^T G T ----
    const float *T0 = vg.T0, *T1 = vg.T1;
    // full-matrix entries (a,b) for a <= b: xx, xy, xz, yy, yz, zz
    const int ia[6] = {0, 0, 0, 1, 1, 2}, ib[6] = {0, 1, 2, 1, 2, 2};
#pragma unroll
    for (int e = 0; e < 6; e++) {
        int p = ia[e], q = ib[e];
        g_S[e] += T0[p] * T0[q] * G00 + (T0[p] * T1[q] + T1[p] * T0[q]) * G01 + T1[p] * T1[q] * G11;
    }
    // dL/dT = 2 G T Sigma
    const float *S = s.S;
    float sT0[3] = {S[0] * T0[0] + S[1] * T0[1] + S[2] * T0[2],
                    S[1] * T0[0] + S[3] * T0[1] + S[4] * T0[2],
                    S[2] * T0[0] + S[4] * T0[1] + S[5] * T0[2]};
    float sT1[3] = {S[0] * T1[0] + S[1] * T1[1] + S[2] * T1[2],
                    S[1] * T1[0] + S[3] * T1[1] + S[4] * T1[2],
                    S[2] * T1[0] + S[4] * T1[1] + S[5] * T1[2]};
    float GT0[3], GT1[3];
#pragma unroll
    for (int k = 0; k < 3; k++) {
        GT0[k] = 2.f * (G00 * sT0[k] + G01 * sT1[k]);
        GT1[k] = 2.f * (G01 * sT0[k] + G11 * sT1[k]);
    }
    // dL/dJ = dL/dT W^T (entries 00, 02, 11, 12)
    const float *W = c.R;
    float GJ00 = GT0[0] * W[0] + GT0[1] * W[1] + GT0[2] * W[2];
    float GJ02 = GT0[0] * W[6] + GT0[1] * W[7] + GT0[2] * W[8];
    float GJ11 = GT1[0] * W[3] + GT1[1] * W[4] + GT1[2] * W[5];
    float GJ12 = GT1[0] * W[6] + GT1[1] * W[7] + GT1[2] * W[8];
    float itz = vg.inv_tz, itz2 = itz * itz;
    float g_tx = 0.f, g_ty = 0.f, g_tz = 0.f;
    g_tz += -c.fx * itz2 * GJ00 - c.fy * itz2 * GJ11;
    // J02 = -fx u / tz, u = clamp(tx / tz)
    float du_dtx = vg.cx_on ? 0.f : itz, du_dtz = vg.cx_on ? 0.f : -vg.tx * itz2;
    float dw_dty = vg.cy_on ? 0.f : itz, dw_dtz = vg.cy_on ? 0.f : -vg.ty * itz2;
    g_tx += GJ02 * (-c.fx * itz) * du_dtx;
    g_tz += GJ02 * (c.fx * vg.u * itz2 - c.fx * itz * du_dtz);
    g_ty += GJ12 * (-c.fy * itz) * dw_dty;
    g_tz += GJ12 * (c.fy * vg.w * itz2 - c.fy * itz * dw_dtz);
    // mean2d = f t / tz + c - 1/2
    g_tx += gmx * c.fx * itz;
    g_ty += gmy * c.fy * itz;
    g_tz += -(gmx * c.fx * vg.tx + gmy * c.fy * vg.ty) * itz2;
    // t = W mu + tau
    g_mu.x += W[0] * g_tx + W[3] * g_ty + W[6] * g_tz;
    g_mu.y += W[1] * g_tx + W[4] * g_ty + W[7] * g_tz;
    g_mu.z += W[2] * g_tx + W[5] * g_ty + W[8] * g_tz;
}

// Parameter gradients of one Gaussian from its summed dL/dSigma, dL/d opacity and per-band
// colour gradients (the latter for the SH band masks).
__device__ __forceinline__ void gauss_backward(const GaussPtrs &g, int64_t i, const GaussState &s,
                                               const float g_S[6], float g_op, const float g_band[4],
                                               float g_q[4], float g_ls[3], float &g_o, float &g_m,
                                               float g_shm[3]) {
    // ---- Sigma = (R S)(R S)^T: dL/d(RS) = (G + G^T)(RS), G symmetric here ----
    const float *R = s.R;
    float Gf[9] = {g_S[0], g_S[1], g_S[2], g_S[1], g_S[3], g_S[4], g_S[2], g_S[4], g_S[5]};
    // Gf holds the full-matrix gradient with both off-diagonal entries equal to the
    // gradient of one entry, so (G + G^T) = 2 Gf.
    float g_s[3] = {0.f, 0.f, 0.f}, GR[9];
#pragma unroll
    for (int rr = 0; rr < 3; rr++)
#pragma unroll
        for (int cc = 0; cc < 3; cc++) {
            float acc2 = 0.f;
#pragma unroll
            for (int k = 0; k < 3; k++) acc2 += 2.f * Gf[3 * rr + k] * R[3 * k + cc] * s.scale[cc];
            g_s[cc] += acc2 * R[3 * rr + cc];
            GR[3 * rr + cc] = acc2 * s.scale[cc];
        }
    // dR/dq for q = (w, x, y, z)
    float w = s.qn[0], x = s.qn[1], y = s.qn[2], z = s.qn[3];
    float gw = 2.f * (-z * GR[1] + y * GR[2] + z * GR[3] - x * GR[5] - y * GR[6] + x * GR[7]);
    float gx = 2.f * (y * GR[1] + z * GR[2] + y * GR[3] - 2.f * x * GR[4] - w * GR[5] + z * GR[6] + w * GR[7] - 2.f * x * GR[8]);
    float gy = 2.f * (-2.f * y * GR[0] + x * GR[1] + w * GR[2] + x * GR[3] + z * GR[5] - w * GR[6] + z * GR[7] - 2.f * y * GR[8]);
    float gz = 2.f * (-2.f * z * GR[0] - w * GR[1] + x * GR[2] + w * GR[3] - 2.f * z * GR[4] + y * GR[5] + x * GR[6] + y * GR[7]);
    float qd = gw * w + gx * x + gy * y + gz * z;
    float iq = 1.f / s.qnorm;
    g_q[0] = (gw - w * qd) * iq;
    g_q[1] = (gx - x * qd) * iq;
    g_q[2] = (gy - y * qd) * iq;
    g_q[3] = (gz - z * qd) * iq;
    float gM = 0.f;
#pragma unroll
    for (int k = 0; k < 3; k++) {
        g_ls[k] = g_s[k] * s.scale[k];
        gM += g_s[k] * s.scale[k];  // exp(l_k) = scale_k since M = 1 here
    }
    g_o = g_op * s.M * s.sig_o * (1.f - s.sig_o);
    gM += g_op * s.sig_o;
    if (g.mask) {
        float sm = sigmoidf_(g.mask[i]);
        g_m = gM * sm * (1.f - sm);
    }
    if (g.shmask)
#pragma unroll
        for (int l = 1; l <= 3; l++) {
            if (l > s.deg) continue;
            float sm = sigmoidf_(g.shmask[3 * i + l - 1]);
            g_shm[l - 1] = g_band[l] * sm * (1.f - sm);
        }
}

constexpr int kBwdThreads = 128;

// Splat gradients of one (view, Gaussian) from its gradient record: either the gradients
// themselves, or (moments != 0) the pixel sums of the blend backward that they are linear in,
// to which the splat's conic (a, b, c) and opacity o' are applied here:
// dL/d mean2d = -o' (Q m), Q = [[a, b], [b, c]], m = (sum u dx, sum u dy);
// dL/d conic a, b, c = -o' (1/2 sum u dx^2, sum u dx dy, 1/2 sum u dy^2).
__device__ __forceinline__ void splat_grads(const float4 &ga, const float4 &gb, int moments, float o,
                                            float ca, float cb, float cc, float &gmx, float &gmy,
                                            float &gca, float &gcb, float &gcc) {
    if (moments) {
        gmx = -o * (ca * ga.x + cb * ga.y);
        gmy = -o * (cb * ga.x + cc * ga.y);
        gca = -0.5f * o * ga.z;
        gcb = -o * ga.w;
        gcc = -0.5f * o * gb.x;
    } else {
        gmx = ga.x;
        gmy = ga.y;
        gca = ga.z;
        gcb = ga.w;
        gcc = gb.x;
    }
}

// The backward as two kernels, so that each holds fewer registers and more
// warps fit on an SM: the colour part (SH coefficient gradients, band-mask gradients and the
// colour term of dL/dmu through the view direction) and then the geometry part (EWA backward,
// opacity, scales, rotation, volume mask, statistics), which adds its dL/dmu to the colour
// kernel's.
__global__ void __launch_bounds__(kBwdThreads) k_preprocess_bwd_colour(GaussPtrs g, const __grid_constant__ CamBatch cb,
                                                        const float4 *__restrict__ sgrads,
                                                        const int32_t *__restrict__ radii,
                                                        GradPtrs out, int no_sh_rest) {
    // a warp's 32 Gaussians have consecutive rows of 45 SH rest coefficients: the rows come in
    // and the gradients go out as one contiguous run per warp through shared memory (stride 45,
    // odd: each thread reads its own row without bank conflicts)
    constexpr int kRest = 45;
    __shared__ float s_rows[kBwdThreads / 32][32 * kRest];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t n = g.n;
    const int64_t i0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t wfirst = i0 - lane;
    if (wfirst >= n) return;  // the whole warp is past the end
    const bool inb = i0 < n;
    const int64_t i = inb ? i0 : wfirst;
    const int wn = (int)min((int64_t)32, n - wfirst);
    float *rows = s_rows[w];
    if (g.sh_rest)
        for (int u = lane; u < kRest * wn; u += 32) rows[u] = g.sh_rest[kRest * wfirst + u];
    __syncwarp();
    const float *rec = reinterpret_cast<const float *>(sgrads);  // 12 floats per (view, Gaussian)
    GaussState s = load_state(g, i);
    if (!inb) s.ok = false;
    ShCoeffs sh;
    float3 g_mu = make_float3(0.f, 0.f, 0.f);
    float3 g_f[16];
#pragma unroll
    for (int k = 0; k < 16; k++) g_f[k] = make_float3(0.f, 0.f, 0.f);
    float g_band[4] = {0.f, 0.f, 0.f, 0.f};
    uint64_t vis = 0;
    if (s.ok) {
#pragma unroll 8
        for (int v = 0; v < cb.V; v++)
            if (radii[(int64_t)v * n + i] > 0) vis |= 1ull << v;
        sh.f[0] = make_float3(g.sh_dc[3 * i], g.sh_dc[3 * i + 1], g.sh_dc[3 * i + 2]);
#pragma unroll
        for (int k = 1; k < 16; k++) {
            const float *r = rows + kRest * lane + 3 * (k - 1);
            sh.f[k] = (g.sh_rest && s.deg >= band_of(k)) ? make_float3(r[0], r[1], r[2]) : make_float3(0.f, 0.f, 0.f);
        }
        float3 nrgb = make_float3(0.f, 0.f, 0.f), nrgb2 = nrgb;
        if (vis & 1ull) nrgb = make_float3(rec[12 * i + 6], rec[12 * i + 7], rec[12 * i + 8]);
        if (cb.V > 1 && (vis & 2ull)) {
            const int64_t rn = 12 * ((int64_t)n + i);
            nrgb2 = make_float3(rec[rn + 6], rec[rn + 7], rec[rn + 8]);
        }
        for (int v = 0; v < cb.V; v++) {
            const float3 g_rgb = nrgb;
            nrgb = nrgb2;
            if (v + 2 < cb.V && ((vis >> (v + 2)) & 1ull)) {
                const int64_t rn = 12 * ((int64_t)(v + 2) * n + i);
                nrgb2 = make_float3(rec[rn + 6], rec[rn + 7], rec[rn + 8]);
            }
            if (!((vis >> v) & 1ull)) continue;
            const DevCam &c = cb.c[v];
            float dx = s.mu.x - c.campos[0], dy = s.mu.y - c.campos[1], dz = s.mu.z - c.campos[2];
            float dn = sqrtf(dx * dx + dy * dy + dz * dz);
            float inv = 1.f / dn;
            float x = dx * inv, y = dy * inv, z = dz * inv;
            float Y[16];
            sh_basis(x, y, z, Y);
            float3 raw = sh_raw(s, sh, Y);
            float3 gr = make_float3(raw.x < 0.f ? 0.f : g_rgb.x, raw.y < 0.f ? 0.f : g_rgb.y,
                                    raw.z < 0.f ? 0.f : g_rgb.z);
            g_f[0].x += Y[0] * gr.x;
            g_f[0].y += Y[0] * gr.y;
            g_f[0].z += Y[0] * gr.z;
            float3 g_dir = make_float3(0.f, 0.f, 0.f);
#pragma unroll
            for (int k = 1; k < 16; k++) {
                const int l = band_of(k);
                if (l > s.deg) continue;
                float sk = sh.f[k].x * gr.x + sh.f[k].y * gr.y + sh.f[k].z * gr.z;
                g_band[l] += Y[k] * sk;
                if (!s.band[l]) continue;
                g_f[k].x += Y[k] * gr.x;
                g_f[k].y += Y[k] * gr.y;
                g_f[k].z += Y[k] * gr.z;
                sh_basis_grad_add(k, x, y, z, sk, g_dir);
            }
            float dd = g_dir.x * x + g_dir.y * y + g_dir.z * z;
            g_mu.x += (g_dir.x - x * dd) * inv;
            g_mu.y += (g_dir.y - y * dd) * inv;
            g_mu.z += (g_dir.z - z * dd) * inv;
        }
    }
    const int acc = out.accumulate;
    float g_shm[3] = {0.f, 0.f, 0.f};
    if (vis && g.shmask)
#pragma unroll
        for (int l = 1; l <= 3; l++) {
            if (l > s.deg) continue;
            const float sm = sigmoidf_(g.shmask[3 * i + l - 1]);
            g_shm[l - 1] = g_band[l] * sm * (1.f - sm);
        }
    if (out.lam_sh_n != 0.f && g.shmask)  // lambda_sh L_sh of Eq. loss3dgs, every Gaussian and band
#pragma unroll
        for (int l = 1; l <= 3; l++) {
            const float sm = sigmoidf_(g.shmask[3 * i + l - 1]);
            g_shm[l - 1] += out.lam_sh_n * ((float)(2 * l + 1) / 15.f) * sm * (1.f - sm);
        }
    if (out.sh_rest && !no_sh_rest) {
        __syncwarp();  // every thread has read its own row
#pragma unroll
        for (int k = 1; k < 16; k++) {
            float *r = rows + kRest * lane + 3 * (k - 1);
            r[0] = g_f[k].x;
            r[1] = g_f[k].y;
            r[2] = g_f[k].z;
        }
        __syncwarp();
        float *dst = out.sh_rest + kRest * wfirst;
        for (int u = lane; u < kRest * wn; u += 32) dst[u] = acc ? dst[u] + rows[u] : rows[u];
    }
    if (!inb) return;  // a lane past the end holds another Gaussian's index
    out_write(out.means, 3 * i + 0, g_mu.x, acc);
    out_write(out.means, 3 * i + 1, g_mu.y, acc);
    out_write(out.means, 3 * i + 2, g_mu.z, acc);
    out_write(out.sh_dc, 3 * i + 0, g_f[0].x, acc);
    out_write(out.sh_dc, 3 * i + 1, g_f[0].y, acc);
    out_write(out.sh_dc, 3 * i + 2, g_f[0].z, acc);
#pragma unroll
    for (int l = 0; l < 3; l++) out_write(out.shmask, 3 * i + l, g_shm[l], acc);
}

__global__ void __launch_bounds__(kBwdThreads, 5) k_preprocess_bwd_geom(GaussPtrs g, const __grid_constant__ CamBatch cb,
                                                      const float4 *__restrict__ sgrads,
                                                      const int32_t *__restrict__ radii,
                                                      GradPtrs out, int moments) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= g.n) return;
    const int64_t n = g.n;
    GaussState s = load_state(g, i);
    float3 g_mu = make_float3(0.f, 0.f, 0.f);
    float g_S[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};  // dL/dSigma (full-matrix entries)
    float g_op = 0.f;
    float st_acc = 0.f;
    int st_cnt = 0, st_max = 0;
    bool any = false;
    if (s.ok) {
        uint64_t vis = 0;
#pragma unroll 8
        for (int v = 0; v < cb.V; v++) {
            const int rad = radii[(int64_t)v * n + i];
            if (rad > 0) {
                vis |= 1ull << v;
                st_max = max(st_max, rad);
            }
        }
        float4 na = make_float4(0.f, 0.f, 0.f, 0.f), nb = na, na2 = na, nb2 = na;
        if (vis & 1ull) {
            na = sgrads[3 * i];
            nb = sgrads[3 * i + 1];
        }
        if (cb.V > 1 && (vis & 2ull)) {
            na2 = sgrads[3 * (n + i)];
            nb2 = sgrads[3 * (n + i) + 1];
        }
        for (int v = 0; v < cb.V; v++) {
            const float4 ga = na, gb4 = nb;
            na = na2;
            nb = nb2;
            if (v + 2 < cb.V && ((vis >> (v + 2)) & 1ull)) {
                const int64_t rn = (int64_t)(v + 2) * n + i;
                na2 = sgrads[3 * rn];
                nb2 = sgrads[3 * rn + 1];
            }
            if (!((vis >> v) & 1ull)) continue;
            const DevCam &c = cb.c[v];
            ViewGeom vg;
            if (!view_geom(s, c, g.near_z, vg)) continue;  // cannot happen when rad > 0
            any = true;
            float gmx, gmy, gca, gcb, gcc;
            splat_grads(ga, gb4, moments, s.op, vg.ca, vg.cb, vg.cc, gmx, gmy, gca, gcb, gcc);
            g_op += gb4.y;
            st_acc += sqrtf(gmx * gmx + gmy * gmy);
            st_cnt += 1;
            view_geom_backward(s, c, vg, gmx, gmy, gca, gcb, gcc, g_S, g_mu);
        }
    }
    const int acc = out.accumulate;
    // ---- statistics (always accumulated) ----
    if (st_cnt > 0) {
        if (out.stat_accum) out.stat_accum[i] += st_acc;
        if (out.stat_count) out.stat_count[i] += st_cnt;
        if (out.stat_maxr) out.stat_maxr[i] = max(out.stat_maxr[i], st_max);
    }
    float g_q[4] = {0.f, 0.f, 0.f, 0.f}, g_ls[3] = {0.f, 0.f, 0.f}, g_o = 0.f, g_m = 0.f;
    float g_shm[3] = {0.f, 0.f, 0.f};
    const float no_band[4] = {0.f, 0.f, 0.f, 0.f};  // the colour kernel did the band masks
    if (any) gauss_backward(g, i, s, g_S, g_op, no_band, g_q, g_ls, g_o, g_m, g_shm);
    if (out.lam_m_n != 0.f && g.mask) {  // lambda_m L_m of Eq. loss3dgs, every Gaussian
        const float sm = sigmoidf_(g.mask[i]);
        g_m += out.lam_m_n * sm * (1.f - sm);
    }
#pragma unroll
    for (int k = 0; k < 3; k++) {
        if (out.means) out.means[3 * i + k] += (k == 0 ? g_mu.x : (k == 1 ? g_mu.y : g_mu.z));
        out_write(out.log_scales, 3 * i + k, g_ls[k], acc);
    }
#pragma unroll
    for (int k = 0; k < 4; k++) out_write(out.quats, 4 * i + k, g_q[k], acc);
    out_write(out.opac, i, g_o, acc);
    out_write(out.mask, i, g_m, acc);
}

// lambda_m L_m + lambda_sh L_sh over the Gaussians (Eq. loss3dgs): per block one partial sum,
// added to *loss; the gradients of the soft masks added to gmask / gshmask when given.
__global__ void __launch_bounds__(256) k_mask_loss(const float *__restrict__ mask, const float *__restrict__ shmask,
                                                   int64_t n, float lam_m, float lam_sh, float inv_n,
                                                   float *__restrict__ loss, float *__restrict__ gmask,
                                                   float *__restrict__ gshmask) {
    float acc = 0.f;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        if (mask) {
            const float sm = sigmoidf_(mask[i]);
            acc += lam_m * sm;
            if (gmask) gmask[i] += lam_m * inv_n * sm * (1.f - sm);
        }
        if (shmask)
#pragma unroll
            for (int l = 1; l <= 3; l++) {
                const float w = (float)(2 * l + 1) / 15.f;
                const float sm = sigmoidf_(shmask[3 * i + l - 1]);
                acc += lam_sh * w * sm;
                if (gshmask) gshmask[3 * i + l - 1] += lam_sh * w * inv_n * sm * (1.f - sm);
            }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    __shared__ float s[8];
    if ((threadIdx.x & 31) == 0) s[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0 && loss) {
        float x = 0.f;
        for (int q = 0; q < (int)(blockDim.x >> 5); q++) x += s[q];
        atomicAdd(loss, x * inv_n);
    }
}

}  // namespace

void launch_mask_loss(const float *mask, const float *shmask, int64_t n, float lam_m, float lam_sh, float *loss,
                      float *gmask, float *gshmask, cudaStream_t st) {
    if (n <= 0 || (!mask && !shmask) || (!loss && !gmask && !gshmask)) return;
    int64_t blocks = (n + 255) / 256;
    if (blocks > 152 * 8) blocks = 152 * 8;
    count_launch();
    k_mask_loss<<<(unsigned)blocks, 256, 0, st>>>(mask, shmask, n, lam_m, lam_sh, (float)(1.0 / (double)n), loss,
                                                   gmask, gshmask);
}

void launch_preprocess(const GaussPtrs &g, const CamBatch &cb, float4 *splats, int32_t *radii,
                       uint32_t *tiles_touched, uint32_t *depth_bits, float *zero_grads,
                       cudaStream_t st) {
    if (g.n <= 0) return;
    const int bs = 128;
    const int64_t grid = (g.n + bs - 1) / bs;
    count_launch();
    if (g.half)
        k_preprocess<__half><<<(unsigned)grid, bs, 0, st>>>(g, cb, splats, radii, tiles_touched, depth_bits,
                                                            reinterpret_cast<float4 *>(zero_grads));
    else
        k_preprocess<float><<<(unsigned)grid, bs, 0, st>>>(g, cb, splats, radii, tiles_touched, depth_bits,
                                                           reinterpret_cast<float4 *>(zero_grads));
}

void launch_preprocess_backward(const GaussPtrs &g, const CamBatch &cb, const float4 *sgrads,
                                const int32_t *radii, const GradPtrs &out, int no_sh_rest,
                                int moments, cudaStream_t st) {
    if (g.n <= 0) return;
    const int bs = kBwdThreads;
    const int64_t grid = (g.n + bs - 1) / bs;
    count_launch();
    k_preprocess_bwd_colour<<<(unsigned)grid, bs, 0, st>>>(g, cb, sgrads, radii, out, no_sh_rest);
    count_launch();
    k_preprocess_bwd_geom<<<(unsigned)grid, bs, 0, st>>>(g, cb, sgrads, radii, out, moments);
}

}  // namespace tgs
