// tgs_bin_noalloc: the binning step (tgs_bin) for callers that cannot allocate device memory.
//
// Its scratch lives in one file-scope __device__ array of fixed size instead of a context's
// arena, so the call needs no tgs_ctx and never calls cudaMalloc or cudaFree. Host code cannot
// use the array's name as a device address (on the host it names a host-side shadow), so the
// device address is looked up once per device with cudaGetSymbolAddress and cached.
#include <cuda_runtime.h>

#include <cstring>
#include <mutex>

#include "tgs_internal.cuh"

using namespace tgs;

namespace {

constexpr int64_t kRec = TGS_NOALLOC_MAX_RECORDS;
constexpr int64_t kKeys = TGS_NOALLOC_MAX_KEYS;
// at least the sizes radix_hist_needed / scan_partials_needed in sort.cu ask for (its sort blocks
// hold at least 2048 items; checked at set-up)
constexpr int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }
constexpr int64_t round4(int64_t a) { return (a + 3) / 4 * 4; }  // 16-byte aligned regions
constexpr int64_t kItems = kRec > kKeys ? kRec : kKeys;
constexpr int64_t kHist = 256 * ceil_div(kItems, 2048) + 256;
constexpr int64_t kPartials = ceil_div(kHist > kItems ? kHist : kItems, 2048) + 1;
constexpr int64_t kBlockOffs = ceil_div(kRec, 2048) + 1;
// word offsets inside the scratch array
constexpr int64_t oTT = 0, oDB = oTT + kRec, oPOS = oDB + kRec, oCK0 = oPOS + kRec,
                  oCV0 = oCK0 + kRec, oCK1 = oCV0 + kRec, oCV1 = oCK1 + kRec,
                  oTK0 = oCV1 + kRec, oTV0 = oTK0 + kKeys, oTK1 = oTV0 + kKeys, oTV1 = oTK1 + kKeys,
                  oKM = oTV1 + kKeys, oOFF = oKM + 2 * kRec, oHIST = round4(oOFF + kBlockOffs),
                  oPART = round4(oHIST + kHist), oCNT = round4(oPART + kPartials), oSTAT = oCNT + 4,
                  kWords = oSTAT + 4;

// The scratch of every tgs_bin_noalloc call on a device (about 13.4 MB, held until exit).
static __device__ __align__(256) uint32_t g_noalloc_scratch[kWords];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
uint32_t *g_dev_ptr[kMaxDevices] = {};

// Device address of the scratch array on the current device (looked up on first use).
tgs_status scratch_ptr(uint32_t **out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        cudaGetLastError();
        return TGS_ERR_CUDA;
    }
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_dev_ptr[dev]) {
        if ((size_t)radix_hist_needed(kItems) > (size_t)kHist ||
            scan_partials_needed(kHist > kItems ? kHist : kItems) > (size_t)kPartials ||
            scan_partials_needed(kRec) > (size_t)kBlockOffs)
            return TGS_ERR_NOT_SUPPORTED;
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            cudaGetLastError();
            return TGS_ERR_CUDA;
        }
        g_dev_ptr[dev] = static_cast<uint32_t *>(p);
    }
    *out = g_dev_ptr[dev];
    return TGS_OK;
}

int bits_for_tiles(int64_t x) {
    int b = 0;
    while (((int64_t)1 << b) < x) b++;
    return b < 1 ? 1 : b;
}

tgs_status cam_batch(const tgs_camera *cams, int V, int tile, CamBatch &cb) {
    if (!cams || V <= 0 || V > kMaxViews) return TGS_ERR_INVALID_ARG;
    if (tile != 8 && tile != 16 && tile != 32) return TGS_ERR_INVALID_ARG;
    memset(&cb, 0, sizeof cb);
    cb.V = V;
    cb.tile = tile;
    int off = 0;
    for (int v = 0; v < V; v++) {
        const tgs_camera &c = cams[v];
        if (c.width <= 0 || c.height <= 0 || c.width > 65535 || c.height > 65535) return TGS_ERR_INVALID_ARG;
        DevCam &d = cb.c[v];
        d.W = c.width;
        d.H = c.height;
        d.gx = (c.width + tile - 1) / tile;
        d.gy = (c.height + tile - 1) / tile;
        d.tile_offset = off;
        off += d.gx * d.gy;
    }
    cb.total_tiles = off;
    return TGS_OK;
}

}  // namespace

extern "C" tgs_status tgs_bin_noalloc(const float *splats, const int32_t *radii, int64_t n,
                                      const tgs_camera *cams, int32_t V, int32_t tile,
                                      uint32_t *sorted_ids, uint64_t *sorted_keys, uint32_t *ranges,
                                      int64_t capacity, int64_t *K_out, tgs_stream stream) {
    if (K_out) *K_out = 0;
    if (!splats || !radii || n < 0 || !sorted_ids || !ranges || capacity < 0) return TGS_ERR_INVALID_ARG;
    CamBatch cb;
    tgs_status s = cam_batch(cams, V, tile, cb);
    if (s != TGS_OK) return s;
    const int64_t nt = n * V;
    if (nt > kRec) return TGS_ERR_SCRATCH_LIMIT;
    uint32_t *w = nullptr;
    s = scratch_ptr(&w);
    if (s != TGS_OK) return s;
    cudaStream_t st = (cudaStream_t)stream;
    uint32_t *cnt = w + oCNT, *status = w + oSTAT;
    // the array keeps the previous call's contents: clear the words read before written
    if (cudaMemsetAsync(cnt, 0, sizeof(uint32_t) * 8, st) != cudaSuccess) return TGS_ERR_CUDA;

    derive_touched(reinterpret_cast<const float4 *>(splats), radii, nt, tile, nullptr, w + oDB, st);
    uint32_t *k = w + oDB, *v = w + oCV0;
    radix_sort_pairs(k, v, w + oCK1, w + oCV1, nullptr, nt, 0, 32, w + oHIST, w + oPART, st, true);
    // the per-record arrays free during the binning hold the key counts of the depth order
    const KeyInfo ki{w + oPOS, reinterpret_cast<uint2 *>(w + oKM), w + oCK0, w + oTT};
    count_keys(v, k, nullptr, nt, reinterpret_cast<const float4 *>(splats), tile, ki, w + oOFF, cnt + 1, st);

    uint32_t hK = 0;
    if (cudaMemcpyAsync(&hK, cnt + 1, sizeof hK, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess) {
        cudaGetLastError();
        return TGS_ERR_CUDA;
    }
    const int64_t K = hK;
    if (K_out) *K_out = K;
    if (K > kKeys) return TGS_ERR_SCRATCH_LIMIT;
    if (K > capacity) return TGS_ERR_CAPACITY;

    const int64_t cap = K > 0 ? K : 1;
    emit_keys(v, w + oOFF, nullptr, nt, ki, reinterpret_cast<const float4 *>(splats), n, cb, w + oTK0, w + oTV0,
              cnt + 1, cap, status, st);
    uint32_t *tk = w + oTK0, *tv = w + oTV0;
    radix_sort_pairs(tk, tv, w + oTK1, w + oTV1, cnt + 1, cap, 0, bits_for_tiles(cb.total_tiles),
                     w + oHIST, w + oPART, st);
    find_ranges(tk, cnt + 1, cap, reinterpret_cast<uint2 *>(ranges), cb.total_tiles, st);
    if (K > 0) {
        if (cudaMemcpyAsync(sorted_ids, tv, sizeof(uint32_t) * (size_t)K, cudaMemcpyDeviceToDevice, st) !=
            cudaSuccess)
            return TGS_ERR_CUDA;
        if (sorted_keys)
            make_full_keys(tk, tv, reinterpret_cast<const float4 *>(splats), cnt + 1, K, sorted_keys, st);
    }
    return cudaGetLastError() == cudaSuccess ? TGS_OK : TGS_ERR_CUDA;
}
