// libtgs host runtime: context, scratch arena, the plain and batched paths, CUDA-graph
// capture of the batched step, and the autotuner. Every entry point is extern "C" and
// returns a tgs_status; no exception crosses the ABI.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "tgs_internal.cuh"

using namespace tgs;

namespace tgs {
thread_local int64_t g_launches = 0;
}

namespace {

struct Buf {
    void *p = nullptr;
    size_t bytes = 0;
};

}  // namespace

struct tgs_ctx {
    tgs_config cfg;
    int device = 0;
    // scratch arena
    Buf splats, radii, tt, dbits, pos, ck0, cv0, ck1, cv1, offsets, tk0, tv0, tk1, tv1, ranges,
        hist, partials, sgrads, counts, status, pixstate, dimg, images, items, kmask, viskeys, ssim, cbuf;
    uint32_t *h_counts = nullptr;   // pinned host copy of (visible, K)
    // binning kept from the last plain forward
    bool state_valid = false;
    tgs_gaussians state_g{};
    tgs_camera state_cam{};
    int state_tile = 0;
    uint32_t *state_ids = nullptr;  // where the sorted ids of that binning live
    uint32_t *sorted_tk = nullptr;  // sorted tile keys of the last binning
    // captured batched steps, keyed by every argument the recorded launches depend on
    // (a few, so that alternating input buffers each keep their graph)
    struct Graph {
        std::vector<unsigned char> key;
        cudaGraphExec_t exec = nullptr;
        uint64_t used = 0;
    };
    std::vector<Graph> graphs;
    uint64_t graph_clock = 0;
    cudaStream_t side = nullptr;
    // tgs_train_step_batched_host: three sets of device copies of a step's inputs, filled on an
    // upload stream while the previous steps compute (the copies of a step may run up to two
    // steps ahead, which absorbs a slow copy)
    struct Stage {
        Buf params, targets;
        cudaEvent_t copied = nullptr, consumed = nullptr;
        bool used = false;
    };
    static constexpr int kStages = 3;
    Stage stage[kStages];
    int stage_next = 0;
    cudaStream_t upload = nullptr;
    Buf lossbuf;
    // measurement
    bool profiling = false;
    cudaEvent_t stage_ev[TGS_MAX_STAGES + 1] = {};
    const char *stage_names[TGS_MAX_STAGES] = {};
    int n_stages = 0;
    int64_t kernels_per_step = 0;
};

namespace {

tgs_status cuda_status(cudaError_t e) { return e == cudaSuccess ? TGS_OK : TGS_ERR_CUDA; }

void drop_graphs(tgs_ctx *c) {
    for (auto &gr : c->graphs)
        if (gr.exec) cudaGraphExecDestroy(gr.exec);
    c->graphs.clear();
}

#define TGS_CHECK(x)                                   \
    do {                                               \
        cudaError_t e_ = (x);                          \
        if (e_ != cudaSuccess) return TGS_ERR_CUDA;    \
    } while (0)

#define TGS_TRY(x)                     \
    do {                               \
        tgs_status s_ = (x);           \
        if (s_ != TGS_OK) return s_;   \
    } while (0)

bool capturing(cudaStream_t st) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cs) != cudaSuccess) return false;
    return cs != cudaStreamCaptureStatusNone;
}

// Grows a scratch buffer; never inside stream capture.
// Bumped on every reallocation of a device buffer: part of every captured graph's key, so that
// no graph holding a freed buffer's address is replayed (it no longer matches and ages out).
std::atomic<uint64_t> g_arena_gen{0};

tgs_status ensure(Buf &b, size_t bytes, cudaStream_t st) {
    if (bytes == 0) bytes = 16;
    if (b.bytes >= bytes) return TGS_OK;
    if (capturing(st)) return TGS_ERR_CAPACITY;
    g_arena_gen.fetch_add(1);
    size_t nb = bytes + bytes / 4;
    if (b.p) {
        cudaStreamSynchronize(st);
        cudaFree(b.p);
        b.p = nullptr;
        b.bytes = 0;
    }
    if (cudaMalloc(&b.p, nb) != cudaSuccess) {
        cudaGetLastError();
        return TGS_ERR_OOM;
    }
    b.bytes = nb;
    return TGS_OK;
}

template <class T>
T *as(Buf &b) { return reinterpret_cast<T *>(b.p); }

bool valid_cfg(const tgs_config &c) {
    return blend_supported(c.tile, c.ppt) && (c.support == TGS_SUPPORT_BOX3 || c.support == TGS_SUPPORT_ALPHA) &&
           c.low_pass >= 0.f && c.eps_mask > 0.f && c.eps_mask < 1.f && c.eps_sh > 0.f && c.eps_sh < 1.f &&
           c.near_plane > 0.f && c.key_capacity >= 0 && c.ssim_lambda >= 0.f && c.ssim_lambda <= 1.f &&
           c.lambda_mask >= 0.f && c.lambda_mask < 1e30f && c.lambda_sh_mask >= 0.f && c.lambda_sh_mask < 1e30f &&
           c.batch >= 0 && c.batch <= 2;
}

tgs_status make_batch(const tgs_config &cfg, const tgs_camera *cams, int V, CamBatch &cb) {
    if (!cams || V <= 0 || V > kMaxViews) return TGS_ERR_INVALID_ARG;
    memset(&cb, 0, sizeof cb);
    cb.V = V;
    cb.tile = cfg.tile;
    int off = 0, poff = 0;
    for (int v = 0; v < V; v++) {
        const tgs_camera &c = cams[v];
        if (c.width <= 0 || c.height <= 0 || c.width > 65535 || c.height > 65535 || !(c.fx > 0.f) ||
            !(c.fy > 0.f))
            return TGS_ERR_INVALID_ARG;
        DevCam &d = cb.c[v];
        for (int r = 0; r < 3; r++) {
            for (int k = 0; k < 3; k++) d.R[3 * r + k] = c.viewmat[4 * r + k];
            d.t[r] = c.viewmat[4 * r + 3];
            d.campos[r] = c.campos[r];
        }
        d.fx = c.fx;
        d.fy = c.fy;
        d.cx = c.cx;
        d.cy = c.cy;
        d.limx = (float)(1.3 * (0.5 * c.width / (double)c.fx));
        d.limy = (float)(1.3 * (0.5 * c.height / (double)c.fy));
        d.s = c.low_pass > 0.f ? c.low_pass : cfg.low_pass;
        d.W = c.width;
        d.H = c.height;
        d.gx = (c.width + cfg.tile - 1) / cfg.tile;
        d.gy = (c.height + cfg.tile - 1) / cfg.tile;
        d.tile_offset = off;
        d.pix_offset = poff;
        off += d.gx * d.gy;
        poff += c.width * c.height;
    }
    cb.total_tiles = off;
    return TGS_OK;
}

float logit_threshold(float eps) { return (float)std::log((double)eps / (1.0 - (double)eps)); }

tgs_status make_gauss(const tgs_config &cfg, const tgs_gaussians *g, GaussPtrs &gp, bool allow_half = false) {
    if (!g || g->n < 0) return TGS_ERR_INVALID_ARG;
    if (g->param_dtype != TGS_PARAM_F32 && g->param_dtype != TGS_PARAM_F16) return TGS_ERR_INVALID_ARG;
    if (g->param_dtype == TGS_PARAM_F16 && !allow_half) return TGS_ERR_NOT_SUPPORTED;
    // an empty scene may come with null pointers
    if (g->n > 0 && (!g->means || !g->log_scales || !g->quats || !g->opacity_logits || !g->sh_dc))
        return TGS_ERR_INVALID_ARG;
    if (g->sh_degree_max < 0 || g->sh_degree_max > 3) return TGS_ERR_INVALID_ARG;
    if (g->n > 0 && g->sh_degree_max > 0 && !g->sh_rest) return TGS_ERR_INVALID_ARG;
    if ((int64_t)g->n * kMaxViews >= (int64_t)1 << 32) return TGS_ERR_INVALID_ARG;
    gp.means = g->means;
    gp.log_scales = g->log_scales;
    gp.quats = g->quats;
    gp.opac = g->opacity_logits;
    gp.sh_dc = g->sh_dc;
    gp.sh_rest = g->sh_rest;
    gp.sh_degree = g->sh_degree;
    gp.mask = g->mask_logits;
    gp.shmask = g->sh_mask_logits;
    gp.n = g->n;
    gp.deg_max = g->sh_degree_max;
    gp.tau_m = logit_threshold(cfg.eps_mask);
    gp.tau_sh = logit_threshold(cfg.eps_sh);
    gp.support = cfg.support;
    gp.near_z = cfg.near_plane;
    gp.half = g->param_dtype == TGS_PARAM_F16 ? 1 : 0;
    return TGS_OK;
}

int bits_for(int64_t x) {
    int b = 0;
    while (((int64_t)1 << b) < x) b++;
    return b < 1 ? 1 : b;
}

// Buffers for V views of n Gaussians (per-record arrays).
tgs_status ensure_records(tgs_ctx *c, int64_t nt, cudaStream_t st) {
    TGS_TRY(ensure(c->splats, sizeof(float) * kSplatWords * (size_t)nt, st));
    TGS_TRY(ensure(c->sgrads, sizeof(float) * 12 * (size_t)nt, st));
    TGS_TRY(ensure(c->radii, sizeof(int32_t) * (size_t)nt, st));
    TGS_TRY(ensure(c->tt, sizeof(uint32_t) * (size_t)nt, st));
    TGS_TRY(ensure(c->dbits, sizeof(uint32_t) * (size_t)nt, st));
    TGS_TRY(ensure(c->pos, sizeof(uint32_t) * (size_t)nt, st));
    TGS_TRY(ensure(c->ck0, sizeof(uint32_t) * (size_t)nt, st));
    TGS_TRY(ensure(c->cv0, sizeof(uint32_t) * (size_t)nt, st));
    TGS_TRY(ensure(c->ck1, sizeof(uint32_t) * (size_t)nt, st));
    TGS_TRY(ensure(c->cv1, sizeof(uint32_t) * (size_t)nt, st));
    TGS_TRY(ensure(c->offsets, sizeof(uint32_t) * scan_partials_needed(nt), st));  // per block of records
    TGS_TRY(ensure(c->kmask, sizeof(uint2) * (size_t)nt, st));
    TGS_TRY(ensure(c->counts, sizeof(uint32_t) * 4, st));
    size_t h = std::max(radix_hist_needed(nt), (size_t)16);
    TGS_TRY(ensure(c->hist, sizeof(uint32_t) * h, st));
    size_t p = std::max(scan_partials_needed(nt), scan_partials_needed((int64_t)h));
    TGS_TRY(ensure(c->partials, sizeof(uint32_t) * p, st));
    return TGS_OK;
}

tgs_status ensure_keys(tgs_ctx *c, int64_t cap, int total_tiles, cudaStream_t st) {
    TGS_TRY(ensure(c->tk0, sizeof(uint32_t) * (size_t)cap, st));
    TGS_TRY(ensure(c->tv0, sizeof(uint32_t) * (size_t)cap, st));
    TGS_TRY(ensure(c->tk1, sizeof(uint32_t) * (size_t)cap, st));
    TGS_TRY(ensure(c->tv1, sizeof(uint32_t) * (size_t)cap, st));
    TGS_TRY(ensure(c->ranges, sizeof(uint2) * (size_t)std::max(total_tiles, 1), st));
    TGS_TRY(ensure(c->viskeys, sizeof(uint16_t) * (size_t)cap, st));  // fused blend's per-key masks
    size_t h = radix_hist_needed(cap);
    TGS_TRY(ensure(c->hist, sizeof(uint32_t) * std::max(h, c->hist.bytes / sizeof(uint32_t)), st));
    size_t p = std::max(scan_partials_needed(cap), scan_partials_needed((int64_t)h));
    TGS_TRY(ensure(c->partials, sizeof(uint32_t) * std::max(p, c->partials.bytes / sizeof(uint32_t)), st));
    return TGS_OK;
}

// Visibility compaction, depth sort and the key-count scan. Leaves the depth-sorted record
// ids in *sorted and the key count in counts[1].
// The per-record arrays free during the binning hold the key counts of the depth order.
KeyInfo key_info(tgs_ctx *c) {
    return KeyInfo{as<uint32_t>(c->pos), as<uint2>(c->kmask), as<uint32_t>(c->ck0), as<uint32_t>(c->tt)};
}

// Depth sort of all records (depth keys from the preprocess; records not visible sort last)
// and the key counts of the depth order. Leaves the sorted record ids in *sorted and the key
// count in counts[1].
void bin_front(tgs_ctx *c, int64_t nt, uint32_t **sorted, cudaStream_t st) {
    uint32_t *cnt = as<uint32_t>(c->counts);
    uint32_t *k = as<uint32_t>(c->dbits), *v = as<uint32_t>(c->cv0);
    radix_sort_pairs(k, v, as<uint32_t>(c->ck1), as<uint32_t>(c->cv1), nullptr, nt, 0, 32,
                     as<uint32_t>(c->hist), as<uint32_t>(c->partials), st, true);
    count_keys(v, k, nullptr, nt, as<float4>(c->splats), c->cfg.tile, key_info(c), as<uint32_t>(c->offsets),
               cnt + 1, st);
    *sorted = v;
}

// Key emission, tile sort and ranges for a key grid of cap. Returns the sorted record ids.
uint32_t *bin_back(tgs_ctx *c, int64_t nt, int64_t n, const uint32_t *sorted, const CamBatch &cb,
                   int64_t cap, cudaStream_t st) {
    uint32_t *cnt = as<uint32_t>(c->counts);
    emit_keys(sorted, as<uint32_t>(c->offsets), nullptr, nt, key_info(c), as<float4>(c->splats), n, cb,
              as<uint32_t>(c->tk0), as<uint32_t>(c->tv0), cnt + 1, cap, as<uint32_t>(c->status), st);
    uint32_t *k = as<uint32_t>(c->tk0), *v = as<uint32_t>(c->tv0);
    radix_sort_pairs(k, v, as<uint32_t>(c->tk1), as<uint32_t>(c->tv1), cnt + 1, cap, 0,
                     bits_for(cb.total_tiles), as<uint32_t>(c->hist), as<uint32_t>(c->partials), st);
    find_ranges(k, cnt + 1, cap, as<uint2>(c->ranges), cb.total_tiles, st);
    c->sorted_tk = k;  // tgs_bin exports the 64-bit keys from these
    return v;
}

// Synchronous read of the key count K after bin_front.
tgs_status read_counts(tgs_ctx *c, cudaStream_t st, int64_t *K) {
    TGS_CHECK(cudaMemcpyAsync(c->h_counts, c->counts.p, sizeof(uint32_t) * 2, cudaMemcpyDeviceToHost, st));
    TGS_CHECK(cudaStreamSynchronize(st));
    if (K) *K = c->h_counts[1];
    return TGS_OK;
}

// Full plain binning of V views whose splat records are already in the arena.
tgs_status bin_plain(tgs_ctx *c, int64_t n, const CamBatch &cb, cudaStream_t st, int64_t *K_out,
                     int64_t cap_limit, uint32_t **ids) {
    const int64_t nt = n * cb.V;
    uint32_t *sorted = nullptr;
    bin_front(c, nt, &sorted, st);
    int64_t K = 0;
    TGS_TRY(read_counts(c, st, &K));
    if (K_out) *K_out = K;
    if (cap_limit >= 0 && K > cap_limit) return TGS_ERR_CAPACITY;
    TGS_TRY(ensure_keys(c, std::max<int64_t>(K, 1), cb.total_tiles, st));
    *ids = bin_back(c, nt, n, sorted, cb, std::max<int64_t>(K, 1), st);
    if (K == 0) {
        cudaMemsetAsync(c->ranges.p, 0, sizeof(uint2) * (size_t)std::max(cb.total_tiles, 1), st);
    }
    return TGS_OK;
}

PixPtrs pix_for(const tgs_view_out *outs, int V, const float *const *dL) {
    PixPtrs p;
    memset(&p, 0, sizeof p);
    for (int v = 0; v < V; v++) {
        p.image[v] = outs[v].image;
        p.T_final[v] = outs[v].T_final;
        p.last[v] = outs[v].last;
        p.n_exam[v] = outs[v].n_examined;
        p.n_contrib[v] = outs[v].n_contrib;
        p.n_eval[v] = outs[v].n_eval;
        p.dL[v] = dL ? dL[v] : nullptr;
    }
    return p;
}

GradPtrs grad_ptrs(const tgs_grads *g, const tgs_stats *s, int acc) {
    GradPtrs o;
    memset(&o, 0, sizeof o);
    if (g) {
        o.means = g->means;
        o.log_scales = g->log_scales;
        o.quats = g->quats;
        o.opac = g->opacity_logits;
        o.sh_dc = g->sh_dc;
        o.sh_rest = g->sh_rest;
        o.mask = g->mask_logits;
        o.shmask = g->sh_mask_logits;
    }
    if (s) {
        o.stat_accum = s->grad_norm_accum;
        o.stat_count = s->vis_count;
        o.stat_maxr = s->max_radius;
    }
    o.accumulate = acc;
    return o;
}

// The mask losses of Eq. loss3dgs folded into the preprocess backward (TGS_MASK_LOSS).
void with_mask_loss(const tgs_config &cfg, int64_t n, GradPtrs &o) {
    if (n <= 0) return;
    o.lam_m_n = (float)((double)cfg.lambda_mask / (double)n);
    o.lam_sh_n = (float)((double)cfg.lambda_sh_mask / (double)n);
}

// Entries of the autotuner's JSON cache, {"key": {"tile": T, "ppt": P, "batch": B}, ...}, with any
// whitespace and field order; "batch" defaults to 1; malformed entries are skipped.
template <class F>
void parse_tune_cache(const std::string &s, F &&emit) {
    size_t i = 0;
    const size_t n = s.size();
    auto skip_ws = [&]() {
        while (i < n && (s[i] == ' ' || s[i] == '\n' || s[i] == '\r' || s[i] == '\t')) i++;
    };
    auto read_str = [&](std::string &out) {
        if (i >= n || s[i] != '"') return false;
        const size_t e = s.find('"', i + 1);
        if (e == std::string::npos) return false;
        out = s.substr(i + 1, e - i - 1);
        i = e + 1;
        return true;
    };
    skip_ws();
    if (i >= n || s[i] != '{') return;
    i++;
    for (;;) {
        skip_ws();
        std::string key;
        if (!read_str(key)) return;
        skip_ws();
        if (i >= n || s[i] != ':') return;
        i++;
        skip_ws();
        if (i >= n || s[i] != '{') return;
        i++;
        int vals[3] = {0, 0, 1};  // tile, ppt, batch
        for (;;) {
            skip_ws();
            if (i < n && s[i] == '}') {
                i++;
                break;
            }
            std::string field;
            if (!read_str(field)) return;
            skip_ws();
            if (i >= n || s[i] != ':') return;
            i++;
            skip_ws();
            char *end = nullptr;
            const long v = strtol(s.c_str() + i, &end, 10);
            if (end == s.c_str() + i) return;
            i = (size_t)(end - s.c_str());
            if (field == "tile") vals[0] = (int)v;
            else if (field == "ppt") vals[1] = (int)v;
            else if (field == "batch") vals[2] = (int)v;
            skip_ws();
            if (i < n && s[i] == ',') i++;
        }
        emit(key, vals[0], vals[1], vals[2]);
        skip_ws();
        if (i < n && s[i] == ',') {
            i++;
            continue;
        }
        return;
    }
}

bool same_cam(const tgs_camera &a, const tgs_camera &b) { return memcmp(&a, &b, sizeof a) == 0; }
bool same_g(const tgs_gaussians &a, const tgs_gaussians &b) { return memcmp(&a, &b, sizeof a) == 0; }

tgs_status last_error() { return cuda_status(cudaGetLastError()); }

// Records the boundary event before stage i (profiling only).
void mark(tgs_ctx *c, int i, const char *name, cudaStream_t st) {
    if (!c->profiling || i > TGS_MAX_STAGES) return;
    // inside stream capture only an external record becomes a node of the graph
    if (capturing(st))
        cudaEventRecordWithFlags(c->stage_ev[i], st, cudaEventRecordExternal);
    else
        cudaEventRecord(c->stage_ev[i], st);
    if (i < TGS_MAX_STAGES) c->stage_names[i] = name;
    c->n_stages = i;
}

}  // namespace

extern "C" {

void tgs_default_config(tgs_config *cfg) {
    if (!cfg) return;
    memset(cfg, 0, sizeof *cfg);
    cfg->tile = 16;
    cfg->ppt = 1;
    cfg->support = TGS_SUPPORT_BOX3;
    cfg->low_pass = 0.3f;
    cfg->eps_mask = 0.05f;
    cfg->eps_sh = 0.1f;
    cfg->near_plane = 0.2f;
    cfg->key_capacity = 0;
    cfg->spin_limit = 0;  // reserved
    cfg->ssim_lambda = 0.2f;
    cfg->lambda_mask = 0.05f;
    cfg->lambda_sh_mask = 0.05f;
}

const char *tgs_status_string(tgs_status s) {
    switch (s) {
        case TGS_OK: return "ok";
        case TGS_ERR_INVALID_ARG: return "invalid argument";
        case TGS_ERR_CUDA: return "CUDA runtime error";
        case TGS_ERR_CAPACITY: return "key capacity exceeded";
        case TGS_ERR_TIMEOUT: return "reserved status (timeout)";
        case TGS_ERR_OOM: return "out of device memory";
        case TGS_ERR_NOT_SUPPORTED: return "not supported";
        case TGS_ERR_SCRATCH_LIMIT: return "input exceeds the fixed scratch of tgs_bin_noalloc";
        case TGS_ERR_INCONSISTENT: return "device consistency check of the key counts failed";
        default: return "unknown status";
    }
}

tgs_status tgs_create(tgs_ctx **out, const tgs_config *cfg) {
    if (!out) return TGS_ERR_INVALID_ARG;
    *out = nullptr;
    tgs_config c;
    if (cfg) c = *cfg; else tgs_default_config(&c);
    if (!valid_cfg(c)) return TGS_ERR_INVALID_ARG;
    tgs_ctx *x = new (std::nothrow) tgs_ctx();
    if (!x) return TGS_ERR_OOM;
    x->cfg = c;
    if (cudaGetDevice(&x->device) != cudaSuccess ||
        cudaMallocHost((void **)&x->h_counts, sizeof(uint32_t) * 4) != cudaSuccess) {
        cudaGetLastError();
        delete x;
        return TGS_ERR_CUDA;
    }
    if (ensure(x->status, sizeof(uint32_t) * 4, nullptr) != TGS_OK ||
        ensure(x->counts, sizeof(uint32_t) * 4, nullptr) != TGS_OK) {
        tgs_destroy(x);
        return TGS_ERR_OOM;
    }
    cudaMemset(x->status.p, 0, x->status.bytes);
    cudaMemset(x->counts.p, 0, x->counts.bytes);
    *out = x;
    return TGS_OK;
}

void tgs_destroy(tgs_ctx *c) {
    if (!c) return;
    cudaDeviceSynchronize();
    Buf *bufs[] = {&c->splats, &c->radii, &c->tt, &c->dbits, &c->pos, &c->ck0, &c->cv0, &c->ck1,
                   &c->cv1, &c->offsets, &c->tk0, &c->tv0, &c->tk1, &c->tv1, &c->ranges, &c->hist,
                   &c->partials, &c->sgrads, &c->counts, &c->status, &c->pixstate, &c->dimg,
                   &c->images, &c->items, &c->kmask, &c->viskeys, &c->ssim, &c->cbuf};
    for (Buf *b : bufs)
        if (b->p) cudaFree(b->p);
    if (c->h_counts) cudaFreeHost(c->h_counts);
    drop_graphs(c);
    for (auto &sg : c->stage) {
        if (sg.params.p) cudaFree(sg.params.p);
        if (sg.targets.p) cudaFree(sg.targets.p);
        if (sg.copied) cudaEventDestroy(sg.copied);
        if (sg.consumed) cudaEventDestroy(sg.consumed);
    }
    if (c->lossbuf.p) cudaFree(c->lossbuf.p);
    if (c->upload) cudaStreamDestroy(c->upload);
    if (c->side) cudaStreamDestroy(c->side);
    for (cudaEvent_t e : c->stage_ev)
        if (e) cudaEventDestroy(e);
    delete c;
}

tgs_status tgs_get_config(const tgs_ctx *c, tgs_config *cfg) {
    if (!c || !cfg) return TGS_ERR_INVALID_ARG;
    *cfg = c->cfg;
    return TGS_OK;
}

tgs_status tgs_set_config(tgs_ctx *c, const tgs_config *cfg) {
    if (!c || !cfg || !valid_cfg(*cfg)) return TGS_ERR_INVALID_ARG;
    c->cfg = *cfg;
    c->state_valid = false;
    drop_graphs(c);
    return TGS_OK;
}

tgs_status tgs_poll_status(tgs_ctx *c, tgs_stream stream) {
    if (!c) return TGS_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    uint32_t h = 0;
    TGS_CHECK(cudaMemcpyAsync(c->h_counts + 2, c->status.p, sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
    TGS_CHECK(cudaStreamSynchronize(st));
    h = c->h_counts[2];
    TGS_CHECK(cudaMemsetAsync(c->status.p, 0, sizeof(uint32_t), st));
    TGS_CHECK(cudaStreamSynchronize(st));
    if (h & kStatusInconsistent) return TGS_ERR_INCONSISTENT;
    if (h & kStatusCapacity) return TGS_ERR_CAPACITY;
    return TGS_OK;
}

int64_t tgs_num_tiles(const tgs_ctx *c, const tgs_camera *cams, int32_t V) {
    if (!c) return -1;
    CamBatch cb;
    if (make_batch(c->cfg, cams, V, cb) != TGS_OK) return -1;
    return cb.total_tiles;
}

size_t tgs_workspace_bytes(const tgs_ctx *c, int64_t n, const tgs_camera *cams, int32_t V) {
    if (!c) return 0;
    CamBatch cb;
    if (make_batch(c->cfg, cams, V, cb) != TGS_OK) return 0;
    const size_t nt = (size_t)n * V;
    size_t pix = 0;
    for (int v = 0; v < V; v++) pix += (size_t)cams[v].width * cams[v].height;
    const size_t cap = (size_t)c->cfg.key_capacity;
    return nt * (kSplatWords * 4 + 12 * 4 + 4 * 9) + cap * 16 + (size_t)cb.total_tiles * 8 +
           radix_hist_needed((int64_t)std::max(nt, cap)) * 4 + pix * 4 * (3 + 2 + 3 + 3);
}

// ---- individual steps -------------------------------------------------------------------

tgs_status tgs_preprocess(tgs_ctx *c, const tgs_gaussians *g, const tgs_camera *cams, int32_t V,
                          float *splats, int32_t *radii, tgs_stream stream) {
    if (!c || !splats || !radii) return TGS_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    CamBatch cb;
    GaussPtrs gp;
    TGS_TRY(make_batch(c->cfg, cams, V, cb));
    TGS_TRY(make_gauss(c->cfg, g, gp, true));
    const int64_t nt = g->n * V;
    TGS_TRY(ensure(c->tt, sizeof(uint32_t) * (size_t)nt, st));
    TGS_TRY(ensure(c->dbits, sizeof(uint32_t) * (size_t)nt, st));
    launch_preprocess(gp, cb, reinterpret_cast<float4 *>(splats), radii, nullptr,
                      as<uint32_t>(c->dbits), nullptr, st);
    return last_error();
}

tgs_status tgs_bin(tgs_ctx *c, const float *splats, const int32_t *radii, int64_t n,
                   const tgs_camera *cams, int32_t V, uint32_t *sorted_ids, uint64_t *sorted_keys,
                   uint32_t *ranges, int64_t capacity, int64_t *K_out, tgs_stream stream) {
    if (!c || !splats || !radii || n < 0 || !sorted_ids || !ranges || capacity < 0) return TGS_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    CamBatch cb;
    TGS_TRY(make_batch(c->cfg, cams, V, cb));
    const int64_t nt = n * V;
    TGS_TRY(ensure_records(c, nt, st));
    // records come from the caller: copy them in and derive tiles touched and depth bits
    TGS_CHECK(cudaMemcpyAsync(c->splats.p, splats, sizeof(float) * kSplatWords * (size_t)nt, cudaMemcpyDeviceToDevice, st));
    TGS_CHECK(cudaMemcpyAsync(c->radii.p, radii, sizeof(int32_t) * (size_t)nt, cudaMemcpyDeviceToDevice, st));
    derive_touched(as<float4>(c->splats), as<int32_t>(c->radii), nt, c->cfg.tile, nullptr,
                   as<uint32_t>(c->dbits), st);
    int64_t K = 0;
    uint32_t *ids = nullptr;
    tgs_status s = bin_plain(c, n, cb, st, &K, capacity, &ids);
    if (K_out) *K_out = K;
    if (s != TGS_OK) return s;
    c->state_valid = false;
    if (K > 0) {
        TGS_CHECK(cudaMemcpyAsync(sorted_ids, ids, sizeof(uint32_t) * (size_t)K, cudaMemcpyDeviceToDevice, st));
        if (sorted_keys)
            make_full_keys(c->sorted_tk, ids, as<float4>(c->splats), as<uint32_t>(c->counts) + 1, K,
                           sorted_keys, st);
    }
    TGS_CHECK(cudaMemcpyAsync(ranges, c->ranges.p, sizeof(uint2) * (size_t)cb.total_tiles, cudaMemcpyDeviceToDevice, st));
    return last_error();
}

tgs_status tgs_blend_forward(tgs_ctx *c, const float *splats, const uint32_t *sorted_ids,
                             const uint32_t *ranges, const tgs_camera *cams, int32_t V,
                             const tgs_view_out *outs, tgs_stream stream) {
    if (!c || !splats || !ranges || !outs) return TGS_ERR_INVALID_ARG;
    CamBatch cb;
    TGS_TRY(make_batch(c->cfg, cams, V, cb));
    for (int v = 0; v < V; v++)
        if (!outs[v].image) return TGS_ERR_INVALID_ARG;
    PixPtrs px = pix_for(outs, V, nullptr);
    launch_blend_forward(c->cfg.tile, c->cfg.ppt, reinterpret_cast<const float4 *>(splats), sorted_ids,
                         reinterpret_cast<const uint2 *>(ranges), cb, px, c->cfg.bg, (cudaStream_t)stream);
    return last_error();
}

tgs_status tgs_blend_backward(tgs_ctx *c, const float *splats, const uint32_t *sorted_ids,
                              const uint32_t *ranges, const tgs_camera *cams, int32_t V,
                              const tgs_view_out *outs, const float *const *dL_dimages,
                              float *splat_grads, tgs_stream stream) {
    if (!c || !splats || !ranges || !outs || !dL_dimages || !splat_grads) return TGS_ERR_INVALID_ARG;
    CamBatch cb;
    TGS_TRY(make_batch(c->cfg, cams, V, cb));
    for (int v = 0; v < V; v++)
        if (!outs[v].T_final || !outs[v].last || !dL_dimages[v]) return TGS_ERR_INVALID_ARG;
    PixPtrs px = pix_for(outs, V, dL_dimages);
    launch_blend_backward(c->cfg.tile, c->cfg.ppt, reinterpret_cast<const float4 *>(splats), sorted_ids,
                          reinterpret_cast<const uint2 *>(ranges), cb, px, c->cfg.bg, splat_grads,
                          (cudaStream_t)stream);
    return last_error();
}

tgs_status tgs_preprocess_backward(tgs_ctx *c, const tgs_gaussians *g, const tgs_camera *cams,
                                   int32_t V, const float *splat_grads, const int32_t *radii,
                                   const tgs_grads *grads, const tgs_stats *stats, uint32_t flags,
                                   tgs_stream stream) {
    if (!c || !splat_grads || !radii) return TGS_ERR_INVALID_ARG;
    CamBatch cb;
    GaussPtrs gp;
    TGS_TRY(make_batch(c->cfg, cams, V, cb));
    TGS_TRY(make_gauss(c->cfg, g, gp));
    GradPtrs o = grad_ptrs(grads, stats, (flags & TGS_ACCUMULATE) ? 1 : 0);
    if (flags & TGS_MASK_LOSS) with_mask_loss(c->cfg, g->n, o);
    launch_preprocess_backward(gp, cb, reinterpret_cast<const float4 *>(splat_grads), radii, o,
                               (flags & TGS_NO_SH_REST_GRAD) ? 1 : 0, 0, (cudaStream_t)stream);
    return last_error();
}

tgs_status tgs_l1_loss(const float *image, const float *target, int64_t count, float scale,
                       float *loss_accum, float *grad, tgs_stream stream) {
    if (!image || !target || count < 0) return TGS_ERR_INVALID_ARG;
    launch_l1(image, target, count, scale, loss_accum, grad, (cudaStream_t)stream);
    return last_error();
}

tgs_status tgs_l1_dssim_loss(tgs_ctx *c, const tgs_camera *cams, int32_t V, const float *const *images,
                             const float *const *targets, float lambda, float *loss_accum, float *const *grads,
                             tgs_stream stream) {
    if (!c || !cams || !images || !targets || !grads || V <= 0 || V > kMaxViews || !(lambda >= 0.f) ||
        !(lambda <= 1.f))
        return TGS_ERR_INVALID_ARG;
    int W[kMaxViews], H[kMaxViews];
    for (int v = 0; v < V; v++) {
        if (!images[v] || !targets[v] || !grads[v] || cams[v].width < 0 || cams[v].height < 0)
            return TGS_ERR_INVALID_ARG;
        W[v] = cams[v].width;
        H[v] = cams[v].height;
    }
    cudaStream_t st = (cudaStream_t)stream;
    TGS_TRY(ensure(c->ssim, sizeof(float) * (size_t)ssim_scratch_floats(W, H, V), st));
    launch_l1_dssim(V, W, H, images, targets, grads, lambda, as<float>(c->ssim), loss_accum, st);
    return last_error();
}

tgs_status tgs_mask_loss(tgs_ctx *c, const tgs_gaussians *g, float *loss_accum, const tgs_grads *grads,
                         tgs_stream stream) {
    if (!c || !g || g->n < 0 || g->param_dtype != TGS_PARAM_F32) return TGS_ERR_INVALID_ARG;
    launch_mask_loss(g->mask_logits, g->sh_mask_logits, g->n, c->cfg.lambda_mask, c->cfg.lambda_sh_mask, loss_accum,
                     (grads && g->mask_logits) ? grads->mask_logits : nullptr,
                     (grads && g->sh_mask_logits) ? grads->sh_mask_logits : nullptr, (cudaStream_t)stream);
    return last_error();
}

// ---- plain path ---------------------------------------------------------------------------

static tgs_status plain_bin_view(tgs_ctx *c, const tgs_gaussians *g, const GaussPtrs &gp,
                                 const tgs_camera *cam, CamBatch &cb, cudaStream_t st, uint32_t **ids) {
    TGS_TRY(make_batch(c->cfg, cam, 1, cb));
    TGS_TRY(ensure_records(c, g->n, st));
    launch_preprocess(gp, cb, as<float4>(c->splats), as<int32_t>(c->radii), nullptr,
                      as<uint32_t>(c->dbits), nullptr, st);
    TGS_TRY(bin_plain(c, g->n, cb, st, nullptr, -1, ids));
    c->state_valid = true;
    c->state_g = *g;
    c->state_cam = *cam;
    c->state_tile = c->cfg.tile;
    c->state_ids = *ids;
    return TGS_OK;
}

tgs_status tgs_forward(tgs_ctx *c, const tgs_gaussians *g, const tgs_camera *cams, int32_t V,
                       const tgs_view_out *outs, uint32_t flags, tgs_stream stream) {
    (void)flags;
    if (!c || !outs || !cams || V <= 0) return TGS_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    GaussPtrs gp;
    TGS_TRY(make_gauss(c->cfg, g, gp, true));
    for (int v = 0; v < V; v++) {
        if (!outs[v].image) return TGS_ERR_INVALID_ARG;
        CamBatch cb;
        uint32_t *ids = nullptr;
        TGS_TRY(plain_bin_view(c, g, gp, cams + v, cb, st, &ids));
        PixPtrs px = pix_for(outs + v, 1, nullptr);
        launch_blend_forward(c->cfg.tile, c->cfg.ppt, as<float4>(c->splats), ids, as<uint2>(c->ranges), cb,
                             px, c->cfg.bg, st);
        if (outs[v].radii)
            TGS_CHECK(cudaMemcpyAsync(outs[v].radii, c->radii.p, sizeof(int32_t) * (size_t)g->n,
                                      cudaMemcpyDeviceToDevice, st));
        TGS_TRY(last_error());
    }
    return TGS_OK;
}

tgs_status tgs_backward(tgs_ctx *c, const tgs_gaussians *g, const tgs_camera *cams, int32_t V,
                        const tgs_view_out *outs, const float *const *dL_dimages,
                        const tgs_grads *grads, const tgs_stats *stats, uint32_t flags,
                        tgs_stream stream) {
    if (!c || !outs || !cams || !dL_dimages || V <= 0) return TGS_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    GaussPtrs gp;
    TGS_TRY(make_gauss(c->cfg, g, gp));
    for (int v = 0; v < V; v++) {
        if (!outs[v].T_final || !outs[v].last || !dL_dimages[v]) return TGS_ERR_INVALID_ARG;
        CamBatch cb;
        uint32_t *ids = nullptr;
        if (c->state_valid && same_g(c->state_g, *g) && same_cam(c->state_cam, cams[v]) &&
            c->state_tile == c->cfg.tile) {
            TGS_TRY(make_batch(c->cfg, cams + v, 1, cb));
            ids = c->state_ids;
        } else {
            TGS_TRY(plain_bin_view(c, g, gp, cams + v, cb, st, &ids));
        }
        TGS_CHECK(cudaMemsetAsync(c->sgrads.p, 0, sizeof(float) * 12 * (size_t)g->n, st));
        PixPtrs px = pix_for(outs + v, 1, dL_dimages + v);
        launch_blend_backward(c->cfg.tile, c->cfg.ppt, as<float4>(c->splats), ids, as<uint2>(c->ranges),
                              cb, px, c->cfg.bg, as<float>(c->sgrads), st);
        const int acc = ((flags & TGS_ACCUMULATE) || v > 0) ? 1 : 0;
        GradPtrs o = grad_ptrs(grads, stats, acc);
        if ((flags & TGS_MASK_LOSS) && v == 0) with_mask_loss(c->cfg, g->n, o);  // once, not per view
        launch_preprocess_backward(gp, cb, as<float4>(c->sgrads), as<int32_t>(c->radii), o,
                                   (flags & TGS_NO_SH_REST_GRAD) ? 1 : 0, 0, st);
        TGS_TRY(last_error());
    }
    return TGS_OK;
}

// ---- significance pruning (Eq. significance-score) -----------------------------------------

tgs_status tgs_count_hits(tgs_ctx *c, const tgs_gaussians *g, const tgs_camera *cams, int32_t V,
                          uint32_t *hit_count, tgs_stream stream) {
    if (!c || !g || !cams || V <= 0 || (!hit_count && g->n > 0)) return TGS_ERR_INVALID_ARG;
    if (g->n == 0) return TGS_OK;
    cudaStream_t st = (cudaStream_t)stream;
    GaussPtrs gp;
    TGS_TRY(make_gauss(c->cfg, g, gp, true));
    // all views at once: one preprocess, one binning (one host read of the key count), one
    // forward blend over every (view, tile) counting hits
    CamBatch cb;
    TGS_TRY(make_batch(c->cfg, cams, V, cb));
    const int64_t nt = g->n * V;
    TGS_TRY(ensure_records(c, nt, st));
    launch_preprocess(gp, cb, as<float4>(c->splats), as<int32_t>(c->radii), nullptr, as<uint32_t>(c->dbits),
                      nullptr, st);
    uint32_t *ids = nullptr;
    c->state_valid = false;  // the binning kept for a backward is not this one's
    TGS_TRY(bin_plain(c, g->n, cb, st, nullptr, -1, &ids));
    PixPtrs px;
    memset(&px, 0, sizeof px);  // nothing but the hits is written
    launch_blend_forward(c->cfg.tile, c->cfg.ppt, as<float4>(c->splats), ids, as<uint2>(c->ranges), cb, px,
                         c->cfg.bg, st, hit_count, g->n);
    return last_error();
}

tgs_status tgs_significance(tgs_ctx *c, const tgs_gaussians *g, const uint32_t *hit_count, double quantile,
                            float *scores, tgs_stream stream) {
    if (!c || !g || !(quantile >= 0.0 && quantile <= 1.0)) return TGS_ERR_INVALID_ARG;
    const int64_t n = g->n;
    if (n == 0) return TGS_OK;
    if (!hit_count || !scores) return TGS_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    GaussPtrs gp;
    TGS_TRY(make_gauss(c->cfg, g, gp));
    TGS_TRY(ensure_records(c, n, st));
    float *vol = as<float>(c->pos);
    uint32_t *k = as<uint32_t>(c->ck0), *v = as<uint32_t>(c->cv0);
    launch_volumes(gp, vol, k, st);
    radix_sort_pairs(k, v, as<uint32_t>(c->ck1), as<uint32_t>(c->cv1), nullptr, n, 0, 32, as<uint32_t>(c->hist),
                     as<uint32_t>(c->partials), st, true);
    const int64_t q_rank = (int64_t)std::floor(quantile * (double)(n - 1));
    launch_scores(gp, hit_count, vol, k, q_rank, scores, st);
    c->state_valid = false;
    return last_error();
}

tgs_status tgs_prune_schedule(int32_t rounds, double first, double decay, double *fractions) {
    if (rounds < 0 || !(first >= 0.0 && first <= 1.0) || !(decay >= 0.0 && decay <= 1.0) ||
        (rounds > 0 && !fractions))
        return TGS_ERR_INVALID_ARG;
    double f = first;
    for (int r = 0; r < rounds; r++) {
        fractions[r] = f;
        f *= decay;
    }
    return TGS_OK;
}

tgs_status tgs_prune_select(tgs_ctx *c, const float *scores, int64_t n, double fraction, uint8_t *prune,
                            tgs_stream stream) {
    if (!c || n < 0 || !(fraction >= 0.0 && fraction <= 1.0)) return TGS_ERR_INVALID_ARG;
    if (n == 0) return TGS_OK;
    if (!scores || !prune) return TGS_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    TGS_TRY(ensure_records(c, n, st));
    uint32_t *k = as<uint32_t>(c->ck0), *v = as<uint32_t>(c->cv0);
    launch_score_keys(scores, n, k, st);
    radix_sort_pairs(k, v, as<uint32_t>(c->ck1), as<uint32_t>(c->cv1), nullptr, n, 0, 32, as<uint32_t>(c->hist),
                     as<uint32_t>(c->partials), st, true);
    TGS_CHECK(cudaMemsetAsync(prune, 0, (size_t)n, st));
    launch_mark(v, (int64_t)std::floor(fraction * (double)n), prune, st);
    c->state_valid = false;
    return last_error();
}

tgs_status tgs_params_to_half(const tgs_gaussians *g, const tgs_half_params *out, tgs_stream stream) {
    if (!g || !out || g->n < 0 || g->param_dtype != TGS_PARAM_F32) return TGS_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    const int64_t n = g->n;
    launch_to_half(g->means, out->means, 3 * n, st);
    launch_to_half(g->log_scales, out->log_scales, 3 * n, st);
    launch_to_half(g->quats, out->quats, 4 * n, st);
    launch_to_half(g->opacity_logits, out->opacity_logits, n, st);
    launch_to_half(g->sh_dc, out->sh_dc, 3 * n, st);
    launch_to_half(g->sh_rest, out->sh_rest, 45 * n, st);
    launch_to_half(g->mask_logits, out->mask_logits, n, st);
    launch_to_half(g->sh_mask_logits, out->sh_mask_logits, 3 * n, st);
    return last_error();
}

tgs_status tgs_compact(tgs_ctx *c, const tgs_gaussians *g, const uint8_t *remove, uint32_t flags,
                       const tgs_grads *out, uint8_t *sh_degree_out, uint32_t *kept_index, int64_t *n_kept,
                       tgs_stream stream) {
    if (!c || !g || !out || !n_kept) return TGS_ERR_INVALID_ARG;
    GaussPtrs gp;
    TGS_TRY(make_gauss(c->cfg, g, gp));
    *n_kept = 0;
    if (g->n == 0) return TGS_OK;
    cudaStream_t st = (cudaStream_t)stream;
    const int64_t nb = compact_blocks(g->n);
    TGS_TRY(ensure(c->cbuf, sizeof(uint32_t) * (size_t)(nb + 1), st));
    uint32_t *counts = as<uint32_t>(c->cbuf);
    launch_compact(gp, remove, (flags & TGS_COMPACT_MASKED) != 0, grad_ptrs(out, nullptr, 0), sh_degree_out,
                   kept_index, counts, counts + nb, st);
    TGS_CHECK(cudaMemcpyAsync(c->h_counts + 3, counts + nb, sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
    TGS_CHECK(cudaStreamSynchronize(st));
    *n_kept = c->h_counts[3];
    return last_error();
}

tgs_status tgs_densify(tgs_ctx *c, const tgs_gaussians *g, const tgs_stats *stats, const float *normals,
                       float grad_threshold, float scale_threshold, const tgs_grads *out, uint8_t *sh_degree_out,
                       uint32_t *src_index, int64_t capacity, int64_t *n_out, int64_t *n_clone, int64_t *n_split,
                       tgs_stream stream) {
    if (!c || !g || !stats || !out || !n_out || capacity < 0 || !(scale_threshold > 0.f)) return TGS_ERR_INVALID_ARG;
    GaussPtrs gp;
    TGS_TRY(make_gauss(c->cfg, g, gp));
    *n_out = g->n;
    if (n_clone) *n_clone = 0;
    if (n_split) *n_split = 0;
    if (g->n == 0) return TGS_OK;
    if (!stats->grad_norm_accum || !stats->vis_count || !normals) return TGS_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    const int64_t nb = compact_blocks(g->n);
    TGS_TRY(ensure(c->cbuf, sizeof(uint32_t) * (size_t)(3 * (nb + 1) + 4), st));
    uint32_t *scratch = as<uint32_t>(c->cbuf), *totals = scratch + 3 * (nb + 1);
    DensifyArgs d{stats->grad_norm_accum, stats->vis_count, normals, grad_threshold,
                  (float)std::log((double)scale_threshold)};
    GradPtrs o = grad_ptrs(out, nullptr, 0);
    launch_densify(gp, d, o, sh_degree_out, src_index, scratch, totals, false, st);
    uint32_t h[3];
    TGS_CHECK(cudaMemcpyAsync(h, totals, sizeof h, cudaMemcpyDeviceToHost, st));
    TGS_CHECK(cudaStreamSynchronize(st));
    const int64_t nn = (int64_t)h[0] + h[1] + 2 * (int64_t)h[2];
    *n_out = nn;
    if (n_clone) *n_clone = h[1];
    if (n_split) *n_split = h[2];
    if (nn > capacity) return TGS_ERR_CAPACITY;
    launch_densify(gp, d, o, sh_degree_out, src_index, scratch, totals, true, st);
    return last_error();
}

// ---- batched path --------------------------------------------------------------------------

tgs_status tgs_plan(tgs_ctx *c, const tgs_gaussians *g, const tgs_camera *cams, int32_t V,
                    double headroom, int64_t *keys_out) {
    if (!c || headroom < 1.0) return TGS_ERR_INVALID_ARG;
    cudaStream_t st = nullptr;
    CamBatch cb;
    GaussPtrs gp;
    TGS_TRY(make_batch(c->cfg, cams, V, cb));
    TGS_TRY(make_gauss(c->cfg, g, gp, true));  // FP16 storage plans the render path
    const int64_t nt = g->n * V;
    TGS_TRY(ensure_records(c, nt, st));
    launch_preprocess(gp, cb, as<float4>(c->splats), as<int32_t>(c->radii), nullptr,
                      as<uint32_t>(c->dbits), nullptr, st);
    uint32_t *sorted = nullptr;
    bin_front(c, nt, &sorted, st);
    int64_t K = 0;
    TGS_TRY(read_counts(c, st, &K));
    c->state_valid = false;
    int64_t cap = (int64_t)std::ceil(headroom * (double)std::max<int64_t>(K, 1));
    c->cfg.key_capacity = cap;
    TGS_TRY(ensure_keys(c, cap, cb.total_tiles, st));
    if (keys_out) *keys_out = K;
    drop_graphs(c);
    return last_error();
}

// The body of one batched step; issues only asynchronous work (capturable).
static tgs_status batched_body(tgs_ctx *c, const tgs_gaussians *g, const GaussPtrs &gp, const CamBatch &cb,
                               const tgs_camera *cams, int V, const float *const *targets,
                               float *const *images, const tgs_grads *grads, const tgs_stats *stats,
                               float *loss_out, uint32_t flags, cudaStream_t st) {
    const int64_t n = g->n, nt = n * V;
    const int64_t cap = c->cfg.key_capacity;
    // the D-SSIM gradient is not pixel-local: forward, loss and backward run as separate kernels
    const bool split = (flags & (TGS_UNFUSED | TGS_LOSS_DSSIM)) != 0;
    // pixel buffers: images (if the caller gives none), T_final, last, dL/dimage
    size_t pix = 0;
    for (int v = 0; v < V; v++) pix += (size_t)cams[v].width * cams[v].height;
    float *imgbuf = as<float>(c->images);
    float *dimg = as<float>(c->dimg);
    float *Tf = as<float>(c->pixstate);
    int32_t *last = reinterpret_cast<int32_t *>(Tf + pix);
    tgs_view_out outs[kMaxViews];
    const float *dls[kMaxViews];
    size_t off = 0;
    for (int v = 0; v < V; v++) {
        const size_t hw = (size_t)cams[v].width * cams[v].height;
        // the fused step needs no image of its own: it writes one only where the caller asks
        outs[v].image = images && images[v] ? images[v] : (split ? imgbuf + 3 * off : nullptr);
        outs[v].T_final = Tf + off;
        outs[v].last = last + off;
        outs[v].n_examined = nullptr;
        outs[v].radii = nullptr;
        outs[v].n_contrib = nullptr;
        outs[v].n_eval = nullptr;
        dls[v] = dimg + 3 * off;
        off += hw;
    }
    const int64_t launches0 = g_launches;
    mark(c, 0, "preprocess", st);
    launch_preprocess(gp, cb, as<float4>(c->splats), as<int32_t>(c->radii), nullptr,
                      as<uint32_t>(c->dbits), as<float>(c->sgrads), st);
    mark(c, 1, "bin", st);
    uint32_t *sorted = nullptr;
    bin_front(c, nt, &sorted, st);
    uint32_t *ids = bin_back(c, nt, n, sorted, cb, cap, st);
    PixPtrs px = pix_for(outs, V, dls);
    for (int v = 0; v < V; v++) px.target[v] = targets[v];
    if (loss_out) TGS_CHECK(cudaMemsetAsync(loss_out, 0, sizeof(float), st));
    int stage = 2;
    if (split) {
        // at tile 32 / 2 px per thread the warp-item kernels take their items heaviest first
        const bool warp_items = c->cfg.tile == 32 && c->cfg.ppt == 2;
        uint32_t *order = nullptr;
        int *ctr = reinterpret_cast<int *>(as<uint32_t>(c->counts) + 2);  // forward, backward
        if (warp_items) {
            mark(c, stage++, "item_order", st);
            uint32_t *it = as<uint32_t>(c->items);
            const size_t T = ((size_t)cb.total_tiles + 3) / 4 * 4;  // 16-byte aligned quarters
            build_item_order(as<uint2>(c->ranges), cb.total_tiles, it, it + T, it + 2 * T, it + 3 * T, &order,
                             as<uint32_t>(c->hist), as<uint32_t>(c->partials), st);
            TGS_CHECK(cudaMemsetAsync(ctr, 0, 2 * sizeof(int), st));
        }
        mark(c, stage++, "blend_forward", st);
        launch_blend_forward(c->cfg.tile, c->cfg.ppt, as<float4>(c->splats), ids, as<uint2>(c->ranges), cb, px,
                             c->cfg.bg, st, stats ? stats->hit_count : nullptr, n, order, order ? ctr : nullptr);
        if (flags & TGS_LOSS_DSSIM) {
            mark(c, stage++, "l1_dssim_loss", st);
            int W[kMaxViews], H[kMaxViews];
            const float *x[kMaxViews];
            float *dx[kMaxViews];
            for (int v = 0; v < V; v++) {
                W[v] = cams[v].width;
                H[v] = cams[v].height;
                x[v] = outs[v].image;
                dx[v] = const_cast<float *>(dls[v]);
            }
            launch_l1_dssim(V, W, H, x, targets, dx, c->cfg.ssim_lambda, as<float>(c->ssim), loss_out, st);
        } else {
            mark(c, stage++, "l1_loss", st);
            for (int v = 0; v < V; v++) {
                const int64_t cnt = 3 * (int64_t)cams[v].width * cams[v].height;
                launch_l1(outs[v].image, targets[v], cnt, (float)(1.0 / ((double)cnt * V)), loss_out,
                          const_cast<float *>(dls[v]), st);
            }
        }
        mark(c, stage++, "blend_backward", st);
        // pixel sums (moments), as the fused kernel leaves them
        launch_blend_backward(c->cfg.tile, c->cfg.ppt, as<float4>(c->splats), ids, as<uint2>(c->ranges), cb, px,
                              c->cfg.bg, as<float>(c->sgrads), st, order, order ? ctr + 1 : nullptr, 1);
    } else {
        mark(c, stage++, "item_order", st);
        uint32_t *it = as<uint32_t>(c->items);
        const size_t T = ((size_t)cb.total_tiles + 3) / 4 * 4;  // 16-byte aligned quarters
        uint32_t *order = nullptr;
        build_item_order(as<uint2>(c->ranges), cb.total_tiles, it, it + T, it + 2 * T, it + 3 * T, &order,
                         as<uint32_t>(c->hist), as<uint32_t>(c->partials), st);
        int *counter = reinterpret_cast<int *>(as<uint32_t>(c->counts) + 2);
        TGS_CHECK(cudaMemsetAsync(counter, 0, sizeof(int), st));
        mark(c, stage++, "fused_blend", st);
        launch_fused_l1(c->cfg.tile, c->cfg.ppt, c->cfg.batch > 1 ? 2 : 1, as<float4>(c->splats), ids, as<uint2>(c->ranges), order, counter,
                        cb, px, c->cfg.bg, as<float>(c->sgrads), loss_out, as<uint16_t>(c->viskeys), st,
                        stats ? stats->hit_count : nullptr, n);
    }
    mark(c, stage++, "preprocess_backward", st);
    GradPtrs o = grad_ptrs(grads, stats, (flags & TGS_ACCUMULATE) ? 1 : 0);
    if (flags & TGS_MASK_LOSS) with_mask_loss(c->cfg, n, o);
    // both blends leave pixel sums (moments) in the gradient records
    launch_preprocess_backward(gp, cb, as<float4>(c->sgrads), as<int32_t>(c->radii), o,
                               (flags & TGS_NO_SH_REST_GRAD) ? 1 : 0, 1, st);
    if ((flags & TGS_MASK_LOSS) && loss_out)  // the value of the mask terms (Eq. loss3dgs)
        launch_mask_loss(g->mask_logits, g->sh_mask_logits, n, c->cfg.lambda_mask, c->cfg.lambda_sh_mask, loss_out,
                         nullptr, nullptr, st);
    mark(c, stage, "end", st);
    c->kernels_per_step = g_launches - launches0;
    return last_error();
}

tgs_status tgs_train_step_batched(tgs_ctx *c, const tgs_gaussians *g, const tgs_camera *cams, int32_t V,
                                  const float *const *targets, float *const *images, const tgs_grads *grads,
                                  const tgs_stats *stats, float *loss_out, uint32_t flags, tgs_stream stream) {
    if (!c || !targets || !cams || V <= 0 || V > kMaxViews) return TGS_ERR_INVALID_ARG;
    for (int v = 0; v < V; v++)
        if (!targets[v]) return TGS_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    CamBatch cb;
    GaussPtrs gp;
    TGS_TRY(make_batch(c->cfg, cams, V, cb));
    TGS_TRY(make_gauss(c->cfg, g, gp));
    if (c->cfg.key_capacity <= 0) {
        if (capturing(st)) return TGS_ERR_CAPACITY;
        TGS_TRY(tgs_plan(c, g, cams, V, 1.25, nullptr));
        TGS_CHECK(cudaDeviceSynchronize());
    }
    const int64_t nt = g->n * V;
    size_t pix = 0;
    for (int v = 0; v < V; v++) pix += (size_t)cams[v].width * cams[v].height;
    TGS_TRY(ensure_records(c, nt, st));
    TGS_TRY(ensure_keys(c, c->cfg.key_capacity, cb.total_tiles, st));
    TGS_TRY(ensure(c->images, sizeof(float) * 3 * pix, st));
    TGS_TRY(ensure(c->dimg, sizeof(float) * 3 * pix, st));
    TGS_TRY(ensure(c->pixstate, sizeof(float) * 2 * pix, st));
    if (flags & TGS_LOSS_DSSIM) {
        int W[kMaxViews], H[kMaxViews];
        for (int v = 0; v < V; v++) {
            W[v] = cams[v].width;
            H[v] = cams[v].height;
        }
        TGS_TRY(ensure(c->ssim, sizeof(float) * (size_t)ssim_scratch_floats(W, H, V), st));
    }
    TGS_TRY(ensure(c->items, sizeof(uint32_t) * 4 * (((size_t)std::max(cb.total_tiles, 1) + 3) / 4 * 4), st));
    c->state_valid = false;

    if (!(flags & TGS_USE_GRAPH) || st == nullptr || capturing(st))
        return batched_body(c, g, gp, cb, cams, V, targets, images, grads, stats, loss_out, flags, st);

    // key of the captured graph: every argument that the recorded launches depend on
    std::vector<unsigned char> key;
    auto put = [&key](const void *p, size_t n) {
        const unsigned char *b = (const unsigned char *)p;
        key.insert(key.end(), b, b + n);
    };
    put(g, sizeof *g);
    put(cams, sizeof(tgs_camera) * V);
    put(&V, sizeof V);
    put(targets, sizeof(float *) * V);
    for (int v = 0; v < V; v++) {
        const float *im = images ? images[v] : nullptr;
        put(&im, sizeof im);
    }
    tgs_grads gz{};
    tgs_stats sz{};
    put(grads ? grads : &gz, sizeof gz);
    put(stats ? stats : &sz, sizeof sz);
    put(&loss_out, sizeof loss_out);
    put(&flags, sizeof flags);
    put(&c->cfg, sizeof c->cfg);
    void *arena[] = {c->splats.p, c->tk0.p, c->hist.p, c->images.p, c->pixstate.p};
    put(arena, sizeof arena);
    const uint64_t gen = g_arena_gen.load();
    put(&gen, sizeof gen);
    tgs_ctx::Graph *hit = nullptr;
    for (auto &gr : c->graphs)
        if (gr.key == key) hit = &gr;
    if (!hit) {
        constexpr size_t kMaxGraphs = 4;
        if (c->graphs.size() >= kMaxGraphs) {  // evict the least recently used
            auto lru = std::min_element(c->graphs.begin(), c->graphs.end(),
                                        [](const tgs_ctx::Graph &a, const tgs_ctx::Graph &b) { return a.used < b.used; });
            cudaGraphExecDestroy(lru->exec);
            c->graphs.erase(lru);
        }
        cudaGraph_t graph = nullptr;
        TGS_CHECK(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
        tgs_status s = batched_body(c, g, gp, cb, cams, V, targets, images, grads, stats, loss_out, flags, st);
        cudaError_t e = cudaStreamEndCapture(st, &graph);
        if (s != TGS_OK) {
            if (graph) cudaGraphDestroy(graph);
            return s;
        }
        TGS_CHECK(e);
        cudaGraphExec_t exec = nullptr;
        e = cudaGraphInstantiate(&exec, graph, 0);
        cudaGraphDestroy(graph);
        TGS_CHECK(e);
        c->graphs.push_back(tgs_ctx::Graph{key, exec, 0});
        hit = &c->graphs.back();
    }
    hit->used = ++c->graph_clock;
    TGS_CHECK(cudaGraphLaunch(hit->exec, st));
    return TGS_OK;
}

tgs_status tgs_train_step_batched_host(tgs_ctx *c, const tgs_gaussians *gh, const tgs_camera *cams, int32_t V,
                                       const float *const *targets_host, const tgs_grads *grads,
                                       const tgs_stats *stats, float *loss_host, uint32_t flags, tgs_stream stream) {
    if (!c || !gh || !cams || !targets_host || V <= 0 || V > kMaxViews || gh->n < 0 ||
        gh->param_dtype != TGS_PARAM_F32)
        return TGS_ERR_INVALID_ARG;
    for (int v = 0; v < V; v++)
        if (!targets_host[v] || cams[v].width <= 0 || cams[v].height <= 0) return TGS_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    if (capturing(st)) return TGS_ERR_NOT_SUPPORTED;
    const int64_t n = gh->n;
    // the parameter arrays, each in a 256-byte aligned segment of one device buffer
    struct Arr {
        const void *src;
        size_t bytes;
    } arr[9] = {{gh->means, 12 * (size_t)n},        {gh->log_scales, 12 * (size_t)n},
                {gh->quats, 16 * (size_t)n},        {gh->opacity_logits, 4 * (size_t)n},
                {gh->sh_dc, 12 * (size_t)n},        {gh->sh_rest, 180 * (size_t)n},
                {gh->mask_logits, 4 * (size_t)n},   {gh->sh_mask_logits, 12 * (size_t)n},
                {gh->sh_degree, (size_t)n}};
    if (gh->sh_degree_max == 0 || !gh->sh_rest) arr[5].src = nullptr;
    size_t off[9], pb = 0;
    for (int i = 0; i < 9; i++) {
        off[i] = pb;
        if (arr[i].src) pb += (arr[i].bytes + 255) / 256 * 256;
    }
    size_t toff[kMaxViews], tb = 0;
    for (int v = 0; v < V; v++) {
        toff[v] = tb;
        tb += (12 * (size_t)cams[v].width * cams[v].height + 255) / 256 * 256;
    }
    tgs_ctx::Stage &sg = c->stage[c->stage_next];
    c->stage_next = (c->stage_next + 1) % tgs_ctx::kStages;
    if (!c->upload) TGS_CHECK(cudaStreamCreateWithFlags(&c->upload, cudaStreamNonBlocking));
    if (!sg.copied) TGS_CHECK(cudaEventCreateWithFlags(&sg.copied, cudaEventDisableTiming));
    if (!sg.consumed) TGS_CHECK(cudaEventCreateWithFlags(&sg.consumed, cudaEventDisableTiming));
    if (sg.params.bytes < pb || sg.targets.bytes < tb) {
        // growing frees the old buffers: no copy or step may still use them
        TGS_CHECK(cudaStreamSynchronize(c->upload));
        TGS_CHECK(cudaStreamSynchronize(st));
        TGS_TRY(ensure(sg.params, pb, st));
        TGS_TRY(ensure(sg.targets, tb, st));
        sg.used = false;
        drop_graphs(c);  // the graphs of the old buffers' addresses
    }
    TGS_TRY(ensure(c->lossbuf, sizeof(float), st));
    // the copies wait for the step that last read this set of buffers
    if (sg.used) TGS_CHECK(cudaStreamWaitEvent(c->upload, sg.consumed, 0));
    unsigned char *pd = as<unsigned char>(sg.params);
    for (int i = 0; i < 9; i++)
        if (arr[i].src && arr[i].bytes)
            TGS_CHECK(cudaMemcpyAsync(pd + off[i], arr[i].src, arr[i].bytes, cudaMemcpyHostToDevice, c->upload));
    unsigned char *td = as<unsigned char>(sg.targets);
    const float *tdev[kMaxViews];
    for (int v = 0; v < V; v++) {
        const size_t bytes = 12 * (size_t)cams[v].width * cams[v].height;
        TGS_CHECK(cudaMemcpyAsync(td + toff[v], targets_host[v], bytes, cudaMemcpyHostToDevice, c->upload));
        tdev[v] = reinterpret_cast<const float *>(td + toff[v]);
    }
    TGS_CHECK(cudaEventRecord(sg.copied, c->upload));
    TGS_CHECK(cudaStreamWaitEvent(st, sg.copied, 0));
    tgs_gaussians gd = *gh;
    auto dp = [&](int i) { return arr[i].src ? reinterpret_cast<const float *>(pd + off[i]) : nullptr; };
    gd.means = dp(0);
    gd.log_scales = dp(1);
    gd.quats = dp(2);
    gd.opacity_logits = dp(3);
    gd.sh_dc = dp(4);
    gd.sh_rest = dp(5);
    gd.mask_logits = dp(6);
    gd.sh_mask_logits = dp(7);
    gd.sh_degree = arr[8].src ? pd + off[8] : nullptr;
    float *loss_dev = as<float>(c->lossbuf);
    const tgs_status s = tgs_train_step_batched(c, &gd, cams, V, tdev, nullptr, grads, stats, loss_dev, flags, stream);
    TGS_CHECK(cudaEventRecord(sg.consumed, st));
    sg.used = true;
    if (s != TGS_OK) return s;
    if (loss_host) TGS_CHECK(cudaMemcpyAsync(loss_host, loss_dev, sizeof(float), cudaMemcpyDeviceToHost, st));
    return last_error();
}

// The body of a batched render; issues only asynchronous work (capturable).
static tgs_status render_body(tgs_ctx *c, const tgs_gaussians *g, const GaussPtrs &gp, const CamBatch &cb,
                              const tgs_view_out *outs, int V, cudaStream_t st) {
    const int64_t n = g->n, nt = n * V;
    const int64_t cap = c->cfg.key_capacity;
    const int64_t launches0 = g_launches;
    launch_preprocess(gp, cb, as<float4>(c->splats), as<int32_t>(c->radii), nullptr, as<uint32_t>(c->dbits),
                      nullptr, st);
    uint32_t *sorted = nullptr;
    bin_front(c, nt, &sorted, st);
    uint32_t *ids = bin_back(c, nt, n, sorted, cb, cap, st);
    PixPtrs px = pix_for(outs, V, nullptr);
    // at tile 32 / 2 px per thread the warp-item kernel takes its items heaviest first
    uint32_t *order = nullptr;
    int *ctr = reinterpret_cast<int *>(as<uint32_t>(c->counts) + 2);
    if (c->cfg.tile == 32 && c->cfg.ppt == 2) {
        uint32_t *it = as<uint32_t>(c->items);
        const size_t T = ((size_t)cb.total_tiles + 3) / 4 * 4;  // 16-byte aligned quarters
        build_item_order(as<uint2>(c->ranges), cb.total_tiles, it, it + T, it + 2 * T, it + 3 * T, &order,
                         as<uint32_t>(c->hist), as<uint32_t>(c->partials), st);
        TGS_CHECK(cudaMemsetAsync(ctr, 0, sizeof(int), st));
    }
    launch_blend_forward(c->cfg.tile, c->cfg.ppt, as<float4>(c->splats), ids, as<uint2>(c->ranges), cb, px,
                         c->cfg.bg, st, nullptr, 0, order, order ? ctr : nullptr);
    c->kernels_per_step = g_launches - launches0;
    return last_error();
}

tgs_status tgs_render_batched(tgs_ctx *c, const tgs_gaussians *g, const tgs_camera *cams, int32_t V,
                              const tgs_view_out *outs, uint32_t flags, tgs_stream stream) {
    if (!c || !cams || !outs || V <= 0 || V > kMaxViews) return TGS_ERR_INVALID_ARG;
    for (int v = 0; v < V; v++)
        if (!outs[v].image) return TGS_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    CamBatch cb;
    GaussPtrs gp;
    TGS_TRY(make_batch(c->cfg, cams, V, cb));
    TGS_TRY(make_gauss(c->cfg, g, gp, true));
    if (c->cfg.key_capacity <= 0) {
        if (capturing(st)) return TGS_ERR_CAPACITY;
        TGS_TRY(tgs_plan(c, g, cams, V, 1.25, nullptr));
        TGS_CHECK(cudaDeviceSynchronize());
    }
    TGS_TRY(ensure_records(c, g->n * V, st));
    TGS_TRY(ensure_keys(c, c->cfg.key_capacity, cb.total_tiles, st));
    TGS_TRY(ensure(c->items, sizeof(uint32_t) * 4 * (((size_t)std::max(cb.total_tiles, 1) + 3) / 4 * 4), st));
    c->state_valid = false;
    if (!(flags & TGS_USE_GRAPH) || st == nullptr || capturing(st)) return render_body(c, g, gp, cb, outs, V, st);
    std::vector<unsigned char> key;
    auto put = [&key](const void *p, size_t n) {
        const unsigned char *b = (const unsigned char *)p;
        key.insert(key.end(), b, b + n);
    };
    const char tag[] = "render";
    put(tag, sizeof tag);
    put(g, sizeof *g);
    put(cams, sizeof(tgs_camera) * V);
    put(&V, sizeof V);
    put(outs, sizeof(tgs_view_out) * V);
    put(&c->cfg, sizeof c->cfg);
    void *arena[] = {c->splats.p, c->tk0.p, c->hist.p};
    put(arena, sizeof arena);
    const uint64_t gen = g_arena_gen.load();
    put(&gen, sizeof gen);
    tgs_ctx::Graph *hit = nullptr;
    for (auto &gr : c->graphs)
        if (gr.key == key) hit = &gr;
    if (!hit) {
        constexpr size_t kMaxGraphs = 4;
        if (c->graphs.size() >= kMaxGraphs) {
            auto lru = std::min_element(c->graphs.begin(), c->graphs.end(),
                                        [](const tgs_ctx::Graph &a, const tgs_ctx::Graph &b) { return a.used < b.used; });
            cudaGraphExecDestroy(lru->exec);
            c->graphs.erase(lru);
        }
        cudaGraph_t graph = nullptr;
        TGS_CHECK(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
        tgs_status s = render_body(c, g, gp, cb, outs, V, st);
        cudaError_t e = cudaStreamEndCapture(st, &graph);
        if (s != TGS_OK) {
            if (graph) cudaGraphDestroy(graph);
            return s;
        }
        TGS_CHECK(e);
        cudaGraphExec_t exec = nullptr;
        e = cudaGraphInstantiate(&exec, graph, 0);
        cudaGraphDestroy(graph);
        TGS_CHECK(e);
        c->graphs.push_back(tgs_ctx::Graph{key, exec, 0});
        hit = &c->graphs.back();
    }
    hit->used = ++c->graph_clock;
    TGS_CHECK(cudaGraphLaunch(hit->exec, st));
    return TGS_OK;
}

tgs_status tgs_set_profiling(tgs_ctx *c, int32_t on) {
    if (!c) return TGS_ERR_INVALID_ARG;
    if (on && !c->stage_ev[0])
        for (auto &e : c->stage_ev) TGS_CHECK(cudaEventCreate(&e));
    if ((bool)on != c->profiling) drop_graphs(c);
    c->profiling = on != 0;
    return TGS_OK;
}

tgs_status tgs_stage_times(tgs_ctx *c, float *ms, int32_t max, int32_t *n_out) {
    if (!c || !ms || !c->profiling) return TGS_ERR_INVALID_ARG;
    const int n = c->n_stages;
    TGS_CHECK(cudaEventSynchronize(c->stage_ev[n]));
    for (int i = 0; i < n && i < max; i++) TGS_CHECK(cudaEventElapsedTime(ms + i, c->stage_ev[i], c->stage_ev[i + 1]));
    if (n_out) *n_out = n;
    return TGS_OK;
}

const char *tgs_stage_name(tgs_ctx *c, int32_t i) {
    if (!c || i < 0 || i >= c->n_stages || i >= TGS_MAX_STAGES) return "";
    return c->stage_names[i] ? c->stage_names[i] : "";
}

int64_t tgs_kernels_per_step(const tgs_ctx *c) { return c ? c->kernels_per_step : -1; }

size_t tgs_arena_bytes(const tgs_ctx *c) {
    if (!c) return 0;
    const Buf *bufs[] = {&c->splats, &c->radii, &c->tt, &c->dbits, &c->pos, &c->ck0, &c->cv0, &c->ck1,
                         &c->cv1, &c->offsets, &c->tk0, &c->tv0, &c->tk1, &c->tv1, &c->ranges, &c->hist,
                         &c->partials, &c->sgrads, &c->counts, &c->status, &c->pixstate, &c->dimg,
                         &c->images, &c->items, &c->kmask, &c->viskeys, &c->ssim, &c->cbuf, &c->lossbuf,
                         &c->stage[0].params, &c->stage[0].targets, &c->stage[1].params, &c->stage[1].targets,
                         &c->stage[2].params, &c->stage[2].targets};
    size_t b = 0;
    for (const Buf *x : bufs) b += x->bytes;
    return b;
}

tgs_status tgs_autotune(tgs_ctx *c, const tgs_gaussians *g, const tgs_camera *cams, int32_t V,
                        const float *const *targets, const char *cache_path, tgs_stream stream) {
    if (!c || !g || !cams || !targets) return TGS_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    // cache key: n, V and the view sizes
    std::string key = "n" + std::to_string(g->n) + "_V" + std::to_string(V);
    for (int v = 0; v < V; v++) key += "_" + std::to_string(cams[v].width) + "x" + std::to_string(cams[v].height);
    struct Entry {
        std::string key;
        int tile, ppt, batch;
    };
    std::vector<Entry> cache;
    if (cache_path) {
        std::string text;
        if (FILE *f = fopen(cache_path, "r")) {
            char buf[4096];
            size_t got;
            while ((got = fread(buf, 1, sizeof buf, f)) > 0) text.append(buf, got);
            fclose(f);
        }
        parse_tune_cache(text, [&cache](const std::string &k, int tl, int pp, int bt) {
            cache.push_back({k, tl, pp, bt});
        });
        for (auto &e : cache)
            if (e.key == key) {  // a cached choice: adopted without timing anything
                tgs_config cf = c->cfg;
                cf.tile = e.tile;
                cf.ppt = e.ppt;
                cf.batch = e.batch;
                cf.key_capacity = 0;
                if (!valid_cfg(cf)) break;
                TGS_TRY(tgs_set_config(c, &cf));
                return tgs_plan(c, g, cams, V, 1.25, nullptr);
            }
    }
    // tile x pixels per thread x Gaussians per shared-memory batch (multiples of the threads)
    const int tiles[3] = {8, 16, 32}, ppts[3] = {1, 2, 4}, batches[2] = {1, 2};
    float best = 1e30f;
    tgs_config best_cfg = c->cfg, base = c->cfg;
    struct Events {  // destroyed on every return path
        cudaEvent_t e[2] = {nullptr, nullptr};
        ~Events() {
            for (cudaEvent_t x : e)
                if (x) cudaEventDestroy(x);
        }
    } ev;
    TGS_CHECK(cudaEventCreate(&ev.e[0]));
    TGS_CHECK(cudaEventCreate(&ev.e[1]));
    cudaEvent_t e0 = ev.e[0], e1 = ev.e[1];
    for (int tl : tiles)
        for (int pp : ppts) {
            tgs_config cf = base;
            cf.tile = tl;
            cf.ppt = pp;
            cf.batch = 1;
            if (!valid_cfg(cf)) continue;
            cf.key_capacity = 0;
            TGS_TRY(tgs_set_config(c, &cf));
            TGS_TRY(tgs_plan(c, g, cams, V, 1.25, nullptr));  // keys depend on the tile only
            const int64_t cap = c->cfg.key_capacity;
            for (int bt : batches) {
                cf.batch = bt;
                cf.key_capacity = cap;
                TGS_TRY(tgs_set_config(c, &cf));
                for (int w = 0; w < 2; w++)
                    TGS_TRY(tgs_train_step_batched(c, g, cams, V, targets, nullptr, nullptr, nullptr, nullptr, 0, st));
                TGS_CHECK(cudaEventRecord(e0, st));
                const int reps = 3;
                for (int r = 0; r < reps; r++)
                    TGS_TRY(tgs_train_step_batched(c, g, cams, V, targets, nullptr, nullptr, nullptr, nullptr, 0, st));
                TGS_CHECK(cudaEventRecord(e1, st));
                TGS_CHECK(cudaEventSynchronize(e1));
                float ms = 0.f;
                TGS_CHECK(cudaEventElapsedTime(&ms, e0, e1));
                if (ms < best) {
                    best = ms;
                    best_cfg = cf;
                }
            }
        }
    best_cfg.key_capacity = 0;
    TGS_TRY(tgs_set_config(c, &best_cfg));
    TGS_TRY(tgs_plan(c, g, cams, V, 1.25, nullptr));
    if (cache_path) {
        bool found = false;
        for (auto &e : cache)
            if (e.key == key) {
                e.tile = best_cfg.tile;
                e.ppt = best_cfg.ppt;
                e.batch = best_cfg.batch;
                found = true;
            }
        if (!found) cache.push_back({key, best_cfg.tile, best_cfg.ppt, best_cfg.batch});
        FILE *f = fopen(cache_path, "w");
        if (f) {
            fprintf(f, "{\n");
            for (size_t i = 0; i < cache.size(); i++)
                fprintf(f, "  \"%s\": {\"tile\": %d, \"ppt\": %d, \"batch\": %d}%s\n", cache[i].key.c_str(),
                        cache[i].tile, cache[i].ppt, cache[i].batch, i + 1 < cache.size() ? "," : "");
            fprintf(f, "}\n");
            fclose(f);
        }
    }
    return TGS_OK;
}

}  // extern "C"
