// kns_api.cu -- the C ABI runtime: contexts, resident grids, argument checks, launches, status.
#include <cuda_runtime.h>

#include <chrono>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "kns.h"
#include "kns_device.cuh"
#include "kns_kernels.h"
#include "kns_tc.cuh"

// Device scratch of the wavefront render, owned by the context and grown on demand.
struct WaveScratch {
    int64_t rays = 0;  // capacity in rays
    int nc = 0;        // capacity in cells
    int cams = 0;      // capacity in cameras
    float *t_ray = nullptr;
    float4 *t_hist = nullptr;  // last evaluated positions of each ray (cycle test)
    int4 *trap = nullptr;      // BF16 renders: each ray's seam-trap tracker (kns_wave.cuh)
    int *steps_ray = nullptr, *cell_ray = nullptr, *q[2] = {nullptr, nullptr}, *qcell[2] = {nullptr, nullptr};
    int *sorted = nullptr, *hits = nullptr;
    int *cellbuf = nullptr;  // count[2], fill[2], off, tile_off (6 * (nc + 1) ints)
    int4 *tiles = nullptr;   // tile descriptors of a round (max_tiles(rays, 2 nc))
    int *pend_r[2] = {nullptr, nullptr};  // per round parity: rays waiting for the occupancy DDA
    float *pend_t[2] = {nullptr, nullptr};
    int *ray_view = nullptr;
    kns::ViewDev *d_views = nullptr;
    kns::WaveCtrl *ctrl = nullptr;
};

// Device scratch of the path tracer (per path: ray, throughput, radiance, trace outputs).
struct PtScratch {
    int64_t cap = 0;  // paths
    int cap_cams = 0;
    float *o = nullptr, *w = nullptr, *beta = nullptr, *L = nullptr, *rgb = nullptr, *depth = nullptr,
          *normal = nullptr, *cams = nullptr;
    uint8_t *alive = nullptr, *hit = nullptr;
};

// Device scratch and saved state of the training step, owned by the context and grown on demand.
struct TrainScratch {
    int64_t cap_B = 0, cap_M = 0;  // capacity: rays, eikonal points
    int cap_S = 0, cap_Ns = 0, cap_keys = 0;
    int64_t cap_rec = 0;           // sorted records
    float *t = nullptr, *d_coarse = nullptr, *d_fd = nullptr, *g_fd = nullptr, *d_c = nullptr, *g_dc = nullptr;
    float *rgb_c = nullptr, *g_rgb = nullptr, *C = nullptr;
    uint8_t *valid = nullptr;
    double *acc = nullptr;
    int *keys = nullptr;           // count, off, fill, chunk_off (4 x (keys + 1))
    float4 *sorted = nullptr;
    int *d_counts = nullptr;       // records: coarse, difference points, centres
    // phase timing (events created on first use)
    cudaEvent_t ev[2 * 8] = {};
    bool timed = false;
    // the forward pass whose state the scratch holds
    uint64_t gen = 0;
    bool pending = false, backward_done = false;
    kns::TrainArgs args{};
};

struct kns_ctx {
    int device = 0;
    int sm_count = 1;
    std::mutex mu;
    std::string err;
    int *d_status = nullptr;  // device status word written by kernels (0 = fine)
    WaveScratch ws;
    TrainScratch ts;
    PtScratch ps;
    int *h_live = nullptr;                 // pinned: per recent round, its live samples and its
                                           // predecessor's pending rays (2 ints per round, 4 rounds)
    cudaEvent_t ev_live[4] = {nullptr, nullptr, nullptr, nullptr};
    cudaStream_t side = nullptr;           // the advance kernel of round k runs here beside round k + 1
    cudaEvent_t ev_scan = nullptr, ev_adv[2] = {nullptr, nullptr};
    // last render's statistics
    bool have_stats = false;
    kns_render_stats stats{};
    cudaStream_t stats_stream = nullptr;
    std::vector<cudaEvent_t> ev_pool;                   // timing events (created on demand)
    struct Mark {
        int cls, ev, round;  // kernel class, index of its begin event, round (-1: outside the rounds)
    };
    std::vector<Mark> ev_marks;
    size_t ev_used = 0;
    int cur_round = -1;                    // round being enqueued (tags timing marks)
    std::vector<int> round_live;           // samples queued per round of the last render (-1: not read)
};

struct kns_grid {
    kns_ctx *ctx = nullptr;
    kns_grid_desc desc{};
    kns::Shape shape{};
    float *d_w = nullptr;   // per-thread layout (shading, field queries, occupancy)
    float *d_wt = nullptr;  // k-major trace layout (wavefront tile GEMM)
    int wt_stride = 0;
    unsigned char *d_wb = nullptr;  // BF16 hi/lo tensor-core trace layout (kns_tc.cuh)
    int wb_stride = 0;              // bytes per cell
    float *d_ws = nullptr;          // shading layout (kns_shade.cu)
    int ws_stride = 0;              // floats per cell
    uint32_t *d_occ = nullptr;
    uint32_t *d_occ_coarse = nullptr;  // 8^3-voxel block mask (res % 8 == 0)
    size_t occ_words64 = 0;
    int occ_box[6] = {0, 0, 0, -1, -1, -1};  // index box of the occupied voxels (lo xyz, hi xyz)
    int n_sub = 1;  // grids in the stack (kns_load_grid_stack): cells, layouts and masks back to back
    int *d_boxes = nullptr;  // a stack: each grid's occupied-voxel index box (6 ints per grid)
    kns::GridView view{};
};

namespace {

thread_local std::string g_create_err;

kns_status set_err(kns_ctx *ctx, kns_status st, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    if (ctx)
        ctx->err = buf;
    else
        g_create_err = buf;
    return st;
}

kns_status cuda_err(kns_ctx *ctx, cudaError_t e, const char *what) {
    return set_err(ctx, e == cudaErrorMemoryAllocation ? KNS_ERR_OUT_OF_MEMORY : KNS_ERR_CUDA, "%s: %s (%s)", what,
                   cudaGetErrorString(e), cudaGetErrorName(e));
}

// Makes the context's device current for the scope and restores the caller's device after.
struct DeviceScope {
    int prev = -1;
    bool ok = true;
    explicit DeviceScope(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != dev) ok = cudaSetDevice(dev) == cudaSuccess;
    }
    ~DeviceScope() {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

int64_t canon_sdf_params(const kns_grid_desc &d) {
    const int64_t in = 3 + 6 * d.pe_pos_L;
    int64_t p = in * d.sdf_width + d.sdf_width;
    p += (int64_t)(d.sdf_hidden - 1) * (d.sdf_width * d.sdf_width + d.sdf_width);
    p += (int64_t)d.sdf_width * (1 + d.feat_dim) + (1 + d.feat_dim);
    return p;
}
int64_t canon_col_in(const kns_grid_desc &d) { return d.feat_dim + 3 + 3 + 6 * d.pe_dir_L + (d.col_use_x ? 3 : 0); }
int64_t canon_col_params(const kns_grid_desc &d) {
    const int64_t in = canon_col_in(d);
    int64_t p = in * d.col_width + d.col_width;
    p += (int64_t)(d.col_hidden - 1) * (d.col_width * d.col_width + d.col_width);
    p += (int64_t)d.col_width * 3 + 3;
    return p;
}

kns_status check_desc(kns_ctx *ctx, const kns_grid_desc &d) {
    if (d.N < 1 || d.N > 64) return set_err(ctx, KNS_ERR_INVALID_ARG, "N=%d out of range [1, 64]", d.N);
    if (d.pe_pos_L < 0 || d.pe_pos_L > 12 || d.pe_dir_L < 0 || d.pe_dir_L > 12)
        return set_err(ctx, KNS_ERR_INVALID_ARG, "encoding frequencies out of range");
    if (d.sdf_hidden < 1 || d.sdf_width < 1 || d.col_hidden < 1 || d.col_width < 1 || d.feat_dim < 0)
        return set_err(ctx, KNS_ERR_INVALID_ARG, "MLP shape out of range");
    if (d.col_use_x != 0 && d.col_use_x != 1) return set_err(ctx, KNS_ERR_INVALID_ARG, "col_use_x must be 0 or 1");
    if (!(d.softplus_beta > 0.f) || !std::isfinite(d.softplus_beta))
        return set_err(ctx, KNS_ERR_INVALID_ARG, "softplus_beta must be positive and finite");
    for (int a = 0; a < 3; ++a)
        if (!std::isfinite(d.bbox_min[a]) || !std::isfinite(d.bbox_max[a]) || !(d.bbox_max[a] > d.bbox_min[a]))
            return set_err(ctx, KNS_ERR_INVALID_ARG, "bounding box axis %d is empty or not finite", a);
    if (d.occ_res < 0 || d.occ_res > 1024 || (d.occ_res > 0 && d.occ_res % d.N != 0))
        return set_err(ctx, KNS_ERR_INVALID_ARG, "occ_res=%d must be 0 or a multiple of N up to 1024", d.occ_res);
    kns::Shape sh{d.sdf_width, d.sdf_hidden, d.pe_pos_L, d.pe_dir_L};
    if (d.feat_dim != kns::FEAT || d.col_hidden != 1 || d.col_width != d.sdf_width || !kns::shape_supported(sh))
        return set_err(ctx, KNS_ERR_UNSUPPORTED,
                       "unsupported grid shape (built: widths 32/64, 2-3 SDF hidden layers, (L, Ld) = (4, 2) or "
                       "(6, 4), feat_dim 15, one colour hidden layer of the SDF width)");
    return KNS_OK;
}

// Canonical FP32 layout -> device layout (see kns_device.cuh), one cell at a time.
void convert_cell(const kns_grid_desc &d, int dev_floats, const float *src, float *dst) {
    const int W = d.sdf_width, H = d.sdf_hidden, IN = 3 + 6 * d.pe_pos_L, INP = kns::round4(IN);
    const int CIN_NOX = d.feat_dim + 3 + 3 + 6 * d.pe_dir_L, CIN_DEV = CIN_NOX + 3, CINP = kns::round4(CIN_DEV);
    std::memset(dst, 0, sizeof(float) * dev_floats);
    int64_t s = 0, o = 0;
    // SDF layer 0
    for (int r = 0; r < W; ++r)
        for (int c = 0; c < IN; ++c) dst[o + r * INP + c] = src[s + r * IN + c];
    s += (int64_t)W * IN;
    o += (int64_t)W * INP;
    for (int r = 0; r < W; ++r) dst[o + r] = src[s + r];
    s += W;
    o += W;
    // hidden layers
    for (int l = 1; l < H; ++l) {
        std::memcpy(dst + o, src + s, sizeof(float) * (W * W + W));
        s += W * W + W;
        o += W * W + W;
    }
    // last SDF layer
    std::memcpy(dst + o, src + s, sizeof(float) * (kns::SDF_OUT * W + kns::SDF_OUT));
    s += kns::SDF_OUT * W + kns::SDF_OUT;
    o += kns::SDF_OUT * W + kns::SDF_OUT;
    // colour layer 0: [z, n, gamma(v)] columns, then the x slot
    const int cin = (int)canon_col_in(d);
    for (int r = 0; r < W; ++r) {
        for (int c = 0; c < CIN_NOX; ++c) dst[o + r * CINP + c] = src[s + r * cin + c];
        if (d.col_use_x)
            for (int c = 0; c < 3; ++c) dst[o + r * CINP + CIN_NOX + c] = src[s + r * cin + CIN_NOX + c];
    }
    s += (int64_t)W * cin;
    o += (int64_t)W * CINP;
    for (int r = 0; r < W; ++r) dst[o + r] = src[s + r];
    s += W;
    o += W;
    // colour last layer (3 rows padded to 4)
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < W; ++c) dst[o + r * W + c] = src[s + r * W + c];
    s += 3 * W;
    o += 4 * W;
    for (int r = 0; r < 3; ++r) dst[o + r] = src[s + r];
}

// Canonical SDF layers -> k-major trace layout (kns_device.cuh, Cfg::tW0..tbL), one cell.
void convert_cell_trace(const kns_grid_desc &d, int dev_floats, const float *src, float *dst) {
    const int W = d.sdf_width, H = d.sdf_hidden, IN = 3 + 6 * d.pe_pos_L, INP = kns::round4(IN);
    std::memset(dst, 0, sizeof(float) * dev_floats);
    int64_t s = 0, o = 0;
    for (int r = 0; r < W; ++r)
        for (int c = 0; c < IN; ++c) dst[o + c * W + r] = src[s + r * IN + c];
    s += (int64_t)W * IN;
    o += (int64_t)W * INP;
    for (int r = 0; r < W; ++r) dst[o + r] = src[s + r];
    s += W;
    o += W;
    for (int l = 1; l < H; ++l) {
        for (int r = 0; r < W; ++r)
            for (int c = 0; c < W; ++c) dst[o + c * W + r] = src[s + r * W + c];
        s += W * W;
        o += W * W;
        for (int r = 0; r < W; ++r) dst[o + r] = src[s + r];
        s += W;
        o += W;
    }
    for (int c = 0; c < W; ++c) dst[o + c] = src[s + c];  // row 0 (d) of the last layer
    o += W;
    dst[o] = src[s + (int64_t)kns::SDF_OUT * W];  // its bias
}

// Canonical SDF layers -> the tensor-core trace layout of kns_tc.cuh, one cell: every weight as a
// BF16 pair hi = bf16(w), lo = bf16(w - hi) in the canonical K-major layout (row = output unit,
// column = input), then the FP32 biases, the d row of the last layer and its bias.
static uint16_t to_bf16(float f) {  // round to nearest even
    uint32_t u;
    std::memcpy(&u, &f, 4);
    if ((u & 0x7f800000u) == 0x7f800000u) return (uint16_t)(u >> 16);  // inf / nan
    u += 0x7fffu + ((u >> 16) & 1u);
    return (uint16_t)(u >> 16);
}
static float from_bf16(uint16_t h) {
    const uint32_t u = (uint32_t)h << 16;
    float f;
    std::memcpy(&f, &u, 4);
    return f;
}
int tc_cell_bytes(const kns_grid_desc &d) {
    return kns::tc::cell_bytes(d.sdf_width, d.sdf_hidden, kns::tc::k0_of(3 + 6 * d.pe_pos_L));
}
void convert_cell_tc(const kns_grid_desc &d, int bytes, const float *src, unsigned char *dst) {
    const int W = d.sdf_width, H = d.sdf_hidden, IN = 3 + 6 * d.pe_pos_L, K0 = kns::tc::k0_of(IN);
    std::memset(dst, 0, bytes);
    auto emit_layer = [&](int l, const float *Wm, int kin) {
        const int K = l == 0 ? K0 : W;
        unsigned char *hi = dst + kns::tc::w_hi(l, W, K0), *lo = dst + kns::tc::w_lo(l, W, K0);
        for (int n = 0; n < W; ++n)
            for (int k = 0; k < kin; ++k) {
                const float x = Wm[n * kin + k];
                const uint16_t h = to_bf16(x), r = to_bf16(x - from_bf16(h));
                std::memcpy(hi + kns::tc::canon_off(n, k, K), &h, 2);
                std::memcpy(lo + kns::tc::canon_off(n, k, K), &r, 2);
            }
    };
    float *bias = reinterpret_cast<float *>(dst + kns::tc::bias_off(W, H, K0));
    float *drow = reinterpret_cast<float *>(dst + kns::tc::drow_off(W, H, K0));
    int64_t s = 0;
    emit_layer(0, src, IN);
    s += (int64_t)W * IN;
    for (int r = 0; r < W; ++r) bias[r] = src[s + r];
    s += W;
    for (int l = 1; l < H; ++l) {
        emit_layer(l, src + s, W);
        s += (int64_t)W * W;
        for (int r = 0; r < W; ++r) bias[l * W + r] = src[s + r];
        s += W;
    }
    for (int c = 0; c < W; ++c) drow[c] = src[s + c];  // row 0 (d) of the last layer
    drow[W] = src[s + (int64_t)kns::SDF_OUT * W];       // its bias
}

// 64-bit words of one grid's occupancy mask, and 32-bit words of its 8^3-block mask (0 without one).
size_t occ_words64_per_grid(const kns_grid_desc &d) {
    const int64_t nvox = (int64_t)d.occ_res * d.occ_res * d.occ_res;
    return d.occ_res > 0 ? (size_t)((nvox + 63) / 64) : 0;
}
size_t coarse_words_per_grid(const kns_grid_desc &d) {
    if (d.occ_res <= 0 || d.occ_res % 8 != 0) return 0;
    const int64_t nb = (int64_t)(d.occ_res / 8) * (d.occ_res / 8) * (d.occ_res / 8);
    return (size_t)((nb + 31) / 32);
}

void fill_view(kns_grid *g) {
    kns::GridView &v = g->view;
    const kns_grid_desc &d = g->desc;
    v.w = g->d_w;
    v.cell_stride = kns::cell_floats(g->shape);
    v.ws = g->d_ws;
    v.ws_stride = g->ws_stride;
    v.N = d.N;
    for (int a = 0; a < 3; ++a) {
        v.bmin[a] = d.bbox_min[a];
        v.bmax[a] = d.bbox_max[a];
        v.cscale[a] = (float)d.N / (d.bbox_max[a] - d.bbox_min[a]);
        v.oscale[a] = d.occ_res > 0 ? (float)d.occ_res / (d.bbox_max[a] - d.bbox_min[a]) : 0.f;
        v.ovox[a] = d.occ_res > 0 ? (d.bbox_max[a] - d.bbox_min[a]) / (float)d.occ_res : 0.f;
    }
    v.occ = g->d_occ;
    v.occ_coarse = g->d_occ_coarse;
    v.cres = d.occ_res / 8;
    for (int a = 0; a < 3; ++a) {
        v.olo[a] = g->occ_box[a];
        v.ohi[a] = g->occ_box[3 + a];
    }
    v.occ_res = d.occ_res;
    v.occ_per_cell = d.occ_res > 0 ? d.occ_res / d.N : 1;
    v.beta = d.softplus_beta;
    v.inv_beta = 1.f / d.softplus_beta;
    v.cell_base = 0;
    v.ncl = d.N * d.N * d.N;
    v.occ_words = (int)(2 * occ_words64_per_grid(d));
    v.coarse_words = (int)coarse_words_per_grid(d);
    v.sub_boxes = g->d_boxes;
}

void free_scratch(WaveScratch &w) {
    cudaFree(w.t_ray);
    cudaFree(w.t_hist);
    cudaFree(w.trap);
    cudaFree(w.steps_ray);
    cudaFree(w.cell_ray);
    cudaFree(w.q[0]);
    cudaFree(w.q[1]);
    cudaFree(w.qcell[0]);
    cudaFree(w.qcell[1]);
    cudaFree(w.sorted);
    cudaFree(w.hits);
    cudaFree(w.cellbuf);
    cudaFree(w.tiles);
    for (int p = 0; p < 2; ++p) {
        cudaFree(w.pend_r[p]);
        cudaFree(w.pend_t[p]);
    }
    cudaFree(w.ray_view);
    cudaFree(w.d_views);
    cudaFree(w.ctrl);
    w = WaveScratch{};
}

// Render tiling: samples per tile (a warp tile, or a 256-thread block tile).
constexpr int kRenderBlockTile = 16;        // samples per warp tile
constexpr int kRenderBlockTiles = 4;        // FP32 renders use 128-sample block tiles of 128 threads
// Defaults picked by the autotuner on the 16^3 / width-32 grid at 8 x 800x800.
constexpr int kRenderInnerSteps = 4;
constexpr int kRenderMinActive = 8;
constexpr int kRenderBlockInnerSteps = 2;  // block tiles: a second evaluation of a tile in the round ...
constexpr int kRenderBlockMinActive = 16;  // ... while at least 16 of its rays stay in its cell
constexpr int kRenderTailRays = 131072;  // rounds this small finish one warp per ray (width 32)
// Cells of all grids of a stack: the BF16 seam trap keeps a cell number in 19 bits.
constexpr int64_t kMaxStackCells = 262144;
// tensor-core tiles (BF16 renders): a second evaluation while at least 16 rays stay in the cell
constexpr int kRenderBf16InnerSteps = 2;        // width 64
constexpr int kRenderBf16InnerStepsNarrow = 4;  // width 32
constexpr int kRenderBf16MinActive = 16;
// BF16 renders hand rounds of at most this many rays (live + pending) to the one-warp-per-ray FP32
// tail: the best of 8K..512K on both 1080p workloads (a tensor-core round costs ~50 us however few its rays);
// FP32 renders of width-64 grids too (their tail warps hold 41 KB of weights each: 5 per SM), the best of
// 8K..512K on the 32^3 width-64 workload (131072 stays best at width 32)
constexpr int kRenderBf16TailRays = 32768;
constexpr int kRenderBf16TailRaysWide = 16384;  // BF16 renders of width-64 grids
constexpr int kRenderBlocksPerSM = 16;
constexpr int kRenderStaticTiles = 2;

// Kernel classes timed by kns_render when opts->timing is set.
enum { kTGen = 0, kTSort = 1, kTEvalF32 = 2, kTEvalBF16 = 3, kTShade = 4 };

// Records a begin event for a kernel class; returns its index (or -1 when timing is off).
int timing_begin(kns_ctx *ctx, bool on, int cls, cudaStream_t s) {
    if (!on) return -1;
    while (ctx->ev_pool.size() < ctx->ev_used + 2) {
        cudaEvent_t e;
        if (cudaEventCreate(&e) != cudaSuccess) return -1;
        ctx->ev_pool.push_back(e);
    }
    const int i = (int)ctx->ev_used;
    ctx->ev_used += 2;
    cudaEventRecord(ctx->ev_pool[i], s);
    ctx->ev_marks.push_back({cls, i, ctx->cur_round});
    return i;
}
void timing_end(kns_ctx *ctx, int i, cudaStream_t s) {
    if (i >= 0) cudaEventRecord(ctx->ev_pool[i + 1], s);
}

// Grows the context's wavefront scratch to hold `rays` rays, `nc` cells and `cams` cameras.
kns_status ensure_scratch(kns_ctx *ctx, int64_t rays, int nc, int cams) {
    WaveScratch &w = ctx->ws;
    if (rays <= w.rays && nc <= w.nc && cams <= w.cams) return KNS_OK;
    cudaDeviceSynchronize();  // earlier renders may still use the old buffers
    const int64_t R = std::max(rays, w.rays);
    const int NC = std::max(nc, w.nc);
    const int NCAM = std::max(cams, w.cams);
    free_scratch(w);
    cudaError_t e = cudaSuccess;
    auto alloc = [&](auto **p, size_t bytes) {
        if (e == cudaSuccess) e = cudaMalloc((void **)p, bytes);
    };
    alloc(&w.t_ray, sizeof(float) * R);
    alloc(&w.t_hist, sizeof(float4) * R);
    alloc(&w.trap, sizeof(int4) * R);
    alloc(&w.steps_ray, sizeof(int) * R);
    alloc(&w.cell_ray, sizeof(int) * R);
    alloc(&w.q[0], sizeof(int) * R);
    alloc(&w.q[1], sizeof(int) * R);
    alloc(&w.qcell[0], sizeof(int) * R);
    alloc(&w.qcell[1], sizeof(int) * R);
    alloc(&w.sorted, sizeof(int) * R);
    alloc(&w.hits, sizeof(int) * R);
    alloc(&w.cellbuf, sizeof(int) * 6 * (size_t)(NC + 1));
    alloc(&w.tiles, sizeof(int4) * (size_t)kns::max_tiles(R, 2 * NC));
    for (int p = 0; p < 2; ++p) {
        alloc(&w.pend_r[p], sizeof(int) * R);
        alloc(&w.pend_t[p], sizeof(float) * R);
    }
    alloc(&w.ray_view, sizeof(int) * R);
    alloc(&w.d_views, sizeof(kns::ViewDev) * NCAM);
    alloc(&w.ctrl, sizeof(kns::WaveCtrl));
    if (e != cudaSuccess) {
        free_scratch(w);
        return cuda_err(ctx, e, "render scratch");
    }
    w.rays = R;
    w.nc = NC;
    w.cams = NCAM;
    return KNS_OK;
}

void free_pt_scratch(PtScratch &p) {
    void *ps[] = {p.o, p.w, p.beta, p.L, p.rgb, p.depth, p.normal, p.cams, p.alive, p.hit};
    for (void *q : ps)
        if (q) cudaFree(q);
    p = PtScratch{};
}

kns_status ensure_pt_scratch(kns_ctx *ctx, int64_t n, int cams) {
    PtScratch &p = ctx->ps;
    if (n <= p.cap && cams <= p.cap_cams) return KNS_OK;
    cudaDeviceSynchronize();
    const int64_t N = std::max(n, p.cap);
    const int NC = std::max(cams, p.cap_cams);
    free_pt_scratch(p);
    cudaError_t e = cudaSuccess;
    auto alloc = [&](auto **q, size_t bytes) {
        if (e == cudaSuccess) e = cudaMalloc((void **)q, bytes);
    };
    const size_t v3 = sizeof(float) * 3 * (size_t)N;
    alloc(&p.o, v3);
    alloc(&p.w, v3);
    alloc(&p.beta, v3);
    alloc(&p.L, v3);
    alloc(&p.rgb, v3);
    alloc(&p.normal, v3);
    alloc(&p.depth, sizeof(float) * (size_t)N);
    alloc(&p.cams, sizeof(float) * 16 * (size_t)NC);
    alloc(&p.alive, (size_t)N);
    alloc(&p.hit, (size_t)N);
    if (e != cudaSuccess) {
        free_pt_scratch(p);
        return cuda_err(ctx, e, "path-tracing scratch");
    }
    p.cap = N;
    p.cap_cams = NC;
    return KNS_OK;
}

void free_train_scratch(TrainScratch &t) {
    void *ps[] = {t.t, t.d_coarse, t.d_fd, t.g_fd, t.d_c, t.g_dc, t.rgb_c, t.g_rgb, t.C, t.valid, t.acc, t.keys,
                  t.sorted, t.d_counts};
    for (void *p : ps)
        if (p) cudaFree(p);
    const uint64_t gen = t.gen;
    cudaEvent_t ev[16];
    for (int i = 0; i < 16; ++i) ev[i] = t.ev[i];
    t = TrainScratch{};
    t.gen = gen;
    for (int i = 0; i < 16; ++i) t.ev[i] = ev[i];
}

// Grows the training scratch for B rays of S samples (Ns stratified), M eikonal points, nkeys keys.
kns_status ensure_train_scratch(kns_ctx *ctx, int64_t B, int S, int Ns, int64_t M, int nkeys) {
    TrainScratch &t = ctx->ts;
    const int64_t nrec = std::max(B * Ns, 6 * (B * S + M) + B * S);
    if (B <= t.cap_B && S <= t.cap_S && Ns <= t.cap_Ns && M <= t.cap_M && nkeys <= t.cap_keys && nrec <= t.cap_rec)
        return KNS_OK;
    cudaDeviceSynchronize();  // earlier steps may still use the old buffers
    const int64_t cB = std::max(B, t.cap_B), cM = std::max(M, t.cap_M);
    const int cS = std::max(S, t.cap_S), cNs = std::max(Ns, t.cap_Ns), cK = std::max(nkeys, t.cap_keys);
    const int64_t cR = std::max(nrec, t.cap_rec);
    free_train_scratch(t);
    cudaError_t e = cudaSuccess;
    auto alloc = [&](auto **p, size_t bytes) {
        if (e == cudaSuccess) e = cudaMalloc((void **)p, bytes > 0 ? bytes : 16);
    };
    const size_t bs = (size_t)cB * cS, fd = 6 * ((size_t)cB * cS + (size_t)cM);
    alloc(&t.t, sizeof(float) * bs);
    alloc(&t.d_coarse, sizeof(float) * (size_t)cB * cNs);
    alloc(&t.d_fd, sizeof(float) * fd);
    alloc(&t.g_fd, sizeof(float) * fd);
    alloc(&t.d_c, sizeof(float) * bs);
    alloc(&t.g_dc, sizeof(float) * bs);
    alloc(&t.rgb_c, sizeof(float) * 3 * bs);
    alloc(&t.g_rgb, sizeof(float) * 3 * bs);
    alloc(&t.C, sizeof(float) * 3 * (size_t)cB);
    alloc(&t.valid, (size_t)cB);
    alloc(&t.acc, 2 * sizeof(double));
    alloc(&t.keys, sizeof(int) * 4 * ((size_t)cK + 1));
    alloc(&t.sorted, sizeof(float4) * (size_t)cR);
    alloc(&t.d_counts, 4 * sizeof(int));
    if (e != cudaSuccess) {
        free_train_scratch(t);
        return cuda_err(ctx, e, "training scratch");
    }
    t.cap_B = cB;
    t.cap_S = cS;
    t.cap_Ns = cNs;
    t.cap_M = cM;
    t.cap_keys = cK;
    t.cap_rec = cR;
    return KNS_OK;
}

}  // namespace

// ------------------------------------------------------------------ allocation-free render
//
// kns_render_noalloc serves callers that must not allocate device memory once they are running:
// an engine that hands all device memory to its own pool allocator up front, or a latency-bound
// loop that cannot afford cudaMalloc's implicit device synchronisation.  Its scratch is one
// file-scope device array sized for KNS_NOALLOC_MAX_RAYS rays, KNS_NOALLOC_MAX_CELLS cells and
// KNS_NOALLOC_MAX_CAMS cameras (about 14 MB: twelve 1 MiB per-ray buffers, the per-cell counters and
// offsets, the tile descriptors, the view table and the control words -- kNoAllocBytes below), held by
// every GPU that loads the library until the process exits.  kns_create loads the array on its device
// and looks up its address there, so the entry point itself allocates nothing.  Every call shares the
// array, so calls that overlap on the GPU race; the counters that must start at zero are cleared by
// each call.
namespace {

constexpr size_t kNoAllocAlign = 256;
constexpr size_t align_up(size_t v) { return (v + kNoAllocAlign - 1) / kNoAllocAlign * kNoAllocAlign; }
constexpr size_t kNoAllocRayBuf = align_up(sizeof(int) * (size_t)KNS_NOALLOC_MAX_RAYS);
constexpr size_t kNoAllocCellBuf = align_up(sizeof(int) * 6 * (size_t)(KNS_NOALLOC_MAX_CELLS + 1));
constexpr size_t kNoAllocViewBuf = align_up(sizeof(kns::ViewDev) * (size_t)KNS_NOALLOC_MAX_CAMS);
constexpr size_t kNoAllocCtrlBuf = align_up(sizeof(kns::WaveCtrl));
constexpr size_t kNoAllocTileBuf =
    align_up(sizeof(int4) * (size_t)(KNS_NOALLOC_MAX_RAYS / 16 + KNS_NOALLOC_MAX_CELLS + 1));
// t_ray, steps_ray, cell_ray, q[2], qcell[2], sorted, hits, ray_view, pend_r, pend_t: twelve per-ray
// int/float buffers
constexpr size_t kNoAllocBytes =
    12 * kNoAllocRayBuf + kNoAllocCellBuf + kNoAllocViewBuf + kNoAllocCtrlBuf + kNoAllocTileBuf;

__device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

std::mutex g_noalloc_mu;
void *g_noalloc_dev_ptr[256] = {};  // device address of g_noalloc_scratch, per device ordinal

// The host-side name g_noalloc_scratch is only a stand-in for the device array: its device address
// is looked up once per device, with that device current -- by kns_create (the lookup loads the module
// and with it the array), or, should that have failed, by the first kns_render_noalloc on the device.
kns_status noalloc_scratch(kns_ctx *ctx, unsigned char **out) {
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (ctx->device < 0 || ctx->device >= 256) return set_err(ctx, KNS_ERR_INVALID_ARG, "device ordinal too large");
    if (!g_noalloc_dev_ptr[ctx->device]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) return cuda_err(ctx, e, "cudaGetSymbolAddress(no-alloc scratch)");
        g_noalloc_dev_ptr[ctx->device] = p;
    }
    *out = (unsigned char *)g_noalloc_dev_ptr[ctx->device];
    return KNS_OK;
}

}  // namespace

extern "C" {

kns_status kns_create(int device, kns_ctx **out) {
    if (!out) return set_err(nullptr, KNS_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    int n = 0;
    cudaError_t e = cudaGetDeviceCount(&n);
    if (e != cudaSuccess) return cuda_err(nullptr, e, "cudaGetDeviceCount");
    if (device < 0 || device >= n) return set_err(nullptr, KNS_ERR_INVALID_ARG, "device %d of %d", device, n);
    kns_ctx *c = new (std::nothrow) kns_ctx();
    if (!c) return set_err(nullptr, KNS_ERR_OUT_OF_MEMORY, "host allocation failed");
    c->device = device;
    DeviceScope ds(device);
    cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, device);
    if (c->sm_count < 1) c->sm_count = 1;
    if ((e = cudaMalloc(&c->d_status, sizeof(int))) != cudaSuccess) {
        delete c;
        return cuda_err(nullptr, e, "cudaMalloc(status)");
    }
    if ((e = cudaMemset(c->d_status, 0, sizeof(int))) != cudaSuccess ||
        (e = cudaHostAlloc((void **)&c->h_live, 8 * sizeof(int), cudaHostAllocDefault)) != cudaSuccess) {
        cudaFree(c->d_status);
        delete c;
        return cuda_err(nullptr, e, "context set-up");
    }
    cudaEvent_t *evs[7] = {&c->ev_live[0], &c->ev_live[1], &c->ev_live[2], &c->ev_live[3], &c->ev_scan,
                           &c->ev_adv[0], &c->ev_adv[1]};
    for (cudaEvent_t *ev : evs)
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(ev, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&c->side, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
        for (cudaEvent_t *ev : evs)
            if (*ev) cudaEventDestroy(*ev);
        cudaFree(c->d_status);
        cudaFreeHost(c->h_live);
        delete c;
        return cuda_err(nullptr, e, "context events and stream");
    }
    // the allocation-free entry point's array: loaded and located now, while allocating is allowed
    unsigned char *scratch = nullptr;
    if (noalloc_scratch(c, &scratch) != KNS_OK) {  // retried by the first kns_render_noalloc
        c->err.clear();
        cudaGetLastError();
    }
    *out = c;
    return KNS_OK;
}

void kns_destroy(kns_ctx *ctx) {
    if (!ctx) return;
    {
        DeviceScope ds(ctx->device);
        cudaDeviceSynchronize();
        free_scratch(ctx->ws);
        free_train_scratch(ctx->ts);
        free_pt_scratch(ctx->ps);
        for (cudaEvent_t ev : ctx->ts.ev)
            if (ev) cudaEventDestroy(ev);
        cudaFree(ctx->d_status);
        cudaFreeHost(ctx->h_live);
        for (int i = 0; i < 4; ++i)
            if (ctx->ev_live[i]) cudaEventDestroy(ctx->ev_live[i]);
        if (ctx->ev_scan) cudaEventDestroy(ctx->ev_scan);
        for (cudaEvent_t ev : ctx->ev_adv)
            if (ev) cudaEventDestroy(ev);
        if (ctx->side) cudaStreamDestroy(ctx->side);
        for (cudaEvent_t ev : ctx->ev_pool) cudaEventDestroy(ev);
    }
    delete ctx;
}

const char *kns_last_error(const kns_ctx *ctx) { return ctx ? ctx->err.c_str() : g_create_err.c_str(); }

kns_status kns_sync(kns_ctx *ctx, void *cuda_stream, int64_t timeout_ms) {
    if (!ctx) return KNS_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(ctx->mu);
    DeviceScope ds(ctx->device);
    cudaStream_t s = (cudaStream_t)cuda_stream;
    const auto start = std::chrono::steady_clock::now();
    for (;;) {
        cudaError_t q = cudaStreamQuery(s);
        if (q == cudaSuccess) break;
        if (q != cudaErrorNotReady) return cuda_err(ctx, q, "stream");
        if (timeout_ms >= 0 &&
            std::chrono::steady_clock::now() - start > std::chrono::milliseconds(timeout_ms))
            return set_err(ctx, KNS_ERR_TIMEOUT, "work on the stream did not finish within %lld ms",
                           (long long)timeout_ms);
        std::this_thread::sleep_for(std::chrono::microseconds(50));
    }
    int status = 0;
    cudaError_t e = cudaMemcpyAsync(&status, ctx->d_status, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_err(ctx, e, "status read");
    if (status != 0) {
        cudaMemsetAsync(ctx->d_status, 0, sizeof(int), s);
        cudaStreamSynchronize(s);
        return set_err(ctx, (kns_status)status, "a kernel reported status %d", status);
    }
    return KNS_OK;
}

// Uploads n_sub grids of one descriptor as one resident object (n_sub = 1: a single grid): their cells
// are numbered back to back (grid k's cell c is k N^3 + c) in every weight layout, and their occupancy
// masks and 8^3-block masks follow each other, each built from its own grid's SDF.
static kns_status load_grid_impl(kns_ctx *ctx, const kns_grid_desc *desc, const float *host_weights,
                                 size_t n_floats, int n_sub, const uint64_t *occ_words, kns_grid **out) {
    if (!desc || !host_weights || !out) return set_err(ctx, KNS_ERR_INVALID_ARG, "NULL desc, weights or out");
    *out = nullptr;
    kns_status st = check_desc(ctx, *desc);
    if (st != KNS_OK) return st;
    const kns_grid_desc d = *desc;
    const int64_t ncl = (int64_t)d.N * d.N * d.N;
    if (n_sub < 1 || (int64_t)n_sub * ncl > kMaxStackCells)
        return set_err(ctx, KNS_ERR_INVALID_ARG, "n_grids=%d: 1 .. %lld cells in all", n_sub,
                       (long long)kMaxStackCells);
    const int64_t ncell = ncl * n_sub;
    const int64_t pcell = canon_sdf_params(d) + canon_col_params(d);
    if ((int64_t)n_floats != ncell * pcell)
        return set_err(ctx, KNS_ERR_INVALID_ARG, "n_floats=%zu, the descriptor needs %lld", n_floats,
                       (long long)(ncell * pcell));
    DeviceScope ds(ctx->device);
    kns_grid *g = new (std::nothrow) kns_grid();
    if (!g) return set_err(ctx, KNS_ERR_OUT_OF_MEMORY, "host allocation failed");
    g->ctx = ctx;
    g->desc = d;
    g->n_sub = n_sub;
    g->shape = kns::Shape{d.sdf_width, d.sdf_hidden, d.pe_pos_L, d.pe_dir_L};
    const int dev_floats = kns::cell_floats(g->shape);
    std::vector<float> host;
    try {
        host.resize((size_t)(ncell * dev_floats));
    } catch (...) {
        delete g;
        return set_err(ctx, KNS_ERR_OUT_OF_MEMORY, "host staging allocation failed");
    }
    for (int64_t c = 0; c < ncell; ++c) convert_cell(d, dev_floats, host_weights + c * pcell, host.data() + c * dev_floats);
    cudaError_t e = cudaMalloc(&g->d_w, host.size() * sizeof(float));
    if (e == cudaSuccess) e = cudaMemcpy(g->d_w, host.data(), host.size() * sizeof(float), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
        g->wt_stride = kns::trace_cell_floats(g->shape);
        std::vector<float> ht;
        try {
            ht.resize((size_t)(ncell * g->wt_stride));
        } catch (...) {
            cudaFree(g->d_w);
            delete g;
            return set_err(ctx, KNS_ERR_OUT_OF_MEMORY, "host staging allocation failed");
        }
        for (int64_t c = 0; c < ncell; ++c)
            convert_cell_trace(d, g->wt_stride, host_weights + c * pcell, ht.data() + c * g->wt_stride);
        e = cudaMalloc(&g->d_wt, ht.size() * sizeof(float));
        if (e == cudaSuccess) e = cudaMemcpy(g->d_wt, ht.data(), ht.size() * sizeof(float), cudaMemcpyHostToDevice);
    }
    if (e == cudaSuccess) {
        g->wb_stride = tc_cell_bytes(d);
        std::vector<unsigned char> hb;
        try {
            hb.resize((size_t)(ncell * g->wb_stride));
        } catch (...) {
            cudaFree(g->d_w);
            cudaFree(g->d_wt);
            delete g;
            return set_err(ctx, KNS_ERR_OUT_OF_MEMORY, "host staging allocation failed");
        }
        for (int64_t c = 0; c < ncell; ++c)
            convert_cell_tc(d, g->wb_stride, host_weights + c * pcell, hb.data() + c * g->wb_stride);
        e = cudaMalloc(&g->d_wb, hb.size());
        if (e == cudaSuccess) e = cudaMemcpy(g->d_wb, hb.data(), hb.size(), cudaMemcpyHostToDevice);
    }
    if (e == cudaSuccess) {  // the shading layout, written on the device from the uploaded weights
        g->ws_stride = kns::shade_cell_floats(g->shape);
        e = cudaMalloc(&g->d_ws, (size_t)ncell * g->ws_stride * sizeof(float));
        if (e == cudaSuccess)
            e = kns::launch_shade_layout(g->shape, g->d_w, dev_floats, ncell, g->d_ws, g->ws_stride, 0);
        if (e == cudaSuccess) e = cudaDeviceSynchronize();
    }
    if (e != cudaSuccess) {
        cudaFree(g->d_w);
        cudaFree(g->d_wt);
        cudaFree(g->d_wb);
        cudaFree(g->d_ws);
        delete g;
        return cuda_err(ctx, e, "grid upload");
    }
    if (d.occ_res > 0) {
        const size_t w64 = occ_words64_per_grid(d), cw = coarse_words_per_grid(d);
        g->occ_words64 = w64 * (size_t)n_sub;
        e = cudaMalloc(&g->d_occ, g->occ_words64 * 8);
        if (e == cudaSuccess) e = cudaMemset(g->d_occ, 0, g->occ_words64 * 8);
        if (e == cudaSuccess && occ_words)
            e = cudaMemcpy(g->d_occ, occ_words, g->occ_words64 * 8, cudaMemcpyHostToDevice);
        if (e == cudaSuccess && cw) e = cudaMalloc(&g->d_occ_coarse, cw * 4 * (size_t)n_sub);
        fill_view(g);
        float diag = 0.f;
        for (int a = 0; a < 3; ++a) diag += g->view.ovox[a] * g->view.ovox[a];
        diag = std::sqrt(diag);
        int box[6] = {d.occ_res, d.occ_res, d.occ_res, -1, -1, -1};  // the union of the grids' boxes
        std::vector<int> boxes((size_t)6 * n_sub);
        for (int k = 0; k < n_sub && e == cudaSuccess; ++k) {
            uint32_t *occ_k = reinterpret_cast<uint32_t *>(g->d_occ) + 2 * w64 * (size_t)k;
            if (!occ_words) {
                kns::GridView v = g->view;
                v.occ = nullptr;
                v.occ_coarse = nullptr;
                v.cell_base = (int)(k * ncl);  // grid k's cells
                e = kns::launch_occupancy_f32(g->shape, v, diag, occ_k, 0);
                if (e == cudaSuccess) e = cudaDeviceSynchronize();
            }
            if (e == cudaSuccess && cw) {
                e = kns::launch_coarse_occupancy(occ_k, d.occ_res, g->d_occ_coarse + cw * (size_t)k, 0);
                if (e == cudaSuccess) e = cudaDeviceSynchronize();
            }
            if (e == cudaSuccess) {
                // the index box of the occupied voxels: the walk leaves (or never enters) it through empty space
                int *d_box = nullptr;
                int init[6] = {d.occ_res, d.occ_res, d.occ_res, -1, -1, -1};
                e = cudaMalloc(&d_box, sizeof(init));
                if (e == cudaSuccess) e = cudaMemcpy(d_box, init, sizeof(init), cudaMemcpyHostToDevice);
                if (e == cudaSuccess) e = kns::launch_occ_bounds(occ_k, d.occ_res, d_box, 0);
                if (e == cudaSuccess) e = cudaMemcpy(init, d_box, sizeof(init), cudaMemcpyDeviceToHost);
                cudaFree(d_box);
                for (int a = 0; a < 3; ++a) {
                    box[a] = std::min(box[a], init[a]);
                    box[3 + a] = std::max(box[3 + a], init[3 + a]);
                }
                for (int a = 0; a < 6; ++a) boxes[6 * k + a] = init[a];
            }
        }
        for (int a = 0; a < 6; ++a) g->occ_box[a] = box[a];
        if (e == cudaSuccess && n_sub > 1) {  // each grid of a stack walks to its own box
            e = cudaMalloc(&g->d_boxes, boxes.size() * sizeof(int));
            if (e == cudaSuccess)
                e = cudaMemcpy(g->d_boxes, boxes.data(), boxes.size() * sizeof(int), cudaMemcpyHostToDevice);
        }
        if (e != cudaSuccess) {
            cudaFree(g->d_w);
            cudaFree(g->d_wt);
            cudaFree(g->d_wb);
            cudaFree(g->d_ws);
            cudaFree(g->d_occ);
            cudaFree(g->d_occ_coarse);
            cudaFree(g->d_boxes);
            delete g;
            return cuda_err(ctx, e, "occupancy");
        }
    }
    fill_view(g);
    *out = g;
    return KNS_OK;
}

kns_status kns_load_grid(kns_ctx *ctx, const kns_grid_desc *desc, const float *host_weights, size_t n_floats,
                         const uint64_t *occ_words, kns_grid **out) {
    if (!ctx) return KNS_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(ctx->mu);
    return load_grid_impl(ctx, desc, host_weights, n_floats, 1, occ_words, out);
}

kns_status kns_load_grid_stack(kns_ctx *ctx, const kns_grid_desc *desc, int32_t n_grids, const float *host_weights,
                               size_t n_floats, const uint64_t *occ_words, kns_grid **out) {
    if (!ctx) return KNS_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(ctx->mu);
    return load_grid_impl(ctx, desc, host_weights, n_floats, n_grids, occ_words, out);
}

kns_status kns_grid_stack_size(const kns_grid *grid, int32_t *n_grids) {
    if (!grid || !n_grids) return KNS_ERR_INVALID_ARG;
    *n_grids = grid->n_sub;
    return KNS_OK;
}

kns_status kns_load_grid_file(kns_ctx *ctx, const char *path, kns_grid **out) {
    if (!ctx) return KNS_ERR_INVALID_ARG;
    if (!path || !out) return set_err(ctx, KNS_ERR_INVALID_ARG, "NULL path or out");
    FILE *f = std::fopen(path, "rb");
    if (!f) return set_err(ctx, KNS_ERR_INVALID_ARG, "cannot open %s", path);
    char magic[4];
    uint32_t version = 0;
    int32_t iv[10];
    float fv[7];
    uint64_t nf = 0, nocc = 0;
    bool ok = std::fread(magic, 1, 4, f) == 4 && std::fread(&version, 4, 1, f) == 1 &&
              std::fread(iv, 4, 10, f) == 10 && std::fread(fv, 4, 7, f) == 7 && std::fread(&nf, 8, 1, f) == 1 &&
              std::fread(&nocc, 8, 1, f) == 1;
    if (!ok || std::memcmp(magic, "KNS1", 4) != 0 || version != 1) {
        std::fclose(f);
        return set_err(ctx, KNS_ERR_FORMAT, "%s: not a version-1 KNS1 grid file", path);
    }
    kns_grid_desc d{};
    d.N = iv[0];
    d.pe_pos_L = iv[1];
    d.pe_dir_L = iv[2];
    d.sdf_hidden = iv[3];
    d.sdf_width = iv[4];
    d.feat_dim = iv[5];
    d.col_hidden = iv[6];
    d.col_width = iv[7];
    d.col_use_x = iv[8];
    d.occ_res = iv[9];
    d.softplus_beta = fv[0];
    for (int a = 0; a < 3; ++a) {
        d.bbox_min[a] = fv[1 + a];
        d.bbox_max[a] = fv[4 + a];
    }
    if (nf > ((uint64_t)1 << 34) || nocc > ((uint64_t)1 << 30)) {
        std::fclose(f);
        return set_err(ctx, KNS_ERR_FORMAT, "%s: implausible sizes in header", path);
    }
    std::vector<float> w;
    std::vector<uint64_t> occ;
    try {
        w.resize(nf);
        occ.resize(nocc);
    } catch (...) {
        std::fclose(f);
        return set_err(ctx, KNS_ERR_OUT_OF_MEMORY, "host allocation failed");
    }
    ok = std::fread(w.data(), 4, nf, f) == nf && std::fread(occ.data(), 8, nocc, f) == nocc;
    std::fclose(f);
    if (!ok) return set_err(ctx, KNS_ERR_FORMAT, "%s: truncated", path);
    if (nocc) {
        const int64_t nvox = (int64_t)d.occ_res * d.occ_res * d.occ_res;
        if (d.occ_res <= 0 || (int64_t)nocc != (nvox + 63) / 64)
            return set_err(ctx, KNS_ERR_FORMAT, "%s: occupancy size does not match occ_res", path);
    }
    return kns_load_grid(ctx, &d, w.data(), w.size(), nocc ? occ.data() : nullptr, out);
}

void kns_free_grid(kns_grid *g) {
    if (!g) return;
    {
        std::lock_guard<std::mutex> lk(g->ctx->mu);
        DeviceScope ds(g->ctx->device);
        cudaDeviceSynchronize();
        cudaFree(g->d_w);
        cudaFree(g->d_wt);
        cudaFree(g->d_wb);
        cudaFree(g->d_ws);
        cudaFree(g->d_occ);
        cudaFree(g->d_occ_coarse);
        cudaFree(g->d_boxes);
    }
    delete g;
}

kns_status kns_grid_get_desc(const kns_grid *g, kns_grid_desc *out) {
    if (!g || !out) return KNS_ERR_INVALID_ARG;
    *out = g->desc;
    return KNS_OK;
}

kns_status kns_copy_occupancy(kns_ctx *ctx, const kns_grid *g, uint64_t *host_words, size_t n_words) {
    if (!ctx) return KNS_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(ctx->mu);
    if (!g || !host_words) return set_err(ctx, KNS_ERR_INVALID_ARG, "NULL grid or buffer");
    if (!g->d_occ) return set_err(ctx, KNS_ERR_INVALID_ARG, "grid has no occupancy mask");
    if (n_words < g->occ_words64)
        return set_err(ctx, KNS_ERR_INVALID_ARG, "buffer holds %zu words, mask needs %zu", n_words, g->occ_words64);
    DeviceScope ds(ctx->device);
    cudaError_t e = cudaMemcpy(host_words, g->d_occ, g->occ_words64 * 8, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_err(ctx, e, "occupancy copy");
    return KNS_OK;
}

}  // extern "C"

namespace {

// Render settings resolved from kns_render_opts.
struct RenderCfg {
    bool bf16 = false, timing = false;
    float eps_coarse = 4e-3f;
    int refine_steps = 2, inner_steps = kRenderInnerSteps, min_active = kRenderMinActive,
        tail_rays = kRenderTailRays, blocks_per_sm = kRenderBlocksPerSM, static_tiles = 1;
    int inner_steps_bf = kRenderBf16InnerSteps, min_active_bf = kRenderBf16MinActive;
    bool persistent = true;  // BF16: every round in one persistent launch
    int block_mode = 1;  // 0 = 16-sample warp tiles; block tiles: 1 = 128 samples x 256 threads,
                         // 3 = 256 x 256, 4 = 128 x 128
};

kns_status resolve_opts(kns_ctx *ctx, const kns_render_opts *opts, float eps, RenderCfg &c, int sdf_width) {
    const int precision = opts ? opts->precision : KNS_FP32;
    if (precision != KNS_FP32 && precision != KNS_BF16)
        return set_err(ctx, KNS_ERR_INVALID_ARG, "unknown precision %d", precision);
    c.bf16 = precision == KNS_BF16;
    // BF16 defaults: the split-BF16 trace is accurate to ~1e-5, so it runs to 0.9 eps itself -- just inside
    // the FP32 threshold, so that the FP32 re-evaluation of its last step at shading confirms the hit (on the
    // 1080p workloads every hit: no FP32 steps follow); FP32 may take one more step (two FP32 evaluations)
    c.eps_coarse = (c.bf16 && opts && opts->eps_coarse > 0.f) ? opts->eps_coarse : 0.9f * eps;
    c.refine_steps = (c.bf16 && opts && opts->refine_steps > 0) ? opts->refine_steps : 2;
    if (c.bf16 && !(c.eps_coarse > 0.f && std::isfinite(c.eps_coarse)))
        return set_err(ctx, KNS_ERR_INVALID_ARG, "eps_coarse must be finite and > 0");
    auto knob = [](int32_t v, int32_t def) { return v == 0 ? def : v; };
    const int bt0 = opts ? knob(opts->block_tiles, kRenderBlockTiles) : kRenderBlockTiles;
    const int def_inner = bt0 == 2 ? kRenderInnerSteps : kRenderBlockInnerSteps;
    const int def_min = bt0 == 2 ? kRenderMinActive : kRenderBlockMinActive;
    c.inner_steps = opts ? knob(opts->inner_steps, def_inner) : def_inner;
    c.min_active = opts ? knob(opts->min_active, def_min) : def_min;
    // the hand-over to the one-warp-per-ray tail and the BF16 tiles' in-tile evaluations, by width (the
    // best of a sweep over 12,288 .. 131,072 rays and 1 .. 8 evaluations at 8 x 1920x1080): FP32 131,072 at
    // width 32, 32,768 at 64; BF16 32,768 rays and 4 evaluations at width 32, 16,384 and 2 at width 64
    const int def_tail = c.bf16 ? (sdf_width >= 64 ? kRenderBf16TailRaysWide : kRenderBf16TailRays)
                                : (sdf_width >= 64 ? kRenderBf16TailRays : kRenderTailRays);
    const int def_inner_bf = sdf_width >= 64 ? kRenderBf16InnerSteps : kRenderBf16InnerStepsNarrow;
    c.tail_rays = opts ? knob(opts->tail_rays, def_tail) : def_tail;
    c.blocks_per_sm = opts ? knob(opts->blocks_per_sm, kRenderBlocksPerSM) : kRenderBlocksPerSM;
    c.static_tiles = (opts ? knob(opts->static_tiles, kRenderStaticTiles) : kRenderStaticTiles) == 1;
    c.inner_steps_bf = opts ? knob(opts->bf16_inner_steps, def_inner_bf) : def_inner_bf;
    c.min_active_bf = opts ? knob(opts->bf16_min_active, kRenderBf16MinActive) : kRenderBf16MinActive;
    if (c.inner_steps_bf < 1 || c.inner_steps_bf > 1024 || c.min_active_bf < 1 || c.min_active_bf > 128)
        return set_err(ctx, KNS_ERR_INVALID_ARG, "bf16 tuning field out of range");
    if (opts && (opts->bf16_rounds < 0 || opts->bf16_rounds > 2))
        return set_err(ctx, KNS_ERR_INVALID_ARG, "bf16_rounds must be 0, 1 or 2");
    c.persistent = !(opts && opts->bf16_rounds == 2);
    if (c.inner_steps < 1 || c.inner_steps > 1024 || c.min_active < 1 || c.min_active > 256 || c.tail_rays < -1 ||
        c.blocks_per_sm < 1 || c.blocks_per_sm > 64 || (opts && (opts->static_tiles < 0 || opts->static_tiles > 2)) ||
        (opts && (opts->block_tiles < 0 || opts->block_tiles > 4)))
        return set_err(ctx, KNS_ERR_INVALID_ARG, "render tuning field out of range");
    const int bt = opts ? knob(opts->block_tiles, kRenderBlockTiles) : kRenderBlockTiles;
    c.block_mode = bt == 2 ? 0 : bt;  // BF16 renders: the FP32 refinement tiles
    if (c.tail_rays < 0) c.tail_rays = 0;
    c.timing = opts && opts->timing == 1;
    return KNS_OK;
}

void begin_stats(kns_ctx *ctx, cudaStream_t s, int64_t rays) {
    ctx->ev_marks.clear();
    ctx->ev_used = 0;
    ctx->round_live.clear();
    ctx->cur_round = -1;
    ctx->stats = kns_render_stats{};
    ctx->stats.rays = rays;
    ctx->stats_stream = s;
    ctx->have_stats = false;
}

// Renders one batch of views (their rays numbered consecutively, fewer than 2^31) with the
// wavefront: generate, rounds of sort + evaluate, shade.  `last` marks the final batch of a call,
// whose device counters kns_get_render_stats reads later; earlier batches add theirs here.
kns_status render_views_impl(kns_ctx *ctx, const kns_grid *grid, const std::vector<kns::ViewDev> &views,
                             int64_t rays, int max_steps, float eps, const RenderCfg &cfg, cudaStream_t s,
                             bool last, const float *ray_o = nullptr, const float *ray_w = nullptr,
                             int64_t n_table = 0) {
    const int NC = grid->n_sub * grid->desc.N * grid->desc.N * grid->desc.N;  // every grid of a stack
    const int nkeys = NC;  // sort keys: cells
    const int nv = (int)views.size();
    kns_status st = ensure_scratch(ctx, rays, nkeys, nv);
    if (st != KNS_OK) return st;
    WaveScratch &w = ctx->ws;
    int max_W = 0, max_H = 0;
    for (const auto &v : views) {
        max_W = std::max(max_W, v.W);
        max_H = std::max(max_H, v.H);
    }
    kns::WaveArgs a{};
    a.n_views = nv;
    a.max_W = max_W;
    a.max_H = max_H;
    a.views = w.d_views;
    a.ray_view = w.ray_view;
    a.ray_o = ray_o;
    a.ray_w = ray_w;
    a.n_table = ray_o ? (int)n_table : 0;
    a.max_steps = max_steps;
    a.eps = eps;
    a.NC = NC;
    a.nkeys = nkeys;
    a.coarse = cfg.bf16 ? 1 : 0;
    a.eps_coarse = cfg.eps_coarse;
    a.refine_steps = cfg.refine_steps;
    a.wb = grid->d_wb;
    a.wb_stride = grid->wb_stride;
    a.btile = kRenderBlockTile;
    a.btile_bf = 128;  // tensor-core tiles: 128 samples
    a.inner_steps = cfg.inner_steps;
    a.tail_max = cfg.tail_rays;
    a.min_active = cfg.min_active;
    a.inner_steps_bf = cfg.inner_steps_bf;
    a.min_active_bf = cfg.min_active_bf;
    a.static_tiles = cfg.static_tiles;
    a.status = ctx->d_status;
    a.wt = grid->d_wt;
    a.wt_stride = grid->wt_stride;
    a.t_ray = w.t_ray;
    a.t_hist = w.t_hist;
    a.trap = cfg.bf16 ? w.trap : nullptr;
    {
        const float ext = std::max(grid->desc.bbox_max[0] - grid->desc.bbox_min[0],
                                   std::max(grid->desc.bbox_max[1] - grid->desc.bbox_min[1],
                                            grid->desc.bbox_max[2] - grid->desc.bbox_min[2]));
        a.trap_span = 0.01f * ext;
    }
    a.steps_ray = w.steps_ray;
    a.cell_ray = w.cell_ray;
    a.q[0] = w.q[0];
    a.q[1] = w.q[1];
    a.qcell[0] = w.qcell[0];
    a.qcell[1] = w.qcell[1];
    a.sorted = w.sorted;
    a.hits = w.hits;
    a.tiles = w.tiles;
    for (int p = 0; p < 2; ++p) {
        a.pend_r[p] = w.pend_r[p];
        a.pend_t[p] = w.pend_t[p];
    }
    a.count[0] = w.cellbuf;
    a.count[1] = w.cellbuf + (nkeys + 1);
    a.fill[0] = w.cellbuf + 2 * (nkeys + 1);
    a.fill[1] = w.cellbuf + 3 * (nkeys + 1);
    a.off = w.cellbuf + 4 * (nkeys + 1);
    a.tile_off = w.cellbuf + 5 * (nkeys + 1);
    a.ctrl = w.ctrl;
    cudaError_t e = cudaMemcpyAsync(w.d_views, views.data(), sizeof(kns::ViewDev) * nv, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(w.ctrl, 0, sizeof(kns::WaveCtrl), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(w.cellbuf, 0, sizeof(int) * 4 * (nkeys + 1), s);
    if (e == cudaSuccess) {
        const int tm = timing_begin(ctx, cfg.timing, kTGen, s);
        e = kns::launch_wave_gen(grid->shape, grid->view, a, s);
        timing_end(ctx, tm, s);
    }
    const int eval_blocks = ctx->sm_count * cfg.blocks_per_sm, scatter_blocks = ctx->sm_count * 4;
    // Rounds.  A ray takes one step per round, except that a step into an empty occupancy voxel
    // puts it on its round's pending list: the advance kernel of round k walks those rays to their
    // next occupied voxel on the side stream while round k + 1 runs (after round k + 1's scan has
    // cleared the counters it adds to) and they rejoin in round k + 2, whose scan waits for it.  So a
    // ray's budget of max_steps steps takes at most 2 max_steps rounds.  The host reads, for round
    // k - 2, its live count and round k - 3's pending count before launching round k, and stops when
    // both are zero (rounds k - 1 and k then hold nothing), so it runs at most two rounds ahead.
    int last_adv = -1;  // the last round whose advance kernel was launched
    const int round0 = (int)ctx->round_live.size();  // rounds of earlier batches of this call
    if (e == cudaSuccess && cfg.bf16 && cfg.persistent) {  // every round on the device, one launch
        a.btile = 128;
        const int tm = timing_begin(ctx, cfg.timing, kTEvalBF16, s);
        e = kns::launch_trace_tc(grid->shape, grid->view, a, ctx->sm_count, s);
        timing_end(ctx, tm, s);
        if (e == cudaSuccess) {  // the rays of the round it left, one warp per ray (nothing when none)
            const int tm2 = timing_begin(ctx, cfg.timing, kTEvalF32, s);
            e = kns::launch_wave_tail(grid->shape, grid->view, a, -1, ctx->sm_count, s);
            timing_end(ctx, tm2, s);
        }
    }
    for (int k = 0; k < 2 * max_steps + 2 && e == cudaSuccess && !(cfg.bf16 && cfg.persistent); ++k) {
        const int cur = k & 1;
        if (k >= 2) {
            e = cudaEventSynchronize(ctx->ev_live[(k - 2) & 3]);
            const int *hl = ctx->h_live + 2 * ((k - 2) & 3);
            if (e == cudaSuccess) ctx->round_live[round0 + k - 2] = hl[0];
            if (e != cudaSuccess || (hl[0] == 0 && hl[1] == 0)) break;
            // round k - 2's advance added to this round's counters
            e = cudaStreamWaitEvent(s, ctx->ev_adv[k & 1], 0);
            if (e != cudaSuccess) break;
        }
        ++ctx->stats.rounds;
        ctx->cur_round = round0 + k;
        ctx->round_live.push_back(-1);
        // the sort cuts tiles of the size the evaluation kernel takes: tensor-core tiles of 128 samples
        // (BF16), block tiles of 128 or 256, or warp tiles of 16
        if (cfg.bf16 || cfg.block_mode == 1 || cfg.block_mode == 4) a.btile = 128;
        else if (cfg.block_mode == 3) a.btile = 256;
        // BF16: the first round always runs on the tensor cores (no one-warp-per-ray tail)
        a.tail_max = (cfg.bf16 && k == 0) ? -1 : cfg.tail_rays;
        int tm = timing_begin(ctx, cfg.timing, kTSort, s);
        e = kns::launch_wave_scan(a, cur, s);
        int *hl = ctx->h_live + 2 * (k & 3);
        if (e == cudaSuccess) e = cudaMemcpyAsync(hl, &w.ctrl->n_live[cur], sizeof(int), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(hl + 1, &w.ctrl->n_pend[cur ^ 1], sizeof(int), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaEventRecord(ctx->ev_live[k & 3], s);
        if (e == cudaSuccess && k >= 1) {  // round k - 1's pending rays, beside this round
            e = cudaEventRecord(ctx->ev_scan, s);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(ctx->side, ctx->ev_scan, 0);
            if (e == cudaSuccess) e = kns::launch_wave_advance(grid->view, a, cur ^ 1, ctx->sm_count, ctx->side);
            if (e == cudaSuccess) e = cudaEventRecord(ctx->ev_adv[cur ^ 1], ctx->side);
            if (e == cudaSuccess) last_adv = k - 1;
        }
        if (e == cudaSuccess) e = kns::launch_wave_scatter(a, cur, scatter_blocks, s);
        timing_end(ctx, tm, s);
        if (e == cudaSuccess && cfg.bf16) {  // tensor-core tiles, or the one-warp-per-ray tail of a small round
            tm = timing_begin(ctx, cfg.timing, kTEvalBF16, s);
            e = kns::launch_wave_eval_tc(grid->shape, grid->view, a, cur, ctx->sm_count, s);
            timing_end(ctx, tm, s);
            tm = timing_begin(ctx, cfg.timing, kTEvalF32, s);
            if (e == cudaSuccess) e = kns::launch_wave_tail(grid->shape, grid->view, a, cur, ctx->sm_count, s);
            timing_end(ctx, tm, s);
        } else if (e == cudaSuccess) {  // FP32 tiles and the one-warp-per-ray tail
            tm = timing_begin(ctx, cfg.timing, kTEvalF32, s);
            e = kns::launch_wave_eval(grid->shape, grid->view, a, cur, eval_blocks, cfg.block_mode, ctx->sm_count, s);
            timing_end(ctx, tm, s);
        }
    }
    ctx->cur_round = -1;
    // the side stream's last advance joins before the shading (it found nothing: the rounds ended)
    if (e == cudaSuccess && last_adv >= 0) e = cudaStreamWaitEvent(s, ctx->ev_adv[last_adv & 1], 0);
    if (e == cudaSuccess) {
        const int tm = timing_begin(ctx, cfg.timing, kTShade, s);
        // hits sorted by cell, shaded on block tiles
        e = kns::launch_hit_sort(a, kns::shade_hit_tile(grid->desc.sdf_width), ctx->sm_count, s);
        if (e == cudaSuccess) e = kns::launch_shade_block(grid->shape, grid->view, a, ctx->sm_count, s);
        // BF16: the hits the shading's FP32 evaluation did not confirm take their last FP32 steps
        if (e == cudaSuccess && cfg.bf16) e = kns::launch_refine(grid->shape, grid->view, a, ctx->sm_count, s);
        timing_end(ctx, tm, s);
    }
    if (e != cudaSuccess) return cuda_err(ctx, e, "render launch");
    if (!last) {
        kns::WaveCtrl hc;
        e = cudaMemcpyAsync(&hc, w.ctrl, sizeof(hc), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return cuda_err(ctx, e, "render counters");
        ctx->stats.hits += hc.n_hits;
        ctx->stats.samples_fp32 += (int64_t)hc.samples_f32;
        ctx->stats.samples_bf16 += (int64_t)hc.samples_bf16;
        ctx->stats.samples_tail += (int64_t)hc.samples_tail;
        ctx->stats.refined += hc.n_refine;
    }
    return KNS_OK;
}

kns::ViewDev make_view(const kns_camera &cam, int W, int H, int64_t ray_base, const kns_frame &out, int grid = 0) {
    kns::ViewDev v{};
    v.grid = grid;
    std::memcpy(v.cam, &cam, sizeof(float) * 16);
    v.rgb = out.rgb;
    v.depth = out.depth;
    v.normal = out.normal;
    v.cell = out.cell;
    v.steps = out.steps;
    v.hit = out.hit;
    v.W = W;
    v.H = H;
    v.ray_base = (int)ray_base;
    return v;
}

}  // namespace

extern "C" {

kns_status kns_render(kns_ctx *ctx, const kns_grid *grid, const kns_camera *cams, int n_cams, int W, int H,
                      int max_steps, float eps, const kns_render_opts *opts, const kns_frame *out,
                      void *cuda_stream) {
    if (!ctx) return KNS_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(ctx->mu);
    if (!grid || !cams || !out) return set_err(ctx, KNS_ERR_INVALID_ARG, "NULL grid, cams or out");
    if (n_cams < 0 || W < 0 || H < 0) return set_err(ctx, KNS_ERR_INVALID_ARG, "negative size");
    if ((int64_t)n_cams * W * H > ((int64_t)1 << 40)) return set_err(ctx, KNS_ERR_INVALID_ARG, "too many rays");
    if (max_steps < 1) return set_err(ctx, KNS_ERR_INVALID_ARG, "max_steps=%d < 1", max_steps);
    if (!(eps > 0.f) || !std::isfinite(eps)) return set_err(ctx, KNS_ERR_INVALID_ARG, "eps must be > 0 and finite");
    if (!out->rgb || !out->depth) return set_err(ctx, KNS_ERR_INVALID_ARG, "rgb and depth buffers are required");
    RenderCfg cfg;
    kns_status st = resolve_opts(ctx, opts, eps, cfg, grid->desc.sdf_width);
    if (st != KNS_OK) return st;
    if (n_cams == 0 || W == 0 || H == 0) return KNS_OK;
    if ((int64_t)W * H > INT32_MAX) return set_err(ctx, KNS_ERR_INVALID_ARG, "W*H exceeds 2^31-1");
    DeviceScope ds(ctx->device);
    cudaStream_t s = (cudaStream_t)cuda_stream;
    begin_stats(ctx, s, (int64_t)n_cams * W * H);
    const int64_t hw = (int64_t)W * H;
    const int per_chunk = (int)std::max<int64_t>(1, std::min<int64_t>(n_cams, (int64_t)INT32_MAX / hw));
    std::vector<kns::ViewDev> views;
    for (int c0 = 0; c0 < n_cams; c0 += per_chunk) {
        const int nc = std::min(per_chunk, n_cams - c0);
        views.clear();
        for (int c = 0; c < nc; ++c) {
            const int64_t base = (int64_t)(c0 + c) * hw;
            kns_frame f{};
            f.rgb = out->rgb + 3 * base;
            f.depth = out->depth + base;
            f.normal = out->normal ? out->normal + 3 * base : nullptr;
            f.cell = out->cell ? out->cell + base : nullptr;
            f.steps = out->steps ? out->steps + base : nullptr;
            f.hit = out->hit ? out->hit + base : nullptr;
            views.push_back(make_view(cams[c0 + c], W, H, (int64_t)c * hw, f));
        }
        st = render_views_impl(ctx, grid, views, (int64_t)nc * hw, max_steps, eps, cfg, s, c0 + per_chunk >= n_cams);
        if (st != KNS_OK) return st;
    }
    ctx->have_stats = true;
    return KNS_OK;
}

kns_status kns_render_views(kns_ctx *ctx, const kns_grid *grid, const kns_view *views, int n_views, int max_steps,
                            float eps, const kns_render_opts *opts, void *cuda_stream) {
    if (!ctx) return KNS_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(ctx->mu);
    if (!grid || (n_views > 0 && !views)) return set_err(ctx, KNS_ERR_INVALID_ARG, "NULL grid or views");
    if (n_views < 0 || n_views > (1 << 16)) return set_err(ctx, KNS_ERR_INVALID_ARG, "n_views out of range");
    if (max_steps < 1) return set_err(ctx, KNS_ERR_INVALID_ARG, "max_steps=%d < 1", max_steps);
    if (!(eps > 0.f) || !std::isfinite(eps)) return set_err(ctx, KNS_ERR_INVALID_ARG, "eps must be > 0 and finite");
    RenderCfg cfg;
    kns_status st = resolve_opts(ctx, opts, eps, cfg, grid->desc.sdf_width);
    if (st != KNS_OK) return st;
    std::vector<kns::ViewDev> dv;
    int64_t rays = 0;
    for (int i = 0; i < n_views; ++i) {
        const kns_view &v = views[i];
        if (v.W < 0 || v.H < 0) return set_err(ctx, KNS_ERR_INVALID_ARG, "view %d: negative size", i);
        const int64_t n = (int64_t)v.W * v.H;
        if (n == 0) continue;
        if (!v.out.rgb || !v.out.depth)
            return set_err(ctx, KNS_ERR_INVALID_ARG, "view %d: rgb and depth buffers are required", i);
        if (v.grid < 0 || v.grid >= grid->n_sub)
            return set_err(ctx, KNS_ERR_INVALID_ARG, "view %d: grid %d of a stack of %d", i, v.grid, grid->n_sub);
        if (rays + n > INT32_MAX) return set_err(ctx, KNS_ERR_INVALID_ARG, "views hold more than 2^31-1 rays");
        dv.push_back(make_view(v.cam, v.W, v.H, rays, v.out, v.grid));
        rays += n;
    }
    if (dv.empty()) return KNS_OK;
    DeviceScope ds(ctx->device);
    cudaStream_t s = (cudaStream_t)cuda_stream;
    begin_stats(ctx, s, rays);
    st = render_views_impl(ctx, grid, dv, rays, max_steps, eps, cfg, s, true);
    if (st != KNS_OK) return st;
    ctx->have_stats = true;
    return KNS_OK;
}

kns_status kns_trace_rays(kns_ctx *ctx, const kns_grid *grid, const float *origins, const float *dirs, int64_t n,
                          int max_steps, float eps, const kns_frame *out, const kns_render_opts *opts,
                          void *cuda_stream) {
    if (!ctx) return KNS_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(ctx->mu);
    if (!grid) return set_err(ctx, KNS_ERR_INVALID_ARG, "NULL grid");
    if (n < 0 || n > INT32_MAX - 4096) return set_err(ctx, KNS_ERR_INVALID_ARG, "n out of range");
    if (n == 0) return KNS_OK;
    if (!origins || !dirs || !out || !out->rgb || !out->depth)
        return set_err(ctx, KNS_ERR_INVALID_ARG, "NULL rays or rgb/depth outputs");
    if (max_steps < 1) return set_err(ctx, KNS_ERR_INVALID_ARG, "max_steps=%d < 1", max_steps);
    if (!(eps > 0.f) || !std::isfinite(eps)) return set_err(ctx, KNS_ERR_INVALID_ARG, "eps must be > 0 and finite");
    RenderCfg cfg;
    kns_status st = resolve_opts(ctx, opts, eps, cfg, grid->desc.sdf_width);
    if (st != KNS_OK) return st;
    DeviceScope ds(ctx->device);
    // one view of rows of 4096 rays; rays past n in the last row are skipped
    const int Wv = (int)std::min<int64_t>(n, 4096), Hv = (int)((n + Wv - 1) / Wv);
    kns_camera cam{};
    std::vector<kns::ViewDev> dv{make_view(cam, Wv, Hv, 0, *out)};
    cudaStream_t s = (cudaStream_t)cuda_stream;
    begin_stats(ctx, s, n);
    st = render_views_impl(ctx, grid, dv, (int64_t)Wv * Hv, max_steps, eps, cfg, s, true, origins, dirs, n);
    if (st != KNS_OK) return st;
    ctx->have_stats = true;
    return KNS_OK;
}

kns_status kns_path_trace(kns_ctx *ctx, const kns_grid *grid, const kns_camera *cams, int n_cams, int W, int H,
                          const kns_pt_opts *pt, int max_steps, float eps, float *rgb_out,
                          const kns_render_opts *opts, void *cuda_stream) {
    if (!ctx) return KNS_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(ctx->mu);
    if (!grid || !pt || (n_cams > 0 && !cams)) return set_err(ctx, KNS_ERR_INVALID_ARG, "NULL grid, opts or cams");
    if (n_cams < 0 || W < 0 || H < 0) return set_err(ctx, KNS_ERR_INVALID_ARG, "negative size");
    if (pt->spp < 1 || pt->max_depth < 1 || pt->max_depth > kns::pt_max_depth())
        return set_err(ctx, KNS_ERR_INVALID_ARG, "need spp >= 1 and 1 <= max_depth <= %d", kns::pt_max_depth());
    if (!(pt->offset >= 0.f) || !std::isfinite(pt->offset))
        return set_err(ctx, KNS_ERR_INVALID_ARG, "offset must be finite and >= 0");
    const int64_t n_pix = (int64_t)n_cams * W * H, n = n_pix * pt->spp;
    if (n == 0) return KNS_OK;
    if (!rgb_out) return set_err(ctx, KNS_ERR_INVALID_ARG, "NULL rgb_out");
    if (n > INT32_MAX - 4096) return set_err(ctx, KNS_ERR_INVALID_ARG, "more than 2^31 - 4097 paths");
    if (max_steps < 1) return set_err(ctx, KNS_ERR_INVALID_ARG, "max_steps=%d < 1", max_steps);
    if (!(eps > 0.f) || !std::isfinite(eps)) return set_err(ctx, KNS_ERR_INVALID_ARG, "eps must be > 0 and finite");
    RenderCfg cfg;
    kns_status st = resolve_opts(ctx, opts, eps, cfg, grid->desc.sdf_width);
    if (st != KNS_OK) return st;
    DeviceScope ds(ctx->device);
    if ((st = ensure_pt_scratch(ctx, n, n_cams)) != KNS_OK) return st;
    PtScratch &p = ctx->ps;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    kns::PtArgs a{};
    a.n_cams = n_cams;
    a.W = W;
    a.H = H;
    a.spp = pt->spp;
    a.max_depth = pt->max_depth;
    a.n_paths = n;
    a.cams = p.cams;
    a.seed = pt->seed;
    a.offset = pt->offset;
    for (int k = 0; k < 3; ++k) {
        a.horizon[k] = pt->horizon[k];
        a.zenith[k] = pt->zenith[k];
        a.bmax[k] = grid->desc.bbox_max[k];
    }
    a.o = p.o;
    a.w = p.w;
    a.beta = p.beta;
    a.L = p.L;
    a.alive = p.alive;
    a.t_rgb = p.rgb;
    a.t_depth = p.depth;
    a.t_normal = p.normal;
    a.t_hit = p.hit;
    a.rgb_out = rgb_out;
    cudaError_t e = cudaMemcpyAsync(p.cams, cams, sizeof(kns_camera) * n_cams, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = kns::pt_primary(a, s);
    if (e != cudaSuccess) return cuda_err(ctx, e, "path-tracing launch");
    // each depth traces every path's ray (finished paths carry a ray that misses the box at once)
    const int Wv = (int)std::min<int64_t>(n, 4096), Hv = (int)((n + Wv - 1) / Wv);
    kns_frame fr{};
    fr.rgb = p.rgb;
    fr.depth = p.depth;
    fr.normal = p.normal;
    fr.hit = p.hit;
    kns_camera cam0{};
    std::vector<kns::ViewDev> dv{make_view(cam0, Wv, Hv, 0, fr)};
    begin_stats(ctx, s, n);
    for (int depth = 0; depth < pt->max_depth; ++depth) {
        st = render_views_impl(ctx, grid, dv, (int64_t)Wv * Hv, max_steps, eps, cfg, s,
                               depth + 1 == pt->max_depth, p.o, p.w, n);
        if (st != KNS_OK) return st;
        if ((e = kns::pt_bounce(a, depth, s)) != cudaSuccess) return cuda_err(ctx, e, "path-tracing launch");
    }
    if ((e = kns::pt_resolve(a, s)) != cudaSuccess) return cuda_err(ctx, e, "path-tracing launch");
    ctx->have_stats = true;
    return KNS_OK;
}

kns_status kns_get_render_stats(kns_ctx *ctx, kns_render_stats *out) {
    if (!ctx) return KNS_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(ctx->mu);
    if (!out) return set_err(ctx, KNS_ERR_INVALID_ARG, "NULL out");
    if (!ctx->have_stats) return set_err(ctx, KNS_ERR_INVALID_ARG, "no render on this context yet");
    DeviceScope ds(ctx->device);
    kns::WaveCtrl hc{};
    cudaError_t e = cudaSuccess;
    if (ctx->ws.ctrl) e = cudaMemcpyAsync(&hc, ctx->ws.ctrl, sizeof(hc), cudaMemcpyDeviceToHost, ctx->stats_stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stats_stream);
    if (e != cudaSuccess) return cuda_err(ctx, e, "render stats");
    kns_render_stats st = ctx->stats;
    st.hits += hc.n_hits;
    st.samples_fp32 += (int64_t)hc.samples_f32;
    st.samples_bf16 += (int64_t)hc.samples_bf16;
    st.samples_tail += (int64_t)hc.samples_tail;
    st.rounds += hc.rounds;  // a persistent BF16 trace counts its rounds on the device
    st.refined += hc.n_refine;
    float *dst[5] = {&st.ms_generate, &st.ms_sort, &st.ms_eval_fp32, &st.ms_eval_bf16, &st.ms_shade};
    for (const auto &m : ctx->ev_marks) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, ctx->ev_pool[m.ev], ctx->ev_pool[m.ev + 1]) == cudaSuccess) *dst[m.cls] += ms;
    }
    st.ms_total = st.ms_generate + st.ms_sort + st.ms_eval_fp32 + st.ms_eval_bf16 + st.ms_shade;
    *out = st;
    return KNS_OK;
}

kns_status kns_measure_peaks(kns_ctx *ctx, void *cuda_stream, kns_peaks *out) {
    if (!ctx) return KNS_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(ctx->mu);
    if (!out) return set_err(ctx, KNS_ERR_INVALID_ARG, "NULL out");
    DeviceScope ds(ctx->device);
    kns_peaks p{};
    p.sm_count = ctx->sm_count;
    cudaError_t e = cudaDeviceGetAttribute(&p.sm_clock_khz, cudaDevAttrClockRate, ctx->device);
    if (e == cudaSuccess) e = kns::measure_peaks(ctx->sm_count, (cudaStream_t)cuda_stream, &p.ffma_flops, &p.mufu_ops);
    if (e != cudaSuccess) return cuda_err(ctx, e, "peak micro-kernels");
    *out = p;
    return KNS_OK;
}

kns_status kns_selftest_timeout(kns_ctx *ctx, int32_t which, void *cuda_stream) {
    if (!ctx) return KNS_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(ctx->mu);
    if (which != 0 && which != 1) return set_err(ctx, KNS_ERR_INVALID_ARG, "which must be 0 or 1");
    DeviceScope ds(ctx->device);
    cudaStream_t s = (cudaStream_t)cuda_stream;
    kns::WaveCtrl *ctrl = nullptr;  // a fresh control block: its barrier words start at zero
    cudaError_t e = cudaMalloc(&ctrl, sizeof(kns::WaveCtrl));
    if (e == cudaSuccess) e = cudaMemsetAsync(ctrl, 0, sizeof(kns::WaveCtrl), s);
    // ~4 ms of polling for the grid barrier, a few ms for the mbarrier's suspending polls
    if (e == cudaSuccess) e = kns::launch_selftest_timeout(ctrl, ctx->d_status, which, which == 0 ? 4096u : 65536u, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFree(ctrl);
    if (e != cudaSuccess) return cuda_err(ctx, e, "wait self-test");
    return KNS_OK;
}

kns_status kns_get_round_trace(kns_ctx *ctx, kns_round_info *out, int32_t max_rounds, int32_t *n_rounds) {
    if (!ctx) return KNS_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(ctx->mu);
    if (!n_rounds || max_rounds < 0 || (max_rounds > 0 && !out))
        return set_err(ctx, KNS_ERR_INVALID_ARG, "NULL n_rounds, or out NULL with max_rounds > 0");
    if (!ctx->have_stats) return set_err(ctx, KNS_ERR_INVALID_ARG, "no render on this context yet");
    DeviceScope ds(ctx->device);
    cudaError_t e = cudaStreamSynchronize(ctx->stats_stream);
    if (e != cudaSuccess) return cuda_err(ctx, e, "round trace");
    kns::WaveCtrl hc{};
    if (ctx->ws.ctrl) e = cudaMemcpy(&hc, ctx->ws.ctrl, sizeof(hc), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_err(ctx, e, "round trace");
    if (hc.rounds > 0) {  // the persistent BF16 trace: its own per-round counts and timer stamps
        const int n = std::min(hc.rounds, kns::kMaxTraceRounds);
        *n_rounds = n;
        auto ms = [](unsigned long long a, unsigned long long b) { return (float)((double)(b - a) * 1e-6); };
        for (int k = 0; k < std::min(n, (int)max_rounds); ++k) {
            const unsigned long long t0 = k == 0 ? hc.start_ns : hc.round_end_ns[k - 1];
            const unsigned long long *ph = hc.round_phase_ns[k];
            out[k] = kns_round_info{hc.round_live[k], ms(t0, ph[2]), 0.f, ms(ph[2], ph[3]), ms(ph[3], hc.round_end_ns[k]),
                                    hc.round_tiles[k]};
        }
        return KNS_OK;
    }
    const int n = (int)ctx->round_live.size();
    // the last rounds' counts were copied to the pinned ring but not read by the render loop
    for (int k = std::max(0, n - 4); k < n; ++k)
        if (ctx->round_live[k] < 0) ctx->round_live[k] = ctx->h_live[2 * (k & 3)];
    *n_rounds = n;
    for (int k = 0; k < std::min(n, (int)max_rounds); ++k) out[k] = kns_round_info{ctx->round_live[k], 0.f, 0.f, 0.f, 0.f, 0};
    for (const auto &m : ctx->ev_marks) {
        if (m.round < 0 || m.round >= std::min(n, (int)max_rounds)) continue;
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, ctx->ev_pool[m.ev], ctx->ev_pool[m.ev + 1]) != cudaSuccess) continue;
        kns_round_info &r = out[m.round];
        if (m.cls == kTSort) r.ms_sort += ms;
        else if (m.cls == kTEvalF32) r.ms_eval_fp32 += ms;
        else if (m.cls == kTEvalBF16) r.ms_eval_bf16 += ms;
    }
    return KNS_OK;
}

kns_status kns_sdf(kns_ctx *ctx, const kns_grid *grid, const float *pts, int64_t n, float *sdf, float *feat,
                   float *grad, void *cuda_stream) {
    if (!ctx) return KNS_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(ctx->mu);
    if (!grid) return set_err(ctx, KNS_ERR_INVALID_ARG, "NULL grid");
    if (n < 0) return set_err(ctx, KNS_ERR_INVALID_ARG, "n < 0");
    if (n == 0) return KNS_OK;
    if (!pts || !sdf) return set_err(ctx, KNS_ERR_INVALID_ARG, "NULL pts or sdf");
    if (n > ((int64_t)1 << 36)) return set_err(ctx, KNS_ERR_INVALID_ARG, "n too large");
    DeviceScope ds(ctx->device);
    cudaError_t e = kns::launch_sdf_f32(grid->shape, grid->view, pts, n, sdf, feat, grad, (cudaStream_t)cuda_stream);
    if (e != cudaSuccess) return cuda_err(ctx, e, "sdf launch");
    return KNS_OK;
}

}  // extern "C"


extern "C" kns_status kns_render_noalloc(kns_ctx *ctx, const kns_grid *grid, const kns_camera *cams, int n_cams,
                                         int W, int H, int max_steps, float eps, const kns_frame *out,
                                         void *cuda_stream) {
    if (!ctx) return KNS_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(ctx->mu);
    if (!grid || !cams || !out) return set_err(ctx, KNS_ERR_INVALID_ARG, "NULL grid, cams or out");
    if (n_cams < 0 || W < 0 || H < 0) return set_err(ctx, KNS_ERR_INVALID_ARG, "negative size");
    if (max_steps < 1) return set_err(ctx, KNS_ERR_INVALID_ARG, "max_steps=%d < 1", max_steps);
    if (!(eps > 0.f) || !std::isfinite(eps)) return set_err(ctx, KNS_ERR_INVALID_ARG, "eps must be > 0 and finite");
    if (!out->rgb || !out->depth) return set_err(ctx, KNS_ERR_INVALID_ARG, "rgb and depth buffers are required");
    const int64_t rays = (int64_t)n_cams * W * H;
    const int NC = grid->desc.N * grid->desc.N * grid->desc.N;
    if (rays > KNS_NOALLOC_MAX_RAYS)
        return set_err(ctx, KNS_ERR_INVALID_ARG, "kns_render_noalloc: %lld rays exceed its scratch limit of %d",
                       (long long)rays, KNS_NOALLOC_MAX_RAYS);
    if (n_cams > KNS_NOALLOC_MAX_CAMS)
        return set_err(ctx, KNS_ERR_INVALID_ARG, "kns_render_noalloc: %d cameras exceed its limit of %d", n_cams,
                       KNS_NOALLOC_MAX_CAMS);
    if (NC > KNS_NOALLOC_MAX_CELLS)
        return set_err(ctx, KNS_ERR_INVALID_ARG, "kns_render_noalloc: %d cells exceed its limit of %d", NC,
                       KNS_NOALLOC_MAX_CELLS);
    if (rays == 0) return KNS_OK;
    DeviceScope ds(ctx->device);
    unsigned char *base = nullptr;
    kns_status st = noalloc_scratch(ctx, &base);
    if (st != KNS_OK) return st;
    unsigned char *p = base;
    auto take = [&](size_t bytes) {
        unsigned char *q = p;
        p += bytes;
        return q;
    };
    kns::WaveArgs a{};
    a.t_ray = (float *)take(kNoAllocRayBuf);
    a.steps_ray = (int *)take(kNoAllocRayBuf);
    a.cell_ray = (int *)take(kNoAllocRayBuf);
    a.q[0] = (int *)take(kNoAllocRayBuf);
    a.q[1] = (int *)take(kNoAllocRayBuf);
    a.qcell[0] = (int *)take(kNoAllocRayBuf);
    a.qcell[1] = (int *)take(kNoAllocRayBuf);
    a.sorted = (int *)take(kNoAllocRayBuf);
    a.hits = (int *)take(kNoAllocRayBuf);
    a.ray_view = (int *)take(kNoAllocRayBuf);
    int *cellbuf = (int *)take(kNoAllocCellBuf);
    kns::ViewDev *d_views = (kns::ViewDev *)take(kNoAllocViewBuf);
    a.ctrl = (kns::WaveCtrl *)take(kNoAllocCtrlBuf);
    a.tiles = (int4 *)take(kNoAllocTileBuf);
    // warp tiles step every ray to its next occupied voxel themselves: nothing goes on the pending
    // lists, which share one buffer pair
    a.pend_r[0] = a.pend_r[1] = (int *)take(kNoAllocRayBuf);
    a.pend_t[0] = a.pend_t[1] = (float *)take(kNoAllocRayBuf);
    a.count[0] = cellbuf;
    a.count[1] = cellbuf + (NC + 1);
    a.fill[0] = cellbuf + 2 * (NC + 1);
    a.fill[1] = cellbuf + 3 * (NC + 1);
    a.off = cellbuf + 4 * (NC + 1);
    a.tile_off = cellbuf + 5 * (NC + 1);
    a.n_views = n_cams;
    a.max_W = W;
    a.max_H = H;
    a.views = d_views;
    a.max_steps = max_steps;
    a.eps = eps;
    a.NC = NC;
    a.nkeys = NC;
    a.btile = kRenderBlockTile;
    a.btile_bf = 128;  // tensor-core tiles: 128 samples
    a.inner_steps = kRenderInnerSteps;
    a.tail_max = kRenderTailRays;
    a.min_active = kRenderMinActive;
    a.static_tiles = kRenderStaticTiles == 1;
    a.status = ctx->d_status;
    a.wt = grid->d_wt;
    a.wt_stride = grid->wt_stride;
    kns::ViewDev hv[KNS_NOALLOC_MAX_CAMS];  // host staging of the view table (no allocation)
    const int64_t hw = (int64_t)W * H;
    for (int c = 0; c < n_cams; ++c) {
        kns_frame f{};
        f.rgb = out->rgb + 3 * c * hw;
        f.depth = out->depth + c * hw;
        f.normal = out->normal ? out->normal + 3 * c * hw : nullptr;
        f.cell = out->cell ? out->cell + c * hw : nullptr;
        f.steps = out->steps ? out->steps + c * hw : nullptr;
        f.hit = out->hit ? out->hit + c * hw : nullptr;
        hv[c] = make_view(cams[c], W, H, c * hw, f);
    }
    cudaStream_t s = (cudaStream_t)cuda_stream;
    // a copy from pageable host memory has read its source when the call returns, so the stack
    // staging array may go out of scope afterwards
    cudaError_t e = cudaMemcpyAsync(d_views, hv, sizeof(kns::ViewDev) * n_cams, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(a.ctrl, 0, sizeof(kns::WaveCtrl), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(cellbuf, 0, sizeof(int) * 4 * (NC + 1), s);
    if (e == cudaSuccess) e = kns::launch_wave_gen(grid->shape, grid->view, a, s);
    const int eval_blocks = ctx->sm_count * kRenderBlocksPerSM, scatter_blocks = ctx->sm_count * 4;
    for (int k = 0; k < max_steps && e == cudaSuccess; ++k) {
        const int cur = k & 1;
        if (k >= 2) {
            e = cudaEventSynchronize(ctx->ev_live[(k - 2) & 3]);
            if (e != cudaSuccess || ctx->h_live[2 * ((k - 2) & 3)] == 0) break;
        }
        e = kns::launch_wave_scan(a, cur, s);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(ctx->h_live + 2 * (k & 3), &a.ctrl->n_live[cur], sizeof(int), cudaMemcpyDeviceToHost,
                                s);
        if (e == cudaSuccess) e = cudaEventRecord(ctx->ev_live[k & 3], s);
        if (e == cudaSuccess) e = kns::launch_wave_scatter(a, cur, scatter_blocks, s);
        if (e == cudaSuccess) e = kns::launch_wave_eval(grid->shape, grid->view, a, cur, eval_blocks, 0, ctx->sm_count, s);
    }
    if (e == cudaSuccess) {
        // the same shading as kns_render (hits sorted by cell, block tiles)
        e = kns::launch_hit_sort(a, kns::shade_hit_tile(grid->desc.sdf_width), ctx->sm_count, s);
        if (e == cudaSuccess) e = kns::launch_shade_block(grid->shape, grid->view, a, ctx->sm_count, s);
    }
    if (e != cudaSuccess) return cuda_err(ctx, e, "render launch");
    return KNS_OK;
}

// ------------------------------------------------------------------ training step
namespace {

kns_status check_train(kns_ctx *ctx, const kns_grid_desc *desc, const float *params, const kns_train_batch *b) {
    if (!desc || !params || !b) return set_err(ctx, KNS_ERR_INVALID_ARG, "NULL descriptor, params or batch");
    kns_status st = check_desc(ctx, *desc);
    if (st != KNS_OK) return st;
    if (desc->sdf_width != 32 || (desc->sdf_hidden != 2 && desc->sdf_hidden != 3) || desc->pe_pos_L != 4 ||
        desc->pe_dir_L != 2 || desc->col_use_x != 0)
        return set_err(ctx, KNS_ERR_UNSUPPORTED,
                       "training supports width 32, 2 or 3 SDF hidden layers, (L, Ld) = (4, 2), no x colour input");
    if (b->n_rays < 0 || b->n_eik < 0) return set_err(ctx, KNS_ERR_INVALID_ARG, "negative ray or point count");
    if (b->n_strat < 2 || b->n_imp < 0 || b->n_strat + b->n_imp > 256)
        return set_err(ctx, KNS_ERR_INVALID_ARG, "need n_strat >= 2, n_imp >= 0, n_strat + n_imp <= 256");
    if (b->n_rays > 0 && (!b->origins || !b->dirs || !b->target ||
                          (!b->t_fixed && (!b->u_strat || (b->n_imp > 0 && !b->u_imp)))))
        return set_err(ctx, KNS_ERR_INVALID_ARG, "NULL ray array");
    if (b->n_eik > 0 && !b->eik_points) return set_err(ctx, KNS_ERR_INVALID_ARG, "NULL eikonal points");
    if (!(b->s > 0.f) || !(b->s_up > 0.f) || !(b->h > 0.f) || !(b->lambda >= 0.f) || !std::isfinite(b->s) ||
        !std::isfinite(b->s_up) || !std::isfinite(b->h) || !std::isfinite(b->lambda))
        return set_err(ctx, KNS_ERR_INVALID_ARG, "need s, s_up, h > 0 and lambda >= 0, all finite");
    const int64_t S = b->n_strat + b->n_imp;
    const int64_t nrec = 6 * (b->n_rays * S + b->n_eik) + b->n_rays * S;
    if (b->n_rays > ((int64_t)1 << 26) || b->n_eik > ((int64_t)1 << 28) || nrec >= ((int64_t)1 << 31))
        return set_err(ctx, KNS_ERR_INVALID_ARG, "batch too large (records must stay below 2^31)");
    return KNS_OK;
}

}  // namespace

extern "C" {

kns_status kns_train_forward(kns_ctx *ctx, const kns_grid_desc *desc, const float *params,
                             const kns_train_batch *batch, float *loss, float *rgb, float *t_samples,
                             uint64_t *token, void *cuda_stream) {
    if (!ctx) return KNS_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(ctx->mu);
    kns_status st = check_train(ctx, desc, params, batch);
    if (st != KNS_OK) return st;
    if (!loss) return set_err(ctx, KNS_ERR_INVALID_ARG, "NULL loss");
    DeviceScope ds(ctx->device);
    const kns_train_batch &b = *batch;
    const int S = b.n_strat + b.n_imp;
    const int NC = desc->N * desc->N * desc->N;
    ctx->ts.pending = false;
    if ((st = ensure_train_scratch(ctx, b.n_rays, S, b.n_strat, b.n_eik, 2 * NC)) != KNS_OK) return st;
    TrainScratch &t = ctx->ts;
    kns::TrainArgs a{};
    a.N = desc->N;
    a.NC = NC;
    a.H = desc->sdf_hidden;
    for (int k = 0; k < 3; ++k) {
        a.bmin[k] = desc->bbox_min[k];
        a.bmax[k] = desc->bbox_max[k];
        a.cscale[k] = (float)desc->N / (desc->bbox_max[k] - desc->bbox_min[k]);
    }
    a.beta = desc->softplus_beta;
    a.inv_beta = 1.f / desc->softplus_beta;
    a.p_sdf = (int)canon_sdf_params(*desc);
    a.p_cell = a.p_sdf + (int)canon_col_params(*desc);
    a.params = params;
    a.B = b.n_rays;
    a.o = b.origins;
    a.w = b.dirs;
    a.target = b.target;
    a.Ns = b.n_strat;
    a.Ni = b.n_imp;
    a.S = S;
    a.u_s = b.u_strat;
    a.u_i = b.u_imp;
    a.M = b.n_eik;
    a.P = b.eik_points;
    a.s = b.s;
    a.s_up = b.s_up;
    a.lambda = b.lambda;
    a.h = b.h;
    a.t = t.t;
    a.valid = t.valid;
    a.d_coarse = t.d_coarse;
    a.d_fd = t.d_fd;
    a.g_fd = t.g_fd;
    a.d_c = t.d_c;
    a.g_dc = t.g_dc;
    a.rgb_c = t.rgb_c;
    a.g_rgb = t.g_rgb;
    a.C = t.C;
    a.acc = t.acc;
    a.loss = loss;
    a.nkeys = NC;  // the coarse sort uses cell keys only
    const size_t kk = (size_t)t.cap_keys + 1;
    a.count = t.keys;
    a.off = t.keys + kk;
    a.fill = t.keys + 2 * kk;
    a.chunk_off = t.keys + 3 * kk;
    a.sorted = t.sorted;
    a.status = ctx->d_status;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    cudaError_t e = cudaSuccess;
    t.timed = b.timing != 0;
    if (t.timed)
        for (int i = 0; i < 16 && e == cudaSuccess; ++i)
            if (!t.ev[i]) e = cudaEventCreate(&t.ev[i]);
    auto mark = [&](int i) {
        if (t.timed && e == cudaSuccess) e = cudaEventRecord(t.ev[i], s);
    };
    if (e == cudaSuccess) e = cudaMemsetAsync(t.d_counts, 0, 4 * sizeof(int), s);
    mark(0);
    if (a.B > 0 && b.t_fixed) {
        a.t = const_cast<float *>(b.t_fixed);  // read only from here on
        if (e == cudaSuccess) e = kns::train_valid(a, s);
    } else if (a.B > 0) {
        if (e == cudaSuccess) e = kns::train_sort(a, kns::TRAIN_COARSE, a.B * a.Ns, ctx->sm_count, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(t.d_counts, a.off + NC, sizeof(int), cudaMemcpyDeviceToDevice, s);
        if (e == cudaSuccess) e = kns::train_coarse_eval(a, ctx->sm_count, s);
        if (e == cudaSuccess) e = kns::train_importance(a, s);
    }
    mark(1);
    a.nkeys = 2 * NC;
    const int64_t nfine = 6 * (a.B * a.S + a.M) + a.B * a.S;
    mark(2);
    if (e == cudaSuccess && nfine > 0) e = kns::train_sort(a, kns::TRAIN_FINE, nfine, ctx->sm_count, s);
    if (e == cudaSuccess && nfine > 0)
        e = cudaMemcpyAsync(t.d_counts + 1, a.off + NC, sizeof(int), cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess && nfine > 0)
        e = cudaMemcpyAsync(t.d_counts + 2, a.off + 2 * NC, sizeof(int), cudaMemcpyDeviceToDevice, s);
    mark(3);
    mark(4);
    if (e == cudaSuccess && nfine > 0) e = kns::train_fd_forward(a, ctx->sm_count, s);
    mark(5);
    mark(6);
    if (e == cudaSuccess && nfine > 0) e = kns::train_centre_forward(a, ctx->sm_count, s);
    mark(7);
    mark(8);
    if (e == cudaSuccess) e = kns::train_loss_forward(a, s);
    mark(9);
    if (e == cudaSuccess && rgb) e = kns::train_rgb_out(a, rgb, s);
    if (e == cudaSuccess && t_samples && a.B > 0)
        e = cudaMemcpyAsync(t_samples, a.t, sizeof(float) * (size_t)a.B * a.S, cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) return cuda_err(ctx, e, "training forward");
    t.args = a;
    t.pending = true;
    t.backward_done = false;
    t.gen += 1;
    if (token) *token = t.gen;
    return KNS_OK;
}

kns_status kns_train_backward(kns_ctx *ctx, uint64_t token, const float *dloss, float *grad, void *cuda_stream) {
    if (!ctx) return KNS_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(ctx->mu);
    TrainScratch &t = ctx->ts;
    if (!t.pending || token != t.gen)
        return set_err(ctx, KNS_ERR_INVALID_ARG, "no pending training forward with this token");
    if (!grad) return set_err(ctx, KNS_ERR_INVALID_ARG, "NULL grad");
    DeviceScope ds(ctx->device);
    kns::TrainArgs a = t.args;
    a.grad = grad;
    a.dloss = dloss;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    cudaError_t e = cudaSuccess;
    auto mark = [&](int i) {
        if (t.timed && e == cudaSuccess) e = cudaEventRecord(t.ev[i], s);
    };
    mark(10);
    e = cudaMemsetAsync(grad, 0, sizeof(float) * (size_t)a.NC * a.p_cell, s);
    if (e == cudaSuccess) e = kns::train_upstream(a, s);
    mark(11);
    mark(12);
    if (e == cudaSuccess) e = kns::train_centre_backward(a, ctx->sm_count, s);
    mark(13);
    mark(14);
    if (e == cudaSuccess) e = kns::train_fd_backward(a, ctx->sm_count, s);
    mark(15);
    t.backward_done = true;
    if (e != cudaSuccess) return cuda_err(ctx, e, "training backward");
    return KNS_OK;
}

kns_status kns_train_get_stats(kns_ctx *ctx, kns_train_stats *out) {
    if (!ctx || !out) return ctx ? set_err(ctx, KNS_ERR_INVALID_ARG, "NULL out") : KNS_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(ctx->mu);
    TrainScratch &t = ctx->ts;
    if (!t.pending) return set_err(ctx, KNS_ERR_INVALID_ARG, "no training forward on this context");
    DeviceScope ds(ctx->device);
    kns_train_stats st{};
    const kns::TrainArgs &a = t.args;
    st.rays = a.B;
    st.samples_per_ray = a.S;
    st.eik_points = a.M;
    int cnt[4] = {0, 0, 0, 0};
    cudaError_t e = cudaMemcpy(cnt, t.d_counts, sizeof(cnt), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_err(ctx, e, "training stats");
    st.records_coarse = cnt[0];
    st.records_fd = cnt[1];
    st.records_centre = cnt[2] - cnt[1];  // off[2 NC] - off[NC]
    if (t.timed) {
        float *dst[8] = {&st.ms_coarse, &st.ms_sort, &st.ms_fd_forward, &st.ms_centre_forward, &st.ms_loss,
                         &st.ms_upstream, &st.ms_centre_backward, &st.ms_fd_backward};
        const int n = t.backward_done ? 8 : 5;
        for (int k = 0; k < n; ++k) {
            if (cudaEventSynchronize(t.ev[2 * k + 1]) != cudaSuccess ||
                cudaEventElapsedTime(dst[k], t.ev[2 * k], t.ev[2 * k + 1]) != cudaSuccess)
                *dst[k] = 0.f;
            st.ms_total += *dst[k];
        }
    }
    *out = st;
    return KNS_OK;
}

kns_status kns_train_step(kns_ctx *ctx, const kns_grid_desc *desc, const float *params, const kns_train_batch *batch,
                          float *loss, float *grad, void *cuda_stream) {
    uint64_t token = 0;
    kns_status st = kns_train_forward(ctx, desc, params, batch, loss, nullptr, nullptr, &token, cuda_stream);
    if (st != KNS_OK) return st;
    if (!grad) return KNS_OK;
    return kns_train_backward(ctx, token, nullptr, grad, cuda_stream);
}

}  // extern "C"
