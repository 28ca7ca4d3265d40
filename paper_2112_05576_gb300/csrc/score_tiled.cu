// Kernel (c), tiled form: exhaustive score map of one pyramid level
// (Sec. II: every pose scored by Eq. (1) over the model points projected by
// Eq. (2), each point taking its best vote over the 3x3 neighbouring-search
// window).
//
// Work decomposition.  A CTA owns a super-tile of translations (SX x SY warp
// tiles) of one image and a group of TG consecutive angles.  One TMA load
// stages the w_hat window that every (angle, pose, point, neighbour) of the
// CTA can touch -- the super-tile grown by the union of the group's rotated
// offset bounding boxes and the 1-pixel search halo -- into shared memory;
// pixels outside the image arrive as zeros, which is exactly Eq. (1)'s
// contribution of a missing edge.  Warps then loop over (angle, warp tile)
// items.
//
// Register blocking.  A thread owns an R x C = 8 x 6 block of poses.  For one
// model point the block's 3x3 windows cover (R+2) x (C+2) pixels; each pixel's
// dot product with the point's direction is computed once (packed FP32x2 FMA
// on a pixel pair) and shared by the up to nine poses whose windows hold it,
// the 3x3 maximum is taken separably with 3-input max, and the result is
// accumulated in FP32 (packed adds).  Per pose-point: ~0.94 shared loads,
// ~1.9 FMA-pipe instructions for the dots, 2.25 max, 0.5 add.
//
// Field layout (pixel pairs).  Pixels 2j, 2j+1 of a row are stored together
// as {wx_2j, wx_2j+1, wy_2j, wy_2j+1}: 16 bytes in FP32, 8 bytes in FP16 or
// BF16 (multiplied by a 16-bit-rounded direction with mixed-precision FMA;
// accumulation stays FP32).  The shared-memory traffic is the kernel's bound (about 15 bytes per
// pose-point in FP32, 7.5 in 16-bit storage), so lanes are laid out to keep
// the loads conflict-free: FP32 uses 128-bit loads with 8 lanes along x, a
// quarter-warp's lanes starting 3 pairs apart (8 distinct 16-byte slots);
// 16-bit storage uses 64-bit loads with 16 lanes along x, a half-warp's lanes
// starting 3 pairs apart (16 distinct 8-byte slots).
//
// Early termination (exact-safe, see kernels_score.cu): every 32 points a warp
// abandons its tile when every pose's partial sum proves M < min_score.

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <mutex>

#include "sam_internal.h"
#include "score_common.cuh"

namespace sam {

// Set (never cleared by the kernels) when a bounded wait for a window's TMA
// copy gives up; read and cleared by the host after a synchronising call.
__device__ int g_score_err;
// Pose-points the tiled scorers actually evaluated (a warp's poses inside the
// map x the points it processed before finishing or pruning), for the
// roofline of the executed work; read and cleared by
// sam_executed_pose_points.
__device__ unsigned long long g_exec_pp;

namespace {

// Device addresses of the flag and the counter on the current device, looked
// up once per device (the kernels receive them as pointers: they are
// compiled in other translation units).
struct DeviceFlags {
    int *err;
    unsigned long long *exec;
};

bool device_flags(DeviceFlags *out) {
    static std::mutex mu;
    static DeviceFlags cache[64];
    static bool have[64] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64)
        return false;
    std::lock_guard<std::mutex> lock(mu);
    if (!have[dev]) {
        void *e = nullptr, *x = nullptr;
        if (cudaGetSymbolAddress(&e, g_score_err) != cudaSuccess || cudaGetSymbolAddress(&x, g_exec_pp) != cudaSuccess)
            return false;
        cache[dev] = DeviceFlags{(int *)e, (unsigned long long *)x};
        have[dev] = true;
    }
    *out = cache[dev];
    return true;
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
    static EncodeTiledFn fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(p);
    });
    return fn;
}

struct Geometry {
    int wtx, wty, xalign, pair_bytes;
};

// Warp tile and TMA geometry of the 8-byte-element pairs layout: FP32 pairs
// are 16 bytes (8 lanes along x, windows start at even pixels), 16-bit pairs
// 8 bytes (16 lanes along x, windows start at multiples of 4 pixels); a
// thread owns kTileRows x tc poses.
Geometry geometry(int precision, int tc) {
    if (precision == SAM_FP32)
        return {kLanesXF32 * tc, (32 / kLanesXF32) * kTileRows, 2, 16};
    // angle codes: scored as FP32 pairs in shared memory, staged as 2-byte
    // codes whose TMA start must be a multiple of 8 pixels
    if (precision == SAM_ANGLE16)
        return {kLanesXF32 * tc, (32 / kLanesXF32) * kTileRows, 8, 16};
    return {kLanesX16 * tc, (32 / kLanesX16) * kTileRows, 4, 8};
}

// Bytes of the staged angle codes of a window (the expanded window is two
// pixels wider than the staged one).
size_t staged_code_bytes(int bxw, int byw) { return (size_t)(bxw - 2) * byw * 2; }

}  // namespace

// Window box for a tiling: the super-tile grown by the largest union of
// rotated offset boxes over any angle group, the 1-pixel search halo, the
// slack of the aligned TMA start and one pixel for odd-start pair loads.
bool tiled_plan(const LevelHost &L, int precision, int sx, int sy, int tg, int tc, int *bxw, int *byw) {
    if (tg < 1 || (tc != 6 && tc != 10))
        return false;
    const Geometry g = geometry(precision, tc);
    int spx = 0, spy = 0;
    for (int k0 = 0; k0 < L.ntheta; k0 += tg) {
        int x0 = 1 << 30, x1 = -(1 << 30), y0 = 1 << 30, y1 = -(1 << 30);
        for (int k = k0; k < std::min(k0 + tg, L.ntheta); ++k) {
            x0 = std::min(x0, L.bbox[k].x);
            x1 = std::max(x1, L.bbox[k].y);
            y0 = std::min(y0, L.bbox[k].z);
            y1 = std::max(y1, L.bbox[k].w);
        }
        spx = std::max(spx, x1 - x0);
        spy = std::max(spy, y1 - y0);
    }
    int bx = sx * g.wtx + spx + 2 + (g.xalign - 1) + 1;
    bx = (bx + g.xalign - 1) / g.xalign * g.xalign;
    const int by = sy * g.wty + spy + 2;
    if (precision == SAM_ANGLE16) {
        // staged: bx codes per row (a multiple of 8, 16-byte TMA rows);
        // expanded: bx + 2 pixels, an odd number of 16-byte pairs per row
        *bxw = bx + 2;
        *byw = by;
        const size_t win = ((size_t)(bx + 2) * by * 8 + 127) & ~(size_t)127;
        const size_t bytes = win + std::max(edge_bitmap_bytes(bx + 2, by), staged_code_bytes(bx + 2, by));
        return bx <= 256 && by <= 256 && bytes <= 200 * 1024;
    }
    // row pitch: an odd number of 16-byte units (FP32 pixel pairs) or twice
    // an odd number of 8-byte units (16-bit pairs), so rows 2 apart fall in
    // other shared-memory banks
    if (g.pair_bytes == 16 ? ((bx / 2) % 2 == 0) : ((bx / 2) % 4 == 0))
        bx += g.xalign;
    *bxw = bx;
    *byw = by;
    const size_t bytes = (((size_t)bx * by * g.pair_bytes / 2 + 15) & ~(size_t)15) + edge_bitmap_bytes(bx, by);
    return bx * g.pair_bytes / 16 <= 256 && by <= 256 && bytes <= 200 * 1024;
}

// Launch over `count` images whose pairs-layout fields start at `field`
// (row pitch wp pixels, a multiple of 4; image stride field_img_px pixels).
size_t drain_queue_bytes(int count, int gw, int gh, int nth) {
    // blocks of every tiling the autotuner tries (super-tiles of up to 3 x 2
    // warp tiles of at most 16 x 4 lanes, angle groups of at most nth)
    const size_t blocks = (size_t)count * (size_t)(2 * nth) * (size_t)(gw / 6 + 49) * (size_t)(gh / 8 + 9);
    const size_t slices = blocks * (kTileRows / kDrainRows);
    return 256 + (slices / 32 + 64) * 16 + slices * 4;
}

cudaError_t launch_score_tiled(const sam_model *m, int level, const void *field, int precision, int wp,
                               size_t field_img_px, int W, int H, int count, int nbhd, int polarity, float min_score,
                               int early, float *map, size_t map_img, const TileConfig &cfg, cudaStream_t st,
                               const PoseWindow *window, const DrainQueue *queue) {
    const LevelHost &L = m->lv[level];
    const PoseWindow pw = window ? *window : PoseWindow{0, 0, W, H, 0, L.ntheta};
    int bxw = 0, byw = 0;
    if (!tiled_plan(L, precision, cfg.sx, cfg.sy, cfg.tg, cfg.tc, &bxw, &byw))
        return cudaErrorInvalidValue;
    EncodeTiledFn enc = encode_fn();
    if (!enc)
        return cudaErrorNotSupported;
    const Geometry g = geometry(precision, cfg.tc);
    DeviceFlags fl;
    if (!device_flags(&fl))
        return cudaErrorUnknown;
    // the field as a 3-D tensor of 8-byte elements: a pixel pair is 2 (FP32)
    // or 1 (16-bit) element(s); angle codes: 2-byte elements, one per pixel,
    // row pitch wp codes, the box two pixels narrower than the expanded window
    CUtensorMap tm;
    const bool codes = precision == SAM_ANGLE16;
    const cuuint64_t dims[3] = {codes ? (cuuint64_t)wp : (cuuint64_t)wp * g.pair_bytes / 16, (cuuint64_t)H,
                                (cuuint64_t)count};
    const cuuint64_t strides[2] = {codes ? (cuuint64_t)wp * 2 : (cuuint64_t)wp * g.pair_bytes / 2,
                                   codes ? (cuuint64_t)field_img_px * 2 : (cuuint64_t)field_img_px * g.pair_bytes / 2};
    const cuuint32_t box[3] = {codes ? (cuuint32_t)(bxw - 2) : (cuuint32_t)(bxw * g.pair_bytes / 16), (cuuint32_t)byw,
                               1};
    const cuuint32_t estr[3] = {1, 1, 1};
    if (enc(&tm, codes ? CU_TENSOR_MAP_DATA_TYPE_UINT16 : CU_TENSOR_MAP_DATA_TYPE_UINT64, 3, const_cast<void *>(field),
            dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
            CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return cudaErrorInvalidValue;
    TiledArgs a;
    a.rot = m->dev[level].rot;
    a.bbox = m->dev[level].bbox;
    a.n = L.n;
    a.nth = L.ntheta;
    a.W = pw.gw;
    a.H = pw.gh;
    a.ox = pw.x0;
    a.oy = pw.y0;
    a.k0 = pw.k0;
    a.nk = pw.nk;
    a.map = map;
    a.map_img = map_img;
    a.sx = cfg.sx;
    a.sy = cfg.sy;
    a.tg = cfg.tg;
    a.tiles_x = (pw.gw + cfg.sx * g.wtx - 1) / (cfg.sx * g.wtx);
    const int tiles_y = (pw.gh + cfg.sy * g.wty - 1) / (cfg.sy * g.wty);
    a.bxw = bxw;
    a.byw = byw;
    a.inv_n = 1.0f / (float)L.n;
    a.thresh = prune_threshold(L.n, min_score, precision);
    a.early = early;
    a.emin = early ? edge_count_threshold(a.thresh, precision) : 0;
    a.err = fl.err;
    a.exec = fl.exec;
    a.tiles_y = tiles_y;
    const int groups = (pw.nk + cfg.tg - 1) / cfg.tg;
    dim3 grid((unsigned)(a.tiles_x * tiles_y), (unsigned)groups, (unsigned)count);
    // persistent form when the bound is on and the storage holds every slice
    a.queue = nullptr;
    a.tasks = nullptr;
    a.qctr = nullptr;
    a.qcap = a.tcap = 0;
    a.units = (int)(grid.x * grid.y * grid.z);
    a.hot_cnt = nullptr;
    a.hot = nullptr;
    a.hot_cap = 0;
    a.hot_thr = 0.f;
    if (queue && queue->base && a.emin > 0 && L.n < 65536) {
        const size_t items = (size_t)cfg.tg * cfg.sx * cfg.sy;
        const size_t rounds = (items + 127) / 128;
        const size_t ch = (size_t)std::min(cfg.warps * 32, kTaskSlices);   // slices per task
        const size_t units = (size_t)a.units;
        const size_t per_item = 32 * (kTileRows / kDrainRows);
        const size_t qcap = units * items * per_item, tcap = units * (items * per_item / ch + rounds);
        const size_t need = 256 + tcap * 16 + qcap * 4;
        if (need <= queue->bytes && qcap < (1u << 31) && tcap < (1u << 31)) {
            char *b = (char *)queue->base;
            a.qctr = (unsigned *)b;
            a.tasks = (int4 *)(b + 256);
            a.queue = (uint32_t *)(b + 256 + tcap * 16);
            a.qcap = (unsigned)qcap;
            a.tcap = (unsigned)tcap;
            // counters and the tasks' publication flags start at zero
            cudaError_t e = cudaMemsetAsync(b, 0, 256 + tcap * 16, st);
            if (e != cudaSuccess)
                return e;
            // the hot list (map indices must fit 32 bits)
            if (queue->hot && queue->hot_cap && map_img <= 0xFFFFFFFFull) {
                a.hot_cnt = a.qctr + kHotCounter;
                a.hot = queue->hot;
                a.hot_cap = queue->hot_cap;
                a.hot_thr = queue->hot_thr;
                if (queue->hot_made)
                    *queue->hot_made = true;
            }
        }
    }
    // the edge bitmaps follow the window; the persistent form reuses their
    // space for the partial sums of split tasks (warps x 32 lanes x slice)
    const size_t red = (size_t)cfg.warps * 32 * kDrainRows * cfg.tc * 4;
    const size_t smem = codes ? (((size_t)bxw * byw * 8 + 127) & ~(size_t)127) +
                                    std::max(std::max(edge_bitmap_bytes(bxw, byw), red), staged_code_bytes(bxw, byw)) +
                                    128
                              : (((size_t)bxw * byw * g.pair_bytes / 2 + 15) & ~(size_t)15) +
                                    std::max(edge_bitmap_bytes(bxw, byw), red) + 128;
    const bool pol = polarity != 0;
    switch (precision) {
    case SAM_FP32:
        return launch_tiled_f32(tm, a, grid, smem, nbhd, pol, cfg.warps, cfg.tc, st);
    case SAM_ANGLE16:
        return launch_tiled_a16(tm, a, grid, smem, nbhd, pol, cfg.warps, cfg.tc, st);
    case SAM_FP16:
        return launch_tiled_f16(tm, a, grid, smem, nbhd, pol, cfg.warps, cfg.tc, st);
    default:
        return launch_tiled_bf16(tm, a, grid, smem, nbhd, pol, cfg.warps, cfg.tc, st);
    }
}

bool level_needs_chunks(const LevelHost &L) {
    int bxw = 0, byw = 0;
    return !tiled_plan(L, SAM_FP32, 1, 1, 1, 6, &bxw, &byw);
}

// Window box of the chunked kernel: CTA tile + largest chunk box + halo +
// aligned-start slack + one pixel for odd-start pair loads.
bool chunked_plan(const LevelHost &L, int precision, int sx, int sy, int *bxw, int *byw) {
    if (L.crot.empty())
        return false;
    const Geometry g = geometry(precision, kChunkCols);
    int bx = sx * g.wtx + L.cspan_x + 2 + (g.xalign - 1) + 1;
    bx = (bx + g.xalign - 1) / g.xalign * g.xalign;
    const int by = sy * g.wty + L.cspan_y + 2;
    *bxw = bx;
    *byw = by;
    const size_t bytes = (size_t)bx * by * g.pair_bytes / 2;
    return bx * g.pair_bytes / 16 <= 256 && by <= 256 && bytes <= 200 * 1024;
}

// The chunked scorer over `count` images (arguments as launch_score_tiled);
// the CTA tile is cfg.sx x cfg.sy warp tiles with cfg.sx * cfg.sy == cfg.warps.
cudaError_t launch_score_chunked(const sam_model *m, int level, const void *field, int precision, int wp,
                                 size_t field_img_px, int W, int H, int count, int nbhd, int polarity,
                                 float min_score, int early, float *map, size_t map_img, const TileConfig &cfg,
                                 cudaStream_t st, const PoseWindow *window) {
    const LevelHost &L = m->lv[level];
    const LevelDev &D = m->dev[level];
    if (cfg.sx * cfg.sy != cfg.warps || (cfg.warps != 4 && cfg.warps != 8) || !D.crot)
        return cudaErrorInvalidValue;
    int bxw = 0, byw = 0;
    if (!chunked_plan(L, precision, cfg.sx, cfg.sy, &bxw, &byw))
        return cudaErrorInvalidValue;
    EncodeTiledFn enc = encode_fn();
    if (!enc)
        return cudaErrorNotSupported;
    const PoseWindow pw = window ? *window : PoseWindow{0, 0, W, H, 0, L.ntheta};
    const Geometry g = geometry(precision, kChunkCols);
    DeviceFlags fl;
    if (!device_flags(&fl))
        return cudaErrorUnknown;
    CUtensorMap tm;
    const cuuint64_t dims[3] = {(cuuint64_t)wp * g.pair_bytes / 16, (cuuint64_t)H, (cuuint64_t)count};
    const cuuint64_t strides[2] = {(cuuint64_t)wp * g.pair_bytes / 2, (cuuint64_t)field_img_px * g.pair_bytes / 2};
    const cuuint32_t box[3] = {(cuuint32_t)(bxw * g.pair_bytes / 16), (cuuint32_t)byw, 1};
    const cuuint32_t estr[3] = {1, 1, 1};
    if (enc(&tm, CU_TENSOR_MAP_DATA_TYPE_UINT64, 3, const_cast<void *>(field), dims, strides, box, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return cudaErrorInvalidValue;
    ChunkArgs a;
    a.rot = D.crot;
    a.cstart = D.cstart;
    a.cbox = D.cbox;
    a.crange = D.crange;
    a.n = L.n;
    a.W = pw.gw;
    a.H = pw.gh;
    a.ox = pw.x0;
    a.oy = pw.y0;
    a.k0 = pw.k0;
    a.map = map;
    a.map_img = map_img;
    a.sx = cfg.sx;
    a.sy = cfg.sy;
    a.tiles_x = (pw.gw + cfg.sx * g.wtx - 1) / (cfg.sx * g.wtx);
    const int tiles_y = (pw.gh + cfg.sy * g.wty - 1) / (cfg.sy * g.wty);
    a.bxw = bxw;
    a.byw = byw;
    a.inv_n = 1.0f / (float)L.n;
    a.thresh = prune_threshold(L.n, min_score, precision);
    a.early = early;
    a.err = fl.err;
    a.exec = fl.exec;
    a.alive = nullptr;
    a.alive_w = 0;
    dim3 grid((unsigned)(a.tiles_x * tiles_y), (unsigned)pw.nk, (unsigned)count);
    const size_t smem = (size_t)bxw * byw * g.pair_bytes / 2 + 128;
    const bool pol = polarity != 0;
    cudaError_t e = cudaSuccess;
    // The edge-presence bound (with early termination): whole-image planes
    // and one alive bit per pose in stream-ordered scratch, freed after the
    // scorer.  Skipped, and every pose scored, when the scratch cannot be had
    // or the stream is being captured.
    void *bound_mem = nullptr;
    const int emin = early ? edge_count_threshold(a.thresh, precision) : 0;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    bool capturing = true;
    if (cudaStreamIsCapturing(st, &cs) == cudaSuccess)
        capturing = cs != cudaStreamCaptureStatusNone;
    else
        (void)cudaGetLastError();   // the query's own error
    const long long bound_tasks = (long long)pw.gh * ((pw.gw + 31) / 32) * pw.nk * count;   // warps, at most
    if (emin > 0 && L.n < 65536 && !capturing && wp % 2 == 0 && field_img_px % 2 == 0 && H + 2 <= 65535 &&
        count * 4 <= 65535 && bound_tasks < 8LL * 0x7fffffffLL &&
        4LL * (H + 2) * ((wp + 2 + 31) / 32) < 0x7fffffffLL) {
        const int nq = pol ? 1 : 4;
        const int ppw = (wp + 2 + 31) / 32;
        const size_t plane_words = (size_t)count * nq * (H + 2) * ppw;
        const int aw = (pw.gw + 31) / 32;
        const size_t alive_words = (size_t)count * pw.nk * pw.gh * aw;
        if (cudaMallocAsync(&bound_mem, (2 * plane_words + alive_words) * 4, st) != cudaSuccess) {
            (void)cudaGetLastError();
            bound_mem = nullptr;
        } else {
            uint32_t *np = static_cast<uint32_t *>(bound_mem);
            ChunkBoundArgs b;
            b.rot = D.crot;
            b.n = L.n;
            b.dplanes = np + plane_words;
            b.H = H;
            b.ppw = ppw;
            b.gx0 = pw.x0;
            b.gy0 = pw.y0;
            b.k0 = pw.k0;
            b.gh = pw.gh;
            b.nk = pw.nk;
            b.count = count;
            b.aw = aw;
            b.lpr = 1;
            while (b.lpr < 32 && b.lpr < aw)
                b.lpr *= 2;
            b.groups = (aw + b.lpr - 1) / b.lpr;
            b.emin = emin;
            b.alive = np + 2 * plane_words;
            switch (precision) {
            case SAM_FP32:
                e = launch_chunk_bound_f32(field, wp, H, field_img_px, pol, np, b, st);
                break;
            case SAM_FP16:
                e = launch_chunk_bound_f16(field, wp, H, field_img_px, pol, np, b, st);
                break;
            default:
                e = launch_chunk_bound_bf16(field, wp, H, field_img_px, pol, np, b, st);
                break;
            }
            a.alive = b.alive;
            a.alive_w = aw;
        }
    }
    if (e == cudaSuccess) {
        switch (precision) {
        case SAM_FP32:
            e = launch_chunked_f32(tm, a, grid, smem, nbhd, pol, cfg.warps, st);
            break;
        case SAM_FP16:
            e = launch_chunked_f16(tm, a, grid, smem, nbhd, pol, cfg.warps, st);
            break;
        default:
            e = launch_chunked_bf16(tm, a, grid, smem, nbhd, pol, cfg.warps, st);
            break;
        }
    }
    if (bound_mem) {
        const cudaError_t fe = cudaFreeAsync(bound_mem, st);
        if (e == cudaSuccess)
            e = fe;
    }
    return e;
}

// 2-D tensor map of one image's pairs-layout field for the persistent kernel
// (written to host memory; the plan copies it to device memory).
bool encode_pair_tmap(void *out, const void *field, int precision, int wp, int H, int bxw, int byw) {
    EncodeTiledFn enc = encode_fn();
    if (!enc)
        return false;
    const Geometry g = geometry(precision, 6);
    const cuuint64_t dims[2] = {(cuuint64_t)wp * g.pair_bytes / 16, (cuuint64_t)H};
    const cuuint64_t strides[1] = {(cuuint64_t)wp * g.pair_bytes / 2};
    const cuuint32_t box[2] = {(cuuint32_t)(bxw * g.pair_bytes / 16), (cuuint32_t)byw};
    const cuuint32_t estr[2] = {1, 1};
    return enc(reinterpret_cast<CUtensorMap *>(out), CU_TENSOR_MAP_DATA_TYPE_UINT64, 2, const_cast<void *>(field), dims,
               strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
               CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

int tiled_warp_tile(int precision, int tc, int *wty) {
    const Geometry g = geometry(precision, tc);
    *wty = g.wty;
    return g.wtx;
}

cudaError_t launch_score_pairs(const PairScore *pairs, int n_pairs, int total_items, int precision, int nbhd,
                               int polarity, int early, const TileConfig &cfg, size_t window_bytes,
                               size_t bitmap_bytes, unsigned *counter, cudaStream_t st) {
    if (total_items <= 0 || n_pairs <= 0)
        return cudaSuccess;
    const size_t smem = ((window_bytes + 15) & ~(size_t)15) + bitmap_bytes + 128;
    const bool pol = polarity != 0;
    DeviceFlags fl;
    if (!device_flags(&fl))
        return cudaErrorUnknown;
    switch (precision) {
    case SAM_FP32:
        return launch_pairs_f32(pairs, n_pairs, total_items, cfg, nbhd, pol, early, smem, window_bytes, counter,
                                fl.err, fl.exec, st);
    case SAM_FP16:
        return launch_pairs_f16(pairs, n_pairs, total_items, cfg, nbhd, pol, early, smem, window_bytes, counter,
                                fl.err, fl.exec, st);
    default:
        return launch_pairs_bf16(pairs, n_pairs, total_items, cfg, nbhd, pol, early, smem, window_bytes, counter,
                                 fl.err, fl.exec, st);
    }
}

cudaError_t score_error_flag_async(int *host, cudaStream_t st) {
    return cudaMemcpyFromSymbolAsync(host, g_score_err, sizeof(int), 0, cudaMemcpyDeviceToHost, st);
}

cudaError_t score_error_clear(cudaStream_t st) {
    static const int zero = 0;
    return cudaMemcpyToSymbolAsync(g_score_err, &zero, sizeof(int), 0, cudaMemcpyHostToDevice, st);
}

}  // namespace sam

extern "C" long long sam_executed_pose_points(int reset) {
    unsigned long long v = 0;
    if (cudaDeviceSynchronize() != cudaSuccess ||
        cudaMemcpyFromSymbol(&v, sam::g_exec_pp, sizeof(v)) != cudaSuccess)
        return -1;
    if (reset) {
        static const unsigned long long zero = 0;
        if (cudaMemcpyToSymbol(sam::g_exec_pp, &zero, sizeof(zero)) != cudaSuccess)
            return -1;
    }
    return (long long)v;
}

namespace {

// One bounded wait that nothing completes (mode 0: the window-copy mbarrier
// wait, 1: the persistent scorer's wait for a task), reported through the
// device error flag.
sam_status selftest_wait(int mode, int limit_us, double *waited_ms) {
    if (limit_us < 1 || limit_us > 1000000)
        return SAM_ERR_ARG;
    sam::DeviceFlags fl;
    if (!sam::device_flags(&fl))
        return SAM_ERR_CUDA;
    unsigned long long *d_ns = nullptr;
    if (cudaMalloc(&d_ns, 64) != cudaSuccess)
        return SAM_ERR_NOMEM;
    unsigned *fake = reinterpret_cast<unsigned *>(reinterpret_cast<char *>(d_ns) + 16);   // task + 5 counters
    sam_status s = SAM_OK;
    unsigned long long ns = 0;
    int flag = 0;
    if (cudaMemset(d_ns, 0, 64) != cudaSuccess ||
        sam::launch_wait_selftest(fl.err, (unsigned long long)limit_us * 1000ull, d_ns, mode, fake, 0) !=
            cudaSuccess ||
        cudaDeviceSynchronize() != cudaSuccess ||
        cudaMemcpy(&ns, d_ns, sizeof(ns), cudaMemcpyDeviceToHost) != cudaSuccess ||
        cudaMemcpy(&flag, fl.err, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
        s = SAM_ERR_CUDA;
    cudaFree(d_ns);
    if (s != SAM_OK)
        return s;
    if (waited_ms)
        *waited_ms = (double)ns * 1e-6;
    if (flag) {
        static const int zero = 0;
        if (cudaMemcpy(fl.err, &zero, sizeof(int), cudaMemcpyHostToDevice) != cudaSuccess)
            return SAM_ERR_CUDA;
        return SAM_ERR_TIMEOUT;
    }
    return SAM_OK;
}

}  // namespace

extern "C" sam_status sam_selftest_wait_timeout(int limit_us, double *waited_ms) {
    return selftest_wait(0, limit_us, waited_ms);
}

extern "C" sam_status sam_selftest_task_wait_timeout(int limit_us, double *waited_ms) {
    return selftest_wait(1, limit_us, waited_ms);
}

extern "C" int sam_take_device_error(void) {
    if (cudaDeviceSynchronize() != cudaSuccess)
        return 1;
    int flag = 0;
    if (cudaMemcpyFromSymbol(&flag, sam::g_score_err, sizeof(int)) != cudaSuccess)
        return 1;
    if (flag) {
        static const int zero = 0;
        cudaMemcpyToSymbol(sam::g_score_err, &zero, sizeof(int));
    }
    return flag != 0;
}
