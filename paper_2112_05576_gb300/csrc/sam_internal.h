// Internal declarations shared by the library's translation units.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "../../include/sam.h"

namespace sam {

constexpr int kMaxLevels = 8;
constexpr int kMaxTopK = 1024;

// One rotated model point in device tables: integer offset (ox, oy) of
// Eq. (2) stored as int bits in x/y, unit direction (px, py) in z/w.
struct RotPt {
    int ox, oy;
    float px, py;
};

// Host-side description of one model level.
struct LevelHost {
    int tw = 0, th = 0;              // template size at this level
    int n = 0;                       // edge points
    int ntheta = 0;                  // tables at this level: scales x angles (rigid model: angles)
    int nangles = 0;                 // angles per scale (table K = j * nangles + k for scale j, angle k)
    double dtheta = 0.0;             // angle step (deg)
    std::vector<int32_t> tx, ty, gx, gy;
    std::vector<RotPt> rot;          // [ntheta][n]
    std::vector<int4> bbox;          // [ntheta] (oxmin, oxmax, oymin, oymax)
    std::vector<int2> shift;         // [ntheta] child shift to level-1 (empty at level 0)
    // Chunked tables, built for levels whose rotated extent is too large for
    // one staged window: per angle the rotated points regrouped by
    // kChunkCell x kChunkCell cell of their offset (crot [ntheta][n], cells
    // in (cy, cx) order); chunk c of angle k is points crange[c] of that
    // angle's list with offset box cbox[c]; angle k owns chunks
    // cstart[k] .. cstart[k+1] - 1.
    std::vector<RotPt> crot;
    std::vector<int> cstart;
    std::vector<int4> cbox;
    std::vector<int2> crange;
    int cspan_x = 0, cspan_y = 0;    // largest chunk box extent (max - min)
};

constexpr int kChunkCell = 16;

// Device copy of one level's tables.
struct LevelDev {
    int tw, th, n, ntheta;
    int nangles;          // angles per scale (ntheta = scales x nangles)
    const RotPt *rot;
    const int4 *bbox;
    const int2 *shift;
    const float4 *base;   // [n] unrotated (tx, ty, gx/|g|, gy/|g|) for the continuous-pose score
    // chunked tables (null when the level has none)
    const RotPt *crot;
    const int *cstart;
    const int4 *cbox;
    const int2 *crange;
    int cspan_x, cspan_y;
};

struct Workspace {
    void *base = nullptr;
    size_t bytes = 0;
    int device = -1;
};

}  // namespace sam

namespace sam {

// Geometry shared by the tiled scorers: a thread owns kTileRows x cols poses
// (cols 6 or 10); FP32 pairs put kLanesXF32 lanes along x, 16-bit pairs
// kLanesX16; the chunked kernel uses kChunkCols columns.
constexpr int kTileRows = 8;
constexpr int kLanesXF32 = 8;
constexpr int kLanesX16 = 16;
constexpr int kChunkCols = 6;
// Pose rows each lane scores of a block that survives the edge-presence
// bound (kTileRows / kDrainRows lanes share the block).
constexpr int kDrainRows = 2;
// Most surviving slices in one task of the persistent scorer (a task that
// fills fewer warps than the CTA has is split over the idle warps by points).
#ifndef SAM_TASK_SLICES
#define SAM_TASK_SLICES 32
#endif
constexpr int kTaskSlices = SAM_TASK_SLICES;

struct TileConfig {
    int sx = 2, sy = 1;   // super-tile in warp tiles (8 x tc lanes-along-x poses wide, 32 rows tall for FP32)
    int tg = 9;           // angles per CTA (0: the chunked kernel)
    int warps = 8;        // warps per CTA (4 or 8)
    int tc = 6;           // pose columns per thread (6 or 10)
};

}  // namespace sam

namespace sam {
// A captured detection pipeline (sam_detect / sam_detect_batch on device
// buffers): replayed while the call's shape, parameters, workspace and
// scorer tiling are unchanged.
struct GraphCache {
    bool valid = false;
    int w = 0, h = 0, count = 0, device = -1;
    sam_detect_params p{};
    unsigned epoch = 0;
    void *ws_base = nullptr;
    size_t ws_bytes = 0;
    cudaGraphExec_t exec = nullptr;
    cudaStream_t cap = nullptr;   // private stream the pipeline is captured on
    long long kernels = 0;
};
}  // namespace sam

struct sam_model {
    sam_model_params p;
    int levels = 0;
    int ntheta0 = 0;
    // scale grid of a scaled model (sam_create_model_scaled): s_j = scale_min
    // + j scale_step, j < nscales; a rigid model has one scale of 1
    int nscales = 1;
    double scale_min = 1.0, scale_step = 0.0;
    std::vector<sam::LevelHost> lv;
    // device state (uploaded on first use)
    int device = -1;
    void *d_tables = nullptr;
    sam::LevelDev dev[sam::kMaxLevels];
    sam::Workspace ws;
    // tiling chosen by sam_autotune for this model, per field precision and
    // batch class (0: one image per call, 1: several), overriding the default
    bool tuned[3][2] = {};
    sam::TileConfig tile[3][2];
    sam::GraphCache gc;
    // orientation-bin tables of the quantised form, per (level, bins,
    // polarity): device uint8 [ntheta][n], built on first use
    struct QuantBins {
        int level, nbins;
        uint8_t *dev;
    };
    std::vector<QuantBins> qbins;
};

namespace sam {

// ---- accounting: every kernel launch of the library calls this ----
void count_launches(int n);

// ---- host model builder (model.cpp) ----
sam_status build_model(const uint8_t *tmpl, int w, int h, int stride, const sam_model_params &p, sam_model *m,
                       int nscales = 1, double scale_min = 1.0, double scale_step = 0.0);
sam_status upload_model(sam_model *m);

// ---- kernels (launchers return cudaGetLastError()) ----
// One image of a job list (images of different sizes in one launch): the
// source level and its destination (next pyramid level, or a field).
struct ImageJob {
    const uint8_t *src;
    int w, h, src_stride;
    int dst_stride;   // pyramid jobs: destination row pitch (bytes)
    void *dst;
    int vec;          // 1 when every pointer and pitch allows 128-bit access
    int pad;
};
cudaError_t launch_pyramid_jobs(const ImageJob *jobs, int n_jobs, int max_w, int max_h, cudaStream_t st);
cudaError_t launch_gradient_jobs(const ImageJob *jobs, int n_jobs, int max_w, int max_h, int low, int precision,
                                 int layout, cudaStream_t st);

// (b) pyramid step; `count` images, image i at src + i*src_img / dst + i*dst_img
cudaError_t launch_pyramid_down(const uint8_t *src, int w, int h, int src_stride, size_t src_img, uint8_t *dst,
                                int dst_stride, size_t dst_img, int count, cudaStream_t st);
// Refinement-level gradients on demand (kernels_image.cu): after candidate
// extraction, the FP32 pixel-layout tiles (gradient_tile_w() x
// gradient_tile_h() pixels) of levels 0 .. nlev - 1 that the refinement of
// some candidate can read are marked and listed, then computed; the others
// are left unwritten.  reach[l] = (xlo, xhi, ylo, yhi): level-l pixel
// offsets, relative to 2^(top - l) times a candidate's top-level position,
// that bound what its refinement reads.
struct TileMarks {
    const int32_t *kyx;        // candidates (k, y, x), K per image
    const int *count;          // candidates per image
    int K, count_images;
    int top, step_x, step_y, nlev;
    int w[kMaxLevels], h[kMaxLevels], tiles_x[kMaxLevels], tiles_y[kMaxLevels];
    size_t tile_base[kMaxLevels];   // first mask bit of level l (image-major)
    int4 reach[kMaxLevels];
    uint32_t *mask;            // one bit per tile; mask, then the list counter, are cleared together
    unsigned *list_cnt;
    uint2 *list;               // {level << 24 | image, ty << 16 | tx}
    unsigned list_cap;         // every tile of every level: cannot overflow
};
struct GradTiles {
    const uint8_t *img[kMaxLevels];
    int w[kMaxLevels], h[kMaxLevels], pitch[kMaxLevels];
    size_t img_bytes[kMaxLevels];
    float2 *field[kMaxLevels];
    size_t field_px[kMaxLevels];
    int low, vec;
    const unsigned *list_cnt;
    const uint2 *list;
    unsigned list_cap;
};
int gradient_tile_w();
int gradient_tile_h();
// Clears clear_bytes at marks.mask (the mask and the counter after it),
// marks, and computes the listed tiles.
cudaError_t launch_refine_fields(const TileMarks &marks, const GradTiles &g, size_t clear_bytes, cudaStream_t st);
// Levels 1 .. D of `count` images in one launch (D <= 6; deeper pyramids take
// one launch per level): dst[l], dst_stride[l], dst_img[l] for l = 1 .. D.
cudaError_t launch_pyramid_levels(const uint8_t *src, int w, int h, int src_stride, size_t src_img, int D,
                                  uint8_t *const *dst, const int *dst_stride, const size_t *dst_img, int count,
                                  cudaStream_t st);
// (a) gradient / threshold / normalise; field image i at field + i*field_img_px pixels
cudaError_t launch_gradient(const uint8_t *img, int w, int h, int stride, size_t img_bytes, int low, int precision,
                            int layout, void *field, size_t field_img_px, int16_t *gx, int16_t *gy, int count,
                            cudaStream_t st);
// Field layouts: SAM_LAYOUT_PIXEL rows of w (wx, wy) pairs; SAM_LAYOUT_PAIRS
// rows of pixel pairs {wx0, wx1, wy0, wy1}, row pitch w rounded up to a
// multiple of 4 pixels (16-byte rows in every precision), padding pixels zero.
__host__ __device__ inline int field_pitch(int w, int layout) {
    return layout == SAM_LAYOUT_PAIRS ? ((w + 3) & ~3) : w;
}
// Angle-code fields (SAM_ANGLE16): one 16-bit code per pixel, row pitch w, or
// w rounded up to a multiple of 8 codes (16-byte rows, the TMA-read layout).
__host__ __device__ inline int code_pitch(int w, int layout) {
    return layout == SAM_LAYOUT_PAIRS ? ((w + 7) & ~7) : w;
}
// Row pitch of a field of any precision, in pixels.
__host__ __device__ inline int any_field_pitch(int w, int layout, int precision) {
    return precision == SAM_ANGLE16 ? code_pitch(w, layout) : field_pitch(w, layout);
}

// (c) exhaustive score map of one level for `count` fields
struct ScoreArgs {
    const void *field;
    size_t field_img_px;
    int w, h;
    int precision;
    int layout;
    int step_x, step_y;
    int nbhd;
    int polarity;
    float min_score;
    int early;
    float *map;
    size_t map_img;   // floats per image
    int count;
    void *queue = nullptr;     // persistent-form storage of the tiled scorer (optional)
    size_t queue_bytes = 0;
    uint2 *hot = nullptr;      // hot list of the persistent form (optional; see TiledArgs)
    unsigned hot_cap = 0;
    float hot_thr = 0.f;
    bool *hot_made = nullptr;  // set true when the scorer fills the hot list
};
cudaError_t launch_score_map_generic(const LevelDev &L, const ScoreArgs &a, cudaStream_t st);

// Tiled scorer (score_tiled.cu): FP32 paired field, step 1.
bool tiled_plan(const LevelHost &L, int precision, int sx, int sy, int tg, int tc, int *bxw, int *byw);
// Whether a level's rotated extent needs the chunked scorer (its whole-angle
// window does not fit shared memory at the smallest tiling).
bool level_needs_chunks(const LevelHost &L);
// Chunked scorer window box for a CTA tile of sx x sy warp tiles.
bool chunked_plan(const LevelHost &L, int precision, int sx, int sy, int *bxw, int *byw);

// A window of the pose space: translations x0 .. x0 + gw - 1, y0 .. y0 + gh - 1
// (step 1) and angles k0 .. k0 + nk - 1; its map is [nk][gh][gw].
struct PoseWindow {
    int x0, y0, gw, gh, k0, nk;
};

// Stage timing (api.cu): events around a stage when sam_profile_enable is on.
void prof_begin(int stage, cudaStream_t st);
void prof_end(int stage, cudaStream_t st);
constexpr int kStageScoreBound = 6;   // the tiled scorer's launch (inside stage 2)

// Device storage of the persistent form (a slice of the caller's workspace).
struct DrainQueue {
    void *base;    // 256-byte aligned
    size_t bytes;
    uint2 *hot = nullptr;        // hot-list entries (optional; see TiledArgs)
    unsigned hot_cap = 0;
    float hot_thr = 0.f;
    bool *hot_made = nullptr;    // set true when the launch fills the hot list
};
// Index of the hot-list counter among the persistent form's counters (the
// one after it counts the 16-bit candidate filter's pass list; both are
// zeroed with the others before every launch).
constexpr int kHotCounter = 8;
// Workspace bytes that cover the persistent form of every tiling the
// autotuner tries for a gw x gh map with nth angles over `count` images.
size_t drain_queue_bytes(int count, int gw, int gh, int nth);

// The tiled scorer; with `queue` (and early termination) in the persistent
// form, else one CTA per work unit.
cudaError_t launch_score_tiled(const sam_model *m, int level, const void *field, int precision, int wp,
                               size_t field_img_px, int W, int H, int count, int nbhd, int polarity, float min_score,
                               int early, float *map, size_t map_img, const TileConfig &cfg, cudaStream_t st,
                               const PoseWindow *window = nullptr, const DrainQueue *queue = nullptr);

// Kernel arguments of the single-level tiled scorer (score_tiled_kernels.cuh).
struct TiledArgs {
    const RotPt *rot;     // [nth][n]
    const int4 *bbox;     // [nth]
    int n, nth;
    int W, H;             // map size in poses (step 1): the pose window
    int ox, oy;           // pose of map element (0, 0)
    int k0, nk;           // angles k0 .. k0 + nk - 1 (map plane k - k0)
    float *map;
    size_t map_img;
    int sx, sy, tg;       // super-tile in warp tiles, angles per group
    int tiles_x;          // super-tiles along x
    int bxw, byw;         // window box (pixels, rows)
    float inv_n;
    float thresh;
    int early;
    int emin;                   // edge-presence bound: fewest edge windows a surviving pose needs
    int *err;                   // device error flag (bounded waits)
    unsigned long long *exec;   // executed pose-point counter
    int tiles_y;                // super-tiles along y
    // Persistent form (queue non-null, bound on): a unit's bound pass
    // appends its surviving slices to `queue` and one task per CTA-sized
    // batch of them to `tasks`; CTAs score the tasks once the units are out.
    uint32_t *queue;            // (item << 7) | (slice << 5) | lane, one contiguous run per CTA round
    int4 *tasks;                // {unit, first entry, entries, published flag}
    unsigned *qctr;             // [0] entries, [1] tasks, [2] next task, [3] next unit, [4] units done
    unsigned qcap, tcap;        // capacities (entries, tasks)
    int units;                  // work units (super-tile x angle group x image)
    // Hot list (persistent form only; hot_cnt null: none): every pose the
    // drain stores with a score >= hot_thr, as {image, map index}; the
    // counter is qctr[8] (zeroed with the other counters).  A count above
    // hot_cap means the list overflowed (entries past it are not written).
    unsigned *hot_cnt;
    uint2 *hot;
    unsigned hot_cap;
    float hot_thr;
};


// Kernel arguments of the chunked scorer.
struct ChunkArgs {
    const RotPt *rot;      // chunk-ordered points [nth][n]
    const int *cstart;     // [nth + 1]
    const int4 *cbox;      // per chunk (oxmin, oxmax, oymin, oymax)
    const int2 *crange;    // per chunk [p0, p1) within the angle's points
    int n;
    int W, H, ox, oy, k0;  // map window (as TiledArgs)
    float *map;
    size_t map_img;
    int sx, sy;            // CTA tile in warp tiles, sx * sy == warps
    int tiles_x;
    int bxw, byw;
    float inv_n, thresh;
    int early;
    int *err;
    unsigned long long *exec;
    const uint32_t *alive; // edge-presence bound: one bit per pose [count][nk][H][alive_w] (null: none)
    int alive_w;
};

// The chunked form's edge-presence bound (score_tiled_kernels.cuh,
// chunk_bound_kernel).
struct ChunkBoundArgs {
    const RotPt *rot;        // points [nth][n] (any order within an angle)
    int n;
    const uint32_t *dplanes; // dilated planes [count][4 or 1][H + 2][ppw]
    int H, ppw;              // field rows; words per plane row
    int gx0, gy0, k0;        // pose window origin (level pixels) and first angle
    int gh, nk, count;
    int aw;                  // alive words per pose row: (gw + 31) / 32
    int lpr;                 // lanes per pose row (32, 16, 8, 4, 2 or 1; >= aw or 32)
    int groups;              // word groups of lpr words per pose row
    int emin;
    uint32_t *alive;         // [count][nk][gh][aw]
};

struct PairScore;
// Per-field-type instantiations (score_tiled_f32.cu, _f16.cu, _bf16.cu).
#define SAM_TILED_LAUNCHERS(suf)                                                                                    \
    cudaError_t launch_tiled_##suf(const CUtensorMap &tm, const TiledArgs &a, dim3 grid, size_t smem, int nbhd,     \
                                   bool pol, int warps, int tc, cudaStream_t st);                                   \
    cudaError_t launch_chunked_##suf(const CUtensorMap &tm, const ChunkArgs &a, dim3 grid, size_t smem, int nbhd,   \
                                     bool pol, int warps, cudaStream_t st);                                         \
    cudaError_t launch_chunk_bound_##suf(const void *field, int wp, int H, size_t img_px, bool pol,                \
                                         uint32_t *nplanes, const ChunkBoundArgs &b, cudaStream_t st);              \
    cudaError_t launch_pairs_##suf(const PairScore *pairs, int n_pairs, int total, const TileConfig &cfg, int nbhd, \
                                   bool pol, int early, size_t smem, size_t win_bytes, unsigned *counter, int *err, \
                                   unsigned long long *exec, cudaStream_t st);
cudaError_t launch_wait_selftest(int *err, unsigned long long limit_ns, unsigned long long *waited_ns, int mode,
                                 unsigned *fake, cudaStream_t st);
SAM_TILED_LAUNCHERS(f32)
SAM_TILED_LAUNCHERS(f16)
SAM_TILED_LAUNCHERS(bf16)
#undef SAM_TILED_LAUNCHERS
// Angle-code fields (score_tiled_a16.cu): the single-level tiled scorer and
// its persistent form only.
cudaError_t launch_tiled_a16(const CUtensorMap &tm, const TiledArgs &a, dim3 grid, size_t smem, int nbhd, bool pol,
                             int warps, int tc, cudaStream_t st);

// Chunked tiled scorer for levels with chunk tables (score_tiled.cu).
cudaError_t launch_score_chunked(const sam_model *m, int level, const void *field, int precision, int wp,
                                 size_t field_img_px, int W, int H, int count, int nbhd, int polarity,
                                 float min_score, int early, float *map, size_t map_img, const TileConfig &cfg,
                                 cudaStream_t st, const PoseWindow *window = nullptr);

// Persistent tiled scorer over many (image, model) pairs (score_tiled.cu).
struct PairScore {
    const void *tmap;   // the pair's 2-D CUtensorMap in device memory (64-byte aligned)
    const RotPt *rot;   // the model's top-level tables
    const int4 *bbox;
    float *map;         // the pair's map [nth][H][W]
    int n, nth, W, H;
    int tiles_x, tiles; // super-tiles along x, in total
    int bxw, byw;       // the pair's window box
    float inv_n, thresh;
    int item_begin;     // first work unit of this pair (units: tiles x angle groups)
    int emin;           // edge-presence bound (as TiledArgs::emin)
    int job;            // the pair's index in caller order (its hot-list entries' first word)
    unsigned *hot_cnt;  // the batch's hot list (null: none; see TiledArgs)
    uint2 *hot;
    unsigned hot_cap;
    float hot_thr;
};
bool encode_pair_tmap(void *out, const void *field, int precision, int wp, int H, int bxw, int byw);
int tiled_warp_tile(int precision, int tc, int *wty);
cudaError_t launch_score_pairs(const PairScore *pairs, int n_pairs, int total_items, int precision, int nbhd,
                               int polarity, int early, const TileConfig &cfg, size_t window_bytes,
                               size_t bitmap_bytes, unsigned *counter, cudaStream_t st);
// Shared memory of the edge bitmaps the tiled scorers build over a window of
// bxw x byw pixels (edge pixels and their 3x3 dilation, one bit per pixel,
// rows padded by 3 words for the funnel shifts of the bound pass).
// Words per bitmap row: the window's pixels, 3 words of slack for the
// four-word loads of a row segment, rounded to an odd count so that rows
// read by consecutive lanes fall in distinct shared-memory banks.
__host__ __device__ inline int edge_bitmap_words(int bxw) { return ((bxw + 31) / 32 + 3) | 1; }
// 4 planes of edge pixels by the quadrants they can serve and their 4 dilated
// copies (score_tiled_kernels.cuh, build_edge_bits).
__host__ __device__ inline size_t edge_bitmap_bytes(int bxw, int byw) { return 8 * (size_t)byw * edge_bitmap_words(bxw) * 4; }

// Score-kernel selection (process-wide; sam_set_score_kernel).
struct ScoreChoice {
    int kernel = 0;   // 0 automatic, 1 generic, 2 tiled
    TileConfig cfg;
};
ScoreChoice &score_choice();
// Device error flag of the tiled scorer (score_tiled.cu).
cudaError_t score_error_flag_async(int *host, cudaStream_t st);
cudaError_t score_error_clear(cudaStream_t st);
// Dispatch: tiled when allowed and possible, else generic.  `err` may be
// null (then the tiled kernel reports into a library-owned flag).
cudaError_t launch_score_map(const sam_model *m, int level, const ScoreArgs &a, int *err, cudaStream_t st);

// FP32 rescoring of a map computed from a 16-bit field (rescore.cu): poses
// within the storage-error bound of min_score get their FP32 score, all
// others -inf.  scratch: rescore_scratch_bytes(poses_cap).
float rescore_delta(int precision);
size_t rescore_scratch_bytes(size_t poses);
cudaError_t launch_rescore(const LevelDev &L, const float2 *field32, size_t field_img_px, int w, int h, int step_x,
                           int step_y, int count, int nbhd, int polarity, float min_score, int precision, float *map,
                           size_t map_img, void *scratch, size_t poses_cap, cudaStream_t st,
                           const PoseWindow *window = nullptr);
// Candidates of a map scored from a 16-bit field, from its scorer's hot list
// (threshold min_score - delta, capacity every pose): the poses whose 16-bit
// score is within 2 delta of every neighbour's are listed (pass_cnt, zeroed
// before the launch; pass_list, room for every hot entry), then rescored in
// FP32 with their whole neighbourhood (field32: the level's FP32
// pixel-layout field) and kept if they are strict local maxima of the FP32
// scores.
cudaError_t launch_candidates_hot16(const float *map, size_t map_img, int nth, int gh, int gw, float min_score,
                                    float delta, int K, int32_t *out_kyx, float *out_s, int *count, void *scratch,
                                    int n_img, const unsigned *hot_cnt, const uint2 *hot, unsigned hot_cap,
                                    const float2 *field32, size_t field_img_px, int w, int h, const LevelDev &L,
                                    int nbhd, int polarity, unsigned *pass_cnt, unsigned *pass_list,
                                    cudaStream_t st, int ns = 1);

// (d) candidates: local maxima + top-K per image
struct Cand {
    float s;
    uint32_t pad;
    unsigned long long key;   // (k * gh + y) * gw + x
};
// nth: planes of the map (scales x angles); ns: scales (1 for a rigid map).
// A candidate's key is its map index (plane * gh + y) * gw + x.
size_t candidates_scratch_bytes(int nth, int gh, int gw, int ns = 1);
size_t candidates_scratch_bytes_batch(int nth, int gh, int gw, int n_img, int ns = 1);
cudaError_t launch_candidates(const float *map, size_t map_img, int nth, int gh, int gw, float min_score, int K,
                              int32_t *out_kyx, float *out_s, int *count, void *scratch, size_t scratch_img,
                              int n_img, cudaStream_t st, int ns = 1);
// The same from a scorer's hot list (hot_cnt, hot, hot_cap; the list's
// threshold at most min_score): the listed poses only, or every map if the
// list overflowed.
cudaError_t launch_candidates_hot(const float *map, size_t map_img, int nth, int gh, int gw, float min_score, int K,
                                  int32_t *out_kyx, float *out_s, int *count, void *scratch, int n_img,
                                  const unsigned *hot_cnt, const uint2 *hot, unsigned hot_cap, cudaStream_t st,
                                  int ns = 1);

// (d) refinement down the pyramid + NMS
struct RefineArgs {
    const float2 *field[kMaxLevels];   // FP32 fields per level, image 0
    size_t field_img_px[kMaxLevels];   // pixels per image per level
    int w[kMaxLevels], h[kMaxLevels];
    int top;                           // top level index (levels-1)
    int step_x, step_y;
    int nbhd, polarity;
    float min_score;
    int K;
    const int32_t *cand_kyx;           // per image: 3*K
    const float *cand_s;               // per image: K
    const int *cand_count;             // per image
    float4 *refined;                   // per image: K (x, y, k, score) level 0
    int count;
    int nscales;                       // scale grid size (1: rigid); k above is the table index
};
cudaError_t launch_refine(const sam_model *m, const RefineArgs &a, cudaStream_t st);

struct NmsArgs {
    const float4 *refined;   // per image K
    const int *cand_count;
    int K;
    int w0, h0;
    int min_side;
    int max_out;
    double angle_step;
    int nang0;               // angles per scale at level 0 (table k = scale * nang0 + angle)
    sam_pose *out;           // per image max_out
    int *n_out;              // per image
    int count;
};
cudaError_t launch_nms(const NmsArgs &a, cudaStream_t st);

// ---- job lists (batches of different sizes and models; device arrays) ----
struct CandJob {
    const float *map;
    int nth, gh, gw;   // planes (scales x angles), rows, columns
    int ns;            // scales (planes j * nth / ns .. : one scale)
    Cand *cand;
    size_t cap;
    int *cnt;          // zeroed before the launch
    int32_t *out_kyx;  // 3*K
    float *out_s;      // K
    int *out_count;
};
// FP32 rescoring of one (image, model) pair's 16-bit map (job-list form).
struct RescoreJob {
    const float2 *field;   // FP32 pixel-layout field of the scored level (pitch w)
    const RotPt *rot;      // the model level's rotated points [nth][n]
    float *map;            // [nth][h][w]
    unsigned *list;        // 2 x cap entries
    unsigned *count;       // zeroed before the launch
    int w, h, n, nth;
    unsigned cap;
};
cudaError_t launch_rescore_jobs(const RescoreJob *jobs, int n_jobs, size_t max_map, int nbhd, int polarity,
                                float min_score, int precision, cudaStream_t st);
// Candidates of a job list from the pairs scorer's hot list (entries {pair,
// map index}): FP32 maps (the list's threshold min_score; a list that
// overflowed sends every map through the full scan), and 16-bit maps decided
// in FP32 as launch_candidates_hot16 does (the list holds every pose at or
// above min_score - delta; the pair's FP32 field and points from rjobs).
cudaError_t launch_candidates_hot_jobs(const CandJob *jobs, int n_jobs, float min_score, int K,
                                       const unsigned *hot_cnt, const uint2 *hot, unsigned hot_cap,
                                       cudaStream_t st);
cudaError_t launch_candidates_hot16_jobs(const CandJob *cjobs, const RescoreJob *rjobs, int n_jobs, float min_score,
                                         float delta, int K, int nbhd, int polarity, const unsigned *hot_cnt,
                                         const uint2 *hot, unsigned hot_cap, unsigned *pass_cnt,
                                         unsigned *pass_list, cudaStream_t st);

struct RefineJob {
    const LevelDev *L;                 // the model's level tables (device)
    const float2 *field[kMaxLevels];   // this image's FP32 pixel-layout fields
    int w[kMaxLevels], h[kMaxLevels];
    int top, step_x, step_y, polarity;
    float min_score;
    const int32_t *kyx;                // candidates (3*K), scores (K), count
    const float *cs;
    const int *count;
    float4 *refined;                   // K
    int nscales;
};
struct NmsJob {
    const float4 *refined;
    const int *count;
    int w0, h0, min_side, max_out;
    double angle_step;
    int nang0;
    sam_pose *out;
    int *n_out;
};
size_t cand_cap(int nth, int gh, int gw, int ns = 1);
cudaError_t launch_candidates_jobs(const CandJob *jobs, int n_jobs, size_t max_total, float min_score, int K,
                                   cudaStream_t st);
cudaError_t launch_refine_jobs(const RefineJob *jobs, int n_jobs, int K, int nbhd, cudaStream_t st);
cudaError_t launch_nms_jobs(const NmsJob *jobs, int n_jobs, int K, cudaStream_t st);

}  // namespace sam
