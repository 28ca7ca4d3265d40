// C ABI of the detector: model lifetime, the full detection pipeline and the
// individual steps.  Every step of the pipeline runs in this library's CUDA
// kernels; host code only validates arguments, plans device buffers and
// orders launches on the caller's stream.

#include <string.h>

#include <algorithm>
#include <atomic>
#include <new>

#include "sam_internal.h"

#ifndef SAM_ARCH
#define SAM_ARCH 0
#endif

namespace sam {

static std::atomic<long long> g_launches{0};
void count_launches(int n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

namespace {

inline size_t al(size_t v) { return (v + 255) & ~(size_t)255; }

}  // namespace

// ---- stage timing ----
// Stage events go to a pool of event pairs; their elapsed times are summed
// only when the totals are read (or the pool is full), so an enabled profiler
// adds two event records per stage to a call and no host work after it.
// Stages may nest (the score map's launches inside the score-map stage).
struct Profiler {
    bool on = false;
    static constexpr int kPool = 4096;
    std::vector<cudaEvent_t> ev;     // 2 per slot
    std::vector<int> stage_of;       // stage of each recorded slot
    int used = 0;                    // slots taken
    int n_open = 0;                  // stages begun and not yet ended
    int open[SAM_NUM_STAGES] = {};   // slot of each open stage (-1: not recorded)
    double ms[SAM_NUM_STAGES] = {};
    int calls[SAM_NUM_STAGES] = {};
};
static Profiler g_prof;

// Sum every recorded pair (waits for the last one) and empty the pool; only
// while no stage is open.
void prof_flush() {
    if (g_prof.used == 0 || g_prof.n_open > 0)
        return;
    cudaEventSynchronize(g_prof.ev[2 * (g_prof.used - 1) + 1]);
    for (int i = 0; i < g_prof.used; ++i) {
        float t = 0.f;
        if (cudaEventElapsedTime(&t, g_prof.ev[2 * i], g_prof.ev[2 * i + 1]) == cudaSuccess) {
            g_prof.ms[g_prof.stage_of[i]] += t;
            g_prof.calls[g_prof.stage_of[i]] += 1;
        }
    }
    g_prof.used = 0;
}

void prof_begin(int stage, cudaStream_t st) {
    if (!g_prof.on || stage < 0 || stage >= SAM_NUM_STAGES)
        return;
    ++g_prof.n_open;
    g_prof.open[stage] = -1;
    if (g_prof.used == Profiler::kPool)
        prof_flush();
    if (g_prof.used == Profiler::kPool)
        return;   // pool full inside an open stage: this one is not recorded
    const int slot = g_prof.used;
    if ((int)g_prof.stage_of.size() <= slot) {
        cudaEvent_t a = nullptr, b = nullptr;
        if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess)
            return;
        g_prof.ev.push_back(a);
        g_prof.ev.push_back(b);
        g_prof.stage_of.push_back(0);
    }
    ++g_prof.used;
    g_prof.open[stage] = slot;
    g_prof.stage_of[slot] = stage;
    cudaEventRecord(g_prof.ev[2 * slot], st);
    cudaEventRecord(g_prof.ev[2 * slot + 1], st);   // replaced by prof_end
}

void prof_end(int stage, cudaStream_t st) {
    if (!g_prof.on || stage < 0 || stage >= SAM_NUM_STAGES)
        return;
    if (g_prof.n_open > 0)
        --g_prof.n_open;
    const int slot = g_prof.open[stage];
    g_prof.open[stage] = -1;
    if (slot >= 0)
        cudaEventRecord(g_prof.ev[2 * slot + 1], st);
}

namespace {

// Device buffers of one detection call (all images of a batch).
struct Plan {
    int L = 0, count = 0;
    int w[kMaxLevels], h[kMaxLevels];
    int pitch[kMaxLevels];           // level image row pitch (bytes)
    size_t img_bytes[kMaxLevels];    // bytes per image per level (level 0: only if copied)
    size_t off_img[kMaxLevels];
    size_t off_field[kMaxLevels];    // FP32 fields
    size_t field_px[kMaxLevels];
    size_t off_top = 0;              // top-level field, pairs layout, detection precision
    size_t top_px = 0;               // its pixels per image (pairs pitch x h, padded to 8)
    int gw = 0, gh = 0, nth = 0;
    size_t map_img = 0, off_map = 0;
    size_t off_scratch = 0;
    size_t off_rescore = 0;          // FP32 rescoring list (16-bit precisions)
    size_t off_kyx = 0, off_cs = 0, off_ccount = 0, off_refined = 0, off_out = 0, off_nout = 0;
    size_t off_queue = 0, queue_bytes = 0;   // persistent-form storage of the tiled scorer
    size_t off_hot = 0, hot_cap = 0;         // the persistent scorer's hot list (entries of 8 bytes)
    size_t off_pass = 0;                     // 16-bit candidate filter's pass list (4 bytes per hot entry)
    // refinement-level gradient tiles computed on demand: one mask bit and
    // one list entry per tile of levels 0 .. L - 2 of every image
    int tiles_x[kMaxLevels] = {}, tiles_y[kMaxLevels] = {};
    size_t tile_base[kMaxLevels] = {};
    size_t tiles = 0, off_tmask = 0, tmask_bytes = 0, off_tlist = 0;
    size_t total = 0;
};

// Level images of one call: level 0 where the caller's (or the copied)
// images are, the others in the workspace.
struct LevelImgs {
    const uint8_t *img[kMaxLevels];
    int pitch[kMaxLevels];
    size_t bytes[kMaxLevels];
};

sam_status check_detect_params(const sam_model *m, const sam_detect_params *p) {
    if (!p || p->step_x < 1 || p->step_y < 1 || (p->neighbourhood != 1 && p->neighbourhood != 3) ||
        p->max_detections < 1 || p->max_detections > kMaxTopK || p->top_k < 1 || p->top_k > kMaxTopK ||
        p->precision < SAM_FP32 || p->precision > SAM_FP16 || !(p->min_score >= -1.0f && p->min_score <= 1.0f))
        return SAM_ERR_ARG;
    (void)m;
    return SAM_OK;
}

Plan make_plan(const sam_model *m, int w, int h, int count, bool copy_level0, const sam_detect_params &p) {
    Plan P;
    P.L = m->levels;
    P.count = count;
    size_t off = 0;
    for (int l = 0; l < P.L; ++l) {
        P.w[l] = l == 0 ? w : P.w[l - 1] / 2;
        P.h[l] = l == 0 ? h : P.h[l - 1] / 2;
        P.pitch[l] = (int)((P.w[l] + 15) & ~15);
        P.img_bytes[l] = al((size_t)P.pitch[l] * P.h[l]);
        // a multiple of 8 pixels keeps every image's field 16-byte aligned
        P.field_px[l] = ((size_t)P.w[l] * P.h[l] + 7) & ~(size_t)7;
    }
    for (int l = 0; l < P.L; ++l) {
        P.off_img[l] = off;
        if (l > 0 || copy_level0)
            off += al(P.img_bytes[l] * count);
    }
    const int top = P.L - 1;
    for (int l = 0; l < P.L; ++l) {
        P.off_field[l] = off;
        // the top level is scored from its pairs-layout field; an FP32 pixel
        // field is also kept there when the 16-bit map is rescored in FP32
        if (l < top || p.precision != SAM_FP32)
            off += al(P.field_px[l] * 8 * count);
    }
    P.top_px = ((size_t)field_pitch(P.w[top], SAM_LAYOUT_PAIRS) * P.h[top] + 7) & ~(size_t)7;
    P.off_top = off;
    off += al(P.top_px * (p.precision == SAM_FP32 ? 8 : 4) * count);
    P.nth = m->lv[top].ntheta;
    P.gw = (P.w[top] + p.step_x - 1) / p.step_x;
    P.gh = (P.h[top] + p.step_y - 1) / p.step_y;
    P.map_img = (size_t)P.nth * P.gw * P.gh;
    P.off_map = off;
    off += al(P.map_img * 4 * count);
    P.off_scratch = off;
    off += al(candidates_scratch_bytes_batch(P.nth, P.gh, P.gw, count, m->nscales));
    P.off_rescore = off;
    if (p.precision != SAM_FP32)
        off += al(rescore_scratch_bytes(P.map_img * count));
    const int K = p.top_k;
    P.off_kyx = off;
    off += al((size_t)3 * K * 4 * count);
    P.off_cs = off;
    off += al((size_t)K * 4 * count);
    P.off_ccount = off;
    off += al((size_t)4 * count);
    P.off_refined = off;
    off += al((size_t)K * 16 * count);
    P.off_out = off;
    off += al((size_t)p.max_detections * sizeof(sam_pose) * count);
    P.off_nout = off;
    off += al((size_t)4 * count);
    if (p.early_termination && p.step_x == 1 && p.step_y == 1) {
        P.off_queue = off;
        P.queue_bytes = drain_queue_bytes(count, P.gw, P.gh, P.nth);
        off += al(P.queue_bytes);
        // hot list: every pose for a 16-bit map (the rescoring must see all
        // of them), a sixteenth of the poses for FP32 (an overflow only
        // sends candidate extraction back to the whole map)
        const size_t poses = P.map_img * count;
        P.hot_cap = p.precision == SAM_FP32 ? std::min(poses, std::max<size_t>(65536, poses / 16)) : poses;
        if (P.hot_cap > 0xFFFFFFFFull)
            P.hot_cap = 0;
        P.off_hot = off;
        off += al(P.hot_cap * 8);
        // the 16-bit candidate filter's pass list (room for every hot entry)
        P.off_pass = off;
        if (p.precision != SAM_FP32)
            off += al(P.hot_cap * 4);
    }
    {
        const int TW = gradient_tile_w(), TH = gradient_tile_h();
        size_t tiles = 0;
        for (int l = 0; l < top; ++l) {
            P.tiles_x[l] = (P.w[l] + TW - 1) / TW;
            P.tiles_y[l] = (P.h[l] + TH - 1) / TH;
            P.tile_base[l] = tiles;
            tiles += (size_t)P.tiles_x[l] * P.tiles_y[l] * count;
        }
        P.tiles = tiles;
        P.off_tmask = off;
        P.tmask_bytes = (tiles + 31) / 32 * 4 + 4;   // the mask words, then the list counter
        off += al(P.tmask_bytes);
        P.off_tlist = off;
        off += al(std::max<size_t>(1, tiles) * 8);
    }
    P.total = off;
    return P;
}

sam_status ensure_workspace(sam_model *m, size_t bytes) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess)
        return SAM_ERR_CUDA;
    if (m->ws.base && m->ws.bytes >= bytes && m->ws.device == dev)
        return SAM_OK;
    if (m->ws.base) {
        cudaFree(m->ws.base);
        m->ws.base = nullptr;
        m->ws.bytes = 0;
    }
    void *p = nullptr;
    if (cudaMalloc(&p, bytes) != cudaSuccess) {
        cudaGetLastError();
        return SAM_ERR_NOMEM;
    }
    m->ws.base = p;
    m->ws.bytes = bytes;
    m->ws.device = dev;
    return SAM_OK;
}

#define SAM_CU(x)                          \
    do {                                   \
        if ((x) != cudaSuccess)            \
            return SAM_ERR_CUDA;           \
    } while (0)

// Pyramid and gradient fields for `count` images whose level-0 copies start
// at img0 (row pitch pitch0, image i at img0 + i * img0_bytes).
sam_status prepare_fields(sam_model *m, const Plan &P, const uint8_t *img0, int pitch0, size_t img0_bytes,
                          const sam_detect_params &p, cudaStream_t st, LevelImgs *li = nullptr) {
    char *ws = (char *)m->ws.base;
    const int count = P.count, top = P.L - 1;
    const uint8_t *lvl_img[kMaxLevels];
    int lvl_pitch[kMaxLevels];
    size_t lvl_bytes[kMaxLevels];
    lvl_img[0] = img0;
    lvl_pitch[0] = pitch0;
    lvl_bytes[0] = img0_bytes;
    // (b) pyramid
    prof_begin(0, st);
    uint8_t *dsts[kMaxLevels] = {};
    for (int l = 1; l < P.L; ++l) {
        dsts[l] = (uint8_t *)(ws + P.off_img[l]);
        lvl_img[l] = dsts[l];
        lvl_pitch[l] = P.pitch[l];
        lvl_bytes[l] = P.img_bytes[l];
    }
    SAM_CU(launch_pyramid_levels(img0, P.w[0], P.h[0], pitch0, img0_bytes, P.L - 1, dsts, lvl_pitch, lvl_bytes, count,
                                 st));
    prof_end(0, st);
    // (a) gradients of the top level: the pairs layout in the detection
    // precision, and for a 16-bit precision the FP32 pixel-layout field that
    // candidate extraction rescores from.  The refinement levels' FP32
    // fields are computed after candidate extraction, where the candidates
    // can reach (run_search), or here in full when no level is refined
    // from a candidate list.
    prof_begin(1, st);
    if (!li) {
        for (int l = 0; l < top; ++l)
            SAM_CU(launch_gradient(lvl_img[l], P.w[l], P.h[l], lvl_pitch[l], lvl_bytes[l], m->p.low, SAM_FP32,
                                   SAM_LAYOUT_PIXEL, ws + P.off_field[l], P.field_px[l], nullptr, nullptr, count, st));
    }
    if (p.precision != SAM_FP32)
        SAM_CU(launch_gradient(lvl_img[top], P.w[top], P.h[top], lvl_pitch[top], lvl_bytes[top], m->p.low, SAM_FP32,
                               SAM_LAYOUT_PIXEL, ws + P.off_field[top], P.field_px[top], nullptr, nullptr, count, st));
    SAM_CU(launch_gradient(lvl_img[top], P.w[top], P.h[top], lvl_pitch[top], lvl_bytes[top], m->p.low, p.precision,
                           SAM_LAYOUT_PAIRS, ws + P.off_top, P.top_px, nullptr, nullptr, count, st));
    prof_end(1, st);
    if (li)
        for (int l = 0; l < P.L; ++l) {
            li->img[l] = lvl_img[l];
            li->pitch[l] = lvl_pitch[l];
            li->bytes[l] = lvl_bytes[l];
        }
    return SAM_OK;
}

// Level-l pixel reach of the coarse-to-fine refinement around 2^(top - l)
// times a candidate's top-level position (refine_body): the search centre
// at level l is 2 x + shift of the level-(l + 1) pose x, which is its own
// centre +-1, so the centre's distance from the scaled candidate is at most
// E(top - 1) = S(top) and E(l) = 2 E(l + 1) + 2 + S(l + 1) (S(l): the
// largest child shift of level l's tables); the pixels read lie within the
// rotated points' extent and 2 more pixels (a +-1 translation and the 3x3
// window), plus one pixel of margin.
void refine_reach(const sam_model *m, int top, int4 *reach) {
    int ex = 0, ey = 0;
    for (int l = top - 1; l >= 0; --l) {
        int sx = 0, sy = 0;
        for (const int2 &v : m->lv[l + 1].shift) {
            sx = std::max(sx, std::abs(v.x));
            sy = std::max(sy, std::abs(v.y));
        }
        if (l == top - 1) {
            ex = sx;
            ey = sy;
        } else {
            ex = 2 * ex + 2 + sx;
            ey = 2 * ey + 2 + sy;
        }
        int x0 = 0, x1 = 0, y0 = 0, y1 = 0;
        bool first = true;
        for (const int4 &b : m->lv[l].bbox) {
            x0 = first ? b.x : std::min(x0, b.x);
            x1 = first ? b.y : std::max(x1, b.y);
            y0 = first ? b.z : std::min(y0, b.z);
            y1 = first ? b.w : std::max(y1, b.w);
            first = false;
        }
        reach[l] = make_int4(-ex + x0 - 3, ex + x1 + 3, -ey + y0 - 3, ey + y1 + 3);
    }
}

ScoreArgs top_score_args(const sam_model *m, const Plan &P, const sam_detect_params &p) {
    char *ws = (char *)m->ws.base;
    const int top = P.L - 1;
    ScoreArgs sa;
    sa.field = ws + P.off_top;
    sa.field_img_px = P.top_px;
    sa.layout = SAM_LAYOUT_PAIRS;
    sa.w = P.w[top];
    sa.h = P.h[top];
    sa.precision = p.precision;
    sa.step_x = p.step_x;
    sa.step_y = p.step_y;
    sa.nbhd = p.neighbourhood;
    sa.polarity = m->p.polarity;
    sa.min_score = p.min_score;
    sa.early = p.early_termination;
    sa.map = (float *)(ws + P.off_map);
    sa.map_img = P.map_img;
    sa.count = P.count;
    sa.queue = P.queue_bytes ? ws + P.off_queue : nullptr;
    sa.queue_bytes = P.queue_bytes;
    if (P.hot_cap) {
        sa.hot = (uint2 *)(ws + P.off_hot);
        sa.hot_cap = (unsigned)P.hot_cap;
        sa.hot_thr = p.precision == SAM_FP32 ? p.min_score : p.min_score - rescore_delta(p.precision);
    }
    return sa;
}

// Exhaustive top-level search, candidates, refinement and NMS on the fields
// prepared by prepare_fields.
sam_status run_search(sam_model *m, const Plan &P, const sam_detect_params &p, cudaStream_t st,
                      const LevelImgs &li) {
    char *ws = (char *)m->ws.base;
    const int count = P.count, top = P.L - 1;
    // (c) exhaustive top-level score map; a 16-bit map is rescored in FP32
    // wherever a pose can reach min_score
    ScoreArgs sa = top_score_args(m, P, p);
    bool hot_made = false;
    sa.hot_made = &hot_made;
    prof_begin(2, st);
    SAM_CU(launch_score_map(m, top, sa, nullptr, st));
    // the persistent scorer's hot list, when it made one: the poses that
    // rescoring and candidate extraction have to look at
    const unsigned *hot_cnt = hot_made ? (const unsigned *)(ws + P.off_queue) + kHotCounter : nullptr;
    // a 16-bit map without a hot list is rescored in FP32 wherever a pose
    // can reach min_score; with one, candidate extraction decides in FP32
    if (p.precision != SAM_FP32 && !hot_cnt)
        SAM_CU(launch_rescore(m->dev[top], (const float2 *)(ws + P.off_field[top]), P.field_px[top], P.w[top],
                              P.h[top], p.step_x, p.step_y, count, p.neighbourhood, m->p.polarity, p.min_score,
                              p.precision, sa.map, P.map_img, ws + P.off_rescore, P.map_img * count, st));
    prof_end(2, st);
    // (d) candidates, refinement, NMS
    const int K = p.top_k;
    int32_t *kyx = (int32_t *)(ws + P.off_kyx);
    float *cs = (float *)(ws + P.off_cs);
    int *ccount = (int *)(ws + P.off_ccount);
    prof_begin(3, st);
    if (hot_cnt && p.precision != SAM_FP32)
        SAM_CU(launch_candidates_hot16(sa.map, P.map_img, P.nth, P.gh, P.gw, p.min_score, rescore_delta(p.precision),
                                       K, kyx, cs, ccount, ws + P.off_scratch, count, hot_cnt, sa.hot, sa.hot_cap,
                                       (const float2 *)(ws + P.off_field[top]), P.field_px[top], P.w[top], P.h[top],
                                       m->dev[top], p.neighbourhood, m->p.polarity,
                                       (unsigned *)(ws + P.off_queue) + kHotCounter + 1, (unsigned *)(ws + P.off_pass),
                                       st, m->nscales));
    else if (hot_cnt)
        SAM_CU(launch_candidates_hot(sa.map, P.map_img, P.nth, P.gh, P.gw, p.min_score, K, kyx, cs, ccount,
                                     ws + P.off_scratch, count, hot_cnt, sa.hot, sa.hot_cap, st, m->nscales));
    else
        SAM_CU(launch_candidates(sa.map, P.map_img, P.nth, P.gh, P.gw, p.min_score, K, kyx, cs, ccount,
                                 ws + P.off_scratch, 0, count, st, m->nscales));
    prof_end(3, st);
    // the refinement levels' FP32 fields where the candidates can reach
    if (top > 0) {
        prof_begin(1, st);
        TileMarks tm;
        memset(&tm, 0, sizeof(tm));
        tm.kyx = kyx;
        tm.count = ccount;
        tm.K = K;
        tm.count_images = count;
        tm.top = top;
        tm.step_x = p.step_x;
        tm.step_y = p.step_y;
        tm.nlev = top;
        refine_reach(m, top, tm.reach);
        GradTiles gt;
        memset(&gt, 0, sizeof(gt));
        bool vec = true;
        for (int l = 0; l < top; ++l) {
            tm.w[l] = P.w[l];
            tm.h[l] = P.h[l];
            tm.tiles_x[l] = P.tiles_x[l];
            tm.tiles_y[l] = P.tiles_y[l];
            tm.tile_base[l] = P.tile_base[l];
            gt.img[l] = li.img[l];
            gt.w[l] = P.w[l];
            gt.h[l] = P.h[l];
            gt.pitch[l] = li.pitch[l];
            gt.img_bytes[l] = li.bytes[l];
            gt.field[l] = (float2 *)(ws + P.off_field[l]);
            gt.field_px[l] = P.field_px[l];
            vec = vec && ((uintptr_t)li.img[l] % 16 == 0) && (li.pitch[l] % 16 == 0) &&
                  (count == 1 || li.bytes[l] % 16 == 0) && ((uintptr_t)gt.field[l] % 16 == 0) &&
                  (count == 1 || (P.field_px[l] * 8) % 16 == 0);
        }
        tm.mask = (uint32_t *)(ws + P.off_tmask);
        tm.list_cnt = (unsigned *)(ws + P.off_tmask + P.tmask_bytes - 4);
        tm.list = (uint2 *)(ws + P.off_tlist);
        tm.list_cap = (unsigned)P.tiles;
        gt.low = m->p.low;
        gt.vec = vec ? 1 : 0;
        gt.list_cnt = tm.list_cnt;
        gt.list = tm.list;
        gt.list_cap = tm.list_cap;
        SAM_CU(launch_refine_fields(tm, gt, P.tmask_bytes, st));
        prof_end(1, st);
    }
    RefineArgs ra;
    memset(&ra, 0, sizeof(ra));
    for (int l = 0; l < P.L; ++l) {
        ra.field[l] = (const float2 *)(ws + P.off_field[l]);
        ra.field_img_px[l] = P.field_px[l];
        ra.w[l] = P.w[l];
        ra.h[l] = P.h[l];
    }
    ra.top = top;
    ra.step_x = p.step_x;
    ra.step_y = p.step_y;
    ra.nbhd = p.neighbourhood;
    ra.polarity = m->p.polarity;
    ra.min_score = p.min_score;
    ra.K = K;
    ra.cand_kyx = kyx;
    ra.cand_s = cs;
    ra.cand_count = ccount;
    ra.refined = (float4 *)(ws + P.off_refined);
    ra.count = count;
    ra.nscales = m->nscales;
    prof_begin(4, st);
    SAM_CU(launch_refine(m, ra, st));
    prof_end(4, st);
    NmsArgs na;
    na.refined = ra.refined;
    na.cand_count = ccount;
    na.K = K;
    na.w0 = P.w[0];
    na.h0 = P.h[0];
    na.min_side = std::min(m->lv[0].tw, m->lv[0].th);
    na.max_out = p.max_detections;
    na.angle_step = m->p.angle_step_deg;
    na.nang0 = m->lv[0].nangles;
    na.out = (sam_pose *)(ws + P.off_out);
    na.n_out = (int *)(ws + P.off_nout);
    na.count = count;
    prof_begin(5, st);
    SAM_CU(launch_nms(na, st));
    prof_end(5, st);
    return SAM_OK;
}

sam_status run_pipeline(sam_model *m, const Plan &P, const uint8_t *img0, int pitch0, size_t img0_bytes,
                        const sam_detect_params &p, cudaStream_t st) {
    LevelImgs li;
    const sam_status s = prepare_fields(m, P, img0, pitch0, img0_bytes, p, st, &li);
    return s != SAM_OK ? s : run_search(m, P, p, st, li);
}

// ---- graph mode ----
// Changes of the scorer's tiling (sam_set_score_kernel, sam_autotune) bump
// the epoch, which invalidates every captured pipeline.
std::atomic<unsigned> g_tiling_epoch{1};
std::atomic<bool> g_graph_mode{true};

void drop_graph(sam_model *m) {
    if (m->gc.exec)
        cudaGraphExecDestroy(m->gc.exec);
    m->gc.exec = nullptr;
    m->gc.valid = false;
}

bool same_params(const sam_detect_params &a, const sam_detect_params &b) {
    return a.step_x == b.step_x && a.step_y == b.step_y && a.neighbourhood == b.neighbourhood &&
           a.min_score == b.min_score && a.max_detections == b.max_detections && a.top_k == b.top_k &&
           a.precision == b.precision && a.early_termination == b.early_termination;
}

// The whole pipeline of a plan whose level-0 images are in the workspace,
// replayed from a captured graph on `st` (captured first if the cached one
// does not match the call).
sam_status run_graph(sam_model *m, const Plan &P, const sam_detect_params &p, cudaStream_t st) {
    GraphCache &g = m->gc;
    int dev = 0;
    SAM_CU(cudaGetDevice(&dev));
    const unsigned epoch = g_tiling_epoch.load();
    if (!(g.valid && g.w == P.w[0] && g.h == P.h[0] && g.count == P.count && g.device == dev && g.epoch == epoch &&
          g.ws_base == m->ws.base && g.ws_bytes == m->ws.bytes && same_params(g.p, p))) {
        drop_graph(m);
        if (g.cap && g.device != dev) {
            cudaStreamDestroy(g.cap);
            g.cap = nullptr;
        }
        if (!g.cap)
            SAM_CU(cudaStreamCreateWithFlags(&g.cap, cudaStreamNonBlocking));
        g.device = dev;
        SAM_CU(cudaStreamBeginCapture(g.cap, cudaStreamCaptureModeRelaxed));
        const char *ws = (const char *)m->ws.base;
        const long long before = sam_kernel_launches();
        const sam_status s = run_pipeline(m, P, (const uint8_t *)(ws + P.off_img[0]), P.pitch[0], P.img_bytes[0], p,
                                          g.cap);
        cudaGraph_t graph = nullptr;
        const cudaError_t e = cudaStreamEndCapture(g.cap, &graph);
        // the capture counted its launches; replays are counted below
        const long long kernels = sam_kernel_launches() - before;
        count_launches(-(int)kernels);
        if (s != SAM_OK || e != cudaSuccess || !graph) {
            if (graph)
                cudaGraphDestroy(graph);
            cudaGetLastError();
            return s != SAM_OK ? s : SAM_ERR_CUDA;
        }
        const cudaError_t ie = cudaGraphInstantiate(&g.exec, graph, 0);
        cudaGraphDestroy(graph);
        if (ie != cudaSuccess) {
            g.exec = nullptr;
            return SAM_ERR_CUDA;
        }
        g.valid = true;
        g.w = P.w[0];
        g.h = P.h[0];
        g.count = P.count;
        g.p = p;
        g.epoch = epoch;
        g.ws_base = m->ws.base;
        g.ws_bytes = m->ws.bytes;
        g.kernels = kernels;
    }
    SAM_CU(cudaGraphLaunch(g.exec, st));
    count_launches((int)g.kernels);
    return SAM_OK;
}

bool graph_path() { return g_graph_mode.load() && !g_prof.on; }

sam_status read_results(sam_model *m, const Plan &P, const sam_detect_params &p, cudaStream_t st, sam_pose *out,
                        int capacity, int *n_out) {
    char *ws = (char *)m->ws.base;
    const int count = P.count;
    // the poses and the counts after them in one copy
    const size_t span = P.off_nout + (size_t)count * sizeof(int) - P.off_out;
    std::vector<char> host(span);
    SAM_CU(cudaMemcpyAsync(host.data(), ws + P.off_out, span, cudaMemcpyDeviceToHost, st));
    const sam_pose *poses = reinterpret_cast<const sam_pose *>(host.data());
    const int *nout = reinterpret_cast<const int *>(host.data() + (P.off_nout - P.off_out));
    int dev_err = 0;
    SAM_CU(score_error_flag_async(&dev_err, st));
    SAM_CU(cudaStreamSynchronize(st));
    if (dev_err) {
        score_error_clear(st);
        cudaStreamSynchronize(st);
        return SAM_ERR_TIMEOUT;
    }
    for (int i = 0; i < count; ++i) {
        const int n = std::min(nout[i], capacity);
        memcpy(out + (size_t)i * capacity, poses + (size_t)i * p.max_detections, (size_t)n * sizeof(sam_pose));
        n_out[i] = n;
    }
    return SAM_OK;
}

}  // namespace

ScoreChoice &score_choice() {
    static ScoreChoice c;
    return c;
}

// Whether the tiled kernel can serve these arguments with this tiling.
bool tiled_ok(const sam_model *m, int level, const ScoreArgs &a, const TileConfig &cfg) {
    int bxw = 0, byw = 0;
    return cfg.tg >= 1 && a.layout == SAM_LAYOUT_PAIRS && a.step_x == 1 && a.step_y == 1 && (a.nbhd == 1 || a.nbhd == 3) &&
           ((uintptr_t)a.field % 16 == 0) &&
           (a.count == 1 || a.field_img_px % (a.precision == SAM_ANGLE16 ? 8 : 4) == 0) &&
           tiled_plan(m->lv[level], a.precision, cfg.sx, cfg.sy, cfg.tg, cfg.tc, &bxw, &byw);
}

// A tiling with tg == 0 selects the chunked scorer (one angle per CTA, CTA
// tile of sx x sy warp tiles, one warp tile per warp).  Its default, 2 x 2
// warp tiles of 4 warps, needs a ~75 KB FP32 window per 16-pixel chunk cell:
// three CTAs per SM.
constexpr TileConfig kChunkCfg = {2, 2, 0, 4, kChunkCols};

bool chunked_ok(const sam_model *m, int level, const ScoreArgs &a, const TileConfig &cfg = kChunkCfg) {
    int bxw = 0, byw = 0;
    return cfg.tg == 0 && cfg.sx * cfg.sy == cfg.warps && (cfg.warps == 4 || cfg.warps == 8) &&
           a.precision != SAM_ANGLE16 && a.layout == SAM_LAYOUT_PAIRS && a.step_x == 1 && a.step_y == 1 && (a.nbhd == 1 || a.nbhd == 3) &&
           ((uintptr_t)a.field % 16 == 0) && (a.count == 1 || a.field_img_px % 4 == 0) && a.count <= 65535 &&
           m->dev[level].crot && m->lv[level].ntheta <= 65535 &&
           chunked_plan(m->lv[level], a.precision, cfg.sx, cfg.sy, &bxw, &byw);
}

// The tiled or chunked scorer for `cfg` over the map (or pose window) of `a`.
cudaError_t launch_fast_scorer(const sam_model *m, int level, const ScoreArgs &a, const TileConfig &cfg,
                               cudaStream_t st, const PoseWindow *window = nullptr) {
    const int wp = any_field_pitch(a.w, SAM_LAYOUT_PAIRS, a.precision);
    if (cfg.tg == 0)
        return launch_score_chunked(m, level, a.field, a.precision, wp, a.field_img_px, a.w, a.h, a.count, a.nbhd,
                                    a.polarity, a.min_score, a.early, a.map, a.map_img, cfg, st, window);
    DrainQueue q{a.queue, a.queue_bytes};
    q.hot = a.hot;
    q.hot_cap = a.hot_cap;
    q.hot_thr = a.hot_thr;
    q.hot_made = a.hot_made;
    return launch_score_tiled(m, level, a.field, a.precision, wp, a.field_img_px, a.w, a.h, a.count, a.nbhd,
                              a.polarity, a.min_score, a.early, a.map, a.map_img, cfg, st, window,
                              a.queue && !window ? &q : nullptr);
}

// The model's tuned tiling for field `precision` and a call over `count`
// images: the one tuned for that batch class (one image / several), else the
// other class's, else none.
const TileConfig *tuned_tiling(const sam_model *m, int precision, int count) {
    // angle codes are scored by the FP32 arithmetic: they use its tuning
    if (precision == SAM_ANGLE16)
        precision = SAM_FP32;
    const int cls = count > 1 ? 1 : 0;
    if (m->tuned[precision][cls])
        return &m->tile[precision][cls];
    if (m->tuned[precision][1 - cls])
        return &m->tile[precision][1 - cls];
    return nullptr;
}

// The scorer a call uses: the model's tuned tiling (or the process-wide
// selection), else the chunked default; false if neither serves the call.
bool pick_fast_scorer(const sam_model *m, int level, const ScoreArgs &a, TileConfig *out) {
    const ScoreChoice &c = score_choice();
    if (c.kernel == 1)
        return false;
    TileConfig cfg = c.cfg;
    const TileConfig *t = tuned_tiling(m, a.precision, a.count);
    if (t && c.kernel == 0)
        cfg = *t;
    if ((cfg.tg >= 1 && tiled_ok(m, level, a, cfg)) || (cfg.tg == 0 && chunked_ok(m, level, a, cfg))) {
        *out = cfg;
        return true;
    }
    if (a.precision == SAM_ANGLE16) {
        // codes have no chunked or generic scorer: the default tiling, or
        // one angle per CTA when its window is too large
        for (const TileConfig &d : {TileConfig{}, TileConfig{1, 1, 1, 4, 6}})
            if (tiled_ok(m, level, a, d)) {
                *out = d;
                return true;
            }
        return false;
    }
    if (chunked_ok(m, level, a)) {
        *out = kChunkCfg;
        return true;
    }
    return false;
}

cudaError_t launch_score_map(const sam_model *m, int level, const ScoreArgs &a, int *err, cudaStream_t st) {
    (void)err;
    TileConfig cfg;
    if (pick_fast_scorer(m, level, a, &cfg))
        return launch_fast_scorer(m, level, a, cfg, st);
    if (a.precision == SAM_ANGLE16)
        return cudaErrorInvalidValue;
    return launch_score_map_generic(m->dev[level], a, st);
}

}  // namespace sam

using namespace sam;

extern "C" {

const char *sam_status_str(sam_status s) {
    switch (s) {
    case SAM_OK:
        return "ok";
    case SAM_ERR_ARG:
        return "invalid argument";
    case SAM_ERR_NOMEM:
        return "out of memory";
    case SAM_ERR_CUDA:
        return "CUDA error";
    case SAM_ERR_TIMEOUT:
        return "device wait timed out";
    case SAM_ERR_EMPTY_MODEL:
        return "template level without edge points";
    case SAM_ERR_CAPACITY:
        return "device buffer capacity exceeded";
    }
    return "unknown status";
}

int sam_version(void) { return 100; }
int sam_compiled_arch(void) { return SAM_ARCH; }

void sam_default_model_params(sam_model_params *p) {
    if (!p)
        return;
    p->low = 30;
    p->high = 60;
    p->levels = 3;
    p->angle_step_deg = 1.0;
    p->polarity = 0;
}

void sam_default_detect_params(sam_detect_params *p) {
    if (!p)
        return;
    p->step_x = p->step_y = 1;
    p->neighbourhood = 3;
    p->min_score = 0.7f;
    p->max_detections = 16;
    p->top_k = 64;
    p->precision = SAM_FP32;
    p->early_termination = 1;
}

sam_status sam_create_model(const uint8_t *tmpl, int w, int h, int stride, const sam_model_params *params,
                            sam_model **out) {
    if (!out || !params)
        return SAM_ERR_ARG;
    *out = nullptr;
    if (params->low > 1024 || params->high > 1024)
        return SAM_ERR_ARG;
    sam_model *m = new (std::nothrow) sam_model();
    if (!m)
        return SAM_ERR_NOMEM;
    const sam_status s = build_model(tmpl, w, h, stride, *params, m);
    if (s != SAM_OK) {
        delete m;
        return s;
    }
    *out = m;
    return SAM_OK;
}

sam_status sam_create_model_scaled(const uint8_t *tmpl, int w, int h, int stride, const sam_model_params *params,
                                   double scale_min, double scale_step, int n_scales, sam_model **out) {
    if (!out || !params)
        return SAM_ERR_ARG;
    *out = nullptr;
    if (params->low > 1024 || params->high > 1024)
        return SAM_ERR_ARG;
    sam_model *m = new (std::nothrow) sam_model();
    if (!m)
        return SAM_ERR_NOMEM;
    const sam_status s = build_model(tmpl, w, h, stride, *params, m, n_scales, scale_min, scale_step);
    if (s != SAM_OK) {
        delete m;
        return s;
    }
    *out = m;
    return SAM_OK;
}

int sam_model_num_scales(const sam_model *m) { return m ? m->nscales : 0; }

double sam_model_scale(const sam_model *m, int j) {
    return (m && j >= 0 && j < m->nscales) ? m->scale_min + j * m->scale_step : 0.0;
}

void sam_free_model(sam_model *m) {
    if (!m)
        return;
    if (m->gc.exec)
        cudaGraphExecDestroy(m->gc.exec);
    if (m->gc.cap)
        cudaStreamDestroy(m->gc.cap);
    if (m->d_tables)
        cudaFree(m->d_tables);
    if (m->ws.base)
        cudaFree(m->ws.base);
    for (auto &q : m->qbins)
        cudaFree(q.dev);
    delete m;
}

int sam_model_levels(const sam_model *m) { return m ? m->levels : 0; }

int sam_model_num_points(const sam_model *m, int level) {
    return (m && level >= 0 && level < m->levels) ? m->lv[level].n : 0;
}

int sam_model_num_angles(const sam_model *m, int level) {
    return (m && level >= 0 && level < m->levels) ? m->lv[level].nangles : 0;
}

int sam_model_template_size(const sam_model *m, int level, int *w, int *h) {
    if (!m || level < 0 || level >= m->levels)
        return 0;
    if (w)
        *w = m->lv[level].tw;
    if (h)
        *h = m->lv[level].th;
    return 1;
}

sam_status sam_model_rotated_points(const sam_model *m, int level, int k, int32_t *ox, int32_t *oy, float *px,
                                    float *py) {
    if (!m || level < 0 || level >= m->levels || k < 0 || k >= m->lv[level].ntheta || !ox || !oy || !px || !py)
        return SAM_ERR_ARG;
    const LevelHost &L = m->lv[level];
    const RotPt *r = L.rot.data() + (size_t)k * L.n;
    for (int i = 0; i < L.n; ++i) {
        ox[i] = r[i].ox;
        oy[i] = r[i].oy;
        px[i] = r[i].px;
        py[i] = r[i].py;
    }
    return SAM_OK;
}

sam_status sam_model_points(const sam_model *m, int level, int32_t *tx, int32_t *ty, int32_t *gx, int32_t *gy) {
    if (!m || level < 0 || level >= m->levels || !tx || !ty || !gx || !gy)
        return SAM_ERR_ARG;
    const LevelHost &L = m->lv[level];
    std::copy(L.tx.begin(), L.tx.end(), tx);
    std::copy(L.ty.begin(), L.ty.end(), ty);
    std::copy(L.gx.begin(), L.gx.end(), gx);
    std::copy(L.gy.begin(), L.gy.end(), gy);
    return SAM_OK;
}

sam_status sam_model_child_shift(const sam_model *m, int level, int k_parent, int32_t *sx, int32_t *sy) {
    if (!m || level < 0 || level + 1 >= m->levels || k_parent < 0 || k_parent >= m->lv[level + 1].ntheta || !sx ||
        !sy)
        return SAM_ERR_ARG;
    *sx = m->lv[level + 1].shift[k_parent].x;
    *sy = m->lv[level + 1].shift[k_parent].y;
    return SAM_OK;
}

sam_status sam_detect(sam_model *m, const uint8_t *img, int w, int h, int stride, int img_on_device,
                      const sam_detect_params *params, void *stream, sam_pose *out, int capacity, int *n_out) {
    if (!m || !img || !out || !n_out || capacity < 0 || stride < w)
        return SAM_ERR_ARG;
    *n_out = 0;
    sam_status s = check_detect_params(m, params);
    if (s != SAM_OK)
        return s;
    if ((w >> (m->levels - 1)) < 1 || (h >> (m->levels - 1)) < 1)
        return SAM_ERR_ARG;
    s = upload_model(m);
    if (s != SAM_OK)
        return s;
    const bool graph = graph_path();
    const Plan P = make_plan(m, w, h, 1, graph || !img_on_device, *params);
    s = ensure_workspace(m, P.total);
    if (s != SAM_OK)
        return s;
    cudaStream_t st = (cudaStream_t)stream;
    if (graph) {
        uint8_t *dst = (uint8_t *)m->ws.base + P.off_img[0];
        SAM_CU(cudaMemcpy2DAsync(dst, P.pitch[0], img, stride, w, h,
                                 img_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, st));
        s = run_graph(m, P, *params, st);
        if (s != SAM_OK)
            return s;
        return read_results(m, P, *params, st, out, capacity, n_out);
    }
    const uint8_t *img0 = img;
    int pitch0 = stride;
    size_t bytes0 = 0;
    if (!img_on_device) {
        uint8_t *dst = (uint8_t *)m->ws.base + P.off_img[0];
        SAM_CU(cudaMemcpy2DAsync(dst, P.pitch[0], img, stride, w, h, cudaMemcpyHostToDevice, st));
        img0 = dst;
        pitch0 = P.pitch[0];
    }
    s = run_pipeline(m, P, img0, pitch0, bytes0, *params, st);
    if (s != SAM_OK)
        return s;
    return read_results(m, P, *params, st, out, capacity, n_out);
}

sam_status sam_detect_batch(sam_model *m, const uint8_t *img, int count, size_t image_bytes, int w, int h,
                            int stride, int img_on_device, const sam_detect_params *params, void *stream,
                            sam_pose *out, int capacity, int *n_out) {
    if (!m || !img || !out || !n_out || count < 1 || capacity < 0 || stride < w ||
        image_bytes < (size_t)stride * (h - 1) + w)
        return SAM_ERR_ARG;
    sam_status s = check_detect_params(m, params);
    if (s != SAM_OK)
        return s;
    if ((w >> (m->levels - 1)) < 1 || (h >> (m->levels - 1)) < 1)
        return SAM_ERR_ARG;
    s = upload_model(m);
    if (s != SAM_OK)
        return s;
    const bool graph = graph_path();
    // the workspace holds the level-0 images in graph mode and for host input
    const bool staged = graph || !img_on_device;
    const Plan P = make_plan(m, w, h, count, staged, *params);
    s = ensure_workspace(m, P.total);
    if (s != SAM_OK)
        return s;
    cudaStream_t st = (cudaStream_t)stream;
    if (staged) {
        // the batch into the workspace's level-0 images (one copy when the
        // rows of all images are evenly spaced), then the pipeline
        const cudaMemcpyKind kind = img_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
        uint8_t *dst = (uint8_t *)m->ws.base + P.off_img[0];
        if (image_bytes == (size_t)stride * h && P.img_bytes[0] == (size_t)P.pitch[0] * h) {
            SAM_CU(cudaMemcpy2DAsync(dst, P.pitch[0], img, stride, w, (size_t)h * count, kind, st));
        } else {
            for (int i = 0; i < count; ++i)
                SAM_CU(cudaMemcpy2DAsync(dst + (size_t)i * P.img_bytes[0], P.pitch[0], img + (size_t)i * image_bytes,
                                         stride, w, h, kind, st));
        }
        if (graph) {
            s = run_graph(m, P, *params, st);
            if (s != SAM_OK)
                return s;
            return read_results(m, P, *params, st, out, capacity, n_out);
        }
        s = run_pipeline(m, P, dst, P.pitch[0], P.img_bytes[0], *params, st);
        if (s != SAM_OK)
            return s;
        return read_results(m, P, *params, st, out, capacity, n_out);
    }
    s = run_pipeline(m, P, img, stride, image_bytes, *params, st);
    if (s != SAM_OK)
        return s;
    return read_results(m, P, *params, st, out, capacity, n_out);
}

sam_status sam_autotune(sam_model *m, const uint8_t *img, int count, size_t image_bytes, int w, int h, int stride,
                        const sam_detect_params *params, void *stream, int32_t *cfg_out, float *ms_out, int max_out,
                        int *n_out) {
    if (!m || !img || count < 1 || stride < w || image_bytes < (size_t)stride * (h - 1) + w || !n_out ||
        max_out < 0 || (max_out > 0 && (!cfg_out || !ms_out)))
        return SAM_ERR_ARG;
    *n_out = 0;
    sam_status s = check_detect_params(m, params);
    if (s != SAM_OK)
        return s;
    if ((w >> (m->levels - 1)) < 1 || (h >> (m->levels - 1)) < 1)
        return SAM_ERR_ARG;
    s = upload_model(m);
    if (s != SAM_OK)
        return s;
    const Plan P = make_plan(m, w, h, count, false, *params);
    s = ensure_workspace(m, P.total);
    if (s != SAM_OK)
        return s;
    cudaStream_t st = (cudaStream_t)stream;
    s = prepare_fields(m, P, img, stride, image_bytes, *params, st);
    if (s != SAM_OK)
        return s;
    const ScoreArgs sa = top_score_args(m, P, *params);
    const int top = P.L - 1;
    const int nth = m->lv[top].ntheta;
    const int tgs[] = {1, 2, 3, 4, 5, 6, 8, 9, 11, 12, 15, 23, nth};
    cudaEvent_t e0, e1;
    SAM_CU(cudaEventCreate(&e0));
    SAM_CU(cudaEventCreate(&e1));
    float best = 1e30f;
    TileConfig bestc;
    bool found = false;
    int n = 0;
    std::vector<TileConfig> cands;
    for (int tc : {6, 10})
        for (int warps : {8, 4})
            for (int sy = 1; sy <= 2; ++sy)
                for (int sx = 1; sx <= 3; ++sx)
                    for (int tg : tgs) {
                        TileConfig c;
                        c.sx = sx;
                        c.sy = sy;
                        c.tg = std::min(tg, nth);
                        c.warps = warps;
                        c.tc = tc;
                        if (tiled_ok(m, top, sa, c))
                            cands.push_back(c);
                    }
    // chunked tilings (tg = 0): one warp tile per warp
    for (const TileConfig &c : {TileConfig{2, 2, 0, 4, kChunkCols}, TileConfig{4, 1, 0, 4, kChunkCols},
                                TileConfig{1, 4, 0, 4, kChunkCols}, TileConfig{2, 4, 0, 8, kChunkCols},
                                TileConfig{4, 2, 0, 8, kChunkCols}})
        if (chunked_ok(m, top, sa, c))
            cands.push_back(c);
    {
        for (const TileConfig &c : cands) {
                    cudaError_t e = launch_fast_scorer(m, top, sa, c, st);
                    cudaEventRecord(e0, st);
                    const int reps = 3;
                    for (int r = 0; r < reps && e == cudaSuccess; ++r)
                        e = launch_fast_scorer(m, top, sa, c, st);
                    cudaEventRecord(e1, st);
                    if (e != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess) {
                        cudaEventDestroy(e0);
                        cudaEventDestroy(e1);
                        return SAM_ERR_CUDA;
                    }
                    float ms = 0.f;
                    cudaEventElapsedTime(&ms, e0, e1);
                    ms /= reps;
                    if (n < max_out) {
                        cfg_out[5 * n] = c.sx;
                        cfg_out[5 * n + 1] = c.sy;
                        cfg_out[5 * n + 2] = c.tg;
                        cfg_out[5 * n + 3] = c.warps;
                        cfg_out[5 * n + 4] = c.tc;
                        ms_out[n] = ms;
                    }
                    ++n;
                    if (ms < best) {
                        best = ms;
                        bestc = c;
                        found = true;
                    }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    *n_out = std::min(n, max_out);
    if (found) {
        const int pr = params->precision;
        const int cls = count > 1 ? 1 : 0;
        m->tuned[pr][cls] = true;
        m->tile[pr][cls] = bestc;
        ++g_tiling_epoch;
    }
    int dev_err = 0;
    SAM_CU(score_error_flag_async(&dev_err, st));
    SAM_CU(cudaStreamSynchronize(st));
    if (dev_err) {
        score_error_clear(st);
        cudaStreamSynchronize(st);
        return SAM_ERR_TIMEOUT;
    }
    return SAM_OK;
}

sam_status sam_model_tiling(const sam_model *m, int precision, int count, int32_t *sx, int32_t *sy, int32_t *tg,
                            int32_t *warps, int32_t *cols) {
    if (!m || !sx || !sy || !tg || !warps || !cols || precision < SAM_FP32 || precision > SAM_FP16 || count < 1)
        return SAM_ERR_ARG;
    // a process-wide tiled selection overrides the model's tuning
    const ScoreChoice &sc = score_choice();
    const TileConfig *t = sc.kernel == 0 ? tuned_tiling(m, precision, count) : nullptr;
    const TileConfig c = t ? *t : sc.cfg;
    *sx = c.sx;
    *sy = c.sy;
    *tg = c.tg;
    *warps = c.warps;
    *cols = c.tc;
    return SAM_OK;
}

sam_status sam_pyramid_down(const uint8_t *src, int w, int h, int src_stride, uint8_t *dst, int dst_stride,
                            void *stream) {
    if (!src || !dst || w < 0 || h < 0 || src_stride < w || dst_stride < w / 2)
        return SAM_ERR_ARG;
    return launch_pyramid_down(src, w, h, src_stride, 0, dst, dst_stride, 0, 1, (cudaStream_t)stream) == cudaSuccess
               ? SAM_OK
               : SAM_ERR_CUDA;
}

sam_status sam_pyramid_levels(const uint8_t *src, int w, int h, int src_stride, int levels, uint8_t *const *dst,
                              const int *dst_stride, void *stream) {
    if (!src || !dst || !dst_stride || w < 0 || h < 0 || src_stride < w || levels < 2 || levels > kMaxLevels)
        return SAM_ERR_ARG;
    uint8_t *d[kMaxLevels] = {};
    int ds[kMaxLevels] = {};
    size_t di[kMaxLevels] = {};
    for (int l = 1; l < levels; ++l) {
        if (!dst[l - 1] || dst_stride[l - 1] < (w >> l))
            return SAM_ERR_ARG;
        d[l] = dst[l - 1];
        ds[l] = dst_stride[l - 1];
    }
    return launch_pyramid_levels(src, w, h, src_stride, 0, levels - 1, d, ds, di, 1, (cudaStream_t)stream) ==
                   cudaSuccess
               ? SAM_OK
               : SAM_ERR_CUDA;
}

sam_status sam_gradient(const uint8_t *img, int w, int h, int stride, int low, int precision, int layout,
                        void *field, int16_t *gx, int16_t *gy, void *stream) {
    if (!img || !field || w < 1 || h < 1 || stride < w || low < 1 || low > 1024 || precision < SAM_FP32 ||
        precision > SAM_ANGLE16 || (layout != SAM_LAYOUT_PIXEL && layout != SAM_LAYOUT_PAIRS) ||
        ((gx == nullptr) != (gy == nullptr)) || (precision == SAM_ANGLE16 && gx) ||
        (layout == SAM_LAYOUT_PAIRS && (gx || (uintptr_t)field % 16)))
        return SAM_ERR_ARG;
    return launch_gradient(img, w, h, stride, 0, low, precision, layout, field,
                           (size_t)any_field_pitch(w, layout, precision) * h, gx, gy, 1,
                           (cudaStream_t)stream) == cudaSuccess
               ? SAM_OK
               : SAM_ERR_CUDA;
}

sam_status sam_score_map(sam_model *m, int level, const void *field, int w, int h, int precision, int layout,
                         int step_x, int step_y, int neighbourhood, float min_score, int early_termination,
                         float *map, void *stream) {
    if (!m || level < 0 || level >= m->levels || !field || !map || w < 1 || h < 1 || step_x < 1 || step_y < 1 ||
        (neighbourhood != 1 && neighbourhood != 3) || precision < SAM_FP32 || precision > SAM_ANGLE16 ||
        (layout != SAM_LAYOUT_PIXEL && layout != SAM_LAYOUT_PAIRS) ||
        (precision == SAM_ANGLE16 && (layout != SAM_LAYOUT_PAIRS || step_x != 1 || step_y != 1)))
        return SAM_ERR_ARG;
    sam_status s = upload_model(m);
    if (s != SAM_OK)
        return s;
    ScoreArgs sa;
    sa.field = field;
    sa.field_img_px = (size_t)any_field_pitch(w, layout, precision) * h;
    sa.w = w;
    sa.h = h;
    sa.precision = precision;
    sa.layout = layout;
    sa.step_x = step_x;
    sa.step_y = step_y;
    sa.nbhd = neighbourhood;
    sa.polarity = m->p.polarity;
    sa.min_score = min_score;
    sa.early = early_termination;
    sa.map = map;
    sa.map_img = 0;
    sa.count = 1;
    cudaStream_t st = (cudaStream_t)stream;
    // early termination at step 1: the tiled scorer's persistent form, its
    // queue in stream-ordered memory of the device's default pool (else one
    // CTA per work unit)
    void *q = nullptr;
    if (early_termination && step_x == 1 && step_y == 1) {
        const size_t qb = drain_queue_bytes(1, w, h, m->lv[level].ntheta);
        if (cudaMallocAsync(&q, qb, st) == cudaSuccess) {
            sa.queue = q;
            sa.queue_bytes = qb;
        } else {
            (void)cudaGetLastError();
            q = nullptr;
        }
    }
    TileConfig probe;
    if (precision == SAM_ANGLE16 && !pick_fast_scorer(m, level, sa, &probe)) {
        if (q)
            cudaFreeAsync(q, st);
        return SAM_ERR_ARG;   // codes are scored by the tiled kernel only
    }
    const cudaError_t e = launch_score_map(m, level, sa, nullptr, st);
    if (q && cudaFreeAsync(q, st) != cudaSuccess)
        return SAM_ERR_CUDA;
    return e == cudaSuccess ? SAM_OK : SAM_ERR_CUDA;
}

size_t sam_score_window_scratch_bytes(size_t max_rescored) { return rescore_scratch_bytes(max_rescored); }

sam_status sam_score_window(sam_model *m, int level, const void *field, int w, int h, int precision, int x0, int y0,
                            int gw, int gh, int k0, int nk, int neighbourhood, float min_score, int early_termination,
                            const float *field32, void *scratch, size_t scratch_bytes, float *map, void *stream) {
    if (!m || level < 0 || level >= m->levels || !field || !map || w < 1 || h < 1 || precision < SAM_FP32 ||
        precision > SAM_ANGLE16 || (neighbourhood != 1 && neighbourhood != 3) || x0 < 0 || y0 < 0 || gw < 1 ||
        gh < 1 || x0 > w - gw || y0 > h - gh || k0 < 0 || nk < 1 || nk > 65535 || k0 > m->lv[level].ntheta - nk ||
        (size_t)nk * gw * gh > 0xFFFFFFFFull || (uintptr_t)field % 16 || (uintptr_t)map % 8)
        return SAM_ERR_ARG;
    const bool rescore = (precision == SAM_BF16 || precision == SAM_FP16) && field32;
    if (rescore && (!scratch || scratch_bytes < rescore_scratch_bytes(1) || (uintptr_t)field32 % 8 ||
                    (uintptr_t)scratch % 8))
        return SAM_ERR_ARG;
    sam_status s = upload_model(m);
    if (s != SAM_OK)
        return s;
    cudaStream_t st = (cudaStream_t)stream;
    ScoreArgs a;
    a.field = field;
    a.field_img_px = (size_t)any_field_pitch(w, SAM_LAYOUT_PAIRS, precision) * h;
    a.w = w;
    a.h = h;
    a.precision = precision;
    a.layout = SAM_LAYOUT_PAIRS;
    a.step_x = 1;
    a.step_y = 1;
    a.nbhd = neighbourhood;
    a.polarity = m->p.polarity;
    a.min_score = min_score;
    a.early = early_termination ? 1 : 0;
    a.map = map;
    a.map_img = (size_t)nk * gw * gh;
    a.count = 1;
    const PoseWindow pw{x0, y0, gw, gh, k0, nk};
    TileConfig cfg;
    if (!pick_fast_scorer(m, level, a, &cfg))
        return SAM_ERR_ARG;
    if (launch_fast_scorer(m, level, a, cfg, st, &pw) != cudaSuccess)
        return SAM_ERR_CUDA;
    if (rescore) {
        const size_t cap = (scratch_bytes - rescore_scratch_bytes(0)) / 8;
        if (launch_rescore(m->dev[level], (const float2 *)field32, (size_t)w * h, w, h, 1, 1, 1, neighbourhood,
                           m->p.polarity, min_score, precision, map, a.map_img, scratch, cap, st, &pw) != cudaSuccess)
            return SAM_ERR_CUDA;
    }
    return SAM_OK;
}

sam_status sam_set_score_kernel(int kernel, int sx, int sy, int tg, int warps, int cols) {
    if (kernel < 0 || kernel > 2 || sx < 1 || sx > 8 || sy < 1 || sy > 8 || tg < 0 || tg > 4096 ||
        (warps != 4 && warps != 8) || (tg == 0 && sx * sy != warps) || (cols != 6 && cols != 10) ||
        (tg == 0 && cols != kChunkCols))
        return SAM_ERR_ARG;
    ScoreChoice &c = score_choice();
    ++g_tiling_epoch;
    c.kernel = kernel;
    c.cfg.sx = sx;
    c.cfg.sy = sy;
    c.cfg.tg = tg;
    c.cfg.warps = warps;
    c.cfg.tc = cols;
    return SAM_OK;
}

void sam_get_score_kernel(int *kernel, int *sx, int *sy, int *tg, int *warps, int *cols) {
    const ScoreChoice &c = score_choice();
    if (kernel)
        *kernel = c.kernel;
    if (sx)
        *sx = c.cfg.sx;
    if (sy)
        *sy = c.cfg.sy;
    if (tg)
        *tg = c.cfg.tg;
    if (warps)
        *warps = c.cfg.warps;
    if (cols)
        *cols = c.cfg.tc;
}

size_t sam_candidates_scratch_bytes(int nth, int gh, int gw) { return candidates_scratch_bytes(nth, gh, gw); }

void sam_profile_enable(int on) { g_prof.on = on != 0; }

void sam_set_graph_mode(int on) { g_graph_mode = on != 0; }

long long sam_kernel_launches(void) { return g_launches.load(); }

int sam_profile_read(float *ms, int *calls, int n) {
    // no call is in flight between API calls: a stage an error path left
    // open has both its events recorded
    g_prof.n_open = 0;
    prof_flush();
    const int m = n < SAM_NUM_STAGES ? n : SAM_NUM_STAGES;
    for (int s = 0; s < m; ++s) {
        if (ms)
            ms[s] = (float)g_prof.ms[s];
        if (calls)
            calls[s] = g_prof.calls[s];
    }
    for (int s = 0; s < SAM_NUM_STAGES; ++s) {
        g_prof.ms[s] = 0.0;
        g_prof.calls[s] = 0;
    }
    return m;
}

size_t sam_candidates_scaled_scratch_bytes(int n_scales, int n_angles, int gh, int gw) {
    if (n_scales < 1 || n_angles < 1 || gh < 1 || gw < 1)
        return 0;
    return candidates_scratch_bytes(n_scales * n_angles, gh, gw, n_scales);
}

sam_status sam_candidates_scaled(const float *map, int n_scales, int n_angles, int gh, int gw, float min_score, int K,
                                 int32_t *out_kyx, float *out_s, int *count, void *scratch, void *stream) {
    if (!map || !out_kyx || !out_s || !count || !scratch || n_scales < 1 || n_angles < 1 || gh < 1 || gw < 1 ||
        K < 1 || K > kMaxTopK || (long long)n_scales * n_angles > (1LL << 30))
        return SAM_ERR_ARG;
    return launch_candidates(map, 0, n_scales * n_angles, gh, gw, min_score, K, out_kyx, out_s, count, scratch, 0, 1,
                             (cudaStream_t)stream, n_scales) == cudaSuccess
               ? SAM_OK
               : SAM_ERR_CUDA;
}

sam_status sam_candidates(const float *map, int nth, int gh, int gw, float min_score, int K, int32_t *out_kyx,
                          float *out_s, int *count, void *scratch, void *stream) {
    if (!map || !out_kyx || !out_s || !count || !scratch || nth < 1 || gh < 1 || gw < 1 || K < 1 || K > kMaxTopK)
        return SAM_ERR_ARG;
    return launch_candidates(map, 0, nth, gh, gw, min_score, K, out_kyx, out_s, count, scratch, 0, 1,
                             (cudaStream_t)stream) == cudaSuccess
               ? SAM_OK
               : SAM_ERR_CUDA;
}

}  // extern "C"
