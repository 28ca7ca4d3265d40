// Batched detection of uneven workloads: many search images of different
// sizes, each matched against one or more models (Sec. II detection, applied
// to (image, model) pairs).  A plan owns every device buffer of the batch and
// its descriptor arrays; one run is a fixed sequence of job-list launches --
// pyramid steps, gradients, one persistent exhaustive scorer over all pairs,
// (for 16-bit fields) FP32 rescoring, candidates, refinement and NMS -- which
// the plan captures once into a CUDA graph and replays.

#include <string.h>

#include <algorithm>
#include <new>
#include <numeric>
#include <vector>

#include "sam_internal.h"
#include "score_common.cuh"

namespace sam {
namespace {

inline size_t al(size_t v) { return (v + 255) & ~(size_t)255; }

struct ImgPlan {
    int L = 1;   // pyramid levels needed (max over the image's pairs)
    int w[kMaxLevels], h[kMaxLevels], pitch[kMaxLevels];
    size_t off_img[kMaxLevels], off_field[kMaxLevels], field_px[kMaxLevels];
};

struct TopField {   // pairs-layout field of one image at one level
    int img, level;
    size_t off, px;
    int wp;
};

struct PairPlan {
    int img, model, top, tf;   // tf: index of its TopField
    int W, H, nth, n;
    size_t off_map, map_img;
    size_t off_cand, cap;
    size_t off_kyx, off_cs, off_refined, off_out, off_nout, off_rescore;
    int bxw = 0, byw = 0, tiles_x = 0, tiles = 0, items = 0;
    double cost = 0;
};

}  // namespace
}  // namespace sam

struct sam_multi {
    std::vector<sam_model *> models;
    std::vector<sam::ImgPlan> imgs;
    std::vector<sam::TopField> tops;
    std::vector<sam::PairPlan> pp;     // in caller order
    std::vector<int> order;            // pair indices, largest scoring cost first
    sam_detect_params p;
    sam::TileConfig cfg;
    int device = -1;
    void *base = nullptr;
    size_t bytes = 0;
    // descriptor region
    size_t off_desc = 0, desc_bytes = 0;
    size_t off_counters = 0;           // [work counter][cand counters, out counts, rescore counts x n_pairs]
    size_t off_rsjobs = 0;
    size_t off_pyr = 0, off_grad = 0, off_gtop = 0, off_pairs = 0, off_tmaps = 0, off_cjobs = 0, off_rjobs = 0,
           off_njobs = 0, off_levels = 0;
    std::vector<int> pyr_count;        // jobs per pyramid step l -> l+1
    std::vector<int> grad_count;       // jobs per FP32 gradient level
    int max_w0 = 0, max_h0 = 0, Lmax = 1;
    int total_items = 0;
    size_t window_bytes = 0;
    size_t bitmap_bytes = 0;           // edge bitmaps of the largest window
    size_t max_map = 0;
    long long pose_points = 0;
    // hot list of the pairs scorer (see TiledArgs): candidates (and, for a
    // 16-bit field, their FP32 decision) from the listed poses only
    bool hot = false;
    size_t off_hot = 0, hot_cap = 0, off_pass = 0;
    bool dirty = true;                 // descriptors / graph must be rebuilt
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    long long graph_kernels = 0;
};

namespace sam {
namespace {

#define MU_CU(x)                     \
    do {                             \
        if ((x) != cudaSuccess)      \
            return SAM_ERR_CUDA;     \
    } while (0)

// Scoring cost and window of every pair for the plan's tiling; false if a
// pair's window does not fit the tiled kernel.
bool plan_tiling(sam_multi *mp) {
    int wty = 0;
    const int wtx = tiled_warp_tile(mp->p.precision, mp->cfg.tc, &wty);
    mp->window_bytes = 0;
    mp->bitmap_bytes = 0;
    const size_t pair_bytes = mp->p.precision == SAM_FP32 ? 16 : 8;
    for (PairPlan &q : mp->pp) {
        const LevelHost &L = mp->models[q.model]->lv[q.top];
        if (!tiled_plan(L, mp->p.precision, mp->cfg.sx, mp->cfg.sy, mp->cfg.tg, mp->cfg.tc, &q.bxw, &q.byw))
            return false;
        q.tiles_x = (q.W + mp->cfg.sx * wtx - 1) / (mp->cfg.sx * wtx);
        const int tiles_y = (q.H + mp->cfg.sy * wty - 1) / (mp->cfg.sy * wty);
        q.tiles = q.tiles_x * tiles_y;
        q.items = q.tiles * ((q.nth + mp->cfg.tg - 1) / mp->cfg.tg);
        q.cost = (double)q.items * mp->cfg.tg * mp->cfg.sx * mp->cfg.sy * q.n;
        mp->window_bytes = std::max(mp->window_bytes, (size_t)q.bxw * q.byw * pair_bytes / 2);
        mp->bitmap_bytes = std::max(mp->bitmap_bytes, edge_bitmap_bytes(q.bxw, q.byw));
    }
    mp->order.resize(mp->pp.size());
    std::iota(mp->order.begin(), mp->order.end(), 0);
    std::stable_sort(mp->order.begin(), mp->order.end(),
                     [&](int a, int b) { return mp->pp[a].cost > mp->pp[b].cost; });
    return true;
}

// Host images of every descriptor array, copied to the device in one go.
sam_status upload_descriptors(sam_multi *mp) {
    std::vector<char> h(mp->desc_bytes, 0);
    auto put = [&](size_t off, const void *src, size_t n) { memcpy(h.data() + (off - mp->off_desc), src, n); };
    char *base = (char *)mp->base;
    const int np = (int)mp->pp.size();
    // pyramid and gradient jobs, grouped by level
    size_t o = mp->off_pyr;
    for (int l = 1; l < mp->Lmax; ++l)
        for (const ImgPlan &I : mp->imgs) {
            if (I.L <= l)
                continue;
            ImageJob j;
            memset(&j, 0, sizeof(j));
            j.src = (const uint8_t *)(base + I.off_img[l - 1]);
            j.w = I.w[l - 1];
            j.h = I.h[l - 1];
            j.src_stride = I.pitch[l - 1];
            j.dst = base + I.off_img[l];
            j.dst_stride = I.pitch[l];
            j.vec = 1;
            put(o, &j, sizeof(j));
            o += sizeof(j);
        }
    o = mp->off_grad;
    for (int l = 0; l < mp->Lmax; ++l)
        for (const ImgPlan &I : mp->imgs) {
            if (I.L <= l)
                continue;
            ImageJob j;
            memset(&j, 0, sizeof(j));
            j.src = (const uint8_t *)(base + I.off_img[l]);
            j.w = I.w[l];
            j.h = I.h[l];
            j.src_stride = I.pitch[l];
            j.dst = base + I.off_field[l];
            j.vec = 1;   // 256-byte aligned buffers, 16-byte pitches
            put(o, &j, sizeof(j));
            o += sizeof(j);
        }
    o = mp->off_gtop;
    for (const TopField &t : mp->tops) {
        const ImgPlan &I = mp->imgs[t.img];
        ImageJob j;
        memset(&j, 0, sizeof(j));
        j.src = (const uint8_t *)(base + I.off_img[t.level]);
        j.w = I.w[t.level];
        j.h = I.h[t.level];
        j.src_stride = I.pitch[t.level];
        j.dst = base + t.off;
        j.vec = 1;
        put(o, &j, sizeof(j));
        o += sizeof(j);
    }
    // scorer descriptors and tensor maps, in scheduling order
    int item = 0;
    for (int r = 0; r < np; ++r) {
        const PairPlan &q = mp->pp[mp->order[r]];
        const TopField &t = mp->tops[q.tf];
        alignas(64) unsigned char tm[128];
        if (!encode_pair_tmap(tm, base + t.off, mp->p.precision, t.wp, q.H, q.bxw, q.byw))
            return SAM_ERR_CUDA;
        put(mp->off_tmaps + (size_t)r * 128, tm, 128);
        const sam_model *m = mp->models[q.model];
        PairScore s;
        memset(&s, 0, sizeof(s));
        s.tmap = base + mp->off_tmaps + (size_t)r * 128;
        s.rot = m->dev[q.top].rot;
        s.bbox = m->dev[q.top].bbox;
        s.map = (float *)(base + q.off_map);
        s.n = q.n;
        s.nth = q.nth;
        s.W = q.W;
        s.H = q.H;
        s.tiles_x = q.tiles_x;
        s.tiles = q.tiles;
        s.bxw = q.bxw;
        s.byw = q.byw;
        s.inv_n = 1.0f / (float)q.n;
        s.thresh = prune_threshold(q.n, mp->p.min_score, mp->p.precision);
        s.emin = mp->p.early_termination ? edge_count_threshold(s.thresh, mp->p.precision) : 0;
        s.item_begin = item;
        item += q.items;
        s.job = mp->order[r];
        if (mp->hot) {
            s.hot_cnt = (unsigned *)(base + mp->off_counters) + 1 + 3 * (size_t)np;
            s.hot = (uint2 *)(base + mp->off_hot);
            s.hot_cap = (unsigned)mp->hot_cap;
            s.hot_thr = mp->p.precision == SAM_FP32 ? mp->p.min_score
                                                     : mp->p.min_score - rescore_delta(mp->p.precision);
        }
        put(mp->off_pairs + (size_t)r * sizeof(PairScore), &s, sizeof(s));
    }
    mp->total_items = item;
    // per-model level tables
    for (size_t mi = 0; mi < mp->models.size(); ++mi)
        put(mp->off_levels + mi * sizeof(LevelDev) * kMaxLevels, mp->models[mi]->dev, sizeof(LevelDev) * kMaxLevels);
    // candidate, refinement and NMS jobs, in caller order
    int *cnt = (int *)(base + mp->off_counters) + 1;
    for (int i = 0; i < np; ++i) {
        const PairPlan &q = mp->pp[i];
        CandJob c;
        memset(&c, 0, sizeof(c));
        c.map = (const float *)(base + q.off_map);
        c.nth = q.nth;
        c.ns = 1;
        c.gh = q.H;
        c.gw = q.W;
        c.cand = (Cand *)(base + q.off_cand);
        c.cap = q.cap;
        c.cnt = cnt + i;
        c.out_kyx = (int32_t *)(base + q.off_kyx);
        c.out_s = (float *)(base + q.off_cs);
        c.out_count = cnt + np + i;
        put(mp->off_cjobs + (size_t)i * sizeof(CandJob), &c, sizeof(c));
        const ImgPlan &I = mp->imgs[q.img];
        RescoreJob rs;
        memset(&rs, 0, sizeof(rs));
        rs.field = (const float2 *)(base + I.off_field[q.top]);
        rs.rot = mp->models[q.model]->dev[q.top].rot;
        rs.map = (float *)(base + q.off_map);
        rs.list = mp->hot ? nullptr : (unsigned *)(base + q.off_rescore + rescore_scratch_bytes(0));
        rs.count = (unsigned *)(cnt + 2 * np + i);
        rs.w = q.W;
        rs.h = q.H;
        rs.n = q.n;
        rs.nth = q.nth;
        rs.cap = (unsigned)std::min<size_t>(q.map_img, 0xFFFFFFFFu);
        put(mp->off_rsjobs + (size_t)i * sizeof(RescoreJob), &rs, sizeof(rs));
        RefineJob rj;
        memset(&rj, 0, sizeof(rj));
        rj.L = (const LevelDev *)(base + mp->off_levels + (size_t)q.model * sizeof(LevelDev) * kMaxLevels);
        for (int l = 0; l < I.L; ++l) {
            rj.field[l] = (const float2 *)(base + I.off_field[l]);
            rj.w[l] = I.w[l];
            rj.h[l] = I.h[l];
        }
        rj.top = q.top;
        rj.step_x = 1;
        rj.step_y = 1;
        rj.polarity = mp->models[q.model]->p.polarity;
        rj.min_score = mp->p.min_score;
        rj.kyx = c.out_kyx;
        rj.cs = c.out_s;
        rj.count = c.out_count;
        rj.refined = (float4 *)(base + q.off_refined);
        rj.nscales = 1;
        put(mp->off_rjobs + (size_t)i * sizeof(RefineJob), &rj, sizeof(rj));
        NmsJob nj;
        memset(&nj, 0, sizeof(nj));
        nj.refined = rj.refined;
        nj.count = c.out_count;
        nj.w0 = I.w[0];
        nj.h0 = I.h[0];
        nj.min_side = std::min(mp->models[q.model]->lv[0].tw, mp->models[q.model]->lv[0].th);
        nj.max_out = mp->p.max_detections;
        nj.angle_step = mp->models[q.model]->p.angle_step_deg;
        nj.nang0 = mp->models[q.model]->ntheta0;
        nj.out = (sam_pose *)(base + q.off_out);
        nj.n_out = (int *)(base + q.off_nout);
        put(mp->off_njobs + (size_t)i * sizeof(NmsJob), &nj, sizeof(nj));
    }
    MU_CU(cudaMemcpy(base + mp->off_desc, h.data(), h.size(), cudaMemcpyHostToDevice));
    return SAM_OK;
}

// The launch sequence of one run (captured into the graph).
sam_status enqueue_run(sam_multi *mp, cudaStream_t st) {
    char *base = (char *)mp->base;
    const int np = (int)mp->pp.size();
    MU_CU(cudaMemsetAsync(base + mp->off_counters, 0, sizeof(int) * (3 + 3 * (size_t)np), st));
    size_t o = mp->off_pyr;
    for (int l = 1; l < mp->Lmax; ++l) {
        const int n = mp->pyr_count[l];
        MU_CU(launch_pyramid_jobs((const ImageJob *)(base + o), n, mp->max_w0 >> (l - 1), mp->max_h0 >> (l - 1), st));
        o += (size_t)n * sizeof(ImageJob);
    }
    o = mp->off_grad;
    for (int l = 0; l < mp->Lmax; ++l) {
        const int n = mp->grad_count[l];
        MU_CU(launch_gradient_jobs((const ImageJob *)(base + o), n, mp->max_w0 >> l, mp->max_h0 >> l,
                                   mp->models[0]->p.low, SAM_FP32, SAM_LAYOUT_PIXEL, st));
        o += (size_t)n * sizeof(ImageJob);
    }
    MU_CU(launch_gradient_jobs((const ImageJob *)(base + mp->off_gtop), (int)mp->tops.size(), mp->max_w0, mp->max_h0,
                               mp->models[0]->p.low, mp->p.precision, SAM_LAYOUT_PAIRS, st));
    MU_CU(launch_score_pairs((const PairScore *)(base + mp->off_pairs), np, mp->total_items, mp->p.precision,
                             mp->p.neighbourhood, mp->models[0]->p.polarity, mp->p.early_termination, mp->cfg,
                             mp->window_bytes, mp->bitmap_bytes, (unsigned *)(base + mp->off_counters), st));
    const unsigned *hot_cnt = (const unsigned *)(base + mp->off_counters) + 1 + 3 * (size_t)np;
    const uint2 *hot = (const uint2 *)(base + mp->off_hot);
    if (mp->hot && mp->p.precision != SAM_FP32) {
        MU_CU(launch_candidates_hot16_jobs((const CandJob *)(base + mp->off_cjobs),
                                           (const RescoreJob *)(base + mp->off_rsjobs), np, mp->p.min_score,
                                           rescore_delta(mp->p.precision), mp->p.top_k, mp->p.neighbourhood,
                                           mp->models[0]->p.polarity, hot_cnt, hot, (unsigned)mp->hot_cap,
                                           (unsigned *)(base + mp->off_counters) + 2 + 3 * (size_t)np,
                                           (unsigned *)(base + mp->off_pass), st));
    } else if (mp->hot) {
        MU_CU(launch_candidates_hot_jobs((const CandJob *)(base + mp->off_cjobs), np, mp->p.min_score, mp->p.top_k,
                                         hot_cnt, hot, (unsigned)mp->hot_cap, st));
    } else {
        if (mp->p.precision != SAM_FP32)
            MU_CU(launch_rescore_jobs((const RescoreJob *)(base + mp->off_rsjobs), np, mp->max_map,
                                      mp->p.neighbourhood, mp->models[0]->p.polarity, mp->p.min_score,
                                      mp->p.precision, st));
        MU_CU(launch_candidates_jobs((const CandJob *)(base + mp->off_cjobs), np, mp->max_map, mp->p.min_score,
                                     mp->p.top_k, st));
    }
    MU_CU(launch_refine_jobs((const RefineJob *)(base + mp->off_rjobs), np, mp->p.top_k, mp->p.neighbourhood, st));
    MU_CU(launch_nms_jobs((const NmsJob *)(base + mp->off_njobs), np, mp->p.top_k, st));
    return SAM_OK;
}

sam_status rebuild(sam_multi *mp) {
    if (!plan_tiling(mp))
        return SAM_ERR_ARG;
    sam_status s = upload_descriptors(mp);
    if (s != SAM_OK)
        return s;
    if (mp->exec) {
        cudaGraphExecDestroy(mp->exec);
        mp->exec = nullptr;
    }
    if (mp->graph) {
        cudaGraphDestroy(mp->graph);
        mp->graph = nullptr;
    }
    mp->dirty = false;
    return SAM_OK;
}

sam_status capture(sam_multi *mp, cudaStream_t st) {
    cudaStream_t cs = nullptr;
    MU_CU(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    const long long k0 = sam_kernel_launches();
    sam_status s = SAM_OK;
    // relaxed: the launchers query occupancy and set function attributes
    if (cudaStreamBeginCapture(cs, cudaStreamCaptureModeRelaxed) != cudaSuccess) {
        cudaStreamDestroy(cs);
        return SAM_ERR_CUDA;
    }
    s = enqueue_run(mp, cs);
    cudaGraph_t g = nullptr;
    const cudaError_t e = cudaStreamEndCapture(cs, &g);
    cudaStreamDestroy(cs);
    if (s != SAM_OK || e != cudaSuccess) {
        if (g)
            cudaGraphDestroy(g);
        return s != SAM_OK ? s : SAM_ERR_CUDA;
    }
    mp->graph_kernels = sam_kernel_launches() - k0;
    cudaGraphExec_t ex = nullptr;
    if (cudaGraphInstantiate(&ex, g, 0) != cudaSuccess) {
        cudaGraphDestroy(g);
        return SAM_ERR_CUDA;
    }
    mp->graph = g;
    mp->exec = ex;
    (void)st;
    return SAM_OK;
}

}  // namespace
}  // namespace sam

using namespace sam;

extern "C" {

sam_status sam_multi_create(sam_model *const *models, int n_models, const int32_t *image_sizes, int n_images,
                            const sam_pair *pairs, int n_pairs, const sam_detect_params *params, sam_multi **out) {
    if (!out)
        return SAM_ERR_ARG;
    *out = nullptr;
    if (!models || n_models < 1 || !image_sizes || n_images < 1 || !pairs || n_pairs < 1 || !params ||
        params->step_x != 1 || params->step_y != 1 || (params->neighbourhood != 1 && params->neighbourhood != 3) ||
        params->top_k < 1 || params->top_k > kMaxTopK || params->max_detections < 1 ||
        params->max_detections > kMaxTopK || params->precision < SAM_FP32 || params->precision > SAM_FP16)
        return SAM_ERR_ARG;
    for (int i = 0; i < n_models; ++i)
        if (!models[i] || models[i]->p.low != models[0]->p.low || models[i]->p.polarity != models[0]->p.polarity ||
            models[i]->nscales != 1 || models[i]->scale_min != 1.0)   // plans take rigid models
            return SAM_ERR_ARG;   // one edge threshold and polarity per plan
    sam_multi *mp = new (std::nothrow) sam_multi();
    if (!mp)
        return SAM_ERR_NOMEM;
    mp->models.assign(models, models + n_models);
    mp->p = *params;
    for (int i = 0; i < n_models; ++i) {
        const sam_status s = upload_model(models[i]);
        if (s != SAM_OK) {
            delete mp;
            return s;
        }
    }
    cudaGetDevice(&mp->device);
    mp->imgs.resize(n_images);
    for (int i = 0; i < n_images; ++i) {
        ImgPlan &I = mp->imgs[i];
        I.w[0] = image_sizes[2 * i];
        I.h[0] = image_sizes[2 * i + 1];
        if (I.w[0] < 1 || I.h[0] < 1) {
            delete mp;
            return SAM_ERR_ARG;
        }
    }
    mp->pp.resize(n_pairs);
    for (int i = 0; i < n_pairs; ++i) {
        const sam_pair &pr = pairs[i];
        if (pr.image < 0 || pr.image >= n_images || pr.model < 0 || pr.model >= n_models) {
            delete mp;
            return SAM_ERR_ARG;
        }
        ImgPlan &I = mp->imgs[pr.image];
        const int L = models[pr.model]->levels;
        if ((I.w[0] >> (L - 1)) < 1 || (I.h[0] >> (L - 1)) < 1) {
            delete mp;
            return SAM_ERR_ARG;
        }
        I.L = std::max(I.L, L);
        PairPlan &q = mp->pp[i];
        q.img = pr.image;
        q.model = pr.model;
        q.top = L - 1;
    }
    // buffers: images and FP32 fields per level, pairs-layout top fields, per-pair maps and outputs
    size_t off = 0;
    for (ImgPlan &I : mp->imgs) {
        for (int l = 0; l < I.L; ++l) {
            if (l > 0) {
                I.w[l] = I.w[l - 1] / 2;
                I.h[l] = I.h[l - 1] / 2;
            }
            I.pitch[l] = (I.w[l] + 15) & ~15;
            I.off_img[l] = off;
            off += al((size_t)I.pitch[l] * I.h[l]);
            I.field_px[l] = (size_t)I.w[l] * I.h[l];
            I.off_field[l] = off;
            off += al(I.field_px[l] * 8);
        }
        mp->max_w0 = std::max(mp->max_w0, I.w[0]);
        mp->max_h0 = std::max(mp->max_h0, I.h[0]);
        mp->Lmax = std::max(mp->Lmax, I.L);
    }
    const size_t esz = params->precision == SAM_FP32 ? 8 : 4;
    for (PairPlan &q : mp->pp) {
        int tf = -1;
        for (size_t t = 0; t < mp->tops.size(); ++t)
            if (mp->tops[t].img == q.img && mp->tops[t].level == q.top)
                tf = (int)t;
        if (tf < 0) {
            const ImgPlan &I = mp->imgs[q.img];
            TopField t;
            t.img = q.img;
            t.level = q.top;
            t.wp = field_pitch(I.w[q.top], SAM_LAYOUT_PAIRS);
            t.px = (size_t)t.wp * I.h[q.top];
            t.off = off;
            off += al(t.px * esz);
            mp->tops.push_back(t);
            tf = (int)mp->tops.size() - 1;
        }
        q.tf = tf;
        const ImgPlan &I = mp->imgs[q.img];
        const sam_model *m = models[q.model];
        q.W = I.w[q.top];
        q.H = I.h[q.top];
        q.nth = m->lv[q.top].ntheta;
        q.n = m->lv[q.top].n;
        q.map_img = (size_t)q.nth * q.W * q.H;
        q.off_map = off;
        off += al(q.map_img * 4);
        mp->max_map = std::max(mp->max_map, q.map_img);
        q.cap = cand_cap(q.nth, q.H, q.W);
        q.off_cand = off;
        off += al(q.cap * sizeof(Cand));
        const int K = params->top_k;
        q.off_kyx = off;
        off += al((size_t)3 * K * 4);
        q.off_cs = off;
        off += al((size_t)K * 4);
        q.off_refined = off;
        off += al((size_t)K * 16);
        q.off_out = off;
        off += al((size_t)params->max_detections * sizeof(sam_pose));
        q.off_nout = off;
        off += al(4);
        mp->pose_points += (long long)q.map_img * q.n;
    }
    // hot list: every pose of every map for a 16-bit field (the FP32
    // decision must see all poses within the storage bound of min_score),
    // a sixteenth for FP32 (an overflow sends candidate extraction back to
    // the whole maps); entries {pair, map index} of 32 bits each.  Plans
    // too large for 32-bit counts rescore every map as before.
    size_t poses = 0;
    bool idx32 = true;
    for (const PairPlan &q : mp->pp) {
        poses += q.map_img;
        idx32 = idx32 && q.map_img <= 0xFFFFFFFFull;
    }
    mp->hot_cap = params->precision == SAM_FP32 ? std::min(poses, std::max<size_t>(65536, poses / 16)) : poses;
    mp->hot = idx32 && mp->hot_cap <= 0xFFFFFFFFull;
    if (mp->hot) {
        mp->off_hot = off;
        off += al(mp->hot_cap * 8);
        mp->off_pass = off;   // the 16-bit candidate filter's pass list
        if (params->precision != SAM_FP32)
            off += al(mp->hot_cap * 4);
    }
    for (PairPlan &q : mp->pp) {
        q.off_rescore = off;
        if (params->precision != SAM_FP32 && !mp->hot)
            off += al(rescore_scratch_bytes(q.map_img));
    }
    // counters: work counter, candidate counts, output counts, rescore
    // counts (one per pair each), hot-list counter, pass-list counter
    mp->off_counters = off;
    off += al(sizeof(int) * (3 + 3 * (size_t)n_pairs));
    // descriptors
    mp->off_desc = off;
    mp->pyr_count.assign(mp->Lmax, 0);
    mp->grad_count.assign(mp->Lmax, 0);
    size_t n_pyr = 0, n_grad = 0;
    for (int l = 0; l < mp->Lmax; ++l)
        for (const ImgPlan &I : mp->imgs)
            if (I.L > l) {
                ++mp->grad_count[l];
                ++n_grad;
                if (l > 0) {
                    ++mp->pyr_count[l];
                    ++n_pyr;
                }
            }
    auto take = [&](size_t bytes) {
        const size_t o = off;
        off += al(bytes);
        return o;
    };
    mp->off_pyr = take(n_pyr * sizeof(ImageJob));
    mp->off_grad = take(n_grad * sizeof(ImageJob));
    mp->off_gtop = take(mp->tops.size() * sizeof(ImageJob));
    mp->off_pairs = take((size_t)n_pairs * sizeof(PairScore));
    mp->off_tmaps = take((size_t)n_pairs * 128);
    mp->off_cjobs = take((size_t)n_pairs * sizeof(CandJob));
    mp->off_rsjobs = take((size_t)n_pairs * sizeof(RescoreJob));
    mp->off_rjobs = take((size_t)n_pairs * sizeof(RefineJob));
    mp->off_njobs = take((size_t)n_pairs * sizeof(NmsJob));
    mp->off_levels = take((size_t)n_models * sizeof(LevelDev) * kMaxLevels);
    mp->desc_bytes = off - mp->off_desc;
    mp->bytes = off;
    if (cudaMalloc(&mp->base, mp->bytes) != cudaSuccess) {
        cudaGetLastError();
        delete mp;
        return SAM_ERR_NOMEM;
    }
    mp->cfg = TileConfig();
    mp->cfg.sx = 1;
    mp->cfg.sy = 1;
    mp->cfg.tg = 3;
    mp->cfg.warps = 8;
    const sam_status s = rebuild(mp);
    if (s != SAM_OK) {
        sam_multi_free(mp);
        return s;
    }
    *out = mp;
    return SAM_OK;
}

void sam_multi_free(sam_multi *mp) {
    if (!mp)
        return;
    if (mp->exec)
        cudaGraphExecDestroy(mp->exec);
    if (mp->graph)
        cudaGraphDestroy(mp->graph);
    if (mp->base)
        cudaFree(mp->base);
    delete mp;
}

uint8_t *sam_multi_image(sam_multi *mp, int i, int *pitch) {
    if (!mp || i < 0 || i >= (int)mp->imgs.size())
        return nullptr;
    if (pitch)
        *pitch = mp->imgs[i].pitch[0];
    return (uint8_t *)mp->base + mp->imgs[i].off_img[0];
}

sam_status sam_multi_set_image(sam_multi *mp, int i, const uint8_t *src, int stride, int on_device, void *stream) {
    if (!mp || !src || i < 0 || i >= (int)mp->imgs.size() || stride < mp->imgs[i].w[0])
        return SAM_ERR_ARG;
    const ImgPlan &I = mp->imgs[i];
    MU_CU(cudaMemcpy2DAsync((char *)mp->base + I.off_img[0], I.pitch[0], src, stride, I.w[0], I.h[0],
                            on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, (cudaStream_t)stream));
    return SAM_OK;
}

sam_status sam_multi_set_tiling(sam_multi *mp, int sx, int sy, int tg, int warps, int cols) {
    if (!mp || sx < 1 || sx > 8 || sy < 1 || sy > 8 || tg < 1 || tg > 4096 || (warps != 4 && warps != 8) ||
        (cols != 6 && cols != 10))
        return SAM_ERR_ARG;
    const TileConfig old = mp->cfg;
    mp->cfg.sx = sx;
    mp->cfg.sy = sy;
    mp->cfg.tg = tg;
    mp->cfg.warps = warps;
    mp->cfg.tc = cols;
    const sam_status s = rebuild(mp);
    if (s != SAM_OK) {
        mp->cfg = old;
        rebuild(mp);
    }
    return s;
}

sam_status sam_multi_run(sam_multi *mp, void *stream, sam_pose *out, int capacity, int *n_out) {
    if (!mp || (capacity > 0 && !out) || capacity < 0 || !n_out)
        return SAM_ERR_ARG;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev != mp->device)
        return SAM_ERR_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    sam_status s = SAM_OK;
    if (mp->dirty && (s = rebuild(mp)) != SAM_OK)
        return s;
    if (!mp->exec && (s = capture(mp, st)) != SAM_OK)
        return s;
    MU_CU(cudaGraphLaunch(mp->exec, st));
    count_launches((int)mp->graph_kernels);
    const int np = (int)mp->pp.size();
    const int md = mp->p.max_detections;
    std::vector<sam_pose> poses((size_t)np * md);
    std::vector<int> nout(np);
    for (int i = 0; i < np; ++i) {
        MU_CU(cudaMemcpyAsync(poses.data() + (size_t)i * md, (char *)mp->base + mp->pp[i].off_out,
                              (size_t)md * sizeof(sam_pose), cudaMemcpyDeviceToHost, st));
        MU_CU(cudaMemcpyAsync(&nout[i], (char *)mp->base + mp->pp[i].off_nout, sizeof(int), cudaMemcpyDeviceToHost,
                              st));
    }
    int dev_err = 0;
    MU_CU(score_error_flag_async(&dev_err, st));
    MU_CU(cudaStreamSynchronize(st));
    if (dev_err) {
        score_error_clear(st);
        cudaStreamSynchronize(st);
        return SAM_ERR_TIMEOUT;
    }
    for (int i = 0; i < np; ++i) {
        const int n = std::min(nout[i], capacity);
        if (n > 0)
            memcpy(out + (size_t)i * capacity, poses.data() + (size_t)i * md, (size_t)n * sizeof(sam_pose));
        n_out[i] = n;
    }
    return SAM_OK;
}

sam_status sam_multi_pair_map(const sam_multi *mp, int pair, float *dst, size_t capacity, int *nth, int *gh,
                              int *gw, int *level, void *stream) {
    if (!mp || !mp->base || pair < 0 || pair >= (int)mp->pp.size())
        return SAM_ERR_ARG;
    const sam::PairPlan &q = mp->pp[pair];
    if (nth)
        *nth = q.nth;
    if (gh)
        *gh = q.H;
    if (gw)
        *gw = q.W;
    if (level)
        *level = q.top;
    if (!dst)
        return SAM_OK;
    if (capacity < q.map_img)
        return SAM_ERR_ARG;
    MU_CU(cudaMemcpyAsync(dst, (const char *)mp->base + q.off_map, q.map_img * sizeof(float),
                          cudaMemcpyDeviceToDevice, (cudaStream_t)stream));
    return SAM_OK;
}

sam_status sam_multi_stats(const sam_multi *mp, long long *pose_points, long long *graph_kernels,
                           size_t *device_bytes) {
    if (!mp)
        return SAM_ERR_ARG;
    if (pose_points)
        *pose_points = mp->pose_points;
    if (graph_kernels)
        *graph_kernels = mp->graph_kernels;
    if (device_bytes)
        *device_bytes = mp->bytes;
    return SAM_OK;
}

sam_status sam_multi_autotune(sam_multi *mp, void *stream, int32_t *cfg_out, float *ms_out, int max_out,
                              int *n_out) {
    if (!mp || !n_out || max_out < 0 || (max_out > 0 && (!cfg_out || !ms_out)))
        return SAM_ERR_ARG;
    *n_out = 0;
    cudaStream_t st = (cudaStream_t)stream;
    // fields once (the full sequence), then the scorer alone per tiling
    sam_status s = SAM_OK;
    if (mp->dirty && (s = rebuild(mp)) != SAM_OK)
        return s;
    if ((s = enqueue_run(mp, st)) != SAM_OK)
        return s;
    cudaEvent_t e0, e1;
    MU_CU(cudaEventCreate(&e0));
    MU_CU(cudaEventCreate(&e1));
    const TileConfig start = mp->cfg;
    TileConfig best = start;
    float best_ms = 1e30f;
    int n = 0;
    const int tgs[] = {1, 3, 5, 9, 15};
    for (int tc : {6, 10})
    for (int warps : {8, 4})
        for (int sy = 1; sy <= 2; ++sy)
            for (int sx = 1; sx <= 2; ++sx)
                for (int tg : tgs) {
                    mp->cfg.sx = sx;
                    mp->cfg.sy = sy;
                    mp->cfg.tg = tg;
                    mp->cfg.warps = warps;
                    mp->cfg.tc = tc;
                    if (rebuild(mp) != SAM_OK)
                        continue;
                    char *base = (char *)mp->base;
                    float ms = 0.f;
                    cudaError_t e = cudaSuccess;
                    for (int rep = 0; rep < 2 && e == cudaSuccess; ++rep) {
                        cudaMemsetAsync(base + mp->off_counters, 0, sizeof(int), st);
                        cudaEventRecord(e0, st);
                        e = launch_score_pairs((const PairScore *)(base + mp->off_pairs), (int)mp->pp.size(),
                                               mp->total_items, mp->p.precision, mp->p.neighbourhood,
                                               mp->models[0]->p.polarity, mp->p.early_termination, mp->cfg,
                                               mp->window_bytes, mp->bitmap_bytes, (unsigned *)(base + mp->off_counters), st);
                        cudaEventRecord(e1, st);
                        if (e == cudaSuccess && cudaEventSynchronize(e1) == cudaSuccess)
                            cudaEventElapsedTime(&ms, e0, e1);   // second repetition counts
                    }
                    if (e != cudaSuccess) {
                        cudaEventDestroy(e0);
                        cudaEventDestroy(e1);
                        mp->cfg = start;
                        rebuild(mp);
                        return SAM_ERR_CUDA;
                    }
                    if (n < max_out) {
                        cfg_out[5 * n] = sx;
                        cfg_out[5 * n + 1] = sy;
                        cfg_out[5 * n + 2] = tg;
                        cfg_out[5 * n + 3] = warps;
                        cfg_out[5 * n + 4] = tc;
                        ms_out[n] = ms;
                    }
                    ++n;
                    if (ms < best_ms) {
                        best_ms = ms;
                        best = mp->cfg;
                    }
                }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    mp->cfg = best;
    s = rebuild(mp);
    *n_out = std::min(n, max_out);
    return s;
}

}  // extern "C"
