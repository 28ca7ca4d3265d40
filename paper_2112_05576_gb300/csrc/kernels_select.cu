// Kernel (d): candidate extraction, top-K, coarse-to-fine refinement and
// non-maximum suppression.  The paper's search keeps the maximum-score pose
// (Sec. II); several instances need local maxima, refined level by level
// down the pyramid with the size-3 neighbouring search in x, y and theta.
//
// Every selection uses one total order: higher score first, then the
// smaller key (k * H + y) * W + x.  Ties therefore resolve identically on
// every run, independent of atomic ordering.
//
// Each stage has a device body shared by two entry points: a uniform batch
// (images of one size, one model) and a job list (per-image or per-pair
// descriptors in device memory, for batches of different sizes and models).

#include <float.h>

#include <algorithm>

#include <cooperative_groups.h>

#include "sam_internal.h"

namespace sam {
namespace {

constexpr int kSortCap = 2048;   // shared-memory sort buffer (entries)
constexpr int RTHREADS = 256;
constexpr int kRefineCluster = 4;   // CTAs per refined candidate

__device__ __forceinline__ bool beats(float sa, unsigned long long ka, float sb, unsigned long long kb) {
    return sa > sb || (sa == sb && ka < kb);
}

// ---------------------------------------------------------------------------
// local maxima
// ---------------------------------------------------------------------------

// Whether map entry idx is a strict local maximum >= min_score over its up to
// 26 neighbours in (theta circular, y, x); with ns > 1 scales the map's nth
// planes are ns blocks of nth / ns angles (plane j * nang + k for scale j,
// angle k) and the neighbours, up to 80, also span scales j - 1 .. j + 1
// inside the grid (not circular).
__device__ __forceinline__ bool is_candidate(const float *__restrict__ map, int nth, int gh, int gw, float min_score,
                                             size_t idx, int ns) {
    const float s = map[idx];
    if (!(s >= min_score))
        return false;
    const size_t plane = (size_t)gh * gw;
    const int kk = (int)(idx / plane);
    const int r = (int)(idx - (size_t)kk * plane);
    const int y = r / gw, x = r - y * gw;
    const int nang = nth / ns;
    const int js = kk / nang, k = kk - js * nang;
    if (ns == 1) {
        // one scale: the 26 neighbours' values are loaded together (one
        // memory round trip), then compared
        float v[27];
#pragma unroll
        for (int q = 0; q < 27; ++q) {
            const int dk = q / 9 - 1, dy = (q / 3) % 3 - 1, dx = q % 3 - 1;
            const int y2 = y + dy, x2 = x + dx;
            const bool in = q != 13 && (dk == 0 || nang > 1) && y2 >= 0 && y2 < gh && x2 >= 0 && x2 < gw;
            const int k2 = (k + dk + nang) % nang;
            v[q] = in ? __ldg(map + (size_t)k2 * plane + (size_t)y2 * gw + x2) : -INFINITY;
        }
        bool ok = true;
#pragma unroll
        for (int q = 0; q < 27; ++q) {
            const int dk = q / 9 - 1, dy = (q / 3) % 3 - 1, dx = q % 3 - 1;
            const int y2 = y + dy, x2 = x + dx;
            const bool in = q != 13 && (dk == 0 || nang > 1) && y2 >= 0 && y2 < gh && x2 >= 0 && x2 < gw;
            const size_t j = (size_t)((k + dk + nang) % nang) * plane + (size_t)y2 * gw + x2;
            ok = ok && (!in || j == idx || beats(s, idx, v[q], j));
        }
        return ok;
    }
    for (int dj = -1; dj <= 1; ++dj) {
        const int j2 = js + dj;
        if (j2 < 0 || j2 >= ns)
            continue;
        for (int dk = -1; dk <= 1; ++dk) {
            if (dk != 0 && nang == 1)
                continue;
            const int k2 = j2 * nang + (k + dk + nang) % nang;
            for (int dy = -1; dy <= 1; ++dy) {
                const int y2 = y + dy;
                if (y2 < 0 || y2 >= gh)
                    continue;
                for (int dx = -1; dx <= 1; ++dx) {
                    const int x2 = x + dx;
                    if (x2 < 0 || x2 >= gw)
                        continue;
                    const size_t j = (size_t)k2 * plane + (size_t)y2 * gw + x2;
                    if (j == idx)
                        continue;
                    if (!beats(s, idx, map[j], j))
                        return false;
                }
            }
        }
    }
    return true;
}

__device__ __forceinline__ void push_candidate(const float *map, size_t idx, Cand *cand, size_t cap, int *cnt) {
    const int pos = atomicAdd(cnt, 1);
    if ((size_t)pos < cap) {
        Cand c;
        c.s = map[idx];
        c.pad = 0;
        c.key = idx;
        cand[pos] = c;
    }
}

// Candidates (the best pose of Sec. II, generalised to every strict 3x3x3
// local maximum at or above min_score) of `count` equal maps, image
// blockIdx.y; appended to the image's list by atomic counter.
// The map is read four entries at a time (one 16-byte load, four loads in
// flight per thread); almost every entry is below min_score (or -inf where
// early termination pruned it), and only the others are tested against
// their neighbours.  vec: the map (and every image's map) is 16-byte aligned.
__global__ void local_max_kernel(const float *__restrict__ map, size_t map_img, int nth, int gh, int gw,
                                 float min_score, Cand *__restrict__ cand, size_t cap, int *__restrict__ cnt,
                                 int ns, int vec) {
    const int img = blockIdx.y;
    map += (size_t)img * map_img;
    cand += (size_t)img * cap;
    cnt += img;
    const size_t total = (size_t)nth * gh * gw;
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    size_t idx0 = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    size_t scalar_from = 0;
    if (vec) {
        const size_t total4 = total / 4;
        const float4 *m4 = reinterpret_cast<const float4 *>(map);
        for (size_t i4 = idx0; i4 < total4; i4 += 4 * stride) {
            float4 v[4];
#pragma unroll
            for (int u = 0; u < 4; ++u)
                v[u] = i4 + u * stride < total4 ? __ldg(m4 + i4 + u * stride)
                                                 : make_float4(-INFINITY, -INFINITY, -INFINITY, -INFINITY);
            // the entries at or above min_score (rare), then one call site
            uint32_t hit = 0u;
#pragma unroll
            for (int u = 0; u < 4; ++u)
                hit |= (v[u].x >= min_score ? 1u : 0u) << (4 * u) | (v[u].y >= min_score ? 2u : 0u) << (4 * u) |
                       (v[u].z >= min_score ? 4u : 0u) << (4 * u) | (v[u].w >= min_score ? 8u : 0u) << (4 * u);
            while (hit) {
                const int b = __ffs(hit) - 1;
                hit &= hit - 1u;
                const size_t idx = 4 * (i4 + (size_t)(b >> 2) * stride) + (b & 3);
                if (is_candidate(map, nth, gh, gw, min_score, idx, ns))
                    push_candidate(map, idx, cand, cap, cnt);
            }
        }
        scalar_from = 4 * total4;   // the last total % 4 entries
    }
    for (size_t idx = scalar_from + idx0; idx < total; idx += stride)
        if (is_candidate(map, nth, gh, gw, min_score, idx, ns))
            push_candidate(map, idx, cand, cap, cnt);
}

// Candidates of `n_img` equal maps from a scorer's hot list: every pose the
// scorer stored at or above the list's threshold (at most min_score), so
// every entry at or above min_score is listed and the test runs on the
// listed poses only.  A list that overflowed (count above hot_cap) is
// ignored and every map scanned instead.  Grid-stride over the entries.
__global__ void local_max_hot_kernel(const float *__restrict__ map, size_t map_img, int nth, int gh, int gw,
                                     float min_score, Cand *__restrict__ cand, size_t cap, int *__restrict__ cnt,
                                     int ns, const unsigned *__restrict__ hot_cnt, const uint2 *__restrict__ hot,
                                     unsigned hot_cap, int n_img) {
    const unsigned total = *hot_cnt;
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    const size_t tid = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (total <= hot_cap) {
        for (size_t e = tid; e < total; e += stride) {
            const uint2 h = hot[e];
            const float *mi = map + (size_t)h.x * map_img;
            if (is_candidate(mi, nth, gh, gw, min_score, h.y, ns))
                push_candidate(mi, h.y, cand + (size_t)h.x * cap, cap, cnt + h.x);
        }
        return;
    }
    const size_t per = (size_t)nth * gh * gw;
    for (size_t g = tid; g < per * (size_t)n_img; g += stride) {
        const size_t img = g / per, idx = g - img * per;
        const float *mi = map + img * map_img;
        if (is_candidate(mi, nth, gh, gw, min_score, idx, ns))
            push_candidate(mi, idx, cand + img * cap, cap, cnt + img);
    }
}

// ---------------------------------------------------------------------------
// candidates of a map scored from a 16-bit field, decided in FP32
// ---------------------------------------------------------------------------
//
// The 16-bit map M16 is within delta (rescore_delta) of the FP32 score M32 at
// every pose it did not prune, and the poses it pruned are below min_score in
// FP32 too.  A pose p can be a strict local maximum of M32 at or above
// min_score only if (i) M16(p) >= min_score - delta, so it is on the hot
// list, and (ii) no neighbour q has M16(q) > M16(p) + 2 delta (else M32(q) >
// M16(p) + delta >= M32(p)).  For each pose passing both, one CTA computes
// M32 of the pose and of all its neighbours (per model point and angle one
// (NB + 2)^2 window of field pixels serves the nine translations) and keeps
// the pose if it beats every neighbour under the total order.  M32 of a pose
// is the same function of the pose in every CTA (point i on thread i mod
// 256, serial per thread, shuffle tree per warp, warps added in order), so
// neighbouring CTAs agree.  The candidates are those of the FP32 map made of
// these values.

constexpr int kC16Threads = 256;

// What the 16-bit candidate test needs of one image's (or pair's) map.
struct C16View {
    const float *map;      // [nth][gh][gw]
    int nth, gh, gw, ns;
    const float2 *field;   // FP32 pixel-layout field of the scored level (w x h, pitch w)
    int w, h;
    const RotPt *rot;      // [nth][n]
    int n;
    Cand *cand;            // the candidate list and its counter
    size_t cap;
    int *cnt;
};

struct Cand16Args {
    const float *map;
    size_t map_img;
    int nth, gh, gw, ns;
    float min_score, delta;
    const unsigned *hot_cnt;
    const uint2 *hot;
    unsigned hot_cap;
    const float2 *field;   // FP32 pixel-layout field of the scored level
    size_t field_img_px;
    int w, h;
    const RotPt *rot;      // [nth][n]
    int n, polarity;
    Cand *cand;
    size_t cap;
    int *cnt;
    unsigned *pass_cnt;    // poses passing the filter (zeroed before the launch) and their hot entries
    unsigned *pass_list;
};

// Whether no neighbour of map entry idx (the neighbourhood of is_candidate)
// holds a value above `above`.
__device__ __forceinline__ bool no_neighbour_above(const float *__restrict__ map, int nth, int gh, int gw, size_t idx,
                                                   int ns, float above) {
    const size_t plane = (size_t)gh * gw;
    const int kk = (int)(idx / plane);
    const int r = (int)(idx - (size_t)kk * plane);
    const int y = r / gw, x = r - y * gw;
    const int nang = nth / ns;
    const int js = kk / nang, k = kk - js * nang;
    if (ns == 1) {
        // one scale: the 26 neighbours loaded together, then compared
        bool ok = true;
#pragma unroll
        for (int q = 0; q < 27; ++q) {
            const int dk = q / 9 - 1, dy = (q / 3) % 3 - 1, dx = q % 3 - 1;
            const int y2 = y + dy, x2 = x + dx;
            const bool in = q != 13 && (dk == 0 || nang > 1) && y2 >= 0 && y2 < gh && x2 >= 0 && x2 < gw;
            const int k2 = (k + dk + nang) % nang;
            const float v = in ? __ldg(map + (size_t)k2 * plane + (size_t)y2 * gw + x2) : -INFINITY;
            ok = ok && !(v > above);
        }
        return ok;
    }
    for (int dj = -1; dj <= 1; ++dj) {
        const int j2 = js + dj;
        if (j2 < 0 || j2 >= ns)
            continue;
        for (int dk = -1; dk <= 1; ++dk) {
            if (dk != 0 && nang == 1)
                continue;
            const int k2 = j2 * nang + (k + dk + nang) % nang;
            for (int dy = -1; dy <= 1; ++dy) {
                const int y2 = y + dy;
                if (y2 < 0 || y2 >= gh)
                    continue;
                for (int dx = -1; dx <= 1; ++dx) {
                    const int x2 = x + dx;
                    if (x2 < 0 || x2 >= gw)
                        continue;
                    const size_t j = (size_t)k2 * plane + (size_t)y2 * gw + x2;
                    if (j != idx && map[j] > above)
                        return false;
                }
            }
        }
    }
    return true;
}

// Filter: every hot entry (entries {view index, map index}; view(i)
// describes map i) at or above min_score - delta whose score is within
// 2 delta of every neighbour's goes to the pass list (grid-stride, one
// thread per entry).
template <typename ViewAt>
__device__ __forceinline__ void cand16_filter(const unsigned *hot_cnt, const uint2 *hot, unsigned hot_cap,
                                              float min_score, float delta, ViewAt view, unsigned *pass_cnt,
                                              unsigned *pass_list) {
    const unsigned total = min(*hot_cnt, hot_cap);
    const float up = 2.f * delta;
    for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
        const uint2 hv = hot[e];
        const C16View V = view(hv.x);
        const float v = V.map[hv.y];
        if (v >= min_score - delta && no_neighbour_above(V.map, V.nth, V.gh, V.gw, hv.y, V.ns, v + up))
            pass_list[atomicAdd(pass_cnt, 1u)] = (unsigned)e;
    }
}

// Decision: one CTA per listed pose (CTA b the entries b, b + grid, ...)
// computes the FP32 scores of the pose and its neighbours and keeps the pose
// if it beats all of them.  All threads of the CTA call it.
template <int NB, typename ViewAt>
__device__ __forceinline__ void cand16_eval(const uint2 *hot, const unsigned *pass_cnt, const unsigned *pass_list,
                                            float min_score, int polarity, ViewAt view) {
    __shared__ float s_red[kC16Threads / 32][81];   // per-warp sums: plane d, translation q at 9 d + q
    __shared__ float s_val[81];
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const unsigned np = *pass_cnt;
    for (unsigned ip = blockIdx.x; ip < np; ip += gridDim.x) {
        const uint2 hv = hot[pass_list[ip]];
        const C16View V = view(hv.x);
        const size_t plane = (size_t)V.gh * V.gw;
        const int nang = V.nth / V.ns;
        const size_t idx = hv.y;
        const int kk = (int)(idx / plane);
        const int rem = (int)(idx - (size_t)kk * plane);
        const int y = rem / V.gw, x = rem - y * V.gw;
        const int js = kk / nang, k = kk - js * nang;
        // the neighbourhood's planes (scale j2, angle k2), the same list
        // on every thread; dc is the pose's own plane
        int kl[9];
        int npl = 0, dc = 0;
        for (int dj = -1; dj <= 1; ++dj) {
            const int j2 = js + dj;
            if (j2 < 0 || j2 >= V.ns)
                continue;
            for (int dk = -1; dk <= 1; ++dk) {
                if (dk != 0 && nang == 1)
                    continue;
                if (dj == 0 && dk == 0)
                    dc = npl;
                kl[npl++] = j2 * nang + (k + dk + nang) % nang;
            }
        }
        const float2 *F = V.field;
        for (int d = 0; d < npl; ++d) {
            const RotPt *P = V.rot + (size_t)kl[d] * V.n;
            float acc[9];
#pragma unroll
            for (int q = 0; q < 9; ++q)
                acc[q] = 0.f;
            for (int i = t; i < V.n; i += kC16Threads) {
                const RotPt p = P[i];
                const int bxp = x + p.ox, byp = y + p.oy;
                constexpr int D = NB + 2;
                float dd[D][D];
#pragma unroll
                for (int yy = 0; yy < D; ++yy)
#pragma unroll
                    for (int xx = 0; xx < D; ++xx) {
                        const int X = bxp + xx - D / 2, Y = byp + yy - D / 2;
                        float v = 0.f;
                        if (X >= 0 && Y >= 0 && X < V.w && Y < V.h) {
                            const float2 f = __ldg(F + (size_t)Y * V.w + X);
                            v = fmaf(p.px, f.x, p.py * f.y);
                            if (polarity)
                                v = fabsf(v);
                        }
                        dd[yy][xx] = v;
                    }
#pragma unroll
                for (int ty = 0; ty < 3; ++ty)
#pragma unroll
                    for (int tx = 0; tx < 3; ++tx) {
                        float mx = -INFINITY;
#pragma unroll
                        for (int b = 0; b < NB; ++b)
#pragma unroll
                            for (int aa = 0; aa < NB; ++aa)
                                mx = fmaxf(mx, dd[ty + b][tx + aa]);
                        acc[ty * 3 + tx] += mx;
                    }
            }
#pragma unroll
            for (int q = 0; q < 9; ++q) {
                float v = acc[q];
#pragma unroll
                for (int o = 16; o > 0; o >>= 1)
                    v += __shfl_xor_sync(0xffffffffu, v, o);
                if (lane == 0)
                    s_red[warp][d * 9 + q] = v;
            }
        }
        __syncthreads();
        if (t < npl * 9) {
            float v = 0.f;
            for (int wv = 0; wv < kC16Threads / 32; ++wv)
                v += s_red[wv][t];
            s_val[t] = v / (float)V.n;
        }
        __syncthreads();
        if (t == 0) {
            const float sp = s_val[dc * 9 + 4];
            bool ok = sp >= min_score;
            for (int d = 0; d < npl && ok; ++d)
                for (int q = 0; q < 9; ++q) {
                    const int X = x + q % 3 - 1, Y = y + q / 3 - 1;
                    if (X < 0 || Y < 0 || X >= V.gw || Y >= V.gh)
                        continue;
                    const size_t key = (size_t)kl[d] * plane + (size_t)Y * V.gw + X;
                    if (key != idx && !beats(sp, idx, s_val[d * 9 + q], key)) {
                        ok = false;
                        break;
                    }
                }
            if (ok) {
                const int pos = atomicAdd(V.cnt, 1);
                if ((size_t)pos < V.cap) {
                    Cand c;
                    c.s = sp;
                    c.pad = 0;
                    c.key = idx;
                    V.cand[pos] = c;
                }
            }
        }
        __syncthreads();   // s_red and s_val are reused by the next pose
    }
}

// A 16-bit map's candidates: the single-model form (image = view index).
__device__ __forceinline__ C16View c16_view(const Cand16Args &a, unsigned img) {
    C16View v;
    v.map = a.map + (size_t)img * a.map_img;
    v.nth = a.nth;
    v.gh = a.gh;
    v.gw = a.gw;
    v.ns = a.ns;
    v.field = a.field + (size_t)img * a.field_img_px;
    v.w = a.w;
    v.h = a.h;
    v.rot = a.rot;
    v.n = a.n;
    v.cand = a.cand + (size_t)img * a.cap;
    v.cap = a.cap;
    v.cnt = a.cnt + img;
    return v;
}

__global__ void __launch_bounds__(256) cand16_filter_kernel(const Cand16Args a) {
    cand16_filter(a.hot_cnt, a.hot, a.hot_cap, a.min_score, a.delta, [&](unsigned i) { return c16_view(a, i); },
                  a.pass_cnt, a.pass_list);
}

template <int NB>
__global__ void __launch_bounds__(kC16Threads) cand16_eval_kernel(const Cand16Args a) {
    cand16_eval<NB>(a.hot, a.pass_cnt, a.pass_list, a.min_score, a.polarity,
                    [&](unsigned i) { return c16_view(a, i); });
}

// The job-list form: pair p's map and candidate list in cj[p], its FP32
// field and model points in rj[p].
__device__ __forceinline__ C16View c16_job_view(const CandJob *cj, const RescoreJob *rj, unsigned p) {
    const CandJob &c = cj[p];
    const RescoreJob &r = rj[p];
    C16View v;
    v.map = c.map;
    v.nth = c.nth;
    v.gh = c.gh;
    v.gw = c.gw;
    v.ns = c.ns;
    v.field = r.field;
    v.w = r.w;
    v.h = r.h;
    v.rot = r.rot;
    v.n = r.n;
    v.cand = c.cand;
    v.cap = c.cap;
    v.cnt = c.cnt;
    return v;
}

__global__ void __launch_bounds__(256) cand16_filter_jobs_kernel(const CandJob *__restrict__ cj,
                                                                 const RescoreJob *__restrict__ rj,
                                                                 const unsigned *hot_cnt, const uint2 *hot,
                                                                 unsigned hot_cap, float min_score, float delta,
                                                                 unsigned *pass_cnt, unsigned *pass_list) {
    cand16_filter(hot_cnt, hot, hot_cap, min_score, delta, [&](unsigned p) { return c16_job_view(cj, rj, p); },
                  pass_cnt, pass_list);
}

template <int NB>
__global__ void __launch_bounds__(kC16Threads) cand16_eval_jobs_kernel(const CandJob *__restrict__ cj,
                                                                       const RescoreJob *__restrict__ rj,
                                                                       const uint2 *hot, const unsigned *pass_cnt,
                                                                       const unsigned *pass_list, float min_score,
                                                                       int polarity) {
    cand16_eval<NB>(hot, pass_cnt, pass_list, min_score, polarity,
                    [&](unsigned p) { return c16_job_view(cj, rj, p); });
}

// Candidates of a job list's maps from the batch's hot list (entries {pair,
// map index}; the list's threshold at most min_score); if the list
// overflowed, every pair's map is scanned instead.
__global__ void local_max_hot_jobs_kernel(const CandJob *__restrict__ jobs, int n_jobs, float min_score,
                                          const unsigned *__restrict__ hot_cnt, const uint2 *__restrict__ hot,
                                          unsigned hot_cap) {
    const unsigned total = *hot_cnt;
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    const size_t tid = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (total <= hot_cap) {
        for (size_t e = tid; e < total; e += stride) {
            const uint2 h = hot[e];
            const CandJob &j = jobs[h.x];
            if (is_candidate(j.map, j.nth, j.gh, j.gw, min_score, h.y, j.ns))
                push_candidate(j.map, h.y, j.cand, j.cap, j.cnt);
        }
        return;
    }
    for (int p = 0; p < n_jobs; ++p) {
        const CandJob &j = jobs[p];
        const size_t per = (size_t)j.nth * j.gh * j.gw;
        for (size_t idx = tid; idx < per; idx += stride)
            if (is_candidate(j.map, j.nth, j.gh, j.gw, min_score, idx, j.ns))
                push_candidate(j.map, idx, j.cand, j.cap, j.cnt);
    }
}

// The same over a job list of maps of different sizes (job blockIdx.y).
__global__ void local_max_jobs_kernel(const CandJob *__restrict__ jobs, float min_score) {
    const CandJob j = jobs[blockIdx.y];
    const size_t total = (size_t)j.nth * j.gh * j.gw;
    for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
         idx += (size_t)gridDim.x * blockDim.x)
        if (is_candidate(j.map, j.nth, j.gh, j.gw, min_score, idx, j.ns))
            push_candidate(j.map, idx, j.cand, j.cap, j.cnt);
}

// Bitonic sort of n (power of two) entries in shared memory, best first.
__device__ void bitonic_sort(float *s, unsigned long long *key, int n) {
    for (int size = 2; size <= n; size <<= 1) {
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            for (int i = threadIdx.x; i < n / 2; i += blockDim.x) {
                const int lo = 2 * i - (i & (stride - 1));
                const int hi = lo + stride;
                const bool up = ((lo & size) == 0);   // ascending block = best first
                const bool swap = up ? beats(s[hi], key[hi], s[lo], key[lo]) : beats(s[lo], key[lo], s[hi], key[hi]);
                if (swap) {
                    const float ts = s[lo];
                    s[lo] = s[hi];
                    s[hi] = ts;
                    const unsigned long long tk = key[lo];
                    key[lo] = key[hi];
                    key[hi] = tk;
                }
            }
            __syncthreads();
        }
    }
}

// The best K of `total` candidates, by repeated sorts of the running top K
// plus the next chunk in shared memory.
__device__ void topk_body(const Cand *__restrict__ cand, int total, int K, int gh, int gw,
                          int32_t *__restrict__ out_kyx, float *__restrict__ out_s, int *__restrict__ out_count) {
    __shared__ float s[kSortCap];
    __shared__ unsigned long long key[kSortCap];
    const int chunk = kSortCap - K;
    int have = 0;   // valid entries at the front of the buffer (sorted)
    for (int start = 0; start < total || (start == 0 && total == 0); start += chunk) {
        const int take = min(chunk, total - start);
        const int used = have + max(take, 0);
        int n2 = 1;
        while (n2 < used)
            n2 <<= 1;
        for (int i = threadIdx.x; i < n2 - have; i += blockDim.x) {
            const int d = have + i;
            if (i < take) {
                const Cand c = cand[start + i];
                s[d] = c.s;
                key[d] = c.key;
            } else {
                s[d] = -INFINITY;
                key[d] = ~0ull;
            }
        }
        __syncthreads();
        if (n2 > 1)
            bitonic_sort(s, key, n2);
        have = min(K, used);
        __syncthreads();
        if (total == 0)
            break;
    }
    const size_t plane = (size_t)gh * gw;
    for (int i = threadIdx.x; i < K; i += blockDim.x) {
        if (i < have) {
            const unsigned long long kk = key[i];
            const int k = (int)(kk / plane);
            const int r = (int)(kk - (unsigned long long)k * plane);
            out_kyx[3 * i] = k;
            out_kyx[3 * i + 1] = r / gw;
            out_kyx[3 * i + 2] = r % gw;
            out_s[i] = s[i];
        }
    }
    if (threadIdx.x == 0)
        *out_count = have;
}

// Best K of each image's candidate list under the total order (one CTA per
// image).
__global__ void __launch_bounds__(1024) topk_kernel(const Cand *__restrict__ cand, size_t cap,
                                                    const int *__restrict__ cnt, int K, int gh, int gw,
                                                    int32_t *__restrict__ out_kyx, float *__restrict__ out_s,
                                                    int *__restrict__ out_count) {
    const int img = blockIdx.x;
    topk_body(cand + (size_t)img * cap, (int)min((size_t)cnt[img], cap), K, gh, gw, out_kyx + (size_t)img * 3 * K,
              out_s + (size_t)img * K, out_count + img);
}

// The same per job.
__global__ void __launch_bounds__(1024) topk_jobs_kernel(const CandJob *__restrict__ jobs, int K) {
    const CandJob j = jobs[blockIdx.x];
    topk_body(j.cand, (int)min((size_t)*j.cnt, j.cap), K, j.gh, j.gw, j.out_kyx, j.out_s, j.out_count);
}

// ---------------------------------------------------------------------------
// refinement: one CTA per (image or pair, candidate), all levels top-1 .. 0
// ---------------------------------------------------------------------------

struct RefineLevels {
    LevelDev L[kMaxLevels];
};

__device__ __forceinline__ float rmax3(float a, float b, float c) {
    float m;
    asm("max.f32 %0, %1, %2, %3;" : "=f"(m) : "f"(a), "f"(b), "f"(c));
    return m;
}

// The D x D dot products of one projected point's unit vector (px, py) with
// the field pixels (x0 .. x0 + D - 1, y0 .. y0 + D - 1) of a W x H level;
// pixels outside the level count 0.  CHECK = false: the caller has checked
// that the whole window lies inside (no per-pixel tests).
template <int D, bool CHECK>
__device__ __forceinline__ void refine_window(const float2 *__restrict__ F, int W, int H, int x0, int y0, float px,
                                              float py, float (&d)[D][D]) {
    if constexpr (!CHECK) {
        const float2 *q = F + (size_t)y0 * W + x0;
#pragma unroll
        for (int yy = 0; yy < D; ++yy)
#pragma unroll
            for (int xx = 0; xx < D; ++xx) {
                const float2 f = __ldg(q + (size_t)yy * W + xx);
                d[yy][xx] = fmaf(px, f.x, py * f.y);
            }
    } else {
#pragma unroll
        for (int yy = 0; yy < D; ++yy)
#pragma unroll
            for (int xx = 0; xx < D; ++xx) {
                const int X = x0 + xx, Y = y0 + yy;
                float v = 0.f;
                if (X >= 0 && Y >= 0 && X < W && Y < H) {
                    const float2 f = __ldg(F + (size_t)Y * W + X);
                    v = fmaf(px, f.x, py * f.y);
                }
                d[yy][xx] = v;
            }
    }
}

// The 9 scores' terms of one model point at one angle: for each pose
// (x, y) of the 3 x 3 around (cx, cy), the maximum of the dot products over
// the point's NB x NB window (Eq. (1)); the point's projection p at that
// angle; pol: absolute dot products.
template <int NB>
__device__ __forceinline__ void refine_maxima(const float2 *__restrict__ F, int W, int H, int cx, int cy,
                                              const RotPt &p, bool pol, float (&m)[9]) {
    constexpr int D = NB + 2;   // window of dot products
    const int x0 = cx + p.ox - D / 2, y0 = cy + p.oy - D / 2;
    float d[D][D];
    if (x0 >= 0 && y0 >= 0 && x0 + D <= W && y0 + D <= H)
        refine_window<D, false>(F, W, H, x0, y0, p.px, p.py, d);
    else
        refine_window<D, true>(F, W, H, x0, y0, p.px, p.py, d);
    if (pol) {
#pragma unroll
        for (int yy = 0; yy < D; ++yy)
#pragma unroll
            for (int xx = 0; xx < D; ++xx)
                d[yy][xx] = fabsf(d[yy][xx]);
    }
    if constexpr (NB == 3) {
        // 3x3 maxima: rows first, then columns
        float hm[D][3];
#pragma unroll
        for (int yy = 0; yy < D; ++yy)
#pragma unroll
            for (int tx = 0; tx < 3; ++tx)
                hm[yy][tx] = rmax3(d[yy][tx], d[yy][tx + 1], d[yy][tx + 2]);
#pragma unroll
        for (int ty = 0; ty < 3; ++ty)
#pragma unroll
            for (int tx = 0; tx < 3; ++tx)
                m[ty * 3 + tx] = rmax3(hm[ty][tx], hm[ty + 1][tx], hm[ty + 2][tx]);
    } else {
#pragma unroll
        for (int ty = 0; ty < 3; ++ty)
#pragma unroll
            for (int tx = 0; tx < 3; ++tx)
                m[ty * 3 + tx] = d[ty][tx];
    }
}

// One thread-block cluster of kRefineCluster CTAs per candidate: each CTA sums
// its share of the model points for the 27 poses and leaves the sums in its
// shared memory; after one cluster barrier every CTA adds the shares of all
// CTAs in rank order through distributed shared memory and picks the
// level's best pose itself (the same sums in the same order, so the same
// choice everywhere; no second barrier to broadcast it).  The share buffer
// alternates between two slots per reduction: a CTA writes slot r & 1 only
// after the barrier of reduction r - 1, which every CTA reaches after it has
// read the shares of reduction r - 2.  Every branch that skips a cluster
// barrier is taken by the whole cluster (same candidate, same state).
template <int NB, typename View>
__device__ void refine_body(const View &j, const LevelDev *lv, int c) {
    namespace cg = cooperative_groups;
    cg::cluster_group cluster = cg::this_cluster();
    __shared__ float red[RTHREADS / 32][27];
    __shared__ float part[2][27];   // this CTA's sums of the 27 poses, slot = reduction parity
    __shared__ int state[4];        // x, y, k, alive
    __shared__ float sbest;
    const int ncand = *j.count();
    float4 *outp = j.refined() + c;
    const unsigned rank = cluster.block_rank();
    if (c >= ncand) {
        if (rank == 0 && threadIdx.x == 0)
            *outp = make_float4(__int_as_float(0), __int_as_float(0), __int_as_float(0), -INFINITY);
        return;
    }
    if (threadIdx.x == 0) {
        const int32_t *kyx = j.kyx() + 3 * c;
        state[0] = kyx[2] * j.step_x();
        state[1] = kyx[1] * j.step_y();
        state[2] = kyx[0];
        state[3] = 1;
        sbest = j.cs()[c];
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int ns = j.nscales();
    int nred = 0;   // reductions so far (share slot parity)
    for (int l = j.top() - 1; l >= 0; --l) {
        const LevelDev &L = lv[l];
        // parent table Kp = scale jp x angles + angle kp at level l + 1
        const int Kp = state[2];
        const int2 sh = lv[l + 1].shift[Kp];
        const int cx = 2 * state[0] + sh.x, cy = 2 * state[1] + sh.y;
        const int nang = L.nangles, jp = Kp / lv[l + 1].nangles, kp = Kp - jp * lv[l + 1].nangles;
        const int W = j.w(l), H = j.h(l);
        const float2 *F = j.field(l);
        // the scales jp - 1 .. jp + 1 inside the grid, one pass of 27 poses
        // each (a rigid model: one pass); warp 0 keeps the best over the passes
        const int last_ds = min(1, ns - 1 - jp);
        float bs = -INFINITY;
        unsigned long long bk = ~0ull;
        int bx = 0, by = 0, bkk = 0;
        bool any = false;
        for (int ds = max(-1, -jp); ds <= last_ds; ++ds) {
            const int js = jp + ds;
            float acc[27];
#pragma unroll
            for (int q = 0; q < 27; ++q)
                acc[q] = 0.f;
            // the three angles' tables of this pass; per point the three
            // projections are loaded together, then each angle's window
            const RotPt *P3[3];
#pragma unroll
            for (int dk = 0; dk < 3; ++dk)
                P3[dk] = L.rot + (size_t)(js * nang + (2 * kp + dk - 1 + nang) % nang) * L.n;
            // whole rounds of kStride points, each thread a point at all three
            // angles; the remaining points as (point, angle) items dealt
            // round-robin over the cluster's threads, so that no thread
            // carries a whole extra point while the others wait
            constexpr int kStride = kRefineCluster * RTHREADS;
            const int self = (int)rank * RTHREADS + threadIdx.x;
            const int full = L.n - L.n % kStride, rest = L.n - full;
            const bool pol = j.polarity() != 0;
            for (int i = self; i < full; i += kStride) {
                RotPt pt[3];
#pragma unroll
                for (int dk = 0; dk < 3; ++dk)
                    pt[dk] = P3[dk][i];
#pragma unroll
                for (int dk = 0; dk < 3; ++dk) {
                    float m[9];
                    refine_maxima<NB>(F, W, H, cx, cy, pt[dk], pol, m);
#pragma unroll
                    for (int q = 0; q < 9; ++q)
                        acc[dk * 9 + q] += m[q];
                }
            }
            // item dk * rest + r (point full + r at angle dk) goes to thread
            // (dk * rest + r) mod kStride
#pragma unroll
            for (int dk = 0; dk < 3; ++dk) {
                int r = (self - dk * rest) % kStride;
                if (r < 0)
                    r += kStride;
                for (; r < rest; r += kStride) {
                    const RotPt pt = P3[dk][full + r];
                    float m[9];
                    refine_maxima<NB>(F, W, H, cx, cy, pt, pol, m);
#pragma unroll
                    for (int q = 0; q < 9; ++q)
                        acc[dk * 9 + q] += m[q];
                }
            }
            // block reduction of the 27 sums into this CTA's share
#pragma unroll
            for (int q = 0; q < 27; ++q) {
                float v = acc[q];
#pragma unroll
                for (int o = 16; o > 0; o >>= 1)
                    v += __shfl_xor_sync(0xffffffffu, v, o);
                if (lane == 0)
                    red[warp][q] = v;
            }
            __syncthreads();
            float *share = part[nred & 1];
            if (threadIdx.x < 27) {
                float v = 0.f;
                for (int wv = 0; wv < RTHREADS / 32; ++wv)
                    v += red[wv][threadIdx.x];
                share[threadIdx.x] = v;
            }
            cluster.sync();   // every CTA's share of this reduction is in its shared memory
            if (warp == 0) {
                // lane q < 27: pose q's sum over the CTAs (in rank order) and
                // its key; the best by the total order by a shuffle reduction
                float M = -INFINITY;
                unsigned long long key = ~0ull;
                int X = 0, Y = 0, kk = 0;
                bool valid = false;
                if (lane < 27) {
                    float tot = 0.f;
                    for (unsigned r = 0; r < (unsigned)kRefineCluster; ++r)
                        tot += cluster.map_shared_rank(share, r)[lane];
                    const int dk = lane / 9, ty = (lane / 3) % 3, tx = lane % 3;
                    kk = js * nang + (2 * kp + dk - 1 + nang) % nang;
                    X = cx + tx - 1;
                    Y = cy + ty - 1;
                    valid = X >= 0 && Y >= 0 && X < W && Y < H;
                    M = tot / (float)L.n;
                    key = ((unsigned long long)kk * H + Y) * W + X;
                }
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    const float oM = __shfl_xor_sync(0xffffffffu, M, o);
                    const unsigned long long okey = __shfl_xor_sync(0xffffffffu, key, o);
                    const int oX = __shfl_xor_sync(0xffffffffu, X, o), oY = __shfl_xor_sync(0xffffffffu, Y, o);
                    const int okk = __shfl_xor_sync(0xffffffffu, kk, o);
                    const bool ovalid = __shfl_xor_sync(0xffffffffu, valid, o);
                    if (ovalid && (!valid || beats(oM, okey, M, key))) {
                        M = oM;
                        key = okey;
                        X = oX;
                        Y = oY;
                        kk = okk;
                        valid = true;
                    }
                }
                if (lane == 0) {
                    if (valid && (!any || beats(M, key, bs, bk))) {
                        any = true;
                        bs = M;
                        bk = key;
                        bx = X;
                        by = Y;
                        bkk = kk;
                    }
                    if (ds == last_ds) {
                        state[0] = bx;
                        state[1] = by;
                        state[2] = bkk;
                        state[3] = any && bs >= j.min_score();
                        sbest = bs;
                    }
                }
            }
            ++nred;
        }
        __syncthreads();   // warp 0's choice is visible to the CTA
        if (!state[3])
            break;
    }
    cluster.sync();   // no CTA leaves while another may still read its shares
    if (rank == 0 && threadIdx.x == 0)
        *outp = make_float4(__int_as_float(state[0]), __int_as_float(state[1]), __int_as_float(state[2]),
                            state[3] ? sbest : -INFINITY);
}

// Which entry `item` is when entry counts weight(i) of n images (or
// pairs) are laid end to end: *img = i and *rel = item less the entries of
// the images before it; false past the last.  One warp (all lanes call it
// with the same arguments): 32 images' counts are loaded at once and
// scanned with shuffles, so the search costs one memory round trip per 32
// images rather than one per image.
template <typename Weight>
__device__ __forceinline__ bool locate_item(int item, int n, Weight weight, int *img, int *rel) {
    const int lane = threadIdx.x & 31;
    int acc = 0;
    for (int base = 0; base < n; base += 32) {
        const int i = base + lane;
        const int w = i < n ? weight(i) : 0;
        int v = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(0xffffffffu, v, o);
            if (lane >= o)
                v += t;
        }
        const int hi = acc + v, lo = hi - w;
        const unsigned hit = __ballot_sync(0xffffffffu, i < n && item >= lo && item < hi);
        if (hit) {
            const int L = __ffs(hit) - 1;
            *img = base + L;
            *rel = item - __shfl_sync(0xffffffffu, lo, L);
            return true;
        }
        acc += __shfl_sync(0xffffffffu, v, 31);
    }
    return false;
}

// Which candidate the cluster's turn cidx refines: the cidx-th of all
// images' (or pairs') candidates in (image, slot) order; false past the last.
// Warp 0 searches, the CTA reads the answer from shared memory.
template <typename CountAt>
__device__ __forceinline__ bool locate_candidate(int cidx, int n, int K, CountAt count_at, int *img, int *slot) {
    __shared__ int s_loc[2];
    if (threadIdx.x < 32) {
        int i = -1, r = 0;
        const bool ok = locate_item(cidx, n, [&](int x) { return min(count_at(x), K); }, &i, &r);
        if (threadIdx.x == 0) {
            s_loc[0] = ok ? i : -1;
            s_loc[1] = r;
        }
    }
    __syncthreads();
    *img = s_loc[0];
    *slot = s_loc[1];
    __syncthreads();   // s_loc is rewritten by the next search
    return *img >= 0;
}

// A candidate's image seen through the kernel's arguments (image img of a
// batch of equal-size images) or through a job of the job list; the
// arguments are read in place (kernel parameter space or global memory),
// never copied to a per-thread structure.
struct ArgsView {
    const RefineArgs *a;
    int img;
    __device__ const float2 *field(int l) const { return a->field[l] + (size_t)img * a->field_img_px[l]; }
    __device__ int w(int l) const { return a->w[l]; }
    __device__ int h(int l) const { return a->h[l]; }
    __device__ int top() const { return a->top; }
    __device__ int step_x() const { return a->step_x; }
    __device__ int step_y() const { return a->step_y; }
    __device__ int polarity() const { return a->polarity; }
    __device__ float min_score() const { return a->min_score; }
    __device__ int nscales() const { return a->nscales; }
    __device__ const int32_t *kyx() const { return a->cand_kyx + (size_t)img * 3 * a->K; }
    __device__ const float *cs() const { return a->cand_s + (size_t)img * a->K; }
    __device__ const int *count() const { return a->cand_count + img; }
    __device__ float4 *refined() const { return a->refined + (size_t)img * a->K; }
};
struct JobView {
    const RefineJob *j;
    __device__ const float2 *field(int l) const { return j->field[l]; }
    __device__ int w(int l) const { return j->w[l]; }
    __device__ int h(int l) const { return j->h[l]; }
    __device__ int top() const { return j->top; }
    __device__ int step_x() const { return j->step_x; }
    __device__ int step_y() const { return j->step_y; }
    __device__ int polarity() const { return j->polarity; }
    __device__ float min_score() const { return j->min_score; }
    __device__ int nscales() const { return j->nscales; }
    __device__ const int32_t *kyx() const { return j->kyx; }
    __device__ const float *cs() const { return j->cs; }
    __device__ const int *count() const { return j->count; }
    __device__ float4 *refined() const { return j->refined; }
};

// Coarse-to-fine refinement (Sec. II: the search starts at the top pyramid
// level; the size-3 neighbouring search in x, y and theta at each lower
// level), all levels down to 0 in one launch: persistent clusters of
// kRefineCluster CTAs take the candidates of all images in turn (cluster c
// the candidates c, c + clusters, ...), so only clusters with a candidate
// run and empty candidate slots cost nothing.  Two CTAs per SM (128
// registers, no spills) measured faster than three (80 registers, with
// spills) and a prefetch of the next point's tables gained nothing.
template <int NB>
__global__ void __cluster_dims__(kRefineCluster, 1, 1) __launch_bounds__(RTHREADS, 2)
    refine_kernel(const __grid_constant__ RefineLevels lv, const __grid_constant__ RefineArgs a) {
    const int clusters = gridDim.x / kRefineCluster;
    for (int cidx = blockIdx.x / kRefineCluster;; cidx += clusters) {
        int img = 0, slot = 0;
        if (!locate_candidate(cidx, a.count, a.K, [&](int i) { return a.cand_count[i]; }, &img, &slot))
            break;
        refine_body<NB>(ArgsView{&a, img}, lv.L, slot);
    }
}

// The same over a job list (pairs of different images and models).
template <int NB>
__global__ void __cluster_dims__(kRefineCluster, 1, 1) __launch_bounds__(RTHREADS, 2)
    refine_jobs_kernel(const RefineJob *__restrict__ jobs, int n_jobs, int K) {
    const int clusters = gridDim.x / kRefineCluster;
    for (int cidx = blockIdx.x / kRefineCluster;; cidx += clusters) {
        int job = 0, slot = 0;
        if (!locate_candidate(cidx, n_jobs, K, [&](int i) { return *jobs[i].count; }, &job, &slot))
            break;
        const RefineJob *j = jobs + job;
        refine_body<NB>(JobView{j}, j->L, slot);
    }
}

// ---------------------------------------------------------------------------
// NMS: one CTA per image or pair
// ---------------------------------------------------------------------------

__device__ void nms_body(const float4 *__restrict__ R, int nc, int w0, int h0, int min_side, int max_out,
                         double angle_step, int nang0, sam_pose *__restrict__ out, int *__restrict__ n_out) {
    __shared__ float s[kMaxTopK];
    __shared__ unsigned long long key[kMaxTopK];
    __shared__ int px[kMaxTopK], py[kMaxTopK], pk[kMaxTopK];
    __shared__ int kx[kMaxTopK], ky[kMaxTopK];   // positions kept so far
    int n2 = 1;
    while (n2 < nc)
        n2 <<= 1;
    for (int i = threadIdx.x; i < n2; i += blockDim.x) {
        if (i < nc) {
            const float4 r = R[i];
            const int x = __float_as_int(r.x), y = __float_as_int(r.y), k = __float_as_int(r.z);
            s[i] = r.w;
            key[i] = ((unsigned long long)k * h0 + y) * w0 + x;
        } else {
            s[i] = -INFINITY;
            key[i] = ~0ull;
        }
    }
    __syncthreads();
    if (n2 > 1)
        bitonic_sort(s, key, n2);
    const unsigned long long plane = (unsigned long long)h0 * w0;
    for (int i = threadIdx.x; i < n2; i += blockDim.x) {
        const unsigned long long kk = key[i];
        if (kk == ~0ull)
            continue;
        pk[i] = (int)(kk / plane);
        const int r = (int)(kk - (unsigned long long)pk[i] * plane);
        py[i] = r / w0;
        px[i] = r - py[i] * w0;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        int kept = 0;
        const long long ms2 = (long long)min_side * min_side;
        for (int i = 0; i < nc && kept < max_out; ++i) {
            if (s[i] == -INFINITY)
                break;   // sorted: the rest are dead too
            bool ok = true;
            for (int q = 0; q < kept; ++q) {
                const long long dx = px[i] - kx[q], dy = py[i] - ky[q];
                if (4 * (dx * dx + dy * dy) < ms2) {
                    ok = false;
                    break;
                }
            }
            if (!ok)
                continue;
            // table index = scale index x angles + angle index
            const int sj = pk[i] / nang0, ak = pk[i] - sj * nang0;
            sam_pose p;
            p.x = (float)px[i];
            p.y = (float)py[i];
            p.theta_deg = (float)(ak * angle_step);
            p.score = s[i];
            p.angle_index = ak;
            p.level0_x = px[i];
            p.level0_y = py[i];
            p.scale_index = sj;
            kx[kept] = px[i];
            ky[kept] = py[i];
            out[kept++] = p;
        }
        *n_out = kept;
    }
}

// Final non-maximum suppression of each image's refined poses (one CTA per
// image): greedy in the total order, dropping poses closer than half the
// smaller template side to a kept one.
__global__ void __launch_bounds__(256) nms_kernel(NmsArgs a) {
    const int img = blockIdx.x;
    nms_body(a.refined + (size_t)img * a.K, min(a.cand_count[img], a.K), a.w0, a.h0, a.min_side, a.max_out,
             a.angle_step, a.nang0, a.out + (size_t)img * a.max_out, a.n_out + img);
}

// The same per job.
__global__ void __launch_bounds__(256) nms_jobs_kernel(const NmsJob *__restrict__ jobs, int K) {
    const NmsJob j = jobs[blockIdx.x];
    nms_body(j.refined, min(*j.count, K), j.w0, j.h0, j.min_side, j.max_out, j.angle_step, j.nang0, j.out,
             j.n_out);
}

}  // namespace

// At most one strict local maximum per 2x2x2 block of (theta, y, x) of one
// scale (mutual neighbours), so per scale ceil(nang / 2) x ceil(gh / 2) x
// ceil(gw / 2).
size_t cand_cap(int nth, int gh, int gw, int ns) {
    const int nang = nth / ns;
    return (size_t)ns * ((nang + 1) / 2) * ((gh + 1) / 2) * ((gw + 1) / 2);
}

size_t candidates_scratch_bytes(int nth, int gh, int gw, int ns) { return 256 + cand_cap(nth, gh, gw, ns) * sizeof(Cand); }

cudaError_t launch_candidates(const float *map, size_t map_img, int nth, int gh, int gw, float min_score, int K,
                              int32_t *out_kyx, float *out_s, int *count, void *scratch, size_t scratch_img,
                              int n_img, cudaStream_t st, int ns) {
    // scratch layout: [n_img int counters, padded to 256 B][n_img x Cand cap]
    const size_t cap = cand_cap(nth, gh, gw, ns);
    int *cnt = reinterpret_cast<int *>(scratch);
    Cand *cand = reinterpret_cast<Cand *>(reinterpret_cast<char *>(scratch) + 256 * ((n_img * sizeof(int) + 255) / 256));
    (void)scratch_img;
    cudaError_t e = cudaMemsetAsync(cnt, 0, sizeof(int) * (size_t)n_img, st);
    if (e != cudaSuccess)
        return e;
    const size_t total = (size_t)nth * gh * gw;
    const int vec = ((uintptr_t)map % 16 == 0) && (n_img == 1 || map_img % 4 == 0);
    // about 32 CTAs of 256 threads per SM over all images (several waves),
    // each thread a few 16-byte loads of 4 entries
    const int per_img = std::max(1, 152 * 32 / std::max(1, n_img));
    const int blocks = (int)std::max<size_t>(1, std::min<size_t>((total / 4 + 255) / 256, (size_t)per_img));
    dim3 grid((unsigned)blocks, (unsigned)n_img);
    local_max_kernel<<<grid, 256, 0, st>>>(map, map_img, nth, gh, gw, min_score, cand, cap, cnt, ns, vec);
    topk_kernel<<<n_img, 1024, 0, st>>>(cand, cap, cnt, K, gh, gw, out_kyx, out_s, count);
    count_launches(2);
    return cudaGetLastError();
}

cudaError_t launch_candidates_hot(const float *map, size_t map_img, int nth, int gh, int gw, float min_score, int K,
                                  int32_t *out_kyx, float *out_s, int *count, void *scratch, int n_img,
                                  const unsigned *hot_cnt, const uint2 *hot, unsigned hot_cap, cudaStream_t st,
                                  int ns) {
    const size_t cap = cand_cap(nth, gh, gw, ns);
    int *cnt = reinterpret_cast<int *>(scratch);
    Cand *cand = reinterpret_cast<Cand *>(reinterpret_cast<char *>(scratch) + 256 * ((n_img * sizeof(int) + 255) / 256));
    cudaError_t e = cudaMemsetAsync(cnt, 0, sizeof(int) * (size_t)n_img, st);
    if (e != cudaSuccess)
        return e;
    // two CTAs per SM: a few thousand listed poses take one pass; the
    // whole-map fallback strides over every map
    local_max_hot_kernel<<<2 * 152, 256, 0, st>>>(map, map_img, nth, gh, gw, min_score, cand, cap, cnt, ns, hot_cnt,
                                                  hot, hot_cap, n_img);
    topk_kernel<<<n_img, 1024, 0, st>>>(cand, cap, cnt, K, gh, gw, out_kyx, out_s, count);
    count_launches(2);
    return cudaGetLastError();
}

cudaError_t launch_candidates_hot16(const float *map, size_t map_img, int nth, int gh, int gw, float min_score,
                                    float delta, int K, int32_t *out_kyx, float *out_s, int *count, void *scratch,
                                    int n_img, const unsigned *hot_cnt, const uint2 *hot, unsigned hot_cap,
                                    const float2 *field32, size_t field_img_px, int w, int h, const LevelDev &L,
                                    int nbhd, int polarity, unsigned *pass_cnt, unsigned *pass_list,
                                    cudaStream_t st, int ns) {
    const size_t cap = cand_cap(nth, gh, gw, ns);
    int *cnt = reinterpret_cast<int *>(scratch);
    Cand *cand = reinterpret_cast<Cand *>(reinterpret_cast<char *>(scratch) + 256 * ((n_img * sizeof(int) + 255) / 256));
    cudaError_t e = cudaMemsetAsync(cnt, 0, sizeof(int) * (size_t)n_img, st);
    if (e != cudaSuccess)
        return e;
    Cand16Args a;
    a.map = map;
    a.map_img = map_img;
    a.nth = nth;
    a.gh = gh;
    a.gw = gw;
    a.ns = ns;
    a.min_score = min_score;
    a.delta = delta;
    a.hot_cnt = hot_cnt;
    a.hot = hot;
    a.hot_cap = hot_cap;
    a.field = field32;
    a.field_img_px = field_img_px;
    a.w = w;
    a.h = h;
    a.rot = L.rot;
    a.n = L.n;
    a.polarity = polarity;
    a.cand = cand;
    a.cap = cap;
    a.cnt = cnt;
    a.pass_cnt = pass_cnt;
    a.pass_list = pass_list;
    // the filter, then the decision with eight resident CTAs per SM: the
    // poses that pass (a few hundred to a few thousand) one or two per CTA
    cand16_filter_kernel<<<2 * 152, 256, 0, st>>>(a);
    if (nbhd == 3)
        cand16_eval_kernel<3><<<8 * 152, kC16Threads, 0, st>>>(a);
    else
        cand16_eval_kernel<1><<<8 * 152, kC16Threads, 0, st>>>(a);
    topk_kernel<<<n_img, 1024, 0, st>>>(cand, cap, cnt, K, gh, gw, out_kyx, out_s, count);
    count_launches(3);
    return cudaGetLastError();
}

cudaError_t launch_candidates_hot_jobs(const CandJob *jobs, int n_jobs, float min_score, int K,
                                       const unsigned *hot_cnt, const uint2 *hot, unsigned hot_cap,
                                       cudaStream_t st) {
    if (n_jobs <= 0)
        return cudaSuccess;
    local_max_hot_jobs_kernel<<<2 * 152, 256, 0, st>>>(jobs, n_jobs, min_score, hot_cnt, hot, hot_cap);
    topk_jobs_kernel<<<n_jobs, 1024, 0, st>>>(jobs, K);
    count_launches(2);
    return cudaGetLastError();
}

cudaError_t launch_candidates_hot16_jobs(const CandJob *cjobs, const RescoreJob *rjobs, int n_jobs, float min_score,
                                         float delta, int K, int nbhd, int polarity, const unsigned *hot_cnt,
                                         const uint2 *hot, unsigned hot_cap, unsigned *pass_cnt,
                                         unsigned *pass_list, cudaStream_t st) {
    if (n_jobs <= 0)
        return cudaSuccess;
    cand16_filter_jobs_kernel<<<2 * 152, 256, 0, st>>>(cjobs, rjobs, hot_cnt, hot, hot_cap, min_score, delta, pass_cnt,
                                                       pass_list);
    if (nbhd == 3)
        cand16_eval_jobs_kernel<3><<<8 * 152, kC16Threads, 0, st>>>(cjobs, rjobs, hot, pass_cnt, pass_list, min_score,
                                                                   polarity);
    else
        cand16_eval_jobs_kernel<1><<<8 * 152, kC16Threads, 0, st>>>(cjobs, rjobs, hot, pass_cnt, pass_list, min_score,
                                                                   polarity);
    topk_jobs_kernel<<<n_jobs, 1024, 0, st>>>(cjobs, K);
    count_launches(3);
    return cudaGetLastError();
}

size_t candidates_scratch_bytes_batch(int nth, int gh, int gw, int n_img, int ns) {
    return 256 * ((n_img * sizeof(int) + 255) / 256) + (size_t)n_img * cand_cap(nth, gh, gw, ns) * sizeof(Cand);
}

cudaError_t launch_candidates_jobs(const CandJob *jobs, int n_jobs, size_t max_total, float min_score, int K,
                                   cudaStream_t st) {
    if (n_jobs <= 0)
        return cudaSuccess;
    const int blocks = (int)std::max<size_t>(1, std::min<size_t>((max_total + 255) / 256, 64));
    local_max_jobs_kernel<<<dim3((unsigned)blocks, (unsigned)n_jobs), 256, 0, st>>>(jobs, min_score);
    topk_jobs_kernel<<<n_jobs, 1024, 0, st>>>(jobs, K);
    count_launches(2);
    return cudaGetLastError();
}

// Clusters of the persistent refinement that fit on the device at once (the
// first query per device; 152 SMs x 3 CTAs if the query fails).
int refine_clusters() {
    static int cached[64] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64)
        return 152 * 3 / kRefineCluster;
    if (cached[dev] > 0)
        return cached[dev];
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr;
    attr.id = cudaLaunchAttributeClusterDimension;
    attr.val.clusterDim.x = kRefineCluster;
    attr.val.clusterDim.y = 1;
    attr.val.clusterDim.z = 1;
    cfg.gridDim = dim3(kRefineCluster * 1024);
    cfg.blockDim = dim3(RTHREADS);
    cfg.attrs = &attr;
    cfg.numAttrs = 1;
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, (void *)refine_kernel<3>, &cfg) != cudaSuccess || n <= 0) {
        cudaGetLastError();
        n = 152 * 3 / kRefineCluster;
    }
    cached[dev] = n;
    return n;
}

cudaError_t launch_refine(const sam_model *m, const RefineArgs &a, cudaStream_t st) {
    RefineLevels lv;
    for (int l = 0; l < kMaxLevels; ++l)
        lv.L[l] = m->dev[l];
    const int clusters = std::max(1, std::min(a.count * a.K, refine_clusters()));
    dim3 grid((unsigned)(clusters * kRefineCluster));
    if (a.nbhd == 3)
        refine_kernel<3><<<grid, RTHREADS, 0, st>>>(lv, a);
    else
        refine_kernel<1><<<grid, RTHREADS, 0, st>>>(lv, a);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_refine_jobs(const RefineJob *jobs, int n_jobs, int K, int nbhd, cudaStream_t st) {
    if (n_jobs <= 0)
        return cudaSuccess;
    const int clusters = std::max(1, std::min(n_jobs * K, refine_clusters()));
    dim3 grid((unsigned)(clusters * kRefineCluster));
    if (nbhd == 3)
        refine_jobs_kernel<3><<<grid, RTHREADS, 0, st>>>(jobs, n_jobs, K);
    else
        refine_jobs_kernel<1><<<grid, RTHREADS, 0, st>>>(jobs, n_jobs, K);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_nms(const NmsArgs &a, cudaStream_t st) {
    nms_kernel<<<a.count, 256, 0, st>>>(a);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_nms_jobs(const NmsJob *jobs, int n_jobs, int K, cudaStream_t st) {
    if (n_jobs <= 0)
        return cudaSuccess;
    nms_jobs_kernel<<<n_jobs, 256, 0, st>>>(jobs, K);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace sam


// ---------------------------------------------------------------------------
// Candidate extraction without run-time allocation.
//
// Some callers cannot call cudaMalloc at the moment they need candidates: a
// control loop with a hard deadline (cudaMalloc can take milliseconds and
// may synchronise the device), or an integration whose device memory is
// budgeted once at start-up and must not grow afterwards.  This entry point
// serves them: its scratch (the local-maximum counter and candidate list)
// lives in the file-scope device array below instead of a caller buffer.
//
// Limit: 4 MiB per device, held by every GPU that loads the library until
// the process exits; maps whose candidate capacity needs more are rejected
// with SAM_ERR_CAPACITY before anything is launched.
// Sharing: every call on a device uses the same array and leaves its
// contents behind; the counter is cleared at the start of each call.  Calls
// whose work overlaps on the GPU (other streams, other host threads) race
// on the array and must be serialised by the caller.
// ---------------------------------------------------------------------------

#include <cuda.h>
#include <mutex>

namespace sam {
namespace {

constexpr size_t kNoAllocScratchBytes = (size_t)4 << 20;
constexpr int kNoAllocMaxDevices = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

std::mutex g_noalloc_mutex;
void *g_noalloc_ptr[kNoAllocMaxDevices] = {};
unsigned long long g_noalloc_ctx[kNoAllocMaxDevices] = {};   // context the cached address belongs to (0: none)

// Unique id of the current CUDA context (never reused within a process), by
// the driver's cuCtxGetCurrent / cuCtxGetId fetched through the runtime, so
// the library needs no link to the driver; 0 if unavailable.
unsigned long long current_context_id() {
    typedef CUresult (*GetCurrent)(CUcontext *);
    typedef CUresult (*GetId)(CUcontext, unsigned long long *);
    static GetCurrent get_current = nullptr;
    static GetId get_id = nullptr;
    static bool looked_up = false;
    if (!looked_up) {
        looked_up = true;
        cudaDriverEntryPointQueryResult q1 = cudaDriverEntryPointSymbolNotFound, q2 = q1;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", (void **)&get_current, 12000, cudaEnableDefault,
                                             &q1) != cudaSuccess ||
            q1 != cudaDriverEntryPointSuccess)
            get_current = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", (void **)&get_id, 12000, cudaEnableDefault, &q2) !=
                cudaSuccess ||
            q2 != cudaDriverEntryPointSuccess)
            get_id = nullptr;
    }
    CUcontext c = nullptr;
    unsigned long long id = 0;
    if (!get_current || !get_id || get_current(&c) != CUDA_SUCCESS || !c || get_id(c, &id) != CUDA_SUCCESS)
        return 0;
    return id;
}

// Device address of g_noalloc_scratch on the current device.  The first call
// on a device looks it up (cudaGetSymbolAddress, with that device current)
// and caches it together with the id of the device's current context; a
// later call whose context id differs (the device was reset and its primary
// context re-created) looks the address up again, as does every call when
// the id cannot be read.
cudaError_t noalloc_scratch(void **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess)
        return e;
    if (dev < 0 || dev >= kNoAllocMaxDevices)
        return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    const unsigned long long ctx = g_noalloc_ptr[dev] ? current_context_id() : 0;
    if (!g_noalloc_ptr[dev] || ctx == 0 || ctx != g_noalloc_ctx[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) {
            g_noalloc_ptr[dev] = nullptr;
            return e;
        }
        g_noalloc_ptr[dev] = p;
        g_noalloc_ctx[dev] = current_context_id();   // after the lookup, which makes the context current
    }
    *out = g_noalloc_ptr[dev];
    return cudaSuccess;
}

}  // namespace
}  // namespace sam

extern "C" sam_status sam_candidates_noalloc(const float *map, int nth, int gh, int gw, float min_score, int K,
                                             int32_t *out_kyx, float *out_s, int *count, void *stream) {
    using namespace sam;
    if (!map || !out_kyx || !out_s || !count || nth < 1 || gh < 1 || gw < 1 || K < 1 || K > kMaxTopK)
        return SAM_ERR_ARG;
    if (candidates_scratch_bytes(nth, gh, gw) > kNoAllocScratchBytes)
        return SAM_ERR_CAPACITY;
    void *scratch = nullptr;
    if (noalloc_scratch(&scratch) != cudaSuccess)
        return SAM_ERR_CUDA;
    return launch_candidates(map, 0, nth, gh, gw, min_score, K, out_kyx, out_s, count, scratch, 0, 1,
                             (cudaStream_t)stream) == cudaSuccess
               ? SAM_OK
               : SAM_ERR_CUDA;
}
