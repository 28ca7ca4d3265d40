// Host-side model builder (Sec. II, the model image's side of the problem).
//
// For every pyramid level of the template: 3x3 Sobel gradients, hysteresis
// edge selection (>= high seeds grown 8-connected through >= low), and the
// edge points t relative to the reference point (floor(W/2), floor(H/2)).
// For every (level, angle index k): the Eq. (2) projection of each point,
// integer offset floor(R(theta_k) t + 1/2) and unit direction R(theta_k) g/|g|,
// computed in FP64 (the host is compiled without FMA contraction so these
// integers are the plain IEEE rounding of the printed expressions).  The
// template is small (at most a few hundred pixels a side), so this runs once
// per model on the CPU; the tables are uploaded to the device on first use.

#include <math.h>
#include <string.h>

#include <algorithm>
#include <deque>
#include <new>

#include "sam_internal.h"

namespace sam {
namespace {

constexpr double kPi = 3.14159265358979323846;

// One pyramid step on the host: rounded 2x2 mean, odd trailing row/col dropped.
std::vector<uint8_t> halve(const std::vector<uint8_t> &img, int w, int h) {
    const int w2 = w / 2, h2 = h / 2;
    std::vector<uint8_t> out((size_t)w2 * h2);
    for (int y = 0; y < h2; ++y) {
        const uint8_t *r0 = img.data() + (size_t)(2 * y) * w;
        const uint8_t *r1 = r0 + w;
        for (int x = 0; x < w2; ++x) {
            const unsigned s = r0[2 * x] + r0[2 * x + 1] + r1[2 * x] + r1[2 * x + 1];
            out[(size_t)y * w2 + x] = (uint8_t)((s + 2u) >> 2);
        }
    }
    return out;
}

// Sobel gradients with a zero 1-pixel border.
void sobel(const std::vector<uint8_t> &img, int w, int h, std::vector<int32_t> &gx, std::vector<int32_t> &gy) {
    gx.assign((size_t)w * h, 0);
    gy.assign((size_t)w * h, 0);
    for (int y = 1; y + 1 < h; ++y) {
        const uint8_t *a = img.data() + (size_t)(y - 1) * w;  // row above
        const uint8_t *b = a + w;                             // centre row
        const uint8_t *c = b + w;                             // row below
        for (int x = 1; x + 1 < w; ++x) {
            const int right = a[x + 1] + 2 * b[x + 1] + c[x + 1];
            const int left = a[x - 1] + 2 * b[x - 1] + c[x - 1];
            const int below = c[x - 1] + 2 * c[x] + c[x + 1];
            const int above = a[x - 1] + 2 * a[x] + a[x + 1];
            gx[(size_t)y * w + x] = right - left;
            gy[(size_t)y * w + x] = below - above;
        }
    }
}

inline bool strong_enough(int32_t gx, int32_t gy, int t) {
    return (int64_t)gx * gx + (int64_t)gy * gy >= (int64_t)16 * t * t;
}

// Hysteresis by breadth-first growth from the strong pixels.
std::vector<uint8_t> hysteresis(const std::vector<int32_t> &gx, const std::vector<int32_t> &gy, int w, int h,
                                int low, int high) {
    std::vector<uint8_t> weak((size_t)w * h), edge((size_t)w * h, 0);
    std::deque<int> q;
    for (size_t i = 0; i < weak.size(); ++i) {
        weak[i] = strong_enough(gx[i], gy[i], low);
        if (strong_enough(gx[i], gy[i], high)) {
            edge[i] = 1;
            q.push_back((int)i);
        }
    }
    while (!q.empty()) {
        const int p = q.front();
        q.pop_front();
        const int py = p / w, px = p - py * w;
        for (int ny = std::max(0, py - 1); ny <= std::min(h - 1, py + 1); ++ny)
            for (int nx = std::max(0, px - 1); nx <= std::min(w - 1, px + 1); ++nx) {
                const int j = ny * w + nx;
                if (weak[j] && !edge[j]) {
                    edge[j] = 1;
                    q.push_back(j);
                }
            }
    }
    return edge;
}

// Eq. (2) table of one level and angle index k.
void rotate_level(LevelHost &L, int k, RotPt *dst, int4 &box) {
    const double th = ((double)k * L.dtheta) * kPi / 180.0;
    const double c = cos(th), s = sin(th);
    box = make_int4(1 << 30, -(1 << 30), 1 << 30, -(1 << 30));
    for (int i = 0; i < L.n; ++i) {
        const double x = (double)L.tx[i], y = (double)L.ty[i];
        const int ox = (int)floor(c * x - s * y + 0.5);
        const int oy = (int)floor(s * x + c * y + 0.5);
        const double g = sqrt((double)L.gx[i] * L.gx[i] + (double)L.gy[i] * L.gy[i]);
        const double ux = L.gx[i] / g, uy = L.gy[i] / g;
        dst[i].ox = ox;
        dst[i].oy = oy;
        dst[i].px = (float)(c * ux - s * uy);
        dst[i].py = (float)(s * ux + c * uy);
        box.x = std::min(box.x, ox);
        box.y = std::max(box.y, ox);
        box.z = std::min(box.z, oy);
        box.w = std::max(box.w, oy);
    }
}

// Scaled table (Eq. (2) with A = s R(theta)) of one level, scale `scale` and
// angle index k: offsets floor(A t + 1/2) with A = [[s c, -(s sn)], [s sn,
// s c]] evaluated exactly as written, directions R(theta) g/|g| (the inverse
// transpose of a similarity turns a gradient as R does).
void scale_level(LevelHost &L, int k, double scale, RotPt *dst, int4 &box) {
    const double th = ((double)k * L.dtheta) * kPi / 180.0;
    const double c = cos(th), sn = sin(th);
    const double a11 = scale * c, a12 = -(scale * sn), a21 = scale * sn, a22 = scale * c;
    box = make_int4(1 << 30, -(1 << 30), 1 << 30, -(1 << 30));
    for (int i = 0; i < L.n; ++i) {
        const double x = (double)L.tx[i], y = (double)L.ty[i];
        const int ox = (int)floor(a11 * x + a12 * y + 0.5);
        const int oy = (int)floor(a21 * x + a22 * y + 0.5);
        const double g = sqrt((double)L.gx[i] * L.gx[i] + (double)L.gy[i] * L.gy[i]);
        const double ux = L.gx[i] / g, uy = L.gy[i] / g;
        dst[i].ox = ox;
        dst[i].oy = oy;
        dst[i].px = (float)(c * ux - sn * uy);
        dst[i].py = (float)(sn * ux + c * uy);
        box.x = std::min(box.x, ox);
        box.y = std::max(box.y, ox);
        box.z = std::min(box.z, oy);
        box.w = std::max(box.w, oy);
    }
}

}  // namespace

// Chunked tables of one level (see LevelHost): for every angle, the rotated
// points sorted by the kChunkCell-sized cell of their offset (floor
// division), one chunk per non-empty cell.
static void build_chunks(LevelHost &L) {
    const size_t n = (size_t)L.n;
    L.crot.resize((size_t)L.ntheta * n);
    L.cstart.assign((size_t)L.ntheta + 1, 0);
    L.cbox.clear();
    L.crange.clear();
    L.cspan_x = L.cspan_y = 0;
    std::vector<std::pair<long long, int>> key(n);
    for (int k = 0; k < L.ntheta; ++k) {
        const RotPt *src = L.rot.data() + (size_t)k * n;
        RotPt *dst = L.crot.data() + (size_t)k * n;
        for (size_t i = 0; i < n; ++i) {
            const long long cx = (long long)floor((double)src[i].ox / kChunkCell);
            const long long cy = (long long)floor((double)src[i].oy / kChunkCell);
            key[i] = std::make_pair(cy * (1LL << 32) + cx, (int)i);
        }
        std::stable_sort(key.begin(), key.end(),
                         [](const std::pair<long long, int> &a, const std::pair<long long, int> &b) {
                             return a.first < b.first;
                         });
        L.cstart[k] = (int)L.cbox.size();
        size_t i = 0;
        while (i < n) {
            size_t j = i;
            int4 b = make_int4(1 << 30, -(1 << 30), 1 << 30, -(1 << 30));
            while (j < n && key[j].first == key[i].first) {
                const RotPt &q = src[key[j].second];
                dst[j] = q;
                b.x = std::min(b.x, q.ox);
                b.y = std::max(b.y, q.ox);
                b.z = std::min(b.z, q.oy);
                b.w = std::max(b.w, q.oy);
                ++j;
            }
            L.cbox.push_back(b);
            L.crange.push_back(make_int2((int)i, (int)j));
            L.cspan_x = std::max(L.cspan_x, b.y - b.x);
            L.cspan_y = std::max(L.cspan_y, b.w - b.z);
            i = j;
        }
    }
    L.cstart[L.ntheta] = (int)L.cbox.size();
}

sam_status build_model(const uint8_t *tmpl, int w, int h, int stride, const sam_model_params &p, sam_model *m,
                       int nscales, double scale_min, double scale_step) {
    if (!tmpl || w < 3 || h < 3 || stride < w || p.levels < 1 || p.levels > kMaxLevels || p.low < 1 ||
        p.high < p.low || !(p.angle_step_deg > 0.0) || (p.polarity != 0 && p.polarity != 1))
        return SAM_ERR_ARG;
    // a scale grid with every s_j in (0, 16]; one scale of 1 is the rigid model
    const bool scaled = !(nscales == 1 && scale_min == 1.0);
    if (nscales < 1 || nscales > 64 || !(scale_min > 0.0) || !(scale_step >= 0.0) ||
        (nscales > 1 && !(scale_step > 0.0)) || !(scale_min + (nscales - 1) * scale_step <= 16.0))
        return SAM_ERR_ARG;
    const double nt = 360.0 / p.angle_step_deg;
    const long n0 = lround(nt);
    if (n0 < 1 || n0 > 1 << 20 || fabs((double)n0 * p.angle_step_deg - 360.0) > 1e-9 ||
        (n0 % (1L << (p.levels - 1))) != 0)
        return SAM_ERR_ARG;
    if ((w >> (p.levels - 1)) < 3 || (h >> (p.levels - 1)) < 3)
        return SAM_ERR_ARG;
    if ((long)nscales * n0 > (1L << 20))
        return SAM_ERR_ARG;
    m->p = p;
    m->levels = p.levels;
    m->ntheta0 = (int)n0;
    m->nscales = nscales;
    m->scale_min = scale_min;
    m->scale_step = scale_step;
    try {
        m->lv.assign(p.levels, LevelHost());
        std::vector<uint8_t> img((size_t)w * h);
        for (int y = 0; y < h; ++y)
            memcpy(img.data() + (size_t)y * w, tmpl + (size_t)y * stride, (size_t)w);
        int cw = w, ch = h;
        for (int l = 0; l < p.levels; ++l) {
            if (l > 0) {
                img = halve(img, cw, ch);
                cw /= 2;
                ch /= 2;
            }
            LevelHost &L = m->lv[l];
            L.tw = cw;
            L.th = ch;
            L.nangles = (int)(n0 >> l);
            L.ntheta = nscales * L.nangles;
            L.dtheta = p.angle_step_deg * (double)(1 << l);
            std::vector<int32_t> gx, gy;
            sobel(img, cw, ch, gx, gy);
            const std::vector<uint8_t> edge = hysteresis(gx, gy, cw, ch, p.low, p.high);
            const int cx = cw / 2, cy = ch / 2;
            for (int y = 0; y < ch; ++y)
                for (int x = 0; x < cw; ++x) {
                    const size_t i = (size_t)y * cw + x;
                    if (!edge[i])
                        continue;
                    L.tx.push_back(x - cx);
                    L.ty.push_back(y - cy);
                    L.gx.push_back(gx[i]);
                    L.gy.push_back(gy[i]);
                }
            L.n = (int)L.tx.size();
            if (L.n == 0)
                return SAM_ERR_EMPTY_MODEL;
            L.rot.resize((size_t)L.ntheta * L.n);
            L.bbox.resize(L.ntheta);
            if (!scaled) {
                for (int k = 0; k < L.ntheta; ++k)
                    rotate_level(L, k, L.rot.data() + (size_t)k * L.n, L.bbox[k]);
            } else {
                for (int j = 0; j < nscales; ++j)
                    for (int k = 0; k < L.nangles; ++k) {
                        const int K = j * L.nangles + k;
                        scale_level(L, k, scale_min + j * scale_step, L.rot.data() + (size_t)K * L.n, L.bbox[K]);
                    }
            }
        }
        // chunk tables for every level: required where the rotated extent
        // exceeds one window, and a tiling choice of the autotuner elsewhere
        for (int l = 0; l < p.levels; ++l)
            build_chunks(m->lv[l]);
        // Coarse-to-fine shifts: a parent pose u' at level l (angle index k')
        // maps to the level-(l-1) pose 2u' + (1/2, 1/2) - R(theta) d with
        // d = 2 c_l + 1/2 - c_{l-1} per axis (c = reference point); the
        // child's search centre is 2u' + nearest integer of the rest.
        for (int l = 1; l < p.levels; ++l) {
            LevelHost &L = m->lv[l];
            const LevelHost &C = m->lv[l - 1];
            const double dx = 2.0 * (double)(L.tw / 2) + 0.5 - (double)(C.tw / 2);
            const double dy = 2.0 * (double)(L.th / 2) + 0.5 - (double)(C.th / 2);
            L.shift.resize(L.ntheta);
            if (!scaled) {
                for (int k = 0; k < L.ntheta; ++k) {
                    const double th = ((double)k * L.dtheta) * kPi / 180.0;
                    const double c = cos(th), s = sin(th);
                    L.shift[k].x = (int)floor(0.5 - (c * dx - s * dy) + 0.5);
                    L.shift[k].y = (int)floor(0.5 - (s * dx + c * dy) + 0.5);
                }
            } else {
                // a scaled parent turns and scales d by its A = s R(theta)
                for (int j = 0; j < nscales; ++j)
                    for (int k = 0; k < L.nangles; ++k) {
                        const double th = ((double)k * L.dtheta) * kPi / 180.0;
                        const double c = cos(th), sn = sin(th), sc = scale_min + j * scale_step;
                        const double a11 = sc * c, a12 = -(sc * sn), a21 = sc * sn, a22 = sc * c;
                        const int K = j * L.nangles + k;
                        L.shift[K].x = (int)floor(0.5 - (a11 * dx + a12 * dy) + 0.5);
                        L.shift[K].y = (int)floor(0.5 - (a21 * dx + a22 * dy) + 0.5);
                    }
            }
        }
    } catch (const std::bad_alloc &) {
        return SAM_ERR_NOMEM;
    }
    return SAM_OK;
}

sam_status upload_model(sam_model *m) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess)
        return SAM_ERR_CUDA;
    if (m->d_tables && m->device == dev)
        return SAM_OK;
    if (m->d_tables) {
        cudaFree(m->d_tables);
        m->d_tables = nullptr;
    }
    size_t bytes = 0;
    auto align = [](size_t v) { return (v + 255) & ~(size_t)255; };
    for (const LevelHost &L : m->lv)
        bytes += align(L.rot.size() * sizeof(RotPt)) + align(L.bbox.size() * sizeof(int4)) +
                 align(std::max<size_t>(1, L.shift.size()) * sizeof(int2)) + align((size_t)L.n * sizeof(float4)) +
                 align(L.crot.size() * sizeof(RotPt)) + align(L.cstart.size() * sizeof(int)) +
                 align(L.cbox.size() * sizeof(int4)) + align(L.crange.size() * sizeof(int2));
    void *base = nullptr;
    if (cudaMalloc(&base, bytes) != cudaSuccess)
        return SAM_ERR_NOMEM;
    char *p = (char *)base;
    for (int l = 0; l < m->levels; ++l) {
        const LevelHost &L = m->lv[l];
        LevelDev &D = m->dev[l];
        D.tw = L.tw;
        D.th = L.th;
        D.n = L.n;
        D.ntheta = L.ntheta;
        D.nangles = L.nangles;
        D.rot = (const RotPt *)p;
        if (cudaMemcpy(p, L.rot.data(), L.rot.size() * sizeof(RotPt), cudaMemcpyHostToDevice) != cudaSuccess)
            goto fail;
        p += align(L.rot.size() * sizeof(RotPt));
        D.bbox = (const int4 *)p;
        if (cudaMemcpy(p, L.bbox.data(), L.bbox.size() * sizeof(int4), cudaMemcpyHostToDevice) != cudaSuccess)
            goto fail;
        p += align(L.bbox.size() * sizeof(int4));
        D.shift = (const int2 *)p;
        if (!L.shift.empty() &&
            cudaMemcpy(p, L.shift.data(), L.shift.size() * sizeof(int2), cudaMemcpyHostToDevice) != cudaSuccess)
            goto fail;
        p += align(std::max<size_t>(1, L.shift.size()) * sizeof(int2));
        {
            std::vector<float4> base((size_t)L.n);
            for (int i = 0; i < L.n; ++i) {
                double mg = sqrt((double)L.gx[i] * L.gx[i] + (double)L.gy[i] * L.gy[i]);
                base[i] = make_float4((float)L.tx[i], (float)L.ty[i], (float)(L.gx[i] / mg), (float)(L.gy[i] / mg));
            }
            D.base = (const float4 *)p;
            if (cudaMemcpy(p, base.data(), base.size() * sizeof(float4), cudaMemcpyHostToDevice) != cudaSuccess)
                goto fail;
            p += align((size_t)L.n * sizeof(float4));
        }
        D.crot = nullptr;
        D.cstart = nullptr;
        D.cbox = nullptr;
        D.crange = nullptr;
        D.cspan_x = L.cspan_x;
        D.cspan_y = L.cspan_y;
        if (!L.crot.empty()) {
            D.crot = (const RotPt *)p;
            if (cudaMemcpy(p, L.crot.data(), L.crot.size() * sizeof(RotPt), cudaMemcpyHostToDevice) != cudaSuccess)
                goto fail;
            p += align(L.crot.size() * sizeof(RotPt));
            D.cstart = (const int *)p;
            if (cudaMemcpy(p, L.cstart.data(), L.cstart.size() * sizeof(int), cudaMemcpyHostToDevice) != cudaSuccess)
                goto fail;
            p += align(L.cstart.size() * sizeof(int));
            D.cbox = (const int4 *)p;
            if (cudaMemcpy(p, L.cbox.data(), L.cbox.size() * sizeof(int4), cudaMemcpyHostToDevice) != cudaSuccess)
                goto fail;
            p += align(L.cbox.size() * sizeof(int4));
            D.crange = (const int2 *)p;
            if (cudaMemcpy(p, L.crange.data(), L.crange.size() * sizeof(int2), cudaMemcpyHostToDevice) != cudaSuccess)
                goto fail;
            p += align(L.crange.size() * sizeof(int2));
        }
    }
    m->d_tables = base;
    m->device = dev;
    return SAM_OK;
fail:
    cudaFree(base);
    return SAM_ERR_CUDA;
}

}  // namespace sam
