/*
 * Plain FP64 CPU oracle of the shape-based alignment detector of
 * T.-S. Le and C.-Y. Lin, "GPU-accelerated image alignment for object
 * detection in industrial applications" (arXiv 2112.05576).
 *
 * TEST INFRASTRUCTURE, NOT PART OF THE PRODUCT.  Only the tests, the smoke
 * check and the benchmark's CPU-baseline leg may load this code.  It shares
 * no source, header, table or helper with the CUDA library; it is written
 * for a reader checking it against the paper, one plain loop per step:
 * single-threaded, FP64, no blocking, no vectorisation.
 *
 * Readings of the paper where it is silent (the paper names no gradient
 * operator, pyramid filter, threshold units, rounding, border rule or
 * coarse-to-fine rule); every one is listed with its justification in the
 * project's design notes:
 *   - gradients: 3x3 Sobel, x to the right, y downwards, integer; the
 *     1-pixel image border has zero gradient (never an edge);
 *   - magnitude unit: |g| / 4 (a step of height h has magnitude h), an edge
 *     is gx^2 + gy^2 >= 16 T^2 (exact integer compare);
 *   - search image: single threshold T_low; model: hysteresis (>= T_high
 *     seeds, grown 8-connected through >= T_low);
 *   - pyramid of intensities, 2x2 mean rounded half up, odd row/col dropped;
 *   - template reference point (floor(W/2), floor(H/2)) at every level;
 *   - projected points rounded to nearest, floor(v + 1/2), in FP64;
 *   - samples outside the image or on non-edge pixels contribute 0.
 *
 * Build: gcc -O2 -fPIC -shared -ffp-contract=off (no -ffast-math, no FMA
 * contraction, so the rounding of projected points is the plain IEEE one).
 */

#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_PI 3.14159265358979323846

/* ------------------------------------------------------------------------ */
/* Sec. II: after edge extraction the method builds an image pyramid.       */
/* One pyramid step: 2x2 block mean, rounded half up; odd trailing row/col   */
/* dropped.  dst is (w/2) x (h/2), row-major, stride w/2.                    */
/* ------------------------------------------------------------------------ */
void or_pyramid_down(const uint8_t *src, int w, int h, uint8_t *dst)
{
    int w2 = w / 2, h2 = h / 2;
    for (int y = 0; y < h2; ++y) {
        for (int x = 0; x < w2; ++x) {
            int s = src[(2 * y) * w + 2 * x] + src[(2 * y) * w + 2 * x + 1] +
                    src[(2 * y + 1) * w + 2 * x] + src[(2 * y + 1) * w + 2 * x + 1];
            dst[y * w2 + x] = (uint8_t)((s + 2) / 4);
        }
    }
}

/* ------------------------------------------------------------------------ */
/* Sec. II: the x and y gradients and the gradient magnitude of every edge  */
/* point are kept.  Operator (unnamed in the paper): 3x3 Sobel, integer:    */
/*   gx = sum_{r=-1..1} w_r (I[y+r][x+1] - I[y+r][x-1]),  w = (1, 2, 1)      */
/*   gy = sum_{c=-1..1} w_c (I[y+1][x+c] - I[y-1][x+c])                      */
/* Border pixels (first/last row and column) get gx = gy = 0.                */
/* ------------------------------------------------------------------------ */
void or_sobel(const uint8_t *img, int w, int h, int32_t *gx, int32_t *gy)
{
    static const int wt[3] = {1, 2, 1};
    for (int y = 0; y < h; ++y) {
        for (int x = 0; x < w; ++x) {
            int32_t sx = 0, sy = 0;
            if (x > 0 && y > 0 && x < w - 1 && y < h - 1) {
                for (int r = -1; r <= 1; ++r)
                    sx += wt[r + 1] * ((int)img[(y + r) * w + x + 1] - (int)img[(y + r) * w + x - 1]);
                for (int c = -1; c <= 1; ++c)
                    sy += wt[c + 1] * ((int)img[(y + 1) * w + x + c] - (int)img[(y - 1) * w + x + c]);
            }
            gx[y * w + x] = sx;
            gy[y * w + x] = sy;
        }
    }
}

/* Edge test of one pixel: magnitude |g|/4 >= T, i.e. gx^2 + gy^2 >= 16 T^2. */
static int or_is_edge(int32_t gx, int32_t gy, int T)
{
    int64_t m2 = (int64_t)gx * gx + (int64_t)gy * gy;
    return m2 >= (int64_t)16 * T * T;
}

/* Sec. II edge thresholds, search image: one threshold T_low.              */
void or_search_mask(const int32_t *gx, const int32_t *gy, int npx, int low, uint8_t *mask)
{
    for (int i = 0; i < npx; ++i)
        mask[i] = (uint8_t)or_is_edge(gx[i], gy[i], low);
}

/* Sec. II edge thresholds, model image: hysteresis.  A pixel is
 * an edge if it is >= T_low and 8-connected through >= T_low pixels to a
 * pixel >= T_high.  Plain flood fill with an explicit stack.               */
void or_hysteresis(const int32_t *gx, const int32_t *gy, int w, int h, int low, int high, uint8_t *mask)
{
    int npx = w * h;
    int *stack = (int *)malloc(sizeof(int) * (size_t)(npx > 0 ? npx : 1));
    int top = 0;
    for (int i = 0; i < npx; ++i)
        mask[i] = 0;
    for (int i = 0; i < npx; ++i) {
        if (mask[i] || !or_is_edge(gx[i], gy[i], high))
            continue;
        mask[i] = 1;
        stack[top++] = i;
        while (top > 0) {
            int p = stack[--top];
            int py = p / w, px = p % w;
            for (int dy = -1; dy <= 1; ++dy) {
                for (int dx = -1; dx <= 1; ++dx) {
                    int qx = px + dx, qy = py + dy;
                    if (qx < 0 || qy < 0 || qx >= w || qy >= h)
                        continue;
                    int q = qy * w + qx;
                    if (!mask[q] && or_is_edge(gx[q], gy[q], low)) {
                        mask[q] = 1;
                        stack[top++] = q;
                    }
                }
            }
        }
    }
    free(stack);
}

/* Eq. (1) normalisation of the search image: w_hat = (gx, gy) / |g| on edge
 * pixels, (0, 0) elsewhere.  field is interleaved (wx, wy) per pixel.     */
void or_unit_field(const int32_t *gx, const int32_t *gy, const uint8_t *mask, int npx, double *field)
{
    for (int i = 0; i < npx; ++i) {
        if (mask[i]) {
            double m = sqrt((double)gx[i] * gx[i] + (double)gy[i] * gy[i]);
            field[2 * i] = gx[i] / m;
            field[2 * i + 1] = gy[i] / m;
        } else {
            field[2 * i] = 0.0;
            field[2 * i + 1] = 0.0;
        }
    }
}

/* Model edge points of one template level (Sec. II): Sobel, hysteresis, then
 * every edge pixel in raster order with t = (col - floor(w/2), row -
 * floor(h/2)) and its integer gradient.  Returns the number of points; the
 * output arrays must hold w*h entries.                                     */
int or_model_points(const uint8_t *tmpl, int w, int h, int low, int high,
                    int32_t *tx, int32_t *ty, int32_t *pgx, int32_t *pgy)
{
    int npx = w * h;
    int32_t *gx = (int32_t *)malloc(sizeof(int32_t) * (size_t)npx);
    int32_t *gy = (int32_t *)malloc(sizeof(int32_t) * (size_t)npx);
    uint8_t *mask = (uint8_t *)malloc((size_t)npx);
    or_sobel(tmpl, w, h, gx, gy);
    or_hysteresis(gx, gy, w, h, low, high, mask);
    int n = 0;
    for (int row = 0; row < h; ++row) {
        for (int col = 0; col < w; ++col) {
            int i = row * w + col;
            if (!mask[i])
                continue;
            tx[n] = col - w / 2;
            ty[n] = row - h / 2;
            pgx[n] = gx[i];
            pgy[n] = gy[i];
            ++n;
        }
    }
    free(gx);
    free(gy);
    free(mask);
    return n;
}

/* Eq. (2): p = R(theta) t + u.  For angle index k at a level whose angle step
 * is dtheta_deg, theta = (k * dtheta_deg) * pi / 180 (FP64).  Offsets are
 * rounded to the nearest pixel, floor(v + 1/2); the model gradient is turned
 * by the same rotation and normalised to a unit vector p_hat.              */
void or_rotate_points(const int32_t *tx, const int32_t *ty, const int32_t *gx, const int32_t *gy, int n,
                      int k, double dtheta_deg, int32_t *ox, int32_t *oy, double *px, double *py)
{
    double th = ((double)k * dtheta_deg) * OR_PI / 180.0;
    double c = cos(th), s = sin(th);
    for (int i = 0; i < n; ++i) {
        double x = (double)tx[i], y = (double)ty[i];
        ox[i] = (int32_t)floor(c * x - s * y + 0.5);
        oy[i] = (int32_t)floor(s * x + c * y + 0.5);
        double m = sqrt((double)gx[i] * gx[i] + (double)gy[i] * gy[i]);
        double ux = gx[i] / m, uy = gy[i] / m;
        px[i] = c * ux - s * uy;
        py[i] = s * ux + c * uy;
    }
}

/* One point's vote (Sec. II neighbouring search + Eq. (1) term): the maximum,
 * over the nbhd x nbhd window around the projected point, of
 * p_hat . w_hat (polarity 0) or |p_hat . w_hat| (polarity 1).  Samples
 * outside the image count as w_hat = 0.                                    */
static double or_vote(const double *field, int w, int h, int x0, int y0, double px, double py,
                      int nbhd, int polarity)
{
    int r = nbhd / 2;
    double best = -INFINITY;
    for (int b = -r; b <= r; ++b) {
        for (int a = -r; a <= r; ++a) {
            int x = x0 + a, y = y0 + b;
            double v = 0.0;
            if (x >= 0 && y >= 0 && x < w && y < h) {
                const double *wv = field + 2 * ((size_t)y * w + x);
                v = px * wv[0] + py * wv[1];
                if (polarity)
                    v = fabs(v);
            }
            if (v > best)
                best = v;
        }
    }
    return best;
}

/* Eq. (1): M(u, theta) = (1/n) sum_i vote_i, the points already rotated for
 * theta (offsets ox, oy and unit directions px, py).                       */
double or_score_pose(const double *field, int w, int h, const int32_t *ox, const int32_t *oy,
                     const double *px, const double *py, int n, int ux, int uy, int nbhd, int polarity)
{
    double sum = 0.0;
    for (int i = 0; i < n; ++i)
        sum += or_vote(field, w, h, ux + ox[i], uy + oy[i], px[i], py[i], nbhd, polarity);
    return sum / n;
}

/* Sec. II CPU design: exhaustive search with three nested loops over
 * x-translation, y-translation and rotation; every pose scored by Eq. (1).
 * Poses are u = (gxi * step_x, gyi * step_y) for the grid gxi < ceil(w /
 * step_x), gyi < ceil(h / step_y), and theta_k for k < ntheta.  The map is
 * written out[(k * gh + gyi) * gw + gxi].  Eq. (2) depends on theta only, so
 * each angle's rotated points are computed once up front.  The _range form
 * scores the angles k_begin .. k_begin + k_count - 1 only (a slice of the
 * same map, written from out[0]).                                          */
void or_score_map_range(const double *field, int w, int h, const int32_t *tx, const int32_t *ty,
                        const int32_t *gx, const int32_t *gy, int n, int k_begin, int k_count, double dtheta_deg,
                        int step_x, int step_y, int nbhd, int polarity, double *out)
{
    int gw = (w + step_x - 1) / step_x, gh = (h + step_y - 1) / step_y;
    int32_t *ox = (int32_t *)malloc(sizeof(int32_t) * (size_t)n * k_count);
    int32_t *oy = (int32_t *)malloc(sizeof(int32_t) * (size_t)n * k_count);
    double *px = (double *)malloc(sizeof(double) * (size_t)n * k_count);
    double *py = (double *)malloc(sizeof(double) * (size_t)n * k_count);
    for (int j = 0; j < k_count; ++j)
        or_rotate_points(tx, ty, gx, gy, n, k_begin + j, dtheta_deg, ox + (size_t)j * n, oy + (size_t)j * n,
                         px + (size_t)j * n, py + (size_t)j * n);
    for (int gxi = 0; gxi < gw; ++gxi) {
        for (int gyi = 0; gyi < gh; ++gyi) {
            for (int j = 0; j < k_count; ++j) {
                size_t o = (size_t)j * n;
                out[((size_t)j * gh + gyi) * gw + gxi] =
                    or_score_pose(field, w, h, ox + o, oy + o, px + o, py + o, n, gxi * step_x, gyi * step_y,
                                  nbhd, polarity);
            }
        }
    }
    free(ox);
    free(oy);
    free(px);
    free(py);
}

/* The full map: all angles k = 0 .. ntheta-1. */
void or_score_map(const double *field, int w, int h, const int32_t *tx, const int32_t *ty,
                  const int32_t *gx, const int32_t *gy, int n, int ntheta, double dtheta_deg,
                  int step_x, int step_y, int nbhd, int polarity, double *out)
{
    or_score_map_range(field, w, h, tx, ty, gx, gy, n, 0, ntheta, dtheta_deg, step_x, step_y, nbhd, polarity, out);
}

/* Total order used for every selection: higher score first, then the
 * smaller key (angle index, y, x) -- the key is the row-major index.       */
static int or_beats(double sa, long ka, double sb, long kb)
{
    return sa > sb || (sa == sb && ka < kb);
}

/* Candidate extraction at the top level (Sec. II keeps the maximum-score
 * pose; several instances need several): poses with M >= min_score that
 * beat each of their up to 26 neighbours in (theta, y, x), theta circular,
 * translations clipped at the grid border; the K best by the order above.
 * Returns the number written (<= K).                                       */
static double *or_sort_scores;
static long *or_sort_keys;
static int or_cmp_idx(const void *a, const void *b)
{
    int i = *(const int *)a, j = *(const int *)b;
    if (or_beats(or_sort_scores[i], or_sort_keys[i], or_sort_scores[j], or_sort_keys[j]))
        return -1;
    if (or_beats(or_sort_scores[j], or_sort_keys[j], or_sort_scores[i], or_sort_keys[i]))
        return 1;
    return 0;
}

int or_candidates(const double *map, int nth, int gh, int gw, double min_score, int K,
                  int32_t *ck, int32_t *cy, int32_t *cx, double *cs)
{
    size_t total = (size_t)nth * gh * gw;
    int cap = 1024, cnt = 0;
    double *sc = (double *)malloc(sizeof(double) * cap);
    long *key = (long *)malloc(sizeof(long) * cap);
    for (int k = 0; k < nth; ++k) {
        for (int y = 0; y < gh; ++y) {
            for (int x = 0; x < gw; ++x) {
                long kp = ((long)k * gh + y) * gw + x;
                double s = map[kp];
                if (!(s >= min_score))
                    continue;
                int ok = 1;
                for (int dk = -1; dk <= 1 && ok; ++dk) {
                    if (dk != 0 && nth == 1)
                        continue;
                    int k2 = ((k + dk) % nth + nth) % nth;
                    for (int dy = -1; dy <= 1 && ok; ++dy) {
                        for (int dx = -1; dx <= 1 && ok; ++dx) {
                            if (dk == 0 && dy == 0 && dx == 0)
                                continue;
                            int y2 = y + dy, x2 = x + dx;
                            if (y2 < 0 || x2 < 0 || y2 >= gh || x2 >= gw)
                                continue;
                            long kq = ((long)k2 * gh + y2) * gw + x2;
                            if (kq == kp)
                                continue;
                            if (!or_beats(s, kp, map[kq], kq))
                                ok = 0;
                        }
                    }
                }
                if (!ok)
                    continue;
                if (cnt == cap) {
                    cap *= 2;
                    sc = (double *)realloc(sc, sizeof(double) * cap);
                    key = (long *)realloc(key, sizeof(long) * cap);
                }
                sc[cnt] = s;
                key[cnt] = kp;
                ++cnt;
            }
        }
    }
    (void)total;
    int *idx = (int *)malloc(sizeof(int) * (size_t)(cnt > 0 ? cnt : 1));
    for (int i = 0; i < cnt; ++i)
        idx[i] = i;
    or_sort_scores = sc;
    or_sort_keys = key;
    qsort(idx, (size_t)cnt, sizeof(int), or_cmp_idx);
    int nout = cnt < K ? cnt : K;
    for (int i = 0; i < nout; ++i) {
        long kp = key[idx[i]];
        cx[i] = (int32_t)(kp % gw);
        cy[i] = (int32_t)((kp / gw) % gh);
        ck[i] = (int32_t)(kp / ((long)gw * gh));
        cs[i] = sc[idx[i]];
    }
    free(idx);
    free(sc);
    free(key);
    return nout;
}

/* Coarse-to-fine shift (the paper only says scoring starts at the top
 * level).  A level-(l+1) pixel X covers level-l pixels 2X and 2X+1, so its
 * centre is 2X + 1/2; a level-(l+1) template point t' has its centre at the
 * level-l template point 2t' + d with d = 2 c_{l+1} + 1/2 - c_l per axis
 * (c = reference point).  A level-(l+1) pose u' therefore maps to the level-l
 * pose 2u' + (1/2, 1/2) - R(theta) d, whose nearest pixel is 2u' + shift.
 * theta is the parent's angle, (k_parent * dtheta_parent_deg) * pi / 180.  */
void or_child_shift(int k_parent, double dtheta_parent_deg, double dx, double dy, int32_t *sx, int32_t *sy)
{
    double th = ((double)k_parent * dtheta_parent_deg) * OR_PI / 180.0;
    double c = cos(th), s = sin(th);
    *sx = (int32_t)floor(0.5 - (c * dx - s * dy) + 0.5);
    *sy = (int32_t)floor(0.5 - (s * dx + c * dy) + 0.5);
}

/* One refinement level (neighbouring-search size 3 in x, y and theta): for
 * each parent pose (x', y', k') at level l+1, evaluate the 27 level-l poses
 * x in cx + {-1,0,1}, y in cy + {-1,0,1}, k in 2k' + {-1,0,1} (mod ntheta),
 * with (cx, cy) = 2 (x', y') + shift(k'), skipping poses outside the image,
 * and keep the best by the total order above.  Writes the refined pose and
 * score; a parent whose best score is below min_score (or that has no pose
 * inside the image) gets score -inf.                                       */
void or_refine_level(const double *field, int w, int h, const int32_t *tx, const int32_t *ty,
                     const int32_t *gx, const int32_t *gy, int n, int ntheta, double dtheta_deg,
                     double dx, double dy, int nbhd, int polarity, double min_score, int ncand,
                     const int32_t *in_x, const int32_t *in_y, const int32_t *in_k,
                     int32_t *out_x, int32_t *out_y, int32_t *out_k, double *out_s)
{
    int32_t *ox = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    int32_t *oy = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    double *px = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    double *py = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    for (int c = 0; c < ncand; ++c) {
        int32_t sx, sy;
        or_child_shift(in_k[c], 2.0 * dtheta_deg, dx, dy, &sx, &sy);
        int cxp = 2 * in_x[c] + sx, cyp = 2 * in_y[c] + sy;
        double best = -INFINITY;
        long bkey = 0;
        int bx = 0, by = 0, bk = 0;
        for (int dk = -1; dk <= 1; ++dk) {
            int k = ((2 * in_k[c] + dk) % ntheta + ntheta) % ntheta;
            or_rotate_points(tx, ty, gx, gy, n, k, dtheta_deg, ox, oy, px, py);
            for (int ddy = -1; ddy <= 1; ++ddy) {
                for (int ddx = -1; ddx <= 1; ++ddx) {
                    int x = cxp + ddx, y = cyp + ddy;
                    if (x < 0 || y < 0 || x >= w || y >= h)
                        continue;
                    double s = or_score_pose(field, w, h, ox, oy, px, py, n, x, y, nbhd, polarity);
                    long key = ((long)k * h + y) * w + x;
                    if (best == -INFINITY || or_beats(s, key, best, bkey)) {
                        best = s;
                        bkey = key;
                        bx = x;
                        by = y;
                        bk = k;
                    }
                }
            }
        }
        out_x[c] = bx;
        out_y[c] = by;
        out_k[c] = bk;
        out_s[c] = (best >= min_score) ? best : -INFINITY;
    }
    free(ox);
    free(oy);
    free(px);
    free(py);
}

/* Final non-maximum suppression over level-0 detections: visit by the total
 * order (score, then key (k, y, x) with the level-0 image width w and height
 * h); keep a detection unless a kept one lies closer than half the smaller
 * template side, compared exactly as 4 (dx^2 + dy^2) < min_side^2.  Entries
 * with score -inf are skipped.  Writes indices of kept entries in order and
 * returns how many (at most max_out).                                      */
int or_nms(int n, const int32_t *x, const int32_t *y, const int32_t *k, const double *s, int w, int h,
           int min_side, int max_out, int32_t *keep)
{
    int *idx = (int *)malloc(sizeof(int) * (size_t)(n > 0 ? n : 1));
    long *key = (long *)malloc(sizeof(long) * (size_t)(n > 0 ? n : 1));
    double *sc = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    for (int i = 0; i < n; ++i) {
        idx[i] = i;
        key[i] = ((long)k[i] * h + y[i]) * w + x[i];
        sc[i] = s[i];
    }
    or_sort_scores = sc;
    or_sort_keys = key;
    qsort(idx, (size_t)n, sizeof(int), or_cmp_idx);
    int nk = 0;
    for (int a = 0; a < n && nk < max_out; ++a) {
        int i = idx[a];
        if (s[i] == -INFINITY)
            continue;
        int ok = 1;
        for (int b = 0; b < nk; ++b) {
            long ddx = x[i] - x[keep[b]], ddy = y[i] - y[keep[b]];
            if (4 * (ddx * ddx + ddy * ddy) < (long)min_side * min_side) {
                ok = 0;
                break;
            }
        }
        if (ok)
            keep[nk++] = i;
    }
    free(idx);
    free(key);
    free(sc);
    return nk;
}

/* ======================================================================== */
/* Differentiable score on a continuous pose (an extension of Eq. (1); the  */
/* paper scores integer poses only).  For a continuous pose u = (x, y) and  */
/* angle theta in degrees, every model point is placed at                   */
/*   p_i = R(theta) t_i + u            (Eq. (2), no rounding)               */
/* and its unit model direction turned to d_i = R(theta) g_i / |g_i|.       */
/* The search field w_hat is sampled by bilinear interpolation at p_i (the  */
/* four surrounding pixels, those outside the image counting as (0, 0)):   */
/*   w_bil(p) = (1-fx)(1-fy) w00 + fx(1-fy) w10 + (1-fx) fy w01 + fx fy w11 */
/* with x0 = floor(px), fx = px - x0 (and the same in y).  No neighbourhood */
/* maximum is taken (it is not differentiable).  The score is              */
/*   M_c = (1/n) sum_i term_i,   term_i = d_i . w_bil(p_i)                  */
/* (polarity 1: |d_i . w_bil(p_i)|).  Inside a pixel cell w_bil is          */
/* bilinear, so its partial derivatives there are                           */
/*   dw/dx = (1-fy)(w10 - w00) + fy(w11 - w01)                              */
/*   dw/dy = (1-fx)(w01 - w00) + fx(w11 - w10)                              */
/* (one-sided at cell borders, the side that floor() selects).  Chain rule: */
/*   d term/dx = d . dw/dx,  d term/dy = d . dw/dy,                         */
/*   d term/dtheta = (R'g/|g|) . w_bil + d . (dw/dx (R't)_x + dw/dy (R't)_y) */
/* with R' = dR/dtheta = [[-s, -c], [c, -s]], times pi/180 per degree.      */
/* Polarity 1 multiplies each derivative by sign(d . w_bil) (0 at 0).       */
/* ======================================================================== */

/* Field vector at integer pixel (x, y); (0, 0) outside the image. */
static void or_field_at(const double *field, int w, int h, int x, int y, double *vx, double *vy)
{
    if (x >= 0 && y >= 0 && x < w && y < h) {
        *vx = field[2 * ((size_t)y * w + x)];
        *vy = field[2 * ((size_t)y * w + x) + 1];
    } else {
        *vx = 0.0;
        *vy = 0.0;
    }
}

/* Score M_c at (x, y, theta_deg).  Optional outputs (NULL to skip), all
 * divided by n like the score:
 *   grad[3] = dM_c / d(x, y, theta_deg);
 *   jtj[6]  = (1/n) sum_i J_i J_i^T  as (xx, xy, xt, yy, yt, tt);
 *   jtr[3]  = (1/n) sum_i J_i (1 - term_i);
 * where J_i = d term_i / d(x, y, theta_deg): the normal equations of the
 * Gauss-Newton fit of every term to 1.                                    */
double or_score_bilinear(const double *field, int w, int h, const int32_t *tx, const int32_t *ty,
                         const int32_t *gx, const int32_t *gy, int n, double x, double y, double theta_deg,
                         int polarity, double *grad, double *jtj, double *jtr)
{
    double th = theta_deg * OR_PI / 180.0;
    double c = cos(th), s = sin(th);
    double sum = 0.0;
    double g[3] = {0.0, 0.0, 0.0};
    double a[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    double b[3] = {0.0, 0.0, 0.0};
    for (int i = 0; i < n; ++i) {
        double txi = (double)tx[i], tyi = (double)ty[i];
        double m = sqrt((double)gx[i] * gx[i] + (double)gy[i] * gy[i]);
        double ux = gx[i] / m, uy = gy[i] / m;
        /* Eq. (2) and the turned direction */
        double px = c * txi - s * tyi + x;
        double py = s * txi + c * tyi + y;
        double dx = c * ux - s * uy;
        double dy = s * ux + c * uy;
        /* bilinear sample */
        double fx0 = floor(px), fy0 = floor(py);
        int x0 = (int)fx0, y0 = (int)fy0;
        double fx = px - fx0, fy = py - fy0;
        double w00x, w00y, w10x, w10y, w01x, w01y, w11x, w11y;
        or_field_at(field, w, h, x0, y0, &w00x, &w00y);
        or_field_at(field, w, h, x0 + 1, y0, &w10x, &w10y);
        or_field_at(field, w, h, x0, y0 + 1, &w01x, &w01y);
        or_field_at(field, w, h, x0 + 1, y0 + 1, &w11x, &w11y);
        double wx = (1 - fx) * (1 - fy) * w00x + fx * (1 - fy) * w10x + (1 - fx) * fy * w01x + fx * fy * w11x;
        double wy = (1 - fx) * (1 - fy) * w00y + fx * (1 - fy) * w10y + (1 - fx) * fy * w01y + fx * fy * w11y;
        double dwx_dx = (1 - fy) * (w10x - w00x) + fy * (w11x - w01x);
        double dwy_dx = (1 - fy) * (w10y - w00y) + fy * (w11y - w01y);
        double dwx_dy = (1 - fx) * (w01x - w00x) + fx * (w11x - w10x);
        double dwy_dy = (1 - fx) * (w01y - w00y) + fx * (w11y - w10y);
        double term = dx * wx + dy * wy;
        /* derivatives of term */
        double jx = dx * dwx_dx + dy * dwy_dx;
        double jy = dx * dwx_dy + dy * dwy_dy;
        double rtx = -s * txi - c * tyi;     /* (R' t)_x */
        double rty = c * txi - s * tyi;      /* (R' t)_y */
        double rdx = -s * ux - c * uy;       /* (R' g/|g|)_x */
        double rdy = c * ux - s * uy;        /* (R' g/|g|)_y */
        double jt = (rdx * wx + rdy * wy + jx * rtx + jy * rty) * (OR_PI / 180.0);
        if (polarity) {
            double sg = term > 0 ? 1.0 : (term < 0 ? -1.0 : 0.0);
            term = fabs(term);
            jx *= sg;
            jy *= sg;
            jt *= sg;
        }
        sum += term;
        g[0] += jx;
        g[1] += jy;
        g[2] += jt;
        a[0] += jx * jx;
        a[1] += jx * jy;
        a[2] += jx * jt;
        a[3] += jy * jy;
        a[4] += jy * jt;
        a[5] += jt * jt;
        b[0] += jx * (1.0 - term);
        b[1] += jy * (1.0 - term);
        b[2] += jt * (1.0 - term);
    }
    if (grad)
        for (int j = 0; j < 3; ++j)
            grad[j] = g[j] / n;
    if (jtj)
        for (int j = 0; j < 6; ++j)
            jtj[j] = a[j] / n;
    if (jtr)
        for (int j = 0; j < 3; ++j)
            jtr[j] = b[j] / n;
    return sum / n;
}

/* Marks (mask[i] = 1) the model points whose sample p_i at (x, y,
 * theta_deg) lies within eps of a pixel-cell border in x or in y, where the
 * one-sided derivative of the bilinear sample may jump.  Returns how many.  */
int or_bilinear_border_mask(const int32_t *tx, const int32_t *ty, int n, double x, double y, double theta_deg,
                            double eps, uint8_t *mask)
{
    double th = theta_deg * OR_PI / 180.0;
    double c = cos(th), s = sin(th);
    int cnt = 0;
    for (int i = 0; i < n; ++i) {
        double px = c * tx[i] - s * ty[i] + x;
        double py = s * tx[i] + c * ty[i] + y;
        double ex = px - floor(px + 0.5), ey = py - floor(py + 0.5);
        mask[i] = (uint8_t)(fabs(ex) < eps || fabs(ey) < eps);
        cnt += mask[i];
    }
    return cnt;
}

/* Solve the symmetric 3x3 system A d = b (A packed as xx, xy, xt, yy, yt,
 * tt) by Cramer's rule.  Returns 0 if the determinant is not positive.    */
static int or_solve3(const double *A, const double *b, double *d)
{
    double a00 = A[0], a01 = A[1], a02 = A[2], a11 = A[3], a12 = A[4], a22 = A[5];
    double c00 = a11 * a22 - a12 * a12;
    double c01 = a02 * a12 - a01 * a22;
    double c02 = a01 * a12 - a02 * a11;
    double det = a00 * c00 + a01 * c01 + a02 * c02;
    if (!(det > 0.0))
        return 0;
    double c11 = a00 * a22 - a02 * a02;
    double c12 = a01 * a02 - a00 * a12;
    double c22 = a00 * a11 - a01 * a01;
    d[0] = (c00 * b[0] + c01 * b[1] + c02 * b[2]) / det;
    d[1] = (c01 * b[0] + c11 * b[1] + c12 * b[2]) / det;
    d[2] = (c02 * b[0] + c12 * b[1] + c22 * b[2]) / det;
    return 1;
}

/* Continuous pose refinement by damped Gauss-Newton (Levenberg-Marquardt)
 * on the terms of M_c, each fitted to 1:
 *   lambda = 1e-3; evaluate M_c, J^T J, J^T r at the pose;
 *   repeat `iterations` times:
 *     A = J^T J + lambda diag(J^T J) + 1e-9 I;  solve A d = J^T r;
 *     scale d down so that max(|dx|, |dy|, |dtheta|) <= 1 (px, px, deg);
 *     evaluate at pose + d; if M_c rose strictly, move there and set
 *     lambda = max(lambda / 3, 1e-7); else lambda = min(4 lambda, 1e7).
 * If the system is singular the iteration only raises lambda.  Every
 * iteration costs exactly one evaluation of M_c and its normal equations.
 * pose[3] = (x, y, theta_deg) in and out; returns the final M_c.           */
double or_refine_gn(const double *field, int w, int h, const int32_t *tx, const int32_t *ty,
                    const int32_t *gx, const int32_t *gy, int n, int polarity, double *pose, int iterations)
{
    double A[6], b[3];
    double lambda = 1e-3;
    double S = or_score_bilinear(field, w, h, tx, ty, gx, gy, n, pose[0], pose[1], pose[2], polarity, NULL, A, b);
    for (int it = 0; it < iterations; ++it) {
        double M[6] = {A[0], A[1], A[2], A[3], A[4], A[5]};
        M[0] += lambda * A[0] + 1e-9;
        M[3] += lambda * A[3] + 1e-9;
        M[5] += lambda * A[5] + 1e-9;
        double d[3];
        if (!or_solve3(M, b, d)) {
            lambda = fmin(4.0 * lambda, 1e7);
            continue;
        }
        double big = fmax(fabs(d[0]), fmax(fabs(d[1]), fabs(d[2])));
        if (big > 1.0) {
            d[0] /= big;
            d[1] /= big;
            d[2] /= big;
        }
        double q[3] = {pose[0] + d[0], pose[1] + d[1], pose[2] + d[2]};
        double A2[6], b2[3];
        double S2 = or_score_bilinear(field, w, h, tx, ty, gx, gy, n, q[0], q[1], q[2], polarity, NULL, A2, b2);
        if (S2 > S) {
            pose[0] = q[0];
            pose[1] = q[1];
            pose[2] = q[2];
            S = S2;
            memcpy(A, A2, sizeof(A));
            memcpy(b, b2, sizeof(b));
            lambda = fmax(lambda / 3.0, 1e-7);
        } else {
            lambda = fmin(4.0 * lambda, 1e7);
        }
    }
    return S;
}

/* Sub-pixel and sub-angle peak of a 3x3x3 neighbourhood of Eq. (1) scores
 * (the quadratic-fit refinement of the digitised pose; not in the paper).
 * s[(dk + 1) * 9 + (dy + 1) * 3 + (dx + 1)] = M at (x + dx, y + dy, k + dk).
 * Gradient g and Hessian H of M at the centre from central differences:
 *   g_a = (M(+a) - M(-a)) / 2,  H_aa = M(+a) - 2 M(0) + M(-a),
 *   H_ab = (M(+a+b) - M(+a-b) - M(-a+b) + M(-a-b)) / 4,
 * the second-order Taylor model of M whose stationary point is
 * delta = -H^-1 g.  That point is used when H is negative definite (the
 * model has a maximum); otherwise every axis with H_aa < 0 takes its own
 * parabola's vertex -g_a / H_aa and the others 0.  Each component is then
 * clamped to [-1/2, 1/2] (a farther peak belongs to a neighbouring cell).
 * delta[] = (dx, dy, dk): pixels, pixels, angle steps.                     */
void or_subpixel_fit(const double *s, double *delta)
{
#define S(dk, dy, dx) s[((dk) + 1) * 9 + ((dy) + 1) * 3 + ((dx) + 1)]
    const double c = S(0, 0, 0);
    double g[3], hxx, hyy, hkk, hxy, hxk, hyk;
    g[0] = 0.5 * (S(0, 0, 1) - S(0, 0, -1));
    g[1] = 0.5 * (S(0, 1, 0) - S(0, -1, 0));
    g[2] = 0.5 * (S(1, 0, 0) - S(-1, 0, 0));
    hxx = S(0, 0, 1) - 2.0 * c + S(0, 0, -1);
    hyy = S(0, 1, 0) - 2.0 * c + S(0, -1, 0);
    hkk = S(1, 0, 0) - 2.0 * c + S(-1, 0, 0);
    hxy = 0.25 * (S(0, 1, 1) - S(0, -1, 1) - S(0, 1, -1) + S(0, -1, -1));
    hxk = 0.25 * (S(1, 0, 1) - S(-1, 0, 1) - S(1, 0, -1) + S(-1, 0, -1));
    hyk = 0.25 * (S(1, 1, 0) - S(-1, 1, 0) - S(1, -1, 0) + S(-1, -1, 0));
#undef S
    /* -H, packed xx, xy, xk, yy, yk, kk */
    const double A[6] = {-hxx, -hxy, -hxk, -hyy, -hyk, -hkk};
    const int definite = A[0] > 0.0 && A[0] * A[3] - A[1] * A[1] > 0.0;
    if (!(definite && or_solve3(A, g, delta))) {
        delta[0] = hxx < 0.0 ? -g[0] / hxx : 0.0;
        delta[1] = hyy < 0.0 ? -g[1] / hyy : 0.0;
        delta[2] = hkk < 0.0 ? -g[2] / hkk : 0.0;
    }
    for (int a = 0; a < 3; ++a)
        delta[a] = fmin(0.5, fmax(-0.5, delta[a]));
}

/* Quantised-direction form (an approximation of Eq. (1); not in the paper).
 * Bin of a unit direction among nbins orientation bins: polarity 0 bins of
 * width 2 pi / nbins centred on b 2 pi / nbins; polarity 1 (a direction and
 * its opposite are one orientation) bins of width pi / nbins centred on
 * b pi / nbins.  b = floor(a / width + 1/2) mod nbins, a = atan2(py, px),
 * taken mod pi for polarity 1.                                             */
int or_quant_bin(double px, double py, int nbins, int polarity)
{
    double a = atan2(py, px);
    double width = (polarity ? OR_PI : 2.0 * OR_PI) / nbins;
    if (polarity && a < 0.0)
        a += OR_PI;
    int b = (int)floor(a / width + 0.5);
    b %= nbins;
    if (b < 0)
        b += nbins;
    return b;
}

/* Unit vector of bin b's centre.                                           */
static void or_bin_centre(int b, int nbins, int polarity, double *ux, double *uy)
{
    double phi = b * (polarity ? OR_PI : 2.0 * OR_PI) / nbins;
    *ux = cos(phi);
    *uy = sin(phi);
}

/* The quantised score: Eq. (1) with every rotated model direction replaced
 * by the unit vector of its bin's centre,
 *   M_q(u, theta_k) = (1/n) sum_i max_window u_{b_i} . w_hat  (|.| for
 *   polarity 1; samples outside the image are 0, as in Eq. (1)),
 * over the full pose grid (out[(k * h + y) * w + x], step 1).              */
void or_score_map_quantized(const double *field, int w, int h, const int32_t *tx, const int32_t *ty,
                            const int32_t *gx, const int32_t *gy, int n, int ntheta, double dtheta_deg,
                            int nbins, int nbhd, int polarity, double *out)
{
    int32_t *ox = malloc(sizeof(int32_t) * (size_t)n), *oy = malloc(sizeof(int32_t) * (size_t)n);
    double *px = malloc(sizeof(double) * (size_t)n), *py = malloc(sizeof(double) * (size_t)n);
    double *qx = malloc(sizeof(double) * (size_t)n), *qy = malloc(sizeof(double) * (size_t)n);
    for (int k = 0; k < ntheta; ++k) {
        or_rotate_points(tx, ty, gx, gy, n, k, dtheta_deg, ox, oy, px, py);
        for (int i = 0; i < n; ++i)
            or_bin_centre(or_quant_bin(px[i], py[i], nbins, polarity), nbins, polarity, &qx[i], &qy[i]);
        for (int y = 0; y < h; ++y)
            for (int x = 0; x < w; ++x) {
                double sum = 0.0;
                for (int i = 0; i < n; ++i)
                    sum += or_vote(field, w, h, x + ox[i], y + oy[i], qx[i], qy[i], nbhd, polarity);
                out[((size_t)k * h + y) * w + x] = sum / n;
            }
    }
    free(ox);
    free(oy);
    free(px);
    free(py);
    free(qx);
    free(qy);
}

/* Response maps of the quantised form: for every bin b and every window
 * centre (x, y) with -1 <= x <= w, -1 <= y <= h,
 *   R_b(x, y) = max_window u_b . w_hat (|.| for polarity 1),
 * out[(b * (h + 2) + y + 1) * (w + 2) + x + 1]; a centre farther outside has
 * an all-outside window, R = 0.                                            */
void or_response_maps(const double *field, int w, int h, int nbhd, int polarity, int nbins, double *out)
{
    for (int b = 0; b < nbins; ++b) {
        double ux, uy;
        or_bin_centre(b, nbins, polarity, &ux, &uy);
        for (int y = -1; y <= h; ++y)
            for (int x = -1; x <= w; ++x)
                out[((size_t)b * (h + 2) + y + 1) * (w + 2) + x + 1] =
                    or_vote(field, w, h, x, y, ux, uy, nbhd, polarity);
    }
}

/* ------------------------------------------------------------------------
 * Angle-only storage of the search field (a storage form; the paper keeps
 * x- and y-gradients, Sec. II).  An edge pixel of the search threshold
 * becomes the 16-bit code 0x8000 | a with
 *     a = round(atan2(gy, gx) * 32768 / (2 pi)) mod 32768,
 * its direction quantised to 2^15 steps of 2 pi / 32768 (round half up);
 * any other pixel becomes 0.  The stored direction is then off by at most
 * half a step, pi / 32768, and an Eq. (1) term by at most 2 sin(pi / 65536).
 * ---------------------------------------------------------------------- */
void or_angle_codes(const int32_t *gx, const int32_t *gy, int npx, int low, uint16_t *codes)
{
    for (int i = 0; i < npx; ++i) {
        if (!or_is_edge(gx[i], gy[i], low)) {
            codes[i] = 0;
            continue;
        }
        double t = atan2((double)gy[i], (double)gx[i]) * 32768.0 / (2.0 * OR_PI);
        long a = (long)floor(t + 0.5) % 32768;
        if (a < 0)
            a += 32768;
        codes[i] = (uint16_t)(0x8000 | a);
    }
}

/* The unit field the codes stand for: (cos phi, sin phi), phi = a 2 pi /
 * 32768, where the edge bit is set; (0, 0) elsewhere.                      */
void or_angle_field(const uint16_t *codes, int npx, double *field)
{
    for (int i = 0; i < npx; ++i) {
        if (codes[i] & 0x8000) {
            double phi = (double)(codes[i] & 0x7fff) * (2.0 * OR_PI) / 32768.0;
            field[2 * i] = cos(phi);
            field[2 * i + 1] = sin(phi);
        } else {
            field[2 * i] = 0.0;
            field[2 * i + 1] = 0.0;
        }
    }
}

/* ------------------------------------------------------------------------
 * Affine projection, a generalisation of Eq. (2) (the paper notes that other
 * kinds of projection could be implemented; a scaled pose is A = s R(theta)):
 * p = A t + u, A = [[a11, a12], [a21, a22]], offsets rounded to the nearest
 * pixel as in Eq. (2), floor(v + 1/2).  The model gradient is carried by the
 * inverse transpose: the gradient of the warped image I(A^-1 x) at A t is
 * A^-T times the gradient of I at t, so p_hat = A^-T g / |A^-T g|, with
 * A^-T = (1 / det A) [[a22, -a21], [-a12, a11]].  Returns 0 (and writes
 * nothing) when det A = 0, else 1.
 * ---------------------------------------------------------------------- */
int or_project_affine(const int32_t *tx, const int32_t *ty, const int32_t *gx, const int32_t *gy, int n,
                      double a11, double a12, double a21, double a22, int32_t *ox, int32_t *oy, double *px,
                      double *py)
{
    double det = a11 * a22 - a12 * a21;
    if (det == 0.0)
        return 0;
    for (int i = 0; i < n; ++i) {
        double x = (double)tx[i], y = (double)ty[i];
        ox[i] = (int32_t)floor(a11 * x + a12 * y + 0.5);
        oy[i] = (int32_t)floor(a21 * x + a22 * y + 0.5);
        double vx = (a22 * gx[i] - a21 * gy[i]) / det;
        double vy = (a11 * gy[i] - a12 * gx[i]) / det;
        double m = sqrt(vx * vx + vy * vy);
        px[i] = vx / m;
        py[i] = vy / m;
    }
    return 1;
}

/* ======================================================================== */
/* Scaled poses: Eq. (2) with R(theta) replaced by A = s R(theta) (the      */
/* paper notes that other kinds of projection could be implemented).  The   */
/* search runs over a grid of scales s_j (j < nscales) as well as angles    */
/* theta_k and translations; the scale grid is the same at every pyramid    */
/* level (a scale is a ratio of sizes).  Readings, listed in the design     */
/* notes: a pose (x, y, k, j) is keyed ((j nth + k) H + y) W + x in every   */
/* selection; candidates are strict local maxima over the up to 80          */
/* neighbours in (j, theta circular, y, x), j not circular; the descent     */
/* searches j - 1 .. j + 1 (clipped to the grid) as well as x, y and theta, */
/* up to 81 poses per level; the child shift turns and scales d by A.       */
/* ======================================================================== */

/* The model points projected for scale `scale` and angle index k (angle as
 * in or_rotate_points): A = [[s c, -(s sn)], [s sn, s c]].                 */
int or_scaled_points(const int32_t *tx, const int32_t *ty, const int32_t *gx, const int32_t *gy, int n, int k,
                     double dtheta_deg, double scale, int32_t *ox, int32_t *oy, double *px, double *py)
{
    double th = ((double)k * dtheta_deg) * OR_PI / 180.0;
    double c = cos(th), sn = sin(th);
    return or_project_affine(tx, ty, gx, gy, n, scale * c, -(scale * sn), scale * sn, scale * c, ox, oy, px, py);
}

/* Exhaustive map over scales, angles and step-1 translations (the three
 * nested loops of Sec. II with a scale loop around them):
 * out[((j * nth + k) * h + y) * w + x] = M(x, y, theta_k, s_j).            */
void or_score_map_scaled(const double *field, int w, int h, const int32_t *tx, const int32_t *ty,
                         const int32_t *gx, const int32_t *gy, int n, const double *scales, int nscales, int nth,
                         double dtheta_deg, int nbhd, int polarity, double *out)
{
    int32_t *ox = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    int32_t *oy = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    double *px = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    double *py = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    for (int j = 0; j < nscales; ++j) {
        for (int k = 0; k < nth; ++k) {
            or_scaled_points(tx, ty, gx, gy, n, k, dtheta_deg, scales[j], ox, oy, px, py);
            for (int y = 0; y < h; ++y)
                for (int x = 0; x < w; ++x)
                    out[(((size_t)j * nth + k) * h + y) * w + x] =
                        or_score_pose(field, w, h, ox, oy, px, py, n, x, y, nbhd, polarity);
        }
    }
    free(ox);
    free(oy);
    free(px);
    free(py);
}

/* Candidates over (scale, angle, y, x): poses with M >= min_score that beat
 * each of their up to 80 neighbours (j +- 1 inside the grid, theta
 * circular, y and x clipped), the K best by the total order.  Returns the
 * number written (<= K).                                                   */
int or_candidates_scaled(const double *map, int ns, int nth, int gh, int gw, double min_score, int K,
                         int32_t *cj, int32_t *ck, int32_t *cy, int32_t *cx, double *cs)
{
    int cap = 1024, cnt = 0;
    double *sc = (double *)malloc(sizeof(double) * cap);
    long *key = (long *)malloc(sizeof(long) * cap);
    for (int j = 0; j < ns; ++j) {
        for (int k = 0; k < nth; ++k) {
            for (int y = 0; y < gh; ++y) {
                for (int x = 0; x < gw; ++x) {
                    long kp = (((long)j * nth + k) * gh + y) * gw + x;
                    double s = map[kp];
                    if (!(s >= min_score))
                        continue;
                    int ok = 1;
                    for (int dj = -1; dj <= 1 && ok; ++dj) {
                        int j2 = j + dj;
                        if (j2 < 0 || j2 >= ns)
                            continue;
                        for (int dk = -1; dk <= 1 && ok; ++dk) {
                            if (dk != 0 && nth == 1)
                                continue;
                            int k2 = ((k + dk) % nth + nth) % nth;
                            for (int dy = -1; dy <= 1 && ok; ++dy) {
                                for (int dx = -1; dx <= 1 && ok; ++dx) {
                                    int y2 = y + dy, x2 = x + dx;
                                    if (y2 < 0 || x2 < 0 || y2 >= gh || x2 >= gw)
                                        continue;
                                    long kq = (((long)j2 * nth + k2) * gh + y2) * gw + x2;
                                    if (kq == kp)
                                        continue;
                                    if (!or_beats(s, kp, map[kq], kq))
                                        ok = 0;
                                }
                            }
                        }
                    }
                    if (!ok)
                        continue;
                    if (cnt == cap) {
                        cap *= 2;
                        sc = (double *)realloc(sc, sizeof(double) * cap);
                        key = (long *)realloc(key, sizeof(long) * cap);
                    }
                    sc[cnt] = s;
                    key[cnt] = kp;
                    ++cnt;
                }
            }
        }
    }
    int *idx = (int *)malloc(sizeof(int) * (size_t)(cnt > 0 ? cnt : 1));
    for (int i = 0; i < cnt; ++i)
        idx[i] = i;
    or_sort_scores = sc;
    or_sort_keys = key;
    qsort(idx, (size_t)cnt, sizeof(int), or_cmp_idx);
    int nout = cnt < K ? cnt : K;
    for (int i = 0; i < nout; ++i) {
        long kp = key[idx[i]];
        cx[i] = (int32_t)(kp % gw);
        cy[i] = (int32_t)((kp / gw) % gh);
        ck[i] = (int32_t)((kp / ((long)gw * gh)) % nth);
        cj[i] = (int32_t)(kp / ((long)gw * gh * nth));
        cs[i] = sc[idx[i]];
    }
    free(idx);
    free(sc);
    free(key);
    return nout;
}

/* Coarse-to-fine shift of a scaled parent (as or_child_shift, with d turned
 * and scaled by the parent's A = s R(theta)).                              */
void or_child_shift_scaled(int k_parent, double dtheta_parent_deg, double scale, double dx, double dy, int32_t *sx,
                           int32_t *sy)
{
    double th = ((double)k_parent * dtheta_parent_deg) * OR_PI / 180.0;
    double c = cos(th), sn = sin(th);
    double a11 = scale * c, a12 = -(scale * sn), a21 = scale * sn, a22 = scale * c;
    *sx = (int32_t)floor(0.5 - (a11 * dx + a12 * dy) + 0.5);
    *sy = (int32_t)floor(0.5 - (a21 * dx + a22 * dy) + 0.5);
}

/* One refinement level with scales: for each level-(l+1) parent (x', y', k',
 * j') the level-l poses x, y in centre +- 1, k in 2k' + {-1, 0, 1} (mod nth)
 * and j in j' + {-1, 0, 1} inside the scale grid, centre = 2 (x', y') +
 * shift(k', s_j'); the best by the total order; -inf below min_score.      */
void or_refine_level_scaled(const double *field, int w, int h, const int32_t *tx, const int32_t *ty,
                            const int32_t *gx, const int32_t *gy, int n, const double *scales, int ns, int nth,
                            double dtheta_deg, double dx, double dy, int nbhd, int polarity, double min_score,
                            int ncand, const int32_t *in_x, const int32_t *in_y, const int32_t *in_j,
                            const int32_t *in_k, int32_t *out_x, int32_t *out_y, int32_t *out_j, int32_t *out_k,
                            double *out_s)
{
    int32_t *ox = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    int32_t *oy = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    double *px = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    double *py = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    for (int c = 0; c < ncand; ++c) {
        int32_t sx, sy;
        or_child_shift_scaled(in_k[c], 2.0 * dtheta_deg, scales[in_j[c]], dx, dy, &sx, &sy);
        int cxp = 2 * in_x[c] + sx, cyp = 2 * in_y[c] + sy;
        double best = -INFINITY;
        long bkey = 0;
        int bx = 0, by = 0, bk = 0, bj = 0;
        for (int dj = -1; dj <= 1; ++dj) {
            int j = in_j[c] + dj;
            if (j < 0 || j >= ns)
                continue;
            for (int dk = -1; dk <= 1; ++dk) {
                int k = ((2 * in_k[c] + dk) % nth + nth) % nth;
                or_scaled_points(tx, ty, gx, gy, n, k, dtheta_deg, scales[j], ox, oy, px, py);
                for (int ddy = -1; ddy <= 1; ++ddy) {
                    for (int ddx = -1; ddx <= 1; ++ddx) {
                        int x = cxp + ddx, y = cyp + ddy;
                        if (x < 0 || y < 0 || x >= w || y >= h)
                            continue;
                        double s = or_score_pose(field, w, h, ox, oy, px, py, n, x, y, nbhd, polarity);
                        long key = (((long)j * nth + k) * h + y) * w + x;
                        if (best == -INFINITY || or_beats(s, key, best, bkey)) {
                            best = s;
                            bkey = key;
                            bx = x;
                            by = y;
                            bk = k;
                            bj = j;
                        }
                    }
                }
            }
        }
        out_x[c] = bx;
        out_y[c] = by;
        out_k[c] = bk;
        out_j[c] = bj;
        out_s[c] = (best >= min_score) ? best : -INFINITY;
    }
    free(ox);
    free(oy);
    free(px);
    free(py);
}
