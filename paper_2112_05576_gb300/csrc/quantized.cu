// Quantised-direction score maps (response maps): an approximation of
// Eq. (1) in which every rotated model direction is replaced by the centre
// of its orientation bin.  The window maximum of Eq. (1) then depends only
// on the bin, so it is precomputed once per image and bin,
//   R_b(x, y) = max over the window at (x, y) of u_b . w_hat  (|.| for
//   polarity 1), for -1 <= x <= w, -1 <= y <= h (0 farther outside),
// and the score of a pose is a gather-add over the model points,
//   M_q(u, theta_k) = (1/n) sum_i R_{b_i(k)}(u + o_i(k)).
// Error bound: |M_q - M| <= 2 sin(bin width / 4).
//
// The bins of the rotated directions are computed on the host in FP64 from
// the model's integer gradients with the same rotation as the offsets
// (theta = k dtheta pi / 180; the direction normalised, then rotated), then
// b = floor(atan2 / width + 1/2) mod nbins (the angle taken mod pi for
// polarity 1), and cached on the model per (level, bins).

#include <math.h>
#include <stdint.h>

#include <algorithm>
#include <mutex>
#include <vector>

#include "sam_internal.h"

namespace sam {
namespace {

constexpr int kMaxBins = 64;

struct BinCentres {
    float2 u[kMaxBins];
};

// One thread per extended pixel (x in [-1, w], y in [-1, h]) of one image:
// the window's w_hat loaded once, then every bin's maximum.
template <int NB>
__global__ void __launch_bounds__(256) response_maps_kernel(const float2 *__restrict__ field, int w, int h,
                                                            int nbins, int polarity, const BinCentres c,
                                                            float *__restrict__ maps) {
    const int we = w + 2, he = h + 2;
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= we * he)
        return;
    const int y = idx / we - 1, x = idx % we - 1;
    float2 win[NB * NB];
#pragma unroll
    for (int a = 0; a < NB; ++a)
#pragma unroll
        for (int b = 0; b < NB; ++b) {
            const int X = x + b - NB / 2, Y = y + a - NB / 2;
            win[a * NB + b] = (X >= 0 && Y >= 0 && X < w && Y < h) ? __ldg(field + (size_t)Y * w + X)
                                                                     : make_float2(0.f, 0.f);
        }
    for (int bin = 0; bin < nbins; ++bin) {
        const float2 u = c.u[bin];
        float m = -INFINITY;
#pragma unroll
        for (int q = 0; q < NB * NB; ++q) {
            float v = fmaf(u.x, win[q].x, u.y * win[q].y);
            if (polarity)
                v = fabsf(v);
            m = fmaxf(m, v);
        }
        maps[(size_t)bin * we * he + idx] = m;
    }
}

// Gather-add: one thread per pose of a row segment (consecutive x in a warp,
// so each point's reads are contiguous), one CTA per (row, angle).
__global__ void __launch_bounds__(256) score_quantized_kernel(const float *__restrict__ maps,
                                                              const RotPt *__restrict__ rot,
                                                              const uint8_t *__restrict__ bins, int n, int w, int h,
                                                              float *__restrict__ out) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y, k = blockIdx.z;
    const int we = w + 2, he = h + 2;
    const RotPt *P = rot + (size_t)k * n;
    const uint8_t *B = bins + (size_t)k * n;
    float sum = 0.f;
    if (x < w) {
        for (int i = 0; i < n; ++i) {
            const RotPt p = P[i];
            const int X = x + p.ox, Y = y + p.oy;
            if (X >= -1 && Y >= -1 && X <= w && Y <= h)
                sum += __ldg(maps + ((size_t)B[i] * he + (Y + 1)) * we + (X + 1));
        }
        out[((size_t)k * h + y) * w + x] = sum / (float)n;
    }
}

// Host: the bins of the rotated directions of one level.
std::vector<uint8_t> quant_bins(const LevelHost &L, int nbins, int polarity) {
    std::vector<uint8_t> out((size_t)L.ntheta * L.n);
    const double width = (polarity ? M_PI : 2.0 * M_PI) / nbins;
    for (int k = 0; k < L.ntheta; ++k) {
        // table k: scale k / nangles (directions do not depend on it), angle k mod nangles
        const double th = ((double)(k % L.nangles) * L.dtheta) * M_PI / 180.0;
        const double c = cos(th), s = sin(th);
        for (int i = 0; i < L.n; ++i) {
            const double m = sqrt((double)L.gx[i] * L.gx[i] + (double)L.gy[i] * L.gy[i]);
            const double ux = L.gx[i] / m, uy = L.gy[i] / m;
            const double px = c * ux - s * uy, py = s * ux + c * uy;
            double a = atan2(py, px);
            if (polarity && a < 0.0)
                a += M_PI;
            int b = (int)floor(a / width + 0.5) % nbins;
            if (b < 0)
                b += nbins;
            out[(size_t)k * L.n + i] = (uint8_t)b;
        }
    }
    return out;
}

// The model's device bin table of (level, nbins), built and uploaded (on
// `st`, behind the call's later launches) on first use; the model's table
// list is guarded so that host threads sharing a model do not race on it.
const uint8_t *bins_table(sam_model *m, int level, int nbins, cudaStream_t st) {
    static std::mutex mu;
    std::lock_guard<std::mutex> lock(mu);
    const int key = nbins * 2 + (m->p.polarity ? 1 : 0);
    for (const auto &q : m->qbins)
        if (q.level == level && q.nbins == key)
            return q.dev;
    const std::vector<uint8_t> h = quant_bins(m->lv[level], nbins, m->p.polarity ? 1 : 0);
    uint8_t *d = nullptr;
    if (cudaMalloc(&d, h.size()) != cudaSuccess)
        return nullptr;
    // pageable source: the copy is staged before the call returns
    if (cudaMemcpyAsync(d, h.data(), h.size(), cudaMemcpyHostToDevice, st) != cudaSuccess) {
        cudaFree(d);
        return nullptr;
    }
    m->qbins.push_back({level, key, d});
    return d;
}

}  // namespace
}  // namespace sam

using namespace sam;

extern "C" size_t sam_response_maps_bytes(int w, int h, int nbins) {
    if (w < 1 || h < 1 || nbins < 1 || nbins > kMaxBins)
        return 0;
    return (size_t)nbins * (size_t)(w + 2) * (size_t)(h + 2) * sizeof(float);
}

extern "C" sam_status sam_score_map_quantized(sam_model *m, int level, const float *field, int w, int h, int nbins,
                                              int neighbourhood, float *maps, size_t maps_bytes, float *map,
                                              void *stream) {
    if (!m || level < 0 || level >= m->levels || !field || !maps || !map || w < 1 || h < 1 || nbins < 2 ||
        nbins > kMaxBins || (neighbourhood != 1 && neighbourhood != 3) ||
        maps_bytes < sam_response_maps_bytes(w, h, nbins) || (uintptr_t)field % 8 || (uintptr_t)maps % 4)
        return SAM_ERR_ARG;
    sam_status s = upload_model(m);
    if (s != SAM_OK)
        return s;
    const uint8_t *bins = bins_table(m, level, nbins, (cudaStream_t)stream);
    if (!bins)
        return SAM_ERR_NOMEM;
    const int pol = m->p.polarity ? 1 : 0;
    BinCentres c;
    for (int b = 0; b < kMaxBins; ++b) {
        const double phi = b * (pol ? M_PI : 2.0 * M_PI) / nbins;
        c.u[b] = make_float2((float)cos(phi), (float)sin(phi));
    }
    cudaStream_t st = (cudaStream_t)stream;
    const int ext = (w + 2) * (h + 2);
    const float2 *f = reinterpret_cast<const float2 *>(field);
    if (neighbourhood == 3)
        response_maps_kernel<3><<<(ext + 255) / 256, 256, 0, st>>>(f, w, h, nbins, pol, c, maps);
    else
        response_maps_kernel<1><<<(ext + 255) / 256, 256, 0, st>>>(f, w, h, nbins, pol, c, maps);
    const LevelHost &L = m->lv[level];
    dim3 grid((unsigned)((w + 255) / 256), (unsigned)h, (unsigned)L.ntheta);
    score_quantized_kernel<<<grid, 256, 0, st>>>(maps, m->dev[level].rot, bins, L.n, w, h, map);
    count_launches(2);
    return cudaGetLastError() == cudaSuccess ? SAM_OK : SAM_ERR_CUDA;
}
