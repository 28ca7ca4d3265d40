// Kernel (c), tiled form: exhaustive score map of one pyramid level
// (Sec. II: every pose scored by Eq. (1) over the model points projected by
// Eq. (2), each point taking its best vote over the 3x3 neighbouring-search
// window).
//
// Work decomposition.  A CTA owns a super-tile of translations (SX x SY warp
// tiles of 48 x 32 poses) of one image and a group of TG consecutive angles.
// One TMA load stages the w_hat window that every (angle, pose, point,
// neighbour) of the CTA can touch -- the super-tile grown by the union of the
// group's rotated offset bounding boxes and the 1-pixel search halo -- into
// shared memory; pixels outside the image arrive as zeros, which is exactly
// Eq. (1)'s contribution of a missing edge.  Warps then loop over (angle,
// warp tile) items.
//
// Register blocking.  A thread owns an R x C = 8 x 6 block of poses.  For one
// model point the block's 3x3 windows cover (R+2) x (C+2) pixels; each pixel's
// dot product with the point's direction is computed once (packed FP32x2 FMA
// on a pixel pair) and shared by the up to nine poses whose windows hold it,
// the 3x3 maximum is taken separably with 3-input max, and the result is
// accumulated in FP32 (packed adds).  Per pose-point: ~0.9 shared loads,
// ~1.9 FMA-pipe instructions for the dots, 2.25 max, 0.5 add.
//
// Field layout (pixel pairs).  The window is FP32 with pixels 2j, 2j+1 of a
// row stored as {wx_2j, wx_2j+1, wy_2j, wy_2j+1} (16 bytes), so one 128-bit
// shared load feeds one packed FMA pair.  Lanes are laid out 8 along x and 4
// along y; the 8 lanes of a quarter-warp start 3 pixel pairs apart, so their
// 128-bit loads fall in 8 distinct 16-byte bank groups.
//
// Early termination (exact-safe, see kernels_score.cu): every 32 points a warp
// abandons its tile when every pose's partial sum proves M < min_score.

#include <cuda.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <mutex>

#include "sam_internal.h"
#include "score_common.cuh"

namespace sam {

// Set (never cleared by the kernel) when a bounded wait for the window's TMA
// copy gives up; read and cleared by the host after a synchronising call.
__device__ int g_score_err;

namespace {

constexpr int TR = 8;            // rows of poses per thread
constexpr int TC = 6;            // columns of poses per thread (TC/2 odd: bank-conflict-free 128-bit loads)
constexpr int LX = 8, LY = 4;    // lanes along x, y
constexpr int WTX = LX * TC;     // warp tile: 48 x 32 poses
constexpr int WTY = LY * TR;
constexpr int PRUNE_EVERY = 32;

struct TiledArgs {
    const RotPt *rot;     // [nth][n]
    const int4 *bbox;     // [nth]
    int n, nth;
    int W, H;             // level size (poses = pixels, step 1)
    float *map;
    size_t map_img;
    int sx, sy, tg;       // super-tile in warp tiles, angles per group
    int tiles_x;          // super-tiles along x
    int bxw, byw;         // window box (pixels, rows)
    float inv_n;
    float thresh;
    int early;
    int polarity;
};



__device__ __forceinline__ float max3(float a, float b, float c) {
    float d;
    asm("max.f32 %0, %1, %2, %3;" : "=f"(d) : "f"(a), "f"(b), "f"(c));
    return d;
}

__device__ __forceinline__ uint32_t smem_addr(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// Bounded wait on an mbarrier phase; false if it did not complete.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
    for (int it = 0; it < (1 << 24); ++it) {
        uint32_t done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(bar), "r"(parity)
            : "memory");
        if (done)
            return true;
    }
    return false;
}

template <int NB, bool POL>
__device__ __forceinline__ void dots_row(const float4 *row, int pair0, float (&d)[TC + 4], int npairs,
                                         float2 pxx, float2 pyy) {
#pragma unroll
    for (int q = 0; q < (TC + 4) / 2; ++q) {
        if (q < npairs) {
            const float4 v = row[pair0 + q];
            float2 t = __fmul2_rn(pxx, make_float2(v.x, v.y));
            t = __ffma2_rn(pyy, make_float2(v.z, v.w), t);
            d[2 * q] = POL ? fabsf(t.x) : t.x;
            d[2 * q + 1] = POL ? fabsf(t.y) : t.y;
        }
    }
}

// One model point over the thread's R x C pose block, 3x3 neighbourhood.
template <bool POL, bool ODD>
__device__ __forceinline__ void point_nb3(const float4 *win, int pp, int row0, int pair0, float2 pxx, float2 pyy,
                                          float2 (&acc)[TR][TC / 2]) {
    constexpr int NP = ODD ? (TC + 4) / 2 : (TC + 2) / 2;   // pixel pairs per row
    constexpr int OFF = ODD ? 1 : 0;
    float hp2[TC], hp1[TC];
#pragma unroll
    for (int r = 0; r < TR + 2; ++r) {
        const float4 *row = win + (row0 + r) * pp;
        float d[TC + 4];
        dots_row<3, POL>(row, pair0, d, NP, pxx, pyy);
        float h[TC];
#pragma unroll
        for (int c = 0; c < TC; ++c)
            h[c] = max3(d[OFF + c], d[OFF + c + 1], d[OFF + c + 2]);
        if (r >= 2) {
#pragma unroll
            for (int j = 0; j < TC / 2; ++j) {
                const float v0 = max3(hp2[2 * j], hp1[2 * j], h[2 * j]);
                const float v1 = max3(hp2[2 * j + 1], hp1[2 * j + 1], h[2 * j + 1]);
                acc[r - 2][j] = __fadd2_rn(acc[r - 2][j], make_float2(v0, v1));
            }
        }
#pragma unroll
        for (int c = 0; c < TC; ++c) {
            hp2[c] = hp1[c];
            hp1[c] = h[c];
        }
    }
}

// One model point, neighbourhood 1 (no search): the centre pixel only.
template <bool POL, bool ODD>
__device__ __forceinline__ void point_nb1(const float4 *win, int pp, int row0, int pair0, float2 pxx, float2 pyy,
                                          float2 (&acc)[TR][TC / 2]) {
    constexpr int NP = ODD ? (TC + 2) / 2 : TC / 2;
#pragma unroll
    for (int r = 0; r < TR; ++r) {
        const float4 *row = win + (row0 + r) * pp;
        float d[TC + 4];
        dots_row<1, POL>(row, pair0, d, NP, pxx, pyy);
#pragma unroll
        for (int j = 0; j < TC / 2; ++j) {
            if (ODD)
                acc[r][j] = __fadd2_rn(acc[r][j], make_float2(d[2 * j + 1], d[2 * j + 2]));
            else
                acc[r][j] = __fadd2_rn(acc[r][j], make_float2(d[2 * j], d[2 * j + 1]));
        }
    }
}

template <int NB, bool POL, int WARPS>
__global__ void __launch_bounds__(WARPS * 32) score_tiled_kernel(const __grid_constant__ CUtensorMap tmap,
                                                                  const TiledArgs a) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    // the TMA destination must be 128-byte aligned: round the base up (the
    // launch adds 128 bytes of slack)
    const uint32_t pad = (128u - (smem_addr(smem_raw) & 127u)) & 127u;
    float4 *win = reinterpret_cast<float4 *>(smem_raw + pad);
    __shared__ __align__(8) unsigned long long mbar;
    __shared__ int s_org[2];   // window origin (pixel x, row y), global coords

    const int img = blockIdx.z;
    const int group = blockIdx.y;
    const int st = blockIdx.x;
    const int stx0 = (st % a.tiles_x) * a.sx * WTX;
    const int sty0 = (st / a.tiles_x) * a.sy * WTY;
    const int k_begin = group * a.tg;
    const int k_end = min(k_begin + a.tg, a.nth);
    const int pp = a.bxw / 2;   // window row pitch in pixel pairs
    const uint32_t bar = smem_addr(&mbar);

    if (threadIdx.x == 0) {
        int xmin = 1 << 30, ymin = 1 << 30;
        for (int k = k_begin; k < k_end; ++k) {
            const int4 b = a.bbox[k];
            xmin = min(xmin, b.x);
            ymin = min(ymin, b.z);
        }
        const int wx0 = (stx0 + xmin - 1) & ~1;   // even: 16-byte aligned TMA start
        const int wy0 = sty0 + ymin - 1;
        s_org[0] = wx0;
        s_org[1] = wy0;
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        const uint32_t bytes = (uint32_t)a.bxw * (uint32_t)a.byw * 8u;
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
        asm volatile(
            "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
            "[%5];" ::"r"(smem_addr(win)),
            "l"(reinterpret_cast<uint64_t>(&tmap)), "r"(wx0), "r"(wy0), "r"(img), "r"(bar)
            : "memory");
    }
    __syncthreads();
    if (!mbar_wait(bar, 0)) {
        if (threadIdx.x == 0)
            atomicExch(&g_score_err, 1);
        return;
    }
    const int wx0 = s_org[0], wy0 = s_org[1];

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int lx = lane & (LX - 1), ly = lane >> 3;
    const int items = (k_end - k_begin) * a.sx * a.sy;
    float *map = a.map + (size_t)img * a.map_img;

    for (int it = warp; it < items; it += WARPS) {
        const int k = k_begin + it / (a.sx * a.sy);
        const int wt = it % (a.sx * a.sy);
        const int x0 = stx0 + (wt % a.sx) * WTX + lx * TC;   // thread's first pose
        const int y0 = sty0 + (wt / a.sx) * WTY + ly * TR;
        // window coordinates of the first needed pixel for offset (0, 0)
        const int bx = x0 - 1 - wx0;
        const int by = y0 - 1 - wy0;
        float2 acc[TR][TC / 2];
#pragma unroll
        for (int r = 0; r < TR; ++r)
#pragma unroll
            for (int j = 0; j < TC / 2; ++j)
                acc[r][j] = make_float2(0.f, 0.f);
        const RotPt *P = a.rot + (size_t)k * a.n;
        bool pruned = false;
        RotPt p = P[0];
        for (int i = 0; i < a.n; ++i) {
            const RotPt cur = p;
            if (i + 1 < a.n)
                p = P[i + 1];
            const float2 pxx = make_float2(cur.px, cur.px);
            const float2 pyy = make_float2(cur.py, cur.py);
            if (NB == 3) {
                const int xs = bx + cur.ox;   // first pixel column (>= 0)
                const int row0 = by + cur.oy;
                if (xs & 1)
                    point_nb3<POL, true>(win, pp, row0, (xs - 1) >> 1, pxx, pyy, acc);
                else
                    point_nb3<POL, false>(win, pp, row0, xs >> 1, pxx, pyy, acc);
            } else {
                const int xs = bx + 1 + cur.ox;   // centre column
                const int row0 = by + 1 + cur.oy;
                if (xs & 1)
                    point_nb1<POL, true>(win, pp, row0, (xs - 1) >> 1, pxx, pyy, acc);
                else
                    point_nb1<POL, false>(win, pp, row0, xs >> 1, pxx, pyy, acc);
            }
            if (a.early && ((i + 1) % PRUNE_EVERY) == 0) {
                const float lim = a.thresh - (float)(a.n - 1 - i);
                bool low = true;
#pragma unroll
                for (int r = 0; r < TR; ++r)
#pragma unroll
                    for (int j = 0; j < TC / 2; ++j)
                        low = low && (acc[r][j].x < lim) && (acc[r][j].y < lim);
                if (__all_sync(0xffffffffu, low)) {
                    pruned = true;
                    break;
                }
            }
        }
        // epilogue: M = sum / n, or -inf where pruned; clip to the level
        float *mk = map + (size_t)k * a.H * a.W;
#pragma unroll
        for (int r = 0; r < TR; ++r) {
            const int y = y0 + r;
            if (y >= a.H)
                break;
            float *row = mk + (size_t)y * a.W;
#pragma unroll
            for (int j = 0; j < TC / 2; ++j) {
                const int x = x0 + 2 * j;
                const float v0 = pruned ? -INFINITY : acc[r][j].x * a.inv_n;
                const float v1 = pruned ? -INFINITY : acc[r][j].y * a.inv_n;
                if (x + 1 < a.W && (a.W & 1) == 0) {
                    *reinterpret_cast<float2 *>(row + x) = make_float2(v0, v1);
                } else {
                    if (x < a.W)
                        row[x] = v0;
                    if (x + 1 < a.W)
                        row[x + 1] = v1;
                }
            }
        }
    }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------

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

template <int NB, bool POL, int WARPS>
cudaError_t launch_t(const CUtensorMap &tm, const TiledArgs &a, dim3 grid, size_t smem, cudaStream_t st) {
    auto kern = score_tiled_kernel<NB, POL, WARPS>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess)
        return e;
    // prefer the largest shared-memory carve-out so window size, not the
    // L1/shared split, limits resident CTAs
    e = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared);
    if (e != cudaSuccess)
        return e;
    kern<<<grid, WARPS * 32, smem, st>>>(tm, a);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace

// Window box for a tiling: the super-tile grown by the largest union of
// rotated offset boxes over any angle group, the 1-pixel search halo, one
// pixel of slack for the even TMA start and one for odd-start pair loads.
bool tiled_plan(const LevelHost &L, int sx, int sy, int tg, int *bxw, int *byw) {
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
    int bx = sx * WTX + spx + 4;
    bx = (bx + 1) & ~1;
    const int by = sy * WTY + spy + 2;
    *bxw = bx;
    *byw = by;
    return bx <= 256 && by <= 256 && (size_t)bx * by * 8 <= 200 * 1024;
}

// Launch over `count` images whose paired FP32 fields start at `field`
// (row pitch wp pixels, image stride field_img_px pixels).
cudaError_t launch_score_tiled(const sam_model *m, int level, const void *field, int wp, size_t field_img_px, int W,
                               int H, int count, int nbhd, int polarity, float min_score, int early, float *map,
                               size_t map_img, int *err, const TileConfig &cfg, cudaStream_t st) {
    const LevelHost &L = m->lv[level];
    int bxw = 0, byw = 0;
    if (!tiled_plan(L, cfg.sx, cfg.sy, cfg.tg, &bxw, &byw))
        return cudaErrorInvalidValue;
    EncodeTiledFn enc = encode_fn();
    if (!enc)
        return cudaErrorNotSupported;
    CUtensorMap tm;
    const cuuint64_t dims[3] = {(cuuint64_t)wp, (cuuint64_t)H, (cuuint64_t)count};
    const cuuint64_t strides[2] = {(cuuint64_t)wp * 8, (cuuint64_t)field_img_px * 8};
    const cuuint32_t box[3] = {(cuuint32_t)bxw, (cuuint32_t)byw, 1};
    const cuuint32_t estr[3] = {1, 1, 1};
    if (enc(&tm, CU_TENSOR_MAP_DATA_TYPE_UINT64, 3, const_cast<void *>(field), dims, strides, box, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return cudaErrorInvalidValue;
    TiledArgs a;
    a.rot = m->dev[level].rot;
    a.bbox = m->dev[level].bbox;
    a.n = L.n;
    a.nth = L.ntheta;
    a.W = W;
    a.H = H;
    a.map = map;
    a.map_img = map_img;
    a.sx = cfg.sx;
    a.sy = cfg.sy;
    a.tg = cfg.tg;
    a.tiles_x = (W + cfg.sx * WTX - 1) / (cfg.sx * WTX);
    const int tiles_y = (H + cfg.sy * WTY - 1) / (cfg.sy * WTY);
    a.bxw = bxw;
    a.byw = byw;
    a.inv_n = 1.0f / (float)L.n;
    a.thresh = prune_threshold(L.n, min_score, SAM_FP32);
    a.early = early;
    a.polarity = polarity;
    (void)err;
    const int groups = (L.ntheta + cfg.tg - 1) / cfg.tg;
    dim3 grid((unsigned)(a.tiles_x * tiles_y), (unsigned)groups, (unsigned)count);
    const size_t smem = (size_t)bxw * byw * 8 + 128;
    const bool pol = polarity != 0;
    switch (cfg.warps) {
    case 4:
        if (nbhd == 3)
            return pol ? launch_t<3, true, 4>(tm, a, grid, smem, st) : launch_t<3, false, 4>(tm, a, grid, smem, st);
        return pol ? launch_t<1, true, 4>(tm, a, grid, smem, st) : launch_t<1, false, 4>(tm, a, grid, smem, st);
    default:
        if (nbhd == 3)
            return pol ? launch_t<3, true, 8>(tm, a, grid, smem, st) : launch_t<3, false, 8>(tm, a, grid, smem, st);
        return pol ? launch_t<1, true, 8>(tm, a, grid, smem, st) : launch_t<1, false, 8>(tm, a, grid, smem, st);
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
