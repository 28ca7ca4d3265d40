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

// Set (never cleared by the kernel) when a bounded wait for the window's TMA
// copy gives up; read and cleared by the host after a synchronising call.
__device__ int g_score_err;

namespace {

constexpr int TR = 8;            // rows of poses per thread
constexpr int TC = 6;            // columns of poses per thread (TC/2 odd: conflict-free loads)
constexpr int PRUNE_EVERY = 32;

// Stored element type of the window: pair size, lane layout, TMA alignment.
template <typename E>
struct Pairs;

template <>
struct Pairs<float> {
    using Raw = float4;
    static constexpr int BYTES = 16;   // one pixel pair
    static constexpr int LX = 8;       // lanes along x
    static constexpr int XALIGN = 2;   // window start (pixels) for a 16-byte TMA start
    static __device__ __forceinline__ float4 get(const Raw *row, int q) { return row[q]; }
};

template <>
struct Pairs<__half> {
    using Raw = uint2;
    static constexpr int BYTES = 8;
    static constexpr int LX = 16;
    static constexpr int XALIGN = 4;
    static __device__ __forceinline__ float4 get(const Raw *row, int q) {
        const uint2 u = row[q];
        const float2 a = __half22float2(*reinterpret_cast<const __half2 *>(&u.x));
        const float2 b = __half22float2(*reinterpret_cast<const __half2 *>(&u.y));
        return make_float4(a.x, a.y, b.x, b.y);
    }
};

template <>
struct Pairs<__nv_bfloat16> {
    using Raw = uint2;
    static constexpr int BYTES = 8;
    static constexpr int LX = 16;
    static constexpr int XALIGN = 4;
    static __device__ __forceinline__ float4 get(const Raw *row, int q) {
        const uint2 u = row[q];
        // bf16 -> fp32 is a 16-bit left shift of the bit pattern
        return make_float4(__uint_as_float(u.x << 16), __uint_as_float(u.x & 0xFFFF0000u),
                           __uint_as_float(u.y << 16), __uint_as_float(u.y & 0xFFFF0000u));
    }
};

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

// Dot products of one pixel pair with the point direction.  FP32 storage:
// packed FP32x2 FMA.  FP16 and BF16 storage: mixed-precision FMA, the 16-bit
// products formed exactly and accumulated in FP32, with the direction
// rounded to the field's type as well (per-term error at most
// 2 sqrt(2) 2^-12 < 7e-4 for FP16, 2 sqrt(2) 2^-9 < 5.6e-3 for BF16, against
// exact arithmetic), which saves the conversions of the stored halves.
template <typename E>
struct PairDot {
    static __device__ __forceinline__ void run(const typename Pairs<E>::Raw *row, int q, float2 pxx, float2 pyy,
                                               float &d0, float &d1) {
        const float4 v = Pairs<E>::get(row, q);
        float2 t = __fmul2_rn(pxx, make_float2(v.x, v.y));
        t = __ffma2_rn(pyy, make_float2(v.z, v.w), t);
        d0 = t.x;
        d1 = t.y;
    }
};

template <>
struct PairDot<__half> {
    static __device__ __forceinline__ void run(const uint2 *row, int q, float2 pxx, float2 pyy, float &d0,
                                               float &d1) {
        const uint2 u = row[q];
        const unsigned short ph = __half_as_ushort(__float2half_rn(pxx.x));
        const unsigned short qh = __half_as_ushort(__float2half_rn(pyy.x));
        asm("{\n .reg .b16 x0, x1, y0, y1;\n .reg .f32 t0, t1;\n mov.b32 {x0, x1}, %2;\n mov.b32 {y0, y1}, %3;\n"
            " fma.rn.f32.f16 t0, %4, x0, 0f00000000;\n fma.rn.f32.f16 t1, %4, x1, 0f00000000;\n"
            " fma.rn.f32.f16 %0, %5, y0, t0;\n fma.rn.f32.f16 %1, %5, y1, t1;\n}"
            : "=f"(d0), "=f"(d1)
            : "r"(u.x), "r"(u.y), "h"(ph), "h"(qh));
    }
};

template <>
struct PairDot<__nv_bfloat16> {
    static __device__ __forceinline__ void run(const uint2 *row, int q, float2 pxx, float2 pyy, float &d0,
                                               float &d1) {
        const uint2 u = row[q];
        const unsigned short ph = __bfloat16_as_ushort(__float2bfloat16_rn(pxx.x));
        const unsigned short qh = __bfloat16_as_ushort(__float2bfloat16_rn(pyy.x));
        asm("{\n .reg .b16 x0, x1, y0, y1;\n .reg .f32 t0, t1;\n mov.b32 {x0, x1}, %2;\n mov.b32 {y0, y1}, %3;\n"
            " fma.rn.f32.bf16 t0, %4, x0, 0f00000000;\n fma.rn.f32.bf16 t1, %4, x1, 0f00000000;\n"
            " fma.rn.f32.bf16 %0, %5, y0, t0;\n fma.rn.f32.bf16 %1, %5, y1, t1;\n}"
            : "=f"(d0), "=f"(d1)
            : "r"(u.x), "r"(u.y), "h"(ph), "h"(qh));
    }
};

template <typename E, bool POL>
__device__ __forceinline__ void dots_row(const typename Pairs<E>::Raw *row, int pair0, float (&d)[TC + 4],
                                         int npairs, float2 pxx, float2 pyy) {
#pragma unroll
    for (int q = 0; q < (TC + 4) / 2; ++q) {
        if (q < npairs) {
            float d0, d1;
            PairDot<E>::run(row, pair0 + q, pxx, pyy, d0, d1);
            d[2 * q] = POL ? fabsf(d0) : d0;
            d[2 * q + 1] = POL ? fabsf(d1) : d1;
        }
    }
}

// One model point over the thread's R x C pose block, 3x3 neighbourhood.
template <typename E, bool POL, bool ODD>
__device__ __forceinline__ void point_nb3(const typename Pairs<E>::Raw *win, int pp, int row0, int pair0,
                                          float2 pxx, float2 pyy, float2 (&acc)[TR][TC / 2]) {
    constexpr int NP = ODD ? (TC + 4) / 2 : (TC + 2) / 2;   // pixel pairs per row
    constexpr int OFF = ODD ? 1 : 0;
    float hp2[TC], hp1[TC];
#pragma unroll
    for (int r = 0; r < TR + 2; ++r) {
        const typename Pairs<E>::Raw *row = win + (row0 + r) * pp;
        float d[TC + 4];
        dots_row<E, POL>(row, pair0, d, NP, pxx, pyy);
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
template <typename E, bool POL, bool ODD>
__device__ __forceinline__ void point_nb1(const typename Pairs<E>::Raw *win, int pp, int row0, int pair0,
                                          float2 pxx, float2 pyy, float2 (&acc)[TR][TC / 2]) {
    constexpr int NP = ODD ? (TC + 2) / 2 : TC / 2;
#pragma unroll
    for (int r = 0; r < TR; ++r) {
        const typename Pairs<E>::Raw *row = win + (row0 + r) * pp;
        float d[TC + 4];
        dots_row<E, POL>(row, pair0, d, NP, pxx, pyy);
#pragma unroll
        for (int j = 0; j < TC / 2; ++j) {
            if (ODD)
                acc[r][j] = __fadd2_rn(acc[r][j], make_float2(d[2 * j + 1], d[2 * j + 2]));
            else
                acc[r][j] = __fadd2_rn(acc[r][j], make_float2(d[2 * j], d[2 * j + 1]));
        }
    }
}

// What a CTA work unit needs besides its window.
struct TileWork {
    const RotPt *rot;
    int n, W, H;
    int ox, oy, k0;   // pose and angle of map element (0, 0, 0)
    float *map;   // the image's (or pair's) map [nk][H][W]
    float inv_n, thresh;
    int early, sx, sy;
};

template <typename E, int NB, bool POL, int WARPS>
__device__ __forceinline__ void score_items(const typename Pairs<E>::Raw *win, int pp, int wx0, int wy0, int stx0,
                                            int sty0, int k_begin, int k_end, const TileWork &a);

template <typename E, int NB, bool POL, int WARPS>
__global__ void __launch_bounds__(WARPS * 32) score_tiled_kernel(const __grid_constant__ CUtensorMap tmap,
                                                                  const TiledArgs a) {
    using Raw = typename Pairs<E>::Raw;
    constexpr int LX = Pairs<E>::LX, LY = 32 / LX;
    constexpr int WTX = LX * TC, WTY = LY * TR;   // warp tile (poses)
    extern __shared__ __align__(128) unsigned char smem_raw[];
    // the TMA destination must be 128-byte aligned: round the base up (the
    // launch adds 128 bytes of slack)
    const uint32_t pad = (128u - (smem_addr(smem_raw) & 127u)) & 127u;
    const Raw *win = reinterpret_cast<const Raw *>(smem_raw + pad);
    __shared__ __align__(8) unsigned long long mbar;
    __shared__ int s_org[2];   // window origin (pixel x, row y), global coords

    const int img = blockIdx.z;
    const int group = blockIdx.y;
    const int st = blockIdx.x;
    const int stx0 = a.ox + (st % a.tiles_x) * a.sx * WTX;
    const int sty0 = a.oy + (st / a.tiles_x) * a.sy * WTY;
    const int k_begin = a.k0 + group * a.tg;
    const int k_end = min(k_begin + a.tg, a.k0 + a.nk);
    const int pp = a.bxw / 2;   // window row pitch in pixel pairs
    const uint32_t bar = smem_addr(&mbar);

    if (threadIdx.x == 0) {
        int xmin = 1 << 30, ymin = 1 << 30;
        for (int k = k_begin; k < k_end; ++k) {
            const int4 b = a.bbox[k];
            xmin = min(xmin, b.x);
            ymin = min(ymin, b.z);
        }
        // aligned start: the TMA x coordinate times the element size must be a
        // multiple of 16 bytes
        const int wx0 = (stx0 + xmin - 1) & ~(Pairs<E>::XALIGN - 1);
        const int wy0 = sty0 + ymin - 1;
        s_org[0] = wx0;
        s_org[1] = wy0;
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        const uint32_t bytes = (uint32_t)a.bxw * (uint32_t)a.byw * (uint32_t)(Pairs<E>::BYTES / 2);
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
        const int xe = wx0 * Pairs<E>::BYTES / 16;   // 8-byte elements
        asm volatile(
            "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
            "[%5];" ::"r"(smem_addr(win)),
            "l"(reinterpret_cast<uint64_t>(&tmap)), "r"(xe), "r"(wy0), "r"(img), "r"(bar)
            : "memory");
    }
    __syncthreads();
    if (!mbar_wait(bar, 0)) {
        if (threadIdx.x == 0)
            atomicExch(&g_score_err, 1);
        return;
    }
    TileWork t;
    t.rot = a.rot;
    t.n = a.n;
    t.W = a.W;
    t.H = a.H;
    t.ox = a.ox;
    t.oy = a.oy;
    t.k0 = a.k0;
    t.map = a.map + (size_t)img * a.map_img;
    t.inv_n = a.inv_n;
    t.thresh = a.thresh;
    t.early = a.early;
    t.sx = a.sx;
    t.sy = a.sy;
    score_items<E, NB, POL, WARPS>(win, pp, s_org[0], s_org[1], stx0, sty0, k_begin, k_end, t);
}

// The (angle, warp tile) items of one CTA work unit over its staged window
// (origin wx0, wy0; row pitch pp pixel pairs), written into t.map.
template <typename E, int NB, bool POL, int WARPS>
__device__ __forceinline__ void score_items(const typename Pairs<E>::Raw *win, int pp, int wx0, int wy0, int stx0,
                                            int sty0, int k_begin, int k_end, const TileWork &a) {
    constexpr int LX = Pairs<E>::LX, LY = 32 / LX;
    constexpr int WTX = LX * TC, WTY = LY * TR;   // warp tile (poses)
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int lx = lane % LX, ly = lane / LX;
    const int items = (k_end - k_begin) * a.sx * a.sy;
    float *map = a.map;

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
                    point_nb3<E, POL, true>(win, pp, row0, (xs - 1) >> 1, pxx, pyy, acc);
                else
                    point_nb3<E, POL, false>(win, pp, row0, xs >> 1, pxx, pyy, acc);
            } else {
                const int xs = bx + 1 + cur.ox;   // centre column
                const int row0 = by + 1 + cur.oy;
                if (xs & 1)
                    point_nb1<E, POL, true>(win, pp, row0, (xs - 1) >> 1, pxx, pyy, acc);
                else
                    point_nb1<E, POL, false>(win, pp, row0, xs >> 1, pxx, pyy, acc);
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
        // epilogue: M = sum / n, or -inf where pruned; clip to the window
        float *mk = map + (size_t)(k - a.k0) * a.H * a.W;
#pragma unroll
        for (int r = 0; r < TR; ++r) {
            const int y = y0 + r - a.oy;
            if (y >= a.H)
                break;
            float *row = mk + (size_t)y * a.W;
#pragma unroll
            for (int j = 0; j < TC / 2; ++j) {
                const int x = x0 + 2 * j - a.ox;
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

// Persistent form for batches of uneven (image, model) pairs: every CTA
// pulls work units (pair, super-tile, angle group) from one atomic counter,
// stages the unit's window with that pair's own 2-D tensor map (box sized for
// the pair), and scores it.  The window buffer and its mbarrier are reused
// unit after unit (the barrier's phase alternates).  Pairs are laid out
// largest first so the dynamic schedule ends with small units.
template <typename E, int NB, bool POL, int WARPS>
__global__ void __launch_bounds__(WARPS * 32) score_pairs_kernel(const PairScore *__restrict__ pairs, int n_pairs,
                                                                  int total, int sx, int sy, int tg, int early,
                                                                  unsigned *__restrict__ counter) {
    using Raw = typename Pairs<E>::Raw;
    constexpr int LX = Pairs<E>::LX, LY = 32 / LX;
    constexpr int WTX = LX * TC, WTY = LY * TR;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    const uint32_t pad = (128u - (smem_addr(smem_raw) & 127u)) & 127u;
    const Raw *win = reinterpret_cast<const Raw *>(smem_raw + pad);
    __shared__ __align__(8) unsigned long long mbar;
    __shared__ int s_unit[6];   // item, pair, super-tile x0, y0, window x0, y0
    const uint32_t bar = smem_addr(&mbar);
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    uint32_t parity = 0;
    for (;;) {
        if (threadIdx.x == 0) {
            const int item = (int)atomicAdd(counter, 1u);
            s_unit[0] = item;
            if (item < total) {
                int lo = 0, hi = n_pairs - 1;   // last pair whose first item <= item
                while (lo < hi) {
                    const int mid = (lo + hi + 1) >> 1;
                    if (pairs[mid].item_begin <= item)
                        lo = mid;
                    else
                        hi = mid - 1;
                }
                const PairScore &P = pairs[lo];
                const int local = item - P.item_begin;
                const int group = local / P.tiles, st = local - group * P.tiles;
                const int stx0 = (st % P.tiles_x) * sx * WTX, sty0 = (st / P.tiles_x) * sy * WTY;
                const int k_begin = group * tg, k_end = min(k_begin + tg, P.nth);
                int xmin = 1 << 30, ymin = 1 << 30;
                for (int k = k_begin; k < k_end; ++k) {
                    const int4 b = P.bbox[k];
                    xmin = min(xmin, b.x);
                    ymin = min(ymin, b.z);
                }
                const int wx0 = (stx0 + xmin - 1) & ~(Pairs<E>::XALIGN - 1);
                const int wy0 = sty0 + ymin - 1;
                s_unit[1] = lo;
                s_unit[2] = stx0;
                s_unit[3] = sty0;
                s_unit[4] = wx0;
                s_unit[5] = wy0;
                const uint32_t bytes = (uint32_t)P.bxw * (uint32_t)P.byw * (uint32_t)(Pairs<E>::BYTES / 2);
                // the previous unit's reads of the window (generic proxy) are
                // ordered before this unit's copy into it (async proxy)
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
                             : "memory");
                const int xe = wx0 * Pairs<E>::BYTES / 16;
                asm volatile(
                    "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], "
                    "[%4];" ::"r"(smem_addr(win)),
                    "l"(reinterpret_cast<uint64_t>(P.tmap)), "r"(xe), "r"(wy0), "r"(bar)
                    : "memory");
            }
        }
        __syncthreads();
        const int item = s_unit[0];
        if (item >= total)
            break;
        const bool ok = mbar_wait(bar, parity);
        parity ^= 1u;
        if (__syncthreads_or(!ok)) {
            if (threadIdx.x == 0)
                atomicExch(&g_score_err, 1);
            break;
        }
        const PairScore &P = pairs[s_unit[1]];
        const int local = item - P.item_begin;
        const int group = local / P.tiles;
        TileWork t;
        t.rot = P.rot;
        t.n = P.n;
        t.W = P.W;
        t.H = P.H;
        t.ox = 0;
        t.oy = 0;
        t.k0 = 0;
        t.map = P.map;
        t.inv_n = P.inv_n;
        t.thresh = P.thresh;
        t.early = early;
        t.sx = sx;
        t.sy = sy;
        score_items<E, NB, POL, WARPS>(win, P.bxw / 2, s_unit[4], s_unit[5], s_unit[2], s_unit[3], group * tg,
                                       min(group * tg + tg, P.nth), t);
        __syncthreads();   // every warp is done with the window before the next copy
    }
}


// Chunked form for templates whose rotated extent is too large for one staged
// window (a 512-pixel template at full resolution spans ~724 pixels).  One
// angle per CTA and one warp tile per warp; the CTA walks the angle's point
// chunks (points grouped by 16 x 16 cell of their offset), staging for each
// chunk by TMA only the window its points reach from the CTA tile: CTA tile
// + chunk box + 3x3 halo.  Accumulators stay in registers across chunks;
// early termination is checked after every chunk, and the CTA stops when
// every warp has pruned.  Each chunk (at most 256 points) is summed into a
// fresh FP32 partial that is then added to the running sum, so the running
// sum takes one rounding per chunk rather than one per point: with ~6000
// points per pose a plain serial FP32 sum drifts by ~1e-5 of the mean.  The window buffer is reused chunk after chunk
// (mbarrier phase alternates; a proxy fence orders the previous chunk's reads
// before the next copy).
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
};

template <typename E, int NB, bool POL, int WARPS>
__global__ void __launch_bounds__(WARPS * 32) score_chunked_kernel(const __grid_constant__ CUtensorMap tmap,
                                                                    const ChunkArgs a) {
    using Raw = typename Pairs<E>::Raw;
    constexpr int LX = Pairs<E>::LX, LY = 32 / LX;
    constexpr int WTX = LX * TC, WTY = LY * TR;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    const uint32_t pad = (128u - (smem_addr(smem_raw) & 127u)) & 127u;
    const Raw *win = reinterpret_cast<const Raw *>(smem_raw + pad);
    __shared__ __align__(8) unsigned long long mbar;
    __shared__ int s_org[2];

    const int img = blockIdx.z;
    const int kl = blockIdx.y;
    const int k = a.k0 + kl;
    const int st = blockIdx.x;
    const int stx0 = a.ox + (st % a.tiles_x) * a.sx * WTX;
    const int sty0 = a.oy + (st / a.tiles_x) * a.sy * WTY;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int lx = lane % LX, ly = lane / LX;
    const int x0 = stx0 + (warp % a.sx) * WTX + lx * TC;   // thread's first pose
    const int y0 = sty0 + (warp / a.sx) * WTY + ly * TR;
    const int pp = a.bxw / 2;
    const uint32_t bar = smem_addr(&mbar);
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();

    float2 acc[TR][TC / 2];
#pragma unroll
    for (int r = 0; r < TR; ++r)
#pragma unroll
        for (int j = 0; j < TC / 2; ++j)
            acc[r][j] = make_float2(0.f, 0.f);
    const RotPt *P = a.rot + (size_t)k * a.n;
    const int c_begin = a.cstart[k], c_end = a.cstart[k + 1];
    bool alive = true;
    int done = 0;
    uint32_t parity = 0;
    for (int c = c_begin; c < c_end; ++c) {
        const int4 b = a.cbox[c];
        const int2 rg = a.crange[c];
        if (threadIdx.x == 0) {
            const int wx0 = (stx0 + b.x - 1) & ~(Pairs<E>::XALIGN - 1);
            const int wy0 = sty0 + b.z - 1;
            s_org[0] = wx0;
            s_org[1] = wy0;
            const uint32_t bytes = (uint32_t)a.bxw * (uint32_t)a.byw * (uint32_t)(Pairs<E>::BYTES / 2);
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
            const int xe = wx0 * Pairs<E>::BYTES / 16;
            asm volatile(
                "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, "
                "%4}], [%5];" ::"r"(smem_addr(win)),
                "l"(reinterpret_cast<uint64_t>(&tmap)), "r"(xe), "r"(wy0), "r"(img), "r"(bar)
                : "memory");
        }
        __syncthreads();
        const bool ok = mbar_wait(bar, parity);
        parity ^= 1u;
        if (__syncthreads_or(!ok)) {
            if (threadIdx.x == 0) {
                atomicExch(&g_score_err, 1);
                mbar_wait(bar, parity ^ 1u);   // let a late copy land before the CTA exits
            }
            return;
        }
        if (alive) {
            const int bx = x0 - 1 - s_org[0];
            const int by = y0 - 1 - s_org[1];
            float2 part[TR][TC / 2];
#pragma unroll
            for (int r = 0; r < TR; ++r)
#pragma unroll
                for (int j = 0; j < TC / 2; ++j)
                    part[r][j] = make_float2(0.f, 0.f);
            RotPt q = P[rg.x];
            for (int i = rg.x; i < rg.y; ++i) {
                const RotPt cur = q;
                if (i + 1 < rg.y)
                    q = P[i + 1];
                const float2 pxx = make_float2(cur.px, cur.px);
                const float2 pyy = make_float2(cur.py, cur.py);
                if (NB == 3) {
                    const int xs = bx + cur.ox;
                    const int row0 = by + cur.oy;
                    if (xs & 1)
                        point_nb3<E, POL, true>(win, pp, row0, (xs - 1) >> 1, pxx, pyy, part);
                    else
                        point_nb3<E, POL, false>(win, pp, row0, xs >> 1, pxx, pyy, part);
                } else {
                    const int xs = bx + 1 + cur.ox;
                    const int row0 = by + 1 + cur.oy;
                    if (xs & 1)
                        point_nb1<E, POL, true>(win, pp, row0, (xs - 1) >> 1, pxx, pyy, part);
                    else
                        point_nb1<E, POL, false>(win, pp, row0, xs >> 1, pxx, pyy, part);
                }
            }
#pragma unroll
            for (int r = 0; r < TR; ++r)
#pragma unroll
                for (int j = 0; j < TC / 2; ++j)
                    acc[r][j] = __fadd2_rn(acc[r][j], part[r][j]);
            done += rg.y - rg.x;
            if (a.early) {
                const float lim = a.thresh - (float)(a.n - done);
                bool low = true;
#pragma unroll
                for (int r = 0; r < TR; ++r)
#pragma unroll
                    for (int j = 0; j < TC / 2; ++j)
                        low = low && (acc[r][j].x < lim) && (acc[r][j].y < lim);
                if (__all_sync(0xffffffffu, low))
                    alive = false;
            }
        }
        // every warp is done with the window before the next copy; stop when
        // all warps have pruned
        if (!__syncthreads_or(alive))
            break;
    }
    float *mk = a.map + (size_t)img * a.map_img + (size_t)kl * a.H * a.W;
#pragma unroll
    for (int r = 0; r < TR; ++r) {
        const int y = y0 + r - a.oy;
        if (y >= a.H)
            break;
        float *row = mk + (size_t)y * a.W;
#pragma unroll
        for (int j = 0; j < TC / 2; ++j) {
            const int x = x0 + 2 * j - a.ox;
            const float v0 = alive ? acc[r][j].x * a.inv_n : -INFINITY;
            const float v1 = alive ? acc[r][j].y * a.inv_n : -INFINITY;
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

struct Geometry {
    int wtx, wty, xalign, pair_bytes;
};

Geometry geometry(int precision) {
    if (precision == SAM_FP32)
        return {Pairs<float>::LX * TC, (32 / Pairs<float>::LX) * TR, Pairs<float>::XALIGN, Pairs<float>::BYTES};
    return {Pairs<__half>::LX * TC, (32 / Pairs<__half>::LX) * TR, Pairs<__half>::XALIGN, Pairs<__half>::BYTES};
}

template <typename E, int NB, bool POL, int WARPS>
cudaError_t launch_t(const CUtensorMap &tm, const TiledArgs &a, dim3 grid, size_t smem, cudaStream_t st) {
    auto kern = score_tiled_kernel<E, NB, POL, WARPS>;
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

template <typename E>
cudaError_t launch_e(const CUtensorMap &tm, const TiledArgs &a, dim3 grid, size_t smem, int nbhd, bool pol,
                     int warps, cudaStream_t st) {
    if (warps == 4) {
        if (nbhd == 3)
            return pol ? launch_t<E, 3, true, 4>(tm, a, grid, smem, st) : launch_t<E, 3, false, 4>(tm, a, grid, smem, st);
        return pol ? launch_t<E, 1, true, 4>(tm, a, grid, smem, st) : launch_t<E, 1, false, 4>(tm, a, grid, smem, st);
    }
    if (nbhd == 3)
        return pol ? launch_t<E, 3, true, 8>(tm, a, grid, smem, st) : launch_t<E, 3, false, 8>(tm, a, grid, smem, st);
    return pol ? launch_t<E, 1, true, 8>(tm, a, grid, smem, st) : launch_t<E, 1, false, 8>(tm, a, grid, smem, st);
}

}  // namespace

// Window box for a tiling: the super-tile grown by the largest union of
// rotated offset boxes over any angle group, the 1-pixel search halo, the
// slack of the aligned TMA start and one pixel for odd-start pair loads.
bool tiled_plan(const LevelHost &L, int precision, int sx, int sy, int tg, int *bxw, int *byw) {
    const Geometry g = geometry(precision);
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
    *bxw = bx;
    *byw = by;
    const size_t bytes = (size_t)bx * by * g.pair_bytes / 2;
    return bx * g.pair_bytes / 16 <= 256 && by <= 256 && bytes <= 200 * 1024;
}

// Launch over `count` images whose pairs-layout fields start at `field`
// (row pitch wp pixels, a multiple of 4; image stride field_img_px pixels).
cudaError_t launch_score_tiled(const sam_model *m, int level, const void *field, int precision, int wp,
                               size_t field_img_px, int W, int H, int count, int nbhd, int polarity, float min_score,
                               int early, float *map, size_t map_img, const TileConfig &cfg, cudaStream_t st,
                               const PoseWindow *window) {
    const LevelHost &L = m->lv[level];
    const PoseWindow pw = window ? *window : PoseWindow{0, 0, W, H, 0, L.ntheta};
    int bxw = 0, byw = 0;
    if (!tiled_plan(L, precision, cfg.sx, cfg.sy, cfg.tg, &bxw, &byw))
        return cudaErrorInvalidValue;
    EncodeTiledFn enc = encode_fn();
    if (!enc)
        return cudaErrorNotSupported;
    const Geometry g = geometry(precision);
    // the field as a 3-D tensor of 8-byte elements: a pixel pair is 2 (FP32)
    // or 1 (16-bit) element(s)
    CUtensorMap tm;
    const cuuint64_t dims[3] = {(cuuint64_t)wp * g.pair_bytes / 16, (cuuint64_t)H, (cuuint64_t)count};
    const cuuint64_t strides[2] = {(cuuint64_t)wp * g.pair_bytes / 2, (cuuint64_t)field_img_px * g.pair_bytes / 2};
    const cuuint32_t box[3] = {(cuuint32_t)(bxw * g.pair_bytes / 16), (cuuint32_t)byw, 1};
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
    const int groups = (pw.nk + cfg.tg - 1) / cfg.tg;
    dim3 grid((unsigned)(a.tiles_x * tiles_y), (unsigned)groups, (unsigned)count);
    const size_t smem = (size_t)bxw * byw * g.pair_bytes / 2 + 128;
    const bool pol = polarity != 0;
    switch (precision) {
    case SAM_FP32:
        return launch_e<float>(tm, a, grid, smem, nbhd, pol, cfg.warps, st);
    case SAM_FP16:
        return launch_e<__half>(tm, a, grid, smem, nbhd, pol, cfg.warps, st);
    default:
        return launch_e<__nv_bfloat16>(tm, a, grid, smem, nbhd, pol, cfg.warps, st);
    }
}

namespace {
template <typename E, int NB, bool POL, int WARPS>
cudaError_t launch_c(const CUtensorMap &tm, const ChunkArgs &a, dim3 grid, size_t smem, cudaStream_t st) {
    auto kern = score_chunked_kernel<E, NB, POL, WARPS>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess)
        return e;
    e = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared);
    if (e != cudaSuccess)
        return e;
    kern<<<grid, WARPS * 32, smem, st>>>(tm, a);
    count_launches(1);
    return cudaGetLastError();
}

template <typename E>
cudaError_t launch_ce(const CUtensorMap &tm, const ChunkArgs &a, dim3 grid, size_t smem, int nbhd, bool pol,
                      int warps, cudaStream_t st) {
    if (warps == 4) {
        if (nbhd == 3)
            return pol ? launch_c<E, 3, true, 4>(tm, a, grid, smem, st) : launch_c<E, 3, false, 4>(tm, a, grid, smem, st);
        return pol ? launch_c<E, 1, true, 4>(tm, a, grid, smem, st) : launch_c<E, 1, false, 4>(tm, a, grid, smem, st);
    }
    if (nbhd == 3)
        return pol ? launch_c<E, 3, true, 8>(tm, a, grid, smem, st) : launch_c<E, 3, false, 8>(tm, a, grid, smem, st);
    return pol ? launch_c<E, 1, true, 8>(tm, a, grid, smem, st) : launch_c<E, 1, false, 8>(tm, a, grid, smem, st);
}
}  // namespace

bool level_needs_chunks(const LevelHost &L) {
    int bxw = 0, byw = 0;
    return !tiled_plan(L, SAM_FP32, 1, 1, 1, &bxw, &byw);
}

// Window box of the chunked kernel: CTA tile + largest chunk box + halo +
// aligned-start slack + one pixel for odd-start pair loads.
bool chunked_plan(const LevelHost &L, int precision, int sx, int sy, int *bxw, int *byw) {
    if (L.crot.empty())
        return false;
    const Geometry g = geometry(precision);
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
    const Geometry g = geometry(precision);
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
    dim3 grid((unsigned)(a.tiles_x * tiles_y), (unsigned)pw.nk, (unsigned)count);
    const size_t smem = (size_t)bxw * byw * g.pair_bytes / 2 + 128;
    const bool pol = polarity != 0;
    switch (precision) {
    case SAM_FP32:
        return launch_ce<float>(tm, a, grid, smem, nbhd, pol, cfg.warps, st);
    case SAM_FP16:
        return launch_ce<__half>(tm, a, grid, smem, nbhd, pol, cfg.warps, st);
    default:
        return launch_ce<__nv_bfloat16>(tm, a, grid, smem, nbhd, pol, cfg.warps, st);
    }
}

// 2-D tensor map of one image's pairs-layout field for the persistent kernel
// (written to host memory; the plan copies it to device memory).
bool encode_pair_tmap(void *out, const void *field, int precision, int wp, int H, int bxw, int byw) {
    EncodeTiledFn enc = encode_fn();
    if (!enc)
        return false;
    const Geometry g = geometry(precision);
    const cuuint64_t dims[2] = {(cuuint64_t)wp * g.pair_bytes / 16, (cuuint64_t)H};
    const cuuint64_t strides[1] = {(cuuint64_t)wp * g.pair_bytes / 2};
    const cuuint32_t box[2] = {(cuuint32_t)(bxw * g.pair_bytes / 16), (cuuint32_t)byw};
    const cuuint32_t estr[2] = {1, 1};
    return enc(reinterpret_cast<CUtensorMap *>(out), CU_TENSOR_MAP_DATA_TYPE_UINT64, 2, const_cast<void *>(field), dims,
               strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
               CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

int tiled_warp_tile(int precision, int *wty) {
    const Geometry g = geometry(precision);
    *wty = g.wty;
    return g.wtx;
}

namespace {
template <typename E, int NB, bool POL, int WARPS>
cudaError_t launch_pairs_t(const PairScore *pairs, int n_pairs, int total, const TileConfig &cfg, int early,
                           size_t smem, unsigned *counter, cudaStream_t st) {
    auto kern = score_pairs_kernel<E, NB, POL, WARPS>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess)
        return e;
    e = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared);
    if (e != cudaSuccess)
        return e;
    int per_sm = 0, dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, WARPS * 32, smem);
    if (e != cudaSuccess)
        return e;
    const int grid = std::max(1, std::min(total, sms * std::max(1, per_sm)));
    kern<<<grid, WARPS * 32, smem, st>>>(pairs, n_pairs, total, cfg.sx, cfg.sy, cfg.tg, early, counter);
    count_launches(1);
    return cudaGetLastError();
}

template <typename E>
cudaError_t launch_pairs_e(const PairScore *pairs, int n_pairs, int total, const TileConfig &cfg, int nbhd, bool pol,
                           int early, size_t smem, unsigned *counter, cudaStream_t st) {
    if (cfg.warps == 4) {
        if (nbhd == 3)
            return pol ? launch_pairs_t<E, 3, true, 4>(pairs, n_pairs, total, cfg, early, smem, counter, st)
                       : launch_pairs_t<E, 3, false, 4>(pairs, n_pairs, total, cfg, early, smem, counter, st);
        return pol ? launch_pairs_t<E, 1, true, 4>(pairs, n_pairs, total, cfg, early, smem, counter, st)
                   : launch_pairs_t<E, 1, false, 4>(pairs, n_pairs, total, cfg, early, smem, counter, st);
    }
    if (nbhd == 3)
        return pol ? launch_pairs_t<E, 3, true, 8>(pairs, n_pairs, total, cfg, early, smem, counter, st)
                   : launch_pairs_t<E, 3, false, 8>(pairs, n_pairs, total, cfg, early, smem, counter, st);
    return pol ? launch_pairs_t<E, 1, true, 8>(pairs, n_pairs, total, cfg, early, smem, counter, st)
               : launch_pairs_t<E, 1, false, 8>(pairs, n_pairs, total, cfg, early, smem, counter, st);
}
}  // namespace

cudaError_t launch_score_pairs(const PairScore *pairs, int n_pairs, int total_items, int precision, int nbhd,
                               int polarity, int early, const TileConfig &cfg, size_t window_bytes, unsigned *counter,
                               cudaStream_t st) {
    if (total_items <= 0 || n_pairs <= 0)
        return cudaSuccess;
    const size_t smem = window_bytes + 128;
    const bool pol = polarity != 0;
    switch (precision) {
    case SAM_FP32:
        return launch_pairs_e<float>(pairs, n_pairs, total_items, cfg, nbhd, pol, early, smem, counter, st);
    case SAM_FP16:
        return launch_pairs_e<__half>(pairs, n_pairs, total_items, cfg, nbhd, pol, early, smem, counter, st);
    default:
        return launch_pairs_e<__nv_bfloat16>(pairs, n_pairs, total_items, cfg, nbhd, pol, early, smem, counter, st);
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
