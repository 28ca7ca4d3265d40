// Device code of the tiled exhaustive scorers (kernel (c)): the
// single-level tiled kernel, the persistent kernel over (image, model) pairs
// and the chunked kernel for large templates.  Included by one translation
// unit per field type (score_tiled_f32.cu, _f16.cu, _bf16.cu), which
// instantiate the kernels for that type; the host side (tiling plans, tensor
// maps, dispatch) is score_tiled.cu.  See score_tiled.cu for the design.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <algorithm>

#include "sam_internal.h"
#include "score_common.cuh"

namespace sam {
namespace {

constexpr int TR = kTileRows;        // rows of poses per thread
constexpr int PRUNE_EVERY = 8;



// Stored element type of the window: pair size, lane layout, TMA alignment.
template <typename E>
struct Pairs;

template <>
struct Pairs<float> {
    using Raw = float4;
    static constexpr int BYTES = 16;   // one pixel pair
    static constexpr int LX = kLanesXF32;   // lanes along x
    static constexpr int XALIGN = 2;   // window start (pixels) for a 16-byte TMA start
    static constexpr bool CODES = false;   // the window is staged as stored
    static __device__ __forceinline__ float4 get(const Raw *row, int q) { return row[q]; }
};

// Angle-only storage (SAM_ANGLE16): the field holds one 16-bit code per
// pixel; the window is staged as codes (2 bytes per pixel, TMA starts at
// multiples of 8 pixels) and expanded in shared memory to FP32 pixel pairs,
// which the FP32 arithmetic then scores.  The expanded window is two pixels
// wider than the staged one (a zero pair column), which keeps its row pitch
// an odd number of 16-byte pairs.
struct AngleCode {};
template <>
struct Pairs<AngleCode> {
    using Raw = float4;
    static constexpr int BYTES = 16;   // one expanded pixel pair in shared memory
    static constexpr int LX = kLanesXF32;
    static constexpr int XALIGN = 8;
    static constexpr bool CODES = true;
    static __device__ __forceinline__ float4 get(const Raw *row, int q) { return row[q]; }
};

template <>
struct Pairs<__half> {
    using Raw = uint2;
    static constexpr int BYTES = 8;
    static constexpr int LX = kLanesX16;
    static constexpr int XALIGN = 4;
    static constexpr bool CODES = false;
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
    static constexpr int LX = kLanesX16;
    static constexpr int XALIGN = 4;
    static constexpr bool CODES = false;
    static __device__ __forceinline__ float4 get(const Raw *row, int q) {
        const uint2 u = row[q];
        // bf16 -> fp32 is a 16-bit left shift of the bit pattern
        return make_float4(__uint_as_float(u.x << 16), __uint_as_float(u.x & 0xFFFF0000u),
                           __uint_as_float(u.y << 16), __uint_as_float(u.y & 0xFFFF0000u));
    }
};

__device__ __forceinline__ float max3(float a, float b, float c) {
    float d;
    asm("max.f32 %0, %1, %2, %3;" : "=f"(d) : "f"(a), "f"(b), "f"(c));
    return d;
}

__device__ __forceinline__ uint32_t smem_addr(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// Bounded wait on an mbarrier phase: true when the phase completed, false
// after `limit_ns` nanoseconds of the global timer (1 s by default; a TMA
// window copy takes microseconds) or 2^26 polls, whichever comes first.
constexpr unsigned long long kWaitLimitNs = 1000000000ull;

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, unsigned long long limit_ns = kWaitLimitNs) {
    const unsigned long long t0 = global_ns();
    for (int it = 0; it < (1 << 26); ++it) {
        uint32_t done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(bar), "r"(parity)
            : "memory");
        if (done)
            return true;
        if (global_ns() - t0 > limit_ns)
            return false;
    }
    return false;
}

// Self-test of the bounded wait: one warp waits on a fresh mbarrier that
// nothing arrives at (no copy is issued), gives up after limit_ns and
// reports it through the error flag exactly as the scorers do.
__device__ int wait_task(const int4 *tasks, unsigned tcap, const unsigned *qctr, unsigned units, unsigned ti,
                          unsigned long long limit_ns);

// mode 0: the mbarrier wait above; mode 1: thread 0's wait for a task of the
// persistent scorer (wait_task) on a task list whose flag nothing sets and
// whose one work unit never completes (`fake`: 16 zero bytes of task, then
// the five zero counters).
__global__ void wait_selftest_kernel(int *err, unsigned long long limit_ns, unsigned long long *waited_ns, int mode,
                                     unsigned *fake) {
    __shared__ __align__(8) unsigned long long mbar;
    const uint32_t bar = smem_addr(&mbar);
    if (mode == 1) {
        if (threadIdx.x == 0) {
            const unsigned long long t0 = global_ns();
            const int r = wait_task(reinterpret_cast<const int4 *>(fake), 1u, fake + 4, 1u, 0u, limit_ns);
            *waited_ns = global_ns() - t0;
            if (r < 0)
                atomicExch(err, 1);
        }
        return;
    }
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    const unsigned long long t0 = global_ns();
    const bool ok = mbar_wait(bar, 0, limit_ns);
    if (threadIdx.x == 0) {
        *waited_ns = global_ns() - t0;
        if (!ok)
            atomicExch(err, 1);
    }
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

template <typename E, bool POL, int TC>
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

// One model point over the thread's R x TC pose block, 3x3 neighbourhood.
template <typename E, bool POL, bool ODD, int TC, int R = TR>
__device__ __forceinline__ void point_nb3(const typename Pairs<E>::Raw *win, int pp, int row0, int pair0,
                                          float2 pxx, float2 pyy, float2 (&acc)[R][TC / 2]) {
    constexpr int NP = ODD ? (TC + 4) / 2 : (TC + 2) / 2;   // pixel pairs per row
    constexpr int OFF = ODD ? 1 : 0;
    if constexpr (R < TC) {
        // fewer rows than columns (the 2-row slices of the drain, 8 x 10
        // blocks): the 3-row maxima of the TC + 2 columns first, then the
        // 3-column maxima, R (TC + 2) + R TC three-input maxima instead of
        // (R + 2) TC + R TC (a maximum is exact in any order)
        float dp2[TC + 2], dp1[TC + 2];
#pragma unroll
        for (int r = 0; r < R + 2; ++r) {
            const typename Pairs<E>::Raw *row = win + (row0 + r) * pp;
            float d[TC + 4];
            dots_row<E, POL, TC>(row, pair0, d, NP, pxx, pyy);
            if (r >= 2) {
                float v[TC + 2];
#pragma unroll
                for (int c = 0; c < TC + 2; ++c)
                    v[c] = max3(dp2[c], dp1[c], d[OFF + c]);
#pragma unroll
                for (int j = 0; j < TC / 2; ++j) {
                    const float v0 = max3(v[2 * j], v[2 * j + 1], v[2 * j + 2]);
                    const float v1 = max3(v[2 * j + 1], v[2 * j + 2], v[2 * j + 3]);
                    acc[r - 2][j] = __fadd2_rn(acc[r - 2][j], make_float2(v0, v1));
                }
            }
#pragma unroll
            for (int c = 0; c < TC + 2; ++c) {
                dp2[c] = dp1[c];
                dp1[c] = d[OFF + c];
            }
        }
    } else {
        float hp2[TC], hp1[TC];
#pragma unroll
        for (int r = 0; r < R + 2; ++r) {
            const typename Pairs<E>::Raw *row = win + (row0 + r) * pp;
            float d[TC + 4];
            dots_row<E, POL, TC>(row, pair0, d, NP, pxx, pyy);
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
}

// One model point, neighbourhood 1 (no search): the centre pixel only.
template <typename E, bool POL, bool ODD, int TC, int R = TR>
__device__ __forceinline__ void point_nb1(const typename Pairs<E>::Raw *win, int pp, int row0, int pair0,
                                          float2 pxx, float2 pyy, float2 (&acc)[R][TC / 2]) {
    constexpr int NP = ODD ? (TC + 2) / 2 : TC / 2;
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const typename Pairs<E>::Raw *row = win + (row0 + r) * pp;
        float d[TC + 4];
        dots_row<E, POL, TC>(row, pair0, d, NP, pxx, pyy);
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
    unsigned long long *exec;   // executed pose-point counter
    int emin;                   // edge-presence bound (0: off)
    int byw;                    // window rows
    uint32_t *bits;             // edge bitmaps of the window (edge_bitmap_bytes: 4 + 4 planes)
    int *err;                   // device error flag
    // persistent form (queue non-null): where the surviving slices go
    uint32_t *queue;
    int4 *tasks;
    unsigned *qctr;
    unsigned qcap, tcap;
    int unit;                   // this CTA's work unit
    // hot list (hot_cnt null: none): see TiledArgs
    unsigned *hot_cnt;
    uint2 *hot;
    unsigned hot_cap;
    float hot_thr;
    unsigned img;               // image (or pair) index of the hot entries
};

// Quadrant of a non-zero vector: 0 for angles in [0, 90) degrees, 1 for
// [90, 180), 2 for [180, 270), 3 for [270, 360), decided by signs alone.  For
// u in quadrant q and v in quadrant q + 2 (mod 4) both products of u . v are
// <= 0 and one is < 0, and a rounded product keeps its sign, so the dot
// product is <= 0 however it is rounded.
__device__ __forceinline__ int quadrant(float x, float y) {
    return y > 0.f ? (x > 0.f ? 0 : 1) : (y < 0.f ? (x < 0.f ? 2 : 3) : (x > 0.f ? 0 : 2));
}

// Edge bitmaps of a staged window (all threads of the CTA; ends with a CTA
// barrier).  Plane q (q < 4, or only q = 0 with POL) of N: bit x of window row
// r is set iff pixel x is an edge pixel (non-zero unit vector) whose
// direction is not in the quadrant opposite q (with POL: any edge pixel).
// C = each plane of N dilated by 3x3: C_q at a point's projected centre is
// set iff its neighbouring-search window holds an edge pixel that can give a
// positive vote to a model direction in quadrant q (Eq. (1): p . w <= 0 for
// opposite quadrants, and pixels that are not edges give 0).
template <typename E, int NTHREADS, bool POL>
__device__ __forceinline__ void build_edge_bits(const typename Pairs<E>::Raw *win, int pp, int byw, uint32_t *nbits,
                                                uint32_t *cbits) {
    constexpr int NQ = POL ? 1 : 4;
    const int dmw = edge_bitmap_words(2 * pp), nw = (2 * pp + 31) / 32;
    const size_t plane = (size_t)byw * dmw;
    for (int idx = threadIdx.x; idx < byw * dmw; idx += NTHREADS) {
        const int r = idx / dmw, wi = idx - r * dmw;
        uint32_t e[NQ];
#pragma unroll
        for (int b = 0; b < NQ; ++b)
            e[b] = 0u;
        if (wi < nw) {
            const typename Pairs<E>::Raw *row = win + (size_t)r * pp;
            // consecutive threads own consecutive words, 16 pixel pairs
            // apart: each thread starts at its own pair of the word (lane
            // rotation) so that one load instruction touches distinct banks
            const int rot = threadIdx.x & 15;
#pragma unroll 4
            for (int qq = 0; qq < 16; ++qq) {
                const int q = (qq + rot) & 15;
                const int pq = wi * 16 + q;
                if (pq < pp) {
                    const float4 v = Pairs<E>::get(row, pq);   // {x0, x1, y0, y1}
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        const float x = h ? v.y : v.x, y = h ? v.w : v.z;
                        if (x != 0.f || y != 0.f) {
                            if (POL) {
                                e[0] |= 1u << (2 * q + h);
                            } else {
                                const int opp = (quadrant(x, y) + 2) & 3;   // the plane it cannot serve
#pragma unroll
                                for (int b = 0; b < NQ; ++b)
                                    if (b != opp)
                                        e[b] |= 1u << (2 * q + h);
                            }
                        }
                    }
                }
            }
        }
#pragma unroll
        for (int b = 0; b < NQ; ++b)
            nbits[b * plane + idx] = e[b];
    }
    __syncthreads();
    for (int idx = threadIdx.x; idx < NQ * byw * dmw; idx += NTHREADS) {
        const int b = idx / (byw * dmw), rest = idx - b * (byw * dmw);
        const int r = rest / dmw, wi = rest - r * dmw;
        uint32_t d = 0;
        for (int dr = -1; dr <= 1; ++dr) {
            const int rr = r + dr;
            if (rr < 0 || rr >= byw)
                continue;
            const uint32_t *er = nbits + b * plane + (size_t)rr * dmw;
            const uint32_t c = er[wi], lw = wi > 0 ? er[wi - 1] : 0u, rw = wi + 1 < dmw ? er[wi + 1] : 0u;
            d |= c | (c << 1) | (lw >> 31) | (c >> 1) | (rw << 31);
        }
        cbits[idx] = d;
    }
    __syncthreads();
}

// Global-memory flag accesses of the persistent form (GPU scope).
__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned *p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release_u32(unsigned *p, unsigned v) {
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
// Thread 0 of a persistent-scorer CTA: waits until task ti is published.
// Returns 1 when it is, 0 when every unit is done (qctr[4] >= units) and no
// task ti exists, -1 after limit_ns (the caller reports it).
__device__ int wait_task(const int4 *tasks, unsigned tcap, const unsigned *qctr, unsigned units, unsigned ti,
                          unsigned long long limit_ns) {
    const unsigned long long t0 = global_ns();
    for (unsigned polls = 0;; ++polls) {
        if (ti < tcap && ld_acquire_u32(reinterpret_cast<const unsigned *>(&tasks[ti].w)) == 1u)
            return 1;
        if (ld_acquire_u32(&qctr[4]) >= units && ti >= ld_acquire_u32(&qctr[1]))
            return 0;
        if ((polls & 15u) == 15u && global_ns() - t0 > limit_ns)
            return -1;
        __nanosleep(64);
    }
}

// Items (angle x warp tile) whose surviving blocks one queue round holds.
constexpr int kQueueItems = 128;
// Pose rows per lane when the surviving blocks are scored (TR / RD lanes
// share one block).
constexpr int RD = kDrainRows;
static_assert(kTileRows / kDrainRows == 4, "queue entries hold the slice index in 2 bits");

// Position of the r-th (0-based) set bit of m; r < popc(m).
__device__ __forceinline__ int nth_set_bit(uint32_t m, int r) {
    int pos = 0;
#pragma unroll
    for (int w = 16; w > 0; w >>= 1) {
        const int c = __popc(m & ((1u << w) - 1u));
        if (r >= c) {
            r -= c;
            m >>= w;
            pos += w;
        }
    }
    return pos;
}

// Where a work unit of the tiled scorer lies: image, super-tile origin
// (poses), angles [k_begin, k_end).  unit = super-tile + tiles * (angle
// group + groups * image), the linear CTA index of the one-CTA-per-unit launch.
struct UnitPos {
    int img, stx0, sty0, k_begin, k_end;
};
template <typename E, int TC>
__device__ __forceinline__ UnitPos unit_pos(const TiledArgs &a, int unit) {
    constexpr int LX = Pairs<E>::LX, LY = 32 / LX;
    constexpr int WTX = LX * TC, WTY = LY * TR;
    const int tiles = a.tiles_x * a.tiles_y, groups = (a.nk + a.tg - 1) / a.tg;
    const int st = unit % tiles, rest = unit / tiles;
    UnitPos u;
    u.img = rest / groups;
    u.stx0 = a.ox + (st % a.tiles_x) * a.sx * WTX;
    u.sty0 = a.oy + (st / a.tiles_x) * a.sy * WTY;
    u.k_begin = a.k0 + (rest % groups) * a.tg;
    u.k_end = min(u.k_begin + a.tg, a.k0 + a.nk);
    return u;
}

// Thread 0: the unit's window origin into s_org and its TMA copy, completing
// on mbarrier `bar`.  The previous reads of the window (generic proxy) are
// ordered before the copy into it (async proxy).
template <typename E>
__device__ __forceinline__ void stage_window(const CUtensorMap &tmap, const TiledArgs &a, const UnitPos &u,
                                             const void *win, uint32_t bar, int *s_org) {
    int xmin = 1 << 30, ymin = 1 << 30;
    for (int k = u.k_begin; k < u.k_end; ++k) {
        const int4 b = a.bbox[k];
        xmin = min(xmin, b.x);
        ymin = min(ymin, b.z);
    }
    // aligned start: the TMA x coordinate times the element size must be a
    // multiple of 16 bytes
    const int wx0 = (u.stx0 + xmin - 1) & ~(Pairs<E>::XALIGN - 1);
    const int wy0 = u.sty0 + ymin - 1;
    s_org[0] = wx0;
    s_org[1] = wy0;
    // codes: (bxw - 2) 2-byte elements per staged row; pairs: 8-byte elements
    const uint32_t bytes = Pairs<E>::CODES ? (uint32_t)(a.bxw - 2) * (uint32_t)a.byw * 2u
                                           : (uint32_t)a.bxw * (uint32_t)a.byw * (uint32_t)(Pairs<E>::BYTES / 2);
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
    const int xe = Pairs<E>::CODES ? wx0 : wx0 * Pairs<E>::BYTES / 16;
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
        "[%5];" ::"r"(smem_addr(win)),
        "l"(reinterpret_cast<uint64_t>(&tmap)), "r"(xe), "r"(wy0), "r"(u.img), "r"(bar)
        : "memory");
}

// Shared-memory layout of the single-level tiled scorers: the window (as
// scored), then the region of the edge bitmaps (and of the persistent form's
// partial sums); with angle codes the staged codes also go to that region,
// 128-byte aligned for the TMA copy, and are expanded before it is used.
template <typename E>
__device__ __forceinline__ size_t window_region_bytes(int bxw, int byw) {
    const size_t b = (size_t)bxw * byw * (Pairs<E>::BYTES / 2);
    return Pairs<E>::CODES ? (b + 127) & ~(size_t)127 : (b + 15) & ~(size_t)15;
}

// One angle code as the unit vector it stands for: (cos, sin)(a 2 pi /
// 32768) = (cospi, sinpi)(a / 16384) on an edge (bit 15), (0, 0) elsewhere.
__device__ __forceinline__ float2 decode_angle(uint32_t c) {
    float sn = 0.f, cs = 0.f;
    if (c & 0x8000u)
        sincospif((float)(c & 0x7FFFu) * (1.0f / 16384.0f), &sn, &cs);
    return make_float2(cs, sn);
}

// Expand the staged codes (byw rows of bxw - 2 codes) into the FP32 pairs
// window (byw rows of bxw / 2 pairs {wx0, wx1, wy0, wy1}, the last pair of a
// row zero).  All threads of the CTA; the caller synchronises afterwards.
__device__ __forceinline__ void expand_codes(const uint32_t *codes, float4 *win, int bxw, int byw) {
    const int pp = bxw / 2, cpp = pp - 1;
    const int warps = blockDim.x >> 5, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int r = warp; r < byw; r += warps) {
        const uint32_t *cr = codes + (size_t)r * cpp;
        float4 *wr = win + (size_t)r * pp;
        for (int j = lane; j < pp; j += 32) {
            float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
            if (j < cpp) {
                const uint32_t c = cr[j];
                const float2 u0 = decode_angle(c & 0xFFFFu), u1 = decode_angle(c >> 16);
                v = make_float4(u0.x, u1.x, u0.y, u1.y);
            }
            wr[j] = v;
        }
    }
}

// The per-image work description of a tiled launch (bits and unit unset).
__device__ __forceinline__ TileWork tile_work(const TiledArgs &a, int img) {
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
    t.exec = a.exec;
    t.emin = a.emin;
    t.byw = a.byw;
    t.bits = nullptr;
    t.err = a.err;
    t.queue = a.queue;
    t.tasks = a.tasks;
    t.qctr = a.qctr;
    t.qcap = a.qcap;
    t.tcap = a.tcap;
    t.unit = 0;
    t.hot_cnt = a.hot_cnt;
    t.hot = a.hot;
    t.hot_cap = a.hot_cap;
    t.hot_thr = a.hot_thr;
    t.img = (unsigned)img;
    return t;
}

template <typename E, int NB, bool POL, int WARPS, int TC>
__device__ __forceinline__ void score_items(const typename Pairs<E>::Raw *win, int pp, int wx0, int wy0, int stx0,
                                            int sty0, int k_begin, int k_end, const TileWork &a);
template <typename E, int NB, bool POL, int TC>
__device__ __forceinline__ void score_slice(const typename Pairs<E>::Raw *win, int pp, int wx0, int wy0, int stx0,
                                            int sty0, int k_begin, int item, int src, int part, bool has,
                                            const TileWork &a, unsigned long long &executed);
template <typename E, int NB, bool POL, int TC>
__device__ __forceinline__ void slice_sum(const typename Pairs<E>::Raw *win, int pp, int wx0, int wy0, int stx0,
                                          int sty0, int k_begin, int item, int src, int part, bool has,
                                          const TileWork &a, int p0, int p1, float2 (&acc)[RD][TC / 2],
                                          unsigned long long &executed);
template <typename E, int TC>
__device__ __forceinline__ void slice_store(int item, int src, int part, int stx0, int sty0, int k_begin,
                                            const TileWork &a, const float2 (&acc)[RD][TC / 2]);

// Exhaustive score (Eq. (1) over the Eq. (2) projections, neighbouring
// search NB) of one work unit per CTA: its TMA-staged window, then
// score_items over the unit's angles and warp tiles.
template <typename E, int NB, bool POL, int WARPS, int TC>
__global__ void __launch_bounds__(WARPS * 32) score_tiled_kernel(const __grid_constant__ CUtensorMap tmap,
                                                                  const TiledArgs a) {
    using Raw = typename Pairs<E>::Raw;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    // the TMA destination must be 128-byte aligned: round the base up (the
    // launch adds 128 bytes of slack)
    const uint32_t pad = (128u - (smem_addr(smem_raw) & 127u)) & 127u;
    const Raw *win = reinterpret_cast<const Raw *>(smem_raw + pad);
    __shared__ __align__(8) unsigned long long mbar;
    __shared__ int s_org[2];   // window origin (pixel x, row y), global coords

    const int unit = blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z);
    const UnitPos u = unit_pos<E, TC>(a, unit);
    const int pp = a.bxw / 2;   // window row pitch in pixel pairs
    const uint32_t bar = smem_addr(&mbar);
    // the region after the window: edge bitmaps (and staged angle codes)
    unsigned char *region = smem_raw + pad + window_region_bytes<E>(a.bxw, a.byw);

    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        stage_window<E>(tmap, a, u, Pairs<E>::CODES ? (const void *)region : (const void *)win, bar, s_org);
    }
    __syncthreads();
    if (!mbar_wait(bar, 0)) {
        if (threadIdx.x == 0)
            atomicExch(a.err, 1);
        return;
    }
    if constexpr (Pairs<E>::CODES) {
        expand_codes(reinterpret_cast<const uint32_t *>(region), const_cast<float4 *>(win), a.bxw, a.byw);
        __syncthreads();
    }
    TileWork t = tile_work(a, u.img);
    t.bits = reinterpret_cast<uint32_t *>(region);
    t.unit = unit;
    score_items<E, NB, POL, WARPS, TC>(win, pp, s_org[0], s_org[1], u.stx0, u.sty0, u.k_begin, u.k_end, t);
}

// One task of the persistent scorer: entries [first, first + cnt) of the
// queue, slices of the staged unit (window origin wx0, wy0; super-tile
// stx0, sty0; first angle k_begin), one per lane.  All threads of the CTA
// call it (it may end with a CTA barrier); `bits` is the bitmap space, free
// while a task is scored.
template <typename E, int NB, bool POL, int WARPS, int TC>
__device__ __forceinline__ void drain_task(const typename Pairs<E>::Raw *win, int pp, int wx0, int wy0, int stx0,
                                           int sty0, int k_begin, const TileWork &t, int first, int cnt,
                                           uint32_t *bits, unsigned long long &executed) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // a task fills ceil(cnt / 32) warps; with G = WARPS / that many warps per
    // 32 slices, each of the G takes 1/G of the points (partial sums reduced
    // in shared memory, in a fixed order)
    const int groups = (cnt + 31) >> 5;
    const int G = max(1, WARPS / groups);
    if (G == 1) {
        for (int e0 = warp * 32; e0 < cnt; e0 += WARPS * 32) {
            const int e = e0 + lane;
            const bool has = e < cnt;
            const uint32_t code = has ? t.queue[first + e] : 0u;
            score_slice<E, NB, POL, TC>(win, pp, wx0, wy0, stx0, sty0, k_begin, (int)(code >> 7), (int)(code & 31u),
                                        (int)((code >> 5) & 3u), has, t, executed);
        }
        return;
    }
    float2 *red = reinterpret_cast<float2 *>(bits);   // [WARPS][RD][TC / 2][32] (the bitmaps are free)
    const int gi = warp / G, g = warp - gi * G;
    const int e = gi * 32 + lane;
    const bool has = gi < groups && e < cnt;
    const uint32_t code = has ? t.queue[first + e] : 0u;
    float2 acc[RD][TC / 2];
    if (gi < groups) {
        const int p0 = (int)(((long long)t.n * g) / G), p1 = (int)(((long long)t.n * (g + 1)) / G);
        slice_sum<E, NB, POL, TC>(win, pp, wx0, wy0, stx0, sty0, k_begin, (int)(code >> 7), (int)(code & 31u),
                                  (int)((code >> 5) & 3u), has, t, p0, p1, acc, executed);
#pragma unroll
        for (int r = 0; r < RD; ++r)
#pragma unroll
            for (int j = 0; j < TC / 2; ++j)
                red[((warp * RD + r) * (TC / 2) + j) * 32 + lane] = acc[r][j];
    }
    __syncthreads();
    if (g == 0 && has) {
        for (int g2 = 1; g2 < G; ++g2)
#pragma unroll
            for (int r = 0; r < RD; ++r)
#pragma unroll
                for (int j = 0; j < TC / 2; ++j)
                    acc[r][j] = __fadd2_rn(acc[r][j], red[(((warp + g2) * RD + r) * (TC / 2) + j) * 32 + lane]);
        slice_store<E, TC>((int)(code >> 7), (int)(code & 31u), (int)((code >> 5) & 3u), stx0, sty0, k_begin, t, acc);
    }
}

// Persistent form (detection with early termination): CTAs pull work from
// two lists.  First the work units of the bound pass (counter qctr[3]): a
// unit's window is staged, every pose's edge-presence bound computed, slices
// with no pose that can reach min_score written -inf and the others queued
// as tasks of CH slices, each published by a release flag.  Once the units
// are handed out, the tasks (counter qctr[2]): the task's unit window is
// staged and its slices scored, one per lane.  A CTA waits for a task that
// is claimed but not yet published; the wait ends when its producer (a
// resident CTA working on a unit) publishes it, when every unit is done
// (qctr[4]) and no such task exists, or after 1 s (error flag).
template <typename E, int NB, bool POL, int WARPS, int TC>
__global__ void __launch_bounds__(WARPS * 32) score_fused_kernel(const __grid_constant__ CUtensorMap tmap,
                                                                  const TiledArgs a) {
    using Raw = typename Pairs<E>::Raw;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    const uint32_t pad = (128u - (smem_addr(smem_raw) & 127u)) & 127u;
    const Raw *win = reinterpret_cast<const Raw *>(smem_raw + pad);
    uint32_t *bits = reinterpret_cast<uint32_t *>(smem_raw + pad + window_region_bytes<E>(a.bxw, a.byw));
    // TMA destination: the window, or (angle codes) the region after it
    const void *dst = Pairs<E>::CODES ? (const void *)bits : (const void *)win;
    __shared__ __align__(8) unsigned long long mbar;
    __shared__ int s_org[2];
    __shared__ int s_job[4];   // kind (0 end, 1 unit, 2 task), unit, first entry, entries
    const uint32_t bar = smem_addr(&mbar);
    const int lane = threadIdx.x & 31;
    const int pp = a.bxw / 2;
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    uint32_t parity = 0;
    bool units_left = true;   // thread 0's view
    unsigned long long executed = 0;
    for (;;) {
        if (threadIdx.x == 0) {
            int kind = 0;
            if (units_left) {
                const unsigned un = atomicAdd(&a.qctr[3], 1u);
                if (un < (unsigned)a.units) {
                    kind = 1;
                    s_job[1] = (int)un;
                    stage_window<E>(tmap, a, unit_pos<E, TC>(a, (int)un), dst, bar, s_org);
                } else {
                    units_left = false;
                }
            }
            if (!units_left) {
                const unsigned ti = atomicAdd(&a.qctr[2], 1u);
                const int w = wait_task(a.tasks, a.tcap, a.qctr, (unsigned)a.units, ti, kWaitLimitNs);
                if (w > 0) {
                    const int4 tk = a.tasks[ti];
                    if (tk.x >= 0 && tk.x < a.units && tk.y >= 0 && tk.z > 0 &&
                        (unsigned)tk.y + (unsigned)tk.z <= a.qcap) {
                        kind = 2;
                        s_job[1] = tk.x;
                        s_job[2] = tk.y;
                        s_job[3] = tk.z;
                        stage_window<E>(tmap, a, unit_pos<E, TC>(a, tk.x), dst, bar, s_org);
                    } else {
                        atomicExch(a.err, 1);
                    }
                } else if (w < 0) {
                    atomicExch(a.err, 1);   // a producer never published (cannot happen)
                }
            }
            s_job[0] = kind;
        }
        __syncthreads();
        const int kind = s_job[0];
        if (kind == 0)
            break;
        const bool ok = mbar_wait(bar, parity);
        parity ^= 1u;
        if (__syncthreads_or(!ok)) {
            if (threadIdx.x == 0)
                atomicExch(a.err, 1);
            break;
        }
        if constexpr (Pairs<E>::CODES) {
            expand_codes(reinterpret_cast<const uint32_t *>(bits), const_cast<float4 *>(win), a.bxw, a.byw);
            __syncthreads();
        }
        const UnitPos u = unit_pos<E, TC>(a, s_job[1]);
        TileWork t = tile_work(a, u.img);
        t.bits = bits;
        t.unit = s_job[1];
        if (kind == 1) {
            // (with the bound on, score_items ends with a CTA barrier after
            // thread 0 published the unit's last tasks)
            score_items<E, NB, POL, WARPS, TC>(win, pp, s_org[0], s_org[1], u.stx0, u.sty0, u.k_begin, u.k_end, t);
            if (threadIdx.x == 0) {
                __threadfence();
                atomicAdd(&a.qctr[4], 1u);   // this unit's tasks are all published
            }
        } else {
            drain_task<E, NB, POL, WARPS, TC>(win, pp, s_org[0], s_org[1], u.stx0, u.sty0, u.k_begin, t, s_job[2],
                                              s_job[3], bits, executed);
        }
        __syncthreads();   // every warp is done with the window before the next copy
    }
    unsigned long long tot = executed;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
        tot += __shfl_xor_sync(0xffffffffu, tot, o);
    if (lane == 0 && tot)
        atomicAdd(a.exec, tot);
}

// One thread's 8 x TC pose block for one angle: the sum of every point's
// 3x3-window vote into acc (all lanes of the warp call it; `work` false
// lanes only keep the warp's loop company).  With early termination a lane
// stops once its block's partial sums prove M < min_score (exact-safe); the
// warp leaves the loop when every lane has stopped.  Returns the points the
// lane processed; `pruned` tells whether it stopped early.
template <typename E, int NB, bool POL, int TC, int R = TR>
__device__ __forceinline__ int block_dot(const typename Pairs<E>::Raw *win, int pp, int bx, int by,
                                         const RotPt *P, int n, bool work, int early, float thresh,
                                         float2 (&acc)[R][TC / 2], bool &pruned) {
#pragma unroll
    for (int r = 0; r < R; ++r)
#pragma unroll
        for (int j = 0; j < TC / 2; ++j)
            acc[r][j] = make_float2(0.f, 0.f);
    pruned = false;
    bool ldone = !work;
    int done = work ? n : 0;
    RotPt p = work ? P[0] : RotPt{0, 0, 0.f, 0.f};
    for (int i = 0; i < n; ++i) {
        const RotPt cur = p;
        if (work && i + 1 < n)
            p = P[i + 1];
        if (!ldone) {
            const float2 pxx = make_float2(cur.px, cur.px);
            const float2 pyy = make_float2(cur.py, cur.py);
            if (NB == 3) {
                const int xs = bx + cur.ox;   // first pixel column (>= 0)
                const int row0 = by + cur.oy;
                if (xs & 1)
                    point_nb3<E, POL, true, TC, R>(win, pp, row0, (xs - 1) >> 1, pxx, pyy, acc);
                else
                    point_nb3<E, POL, false, TC, R>(win, pp, row0, xs >> 1, pxx, pyy, acc);
            } else {
                const int xs = bx + 1 + cur.ox;   // centre column
                const int row0 = by + 1 + cur.oy;
                if (xs & 1)
                    point_nb1<E, POL, true, TC, R>(win, pp, row0, (xs - 1) >> 1, pxx, pyy, acc);
                else
                    point_nb1<E, POL, false, TC, R>(win, pp, row0, xs >> 1, pxx, pyy, acc);
            }
        }
        if (early && ((i + 1) % PRUNE_EVERY) == 0) {
            if (!ldone) {
                const float lim = thresh - (float)(n - 1 - i);
                bool low = true;
#pragma unroll
                for (int r = 0; r < R; ++r)
#pragma unroll
                    for (int j = 0; j < TC / 2; ++j)
                        low = low && (acc[r][j].x < lim) && (acc[r][j].y < lim);
                if (low) {
                    ldone = true;
                    pruned = true;
                    done = i + 1;
                }
            }
            if (__all_sync(0xffffffffu, ldone))
                break;
        }
    }
    return done;
}

// Scores (or -inf) of one thread's block into the map, clipped to the map.
template <int TC, int R = TR>
__device__ __forceinline__ void block_store(float *mk, int W, int H, int xl, int yl, const float2 (&acc)[R][TC / 2],
                                            float inv_n, bool neg) {
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int y = yl + r;
        if (y >= H)
            break;
        float *row = mk + (size_t)y * W;
#pragma unroll
        for (int j = 0; j < TC / 2; ++j) {
            const int x = xl + 2 * j;
            const float v0 = neg ? -INFINITY : acc[r][j].x * inv_n;
            const float v1 = neg ? -INFINITY : acc[r][j].y * inv_n;
            if (x + 1 < W && (W & 1) == 0) {
                *reinterpret_cast<float2 *>(row + x) = make_float2(v0, v1);
            } else {
                if (x < W)
                    row[x] = v0;
                if (x + 1 < W)
                    row[x + 1] = v1;
            }
        }
    }
}

// The poses of one lane's stored block (R rows of TC poses at map position
// xl, yl of angle k) whose score, rounded exactly as block_store stores it,
// is at least t.hot_thr, appended to the hot list as {image, map index}: one
// atomic per row that has such poses.  Entries past the capacity are
// counted, not written (the readers then fall back to the whole map).
template <int TC, int R>
__device__ __forceinline__ void hot_append(const TileWork &t, int k, int xl, int yl, const float2 (&acc)[R][TC / 2]) {
    const size_t plane = (size_t)(k - t.k0) * t.H * t.W;
#pragma unroll
    for (int r = 0; r < R; ++r) {
        if (yl + r >= t.H)
            break;
        uint32_t m = 0u;
#pragma unroll
        for (int j = 0; j < TC / 2; ++j) {
            const int x = xl + 2 * j;
            if (x < t.W && acc[r][j].x * t.inv_n >= t.hot_thr)
                m |= 1u << (2 * j);
            if (x + 1 < t.W && acc[r][j].y * t.inv_n >= t.hot_thr)
                m |= 1u << (2 * j + 1);
        }
        if (!m)
            continue;
        unsigned pos = atomicAdd(t.hot_cnt, (unsigned)__popc(m));
        const size_t row = plane + (size_t)(yl + r) * t.W + xl;
        while (m) {
            const int c = __ffs(m) - 1;
            m &= m - 1u;
            if (pos < t.hot_cap)
                t.hot[pos] = make_uint2(t.img, (unsigned)(row + c));
            ++pos;
        }
    }
}

// -inf over a WTX x WTY region of the map at (xl, yl), clipped to the map,
// by the 32 lanes of a warp: rows in 16-byte chunks (one float4 store per
// lane and chunk, a warp instruction covering 512 contiguous bytes of a row
// where the region is as wide) when the region and the map rows are
// 16-byte aligned, else element by element in row order.
template <int WTX, int WTY>
__device__ __forceinline__ void warp_fill_neg(float *mk, int W, int H, int xl, int yl, int lane) {
    const int cols = min(WTX, W - xl), rows = min(WTY, H - yl);
    if (cols <= 0 || rows <= 0)
        return;
    float *base = mk + (size_t)yl * W + xl;
    if (((uintptr_t)base & 15) == 0 && (W & 3) == 0) {   // every row start 16-byte aligned
        const int c4 = (cols + 3) >> 2;   // 16-byte chunks per row (the last may be partial)
        for (int idx = lane; idx < rows * c4; idx += 32) {
            const int r = idx / c4, c = (idx - r * c4) * 4;
            float *p = base + (size_t)r * W + c;
            if (c + 4 <= cols) {
                *reinterpret_cast<float4 *>(p) = make_float4(-INFINITY, -INFINITY, -INFINITY, -INFINITY);
            } else {
                for (int e = 0; e < cols - c; ++e)
                    p[e] = -INFINITY;
            }
        }
    } else {
        for (int idx = lane; idx < rows * cols; idx += 32) {
            const int r = idx / cols;
            base[(size_t)r * W + (idx - r * cols)] = -INFINITY;
        }
    }
}

// One lane's RD-row slice `part` of surviving block `src` (lane index within
// the warp tile) of item `item` (angle k_begin + item / tiles, warp tile
// item % tiles): scored and stored; `has` false lanes only keep the warp's
// loop company.
template <typename E, int NB, bool POL, int TC>
__device__ __forceinline__ void score_slice(const typename Pairs<E>::Raw *win, int pp, int wx0, int wy0, int stx0,
                                            int sty0, int k_begin, int item, int src, int part, bool has,
                                            const TileWork &a, unsigned long long &executed) {
    constexpr int LX = Pairs<E>::LX, LY = 32 / LX;
    constexpr int WTX = LX * TC, WTY = LY * TR;
    const int tiles = a.sx * a.sy;
    const int k = k_begin + item / tiles;
    const int wt = item % tiles;
    const int x0 = stx0 + (wt % a.sx) * WTX + (src % LX) * TC;
    const int y0 = sty0 + (wt / a.sx) * WTY + (src / LX) * TR + part * RD;
    bool pruned;
    float2 acc[RD][TC / 2];
    const int done = block_dot<E, NB, POL, TC, RD>(win, pp, x0 - 1 - wx0, y0 - 1 - wy0, a.rot + (size_t)k * a.n, a.n,
                                                   has, a.early, a.thresh, acc, pruned);
    if (has) {
        const int vx = max(0, min(TC, a.W - (x0 - a.ox))), vy = max(0, min(RD, a.H - (y0 - a.oy)));
        executed += (unsigned long long)done * (vx * vy);
        block_store<TC, RD>(a.map + (size_t)(k - a.k0) * a.H * a.W, a.W, a.H, x0 - a.ox, y0 - a.oy, acc, a.inv_n,
                            pruned);
        if (a.hot_cnt && !pruned)
            hot_append<TC, RD>(a, k, x0 - a.ox, y0 - a.oy, acc);
    }
}

// Partial sums of one lane's slice (as score_slice) over points [p0, p1),
// without early termination.
template <typename E, int NB, bool POL, int TC>
__device__ __forceinline__ void slice_sum(const typename Pairs<E>::Raw *win, int pp, int wx0, int wy0, int stx0,
                                          int sty0, int k_begin, int item, int src, int part, bool has,
                                          const TileWork &a, int p0, int p1, float2 (&acc)[RD][TC / 2],
                                          unsigned long long &executed) {
    constexpr int LX = Pairs<E>::LX, LY = 32 / LX;
    constexpr int WTX = LX * TC, WTY = LY * TR;
    const int tiles = a.sx * a.sy;
    const int k = k_begin + item / tiles;
    const int wt = item % tiles;
    const int x0 = stx0 + (wt % a.sx) * WTX + (src % LX) * TC;
    const int y0 = sty0 + (wt / a.sx) * WTY + (src / LX) * TR + part * RD;
    bool pruned;
    const int done = block_dot<E, NB, POL, TC, RD>(win, pp, x0 - 1 - wx0, y0 - 1 - wy0,
                                                   a.rot + (size_t)k * a.n + p0, p1 - p0, has && p1 > p0, 0, 0.f, acc,
                                                   pruned);
    if (has) {
        const int vx = max(0, min(TC, a.W - (x0 - a.ox))), vy = max(0, min(RD, a.H - (y0 - a.oy)));
        executed += (unsigned long long)done * (vx * vy);
    }
}

// Scores of one lane's slice (complete sums in acc) into the map.
template <typename E, int TC>
__device__ __forceinline__ void slice_store(int item, int src, int part, int stx0, int sty0, int k_begin,
                                            const TileWork &a, const float2 (&acc)[RD][TC / 2]) {
    constexpr int LX = Pairs<E>::LX, LY = 32 / LX;
    constexpr int WTX = LX * TC, WTY = LY * TR;
    const int tiles = a.sx * a.sy;
    const int k = k_begin + item / tiles;
    const int wt = item % tiles;
    const int x0 = stx0 + (wt % a.sx) * WTX + (src % LX) * TC;
    const int y0 = sty0 + (wt / a.sx) * WTY + (src / LX) * TR + part * RD;
    block_store<TC, RD>(a.map + (size_t)(k - a.k0) * a.H * a.W, a.W, a.H, x0 - a.ox, y0 - a.oy, acc, a.inv_n, false);
    if (a.hot_cnt)
        hot_append<TC, RD>(a, k, x0 - a.ox, y0 - a.oy, acc);
}

// One lane's edge-presence masks of 8 model points i0 .. i0 + 7 for its BW
// poses (bit c: the window of the pose c columns right of the first holds an
// edge pixel the point can take a positive vote from), from the dilated
// plane row words.  qo holds, in lane i0 + j (mod 32), point i0 + j's word
// offset and bit shift (UNI: one lane per pose row), or 32 times the word
// offset plus the shift for the first lane of a row, to which a lane adds
// xoff, its own first pose's column less the first lane's.  Bits past BW
// are left as they come (the caller masks them); CHECK: points past n give
// empty masks.
template <bool UNI, bool CHECK, int BW>
__device__ __forceinline__ void bound_masks8(const uint32_t *rbase, int xoff, int2 qo, int i0, int n,
                                             uint32_t (&mm0)[8], uint32_t (&mm1)[8], uint32_t (&mm2)[8]) {
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        const int q0 = __shfl_sync(0xffffffffu, qo.x, (i0 + j) & 31);
        const int q1 = UNI ? __shfl_sync(0xffffffffu, qo.y, (i0 + j) & 31) : 0;
        const uint32_t *row;
        int sh;
        if (UNI) {
            row = rbase + q0;
            sh = q1;
        } else {
            const int b = q0 + xoff;   // 32 * word offset + shift of this lane's first pose
            row = rbase + (b >> 5);
            sh = b & 31;
        }
        const uint32_t w0 = row[0], w1 = row[1], w2 = row[2];
        uint32_t m0 = __funnelshift_r(w0, w1, sh), m1 = __funnelshift_r(w1, w2, sh), m2 = 0u;
        if (BW > 64)
            m2 = __funnelshift_r(w2, row[3], sh);
        if (CHECK) {
            const bool in = i0 + j < n;
            m0 = in ? m0 : 0u;
            m1 = in ? m1 : 0u;
            m2 = in ? m2 : 0u;
        }
        mm0[j] = m0;
        mm1[j] = m1;
        mm2[j] = m2;
    }
}

// The (angle, warp tile) items of one CTA work unit over its staged window
// (origin wx0, wy0; row pitch pp pixel pairs), written into t.map.
//
// With the edge-presence bound (early termination on) a bound pass over the
// CTA's items first marks which 8 x TC thread blocks can still hold a pose
// reaching min_score; blocks that cannot are written -inf without a dot
// product.  The surviving blocks, in (angle, tile, lane) order, are then
// packed 32 to a warp, one per lane, so the vote loops run on full warps
// (consecutive lanes mostly share an angle, hence the point offsets).
template <typename E, int NB, bool POL, int WARPS, int TC>
__device__ __forceinline__ void score_items(const typename Pairs<E>::Raw *win, int pp, int wx0, int wy0, int stx0,
                                            int sty0, int k_begin, int k_end, const TileWork &a) {
    constexpr int LX = Pairs<E>::LX, LY = 32 / LX;
    constexpr int WTX = LX * TC, WTY = LY * TR;   // warp tile (poses)
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int lx = lane % LX, ly = lane / LX;
    const int tiles = a.sx * a.sy;
    const int items = (k_end - k_begin) * tiles;
    // edge-presence bound (with early termination; counts in 16 bit planes)
    const bool bound = a.early && a.emin > 0 && a.n < 65536;
    const int dmw = edge_bitmap_words(2 * pp);
    const size_t plane = (size_t)a.byw * dmw;
    const uint32_t *cbits = a.bits + 4 * plane;   // dilated planes, one per model-direction quadrant
    if (bound)
        build_edge_bits<E, WARPS * 32, POL>(win, pp, a.byw, a.bits, a.bits + 4 * plane);
    unsigned long long executed = 0;
    float2 acc[TR][TC / 2];
    constexpr int SPLIT = TR / RD;                 // slices per thread block (4)
    __shared__ uint32_t s_mask[kQueueItems][4];    // surviving slices of each item (see the bound pass)
    __shared__ int s_off[kQueueItems + 1];     // their first queue slot

    if (!bound) {
        for (int it = warp; it < items; it += WARPS) {
            const int k = k_begin + it / tiles;
            const int wt = it % tiles;
            const int x0 = stx0 + (wt % a.sx) * WTX + lx * TC;   // thread's first pose
            const int y0 = sty0 + (wt / a.sx) * WTY + ly * TR;
            const int vx = max(0, min(TC, a.W - (x0 - a.ox))), vy = max(0, min(TR, a.H - (y0 - a.oy)));
            bool pruned;
            const int done = block_dot<E, NB, POL, TC>(win, pp, x0 - 1 - wx0, y0 - 1 - wy0, a.rot + (size_t)k * a.n,
                                                       a.n, true, a.early, a.thresh, acc, pruned);
            executed += (unsigned long long)done * (vx * vy);
            block_store<TC>(a.map + (size_t)(k - a.k0) * a.H * a.W, a.W, a.H, x0 - a.ox, y0 - a.oy, acc, a.inv_n,
                            pruned);
            if (a.hot_cnt && !pruned)
                hot_append<TC, TR>(a, k, x0 - a.ox, y0 - a.oy, acc);
        }
    }
    for (int r0 = 0; bound && r0 < items; r0 += kQueueItems) {
        const int ni = min(kQueueItems, items - r0);
        for (int it = warp; it < ni; it += WARPS) {
            const int k = k_begin + (r0 + it) / tiles;
            const int wt = (r0 + it) % tiles;
            const RotPt *P = a.rot + (size_t)k * a.n;
            // Bound pass: lane L counts, for the BW poses of one pose row
            // it owns, how many points have an edge pixel in their window
            // (bit-sliced counters, one bit per pose), then marks the poses
            // whose count can still reach min_score.
            constexpr int LPR = 32 / WTY;       // lanes per pose row
            constexpr int BW = WTX / LPR;       // poses per lane (8 TC <= 80)
            const int xseg = stx0 + (wt % a.sx) * WTX + (lane % LPR) * BW;
            const int yrow = sty0 + (wt / a.sx) * WTY + lane / LPR;
            // Counts over all points with carry-save adders
            // (Harley-Seal): ones, twos, fours hold the low bits of every
            // pose's count, pl the count of eights in bit planes 3 ..
            uint32_t ones0 = 0u, ones1 = 0u, ones2 = 0u, twos0 = 0u, twos1 = 0u, twos2 = 0u;
            uint32_t fours0 = 0u, fours1 = 0u, fours2 = 0u;
            uint32_t pl[16][3];
#pragma unroll
            for (int q = 0; q < 16; ++q)
                pl[q][0] = pl[q][1] = pl[q][2] = 0u;
            // the points' offsets 32 at a time: one coalesced load, then a
            // warp broadcast per point
            int2 qo = make_int2(0, 0);
            const int np8 = (a.n + 7) & ~7;
            // this lane's pose row in the bitmaps and its first pose's column
            const uint32_t *rbase = cbits + (size_t)(yrow - wy0) * dmw;
            const int xb = xseg - wx0;
            const int xb0 = xb - (lane % LPR) * BW;   // the first lane of the row's column
            // Early exit: after point i a pose still needs E_i >= need_i =
            // emin - (n - i) edge hits (every remaining point adds at most
            // one).  Every 32 points the lane checks, from its top count
            // planes, whether all its poses are below 2^m <= need_i; once
            // every lane of the warp is, no pose of the item can reach emin
            // and the count stops (the poses are dead exactly as a complete
            // count would find them).
            bool all_dead = false;
            for (int i0 = 0; i0 < np8; i0 += 8) {
                if ((i0 & 31) == 0) {
                    const int ii = i0 + lane;
                    qo = make_int2(0, 0);
                    if (ii < a.n) {
                        // the word offset of the row offset in the bitmap
                        // plane of the quadrant of the point's rotated
                        // direction, and the column offset; with one lane
                        // per pose row every lane starts at column xb, and
                        // the loading lane resolves the column into the
                        // word offset and the bit shift once for the warp
                        const RotPt t = P[ii];
                        const int qpo = (POL ? 0 : quadrant(t.px, t.py)) * (int)plane + t.oy * dmw;
                        if (LPR == 1) {
                            const int b = xb + t.ox;   // window column of the first pose's centre
                            qo = make_int2(qpo + (b >> 5), b & 31);
                        } else {
                            // for the first lane of each pose row: word
                            // offset * 32 + shift in one (all terms >= 0)
                            qo = make_int2(32 * qpo + xb0 + t.ox, 0);
                        }
                    }
                }
                uint32_t mm0[8], mm1[8], mm2[8];
                if (i0 + 8 <= a.n)
                    bound_masks8<LPR == 1, false, BW>(rbase, xb - xb0, qo, i0, a.n, mm0, mm1, mm2);
                else
                    bound_masks8<LPR == 1, true, BW>(rbase, xb - xb0, qo, i0, a.n, mm0, mm1, mm2);
                // carry-save tree over the 8 masks
                auto csa = [](uint32_t &h, uint32_t &l, uint32_t a_, uint32_t b_, uint32_t c_) {
                    const uint32_t u = a_ ^ b_;
                    h = (a_ & b_) | (u & c_);
                    l = u ^ c_;
                };
                uint32_t e0, e1, e2;
                {
                    uint32_t t1, t2, t3, t4, f1, f2;
                    csa(t1, ones0, ones0, mm0[0], mm0[1]);
                    csa(t2, ones0, ones0, mm0[2], mm0[3]);
                    csa(f1, twos0, twos0, t1, t2);
                    csa(t3, ones0, ones0, mm0[4], mm0[5]);
                    csa(t4, ones0, ones0, mm0[6], mm0[7]);
                    csa(f2, twos0, twos0, t3, t4);
                    csa(e0, fours0, fours0, f1, f2);
                }
                {
                    uint32_t t1, t2, t3, t4, f1, f2;
                    csa(t1, ones1, ones1, mm1[0], mm1[1]);
                    csa(t2, ones1, ones1, mm1[2], mm1[3]);
                    csa(f1, twos1, twos1, t1, t2);
                    csa(t3, ones1, ones1, mm1[4], mm1[5]);
                    csa(t4, ones1, ones1, mm1[6], mm1[7]);
                    csa(f2, twos1, twos1, t3, t4);
                    csa(e1, fours1, fours1, f1, f2);
                }
                if (BW > 64) {
                    uint32_t t1, t2, t3, t4, f1, f2;
                    csa(t1, ones2, ones2, mm2[0], mm2[1]);
                    csa(t2, ones2, ones2, mm2[2], mm2[3]);
                    csa(f1, twos2, twos2, t1, t2);
                    csa(t3, ones2, ones2, mm2[4], mm2[5]);
                    csa(t4, ones2, ones2, mm2[6], mm2[7]);
                    csa(f2, twos2, twos2, t3, t4);
                    csa(e2, fours2, fours2, f1, f2);
                } else {
                    e2 = 0u;
                }
                // eights into the bit planes (short carry chains)
#pragma unroll
                for (int pq = 3; pq < 16; ++pq) {
                    if ((e0 | e1 | e2) == 0u)
                        break;
                    const uint32_t c0 = pl[pq][0] & e0, c1 = pl[pq][1] & e1, c2 = pl[pq][2] & e2;
                    pl[pq][0] ^= e0;
                    pl[pq][1] ^= e1;
                    pl[pq][2] ^= e2;
                    e0 = c0;
                    e1 = c1;
                    e2 = c2;
                }
                if (((i0 + 8) & 31) == 0) {
                    const int need = a.emin - max(0, a.n - (i0 + 8));
                    if (need > 0) {
                        // every count < 2^m <= need when planes m .. 15 are clear
                        const int m = 31 - __clz(need);
                        // (bits past the lane's BW poses hold no count)
                        constexpr uint32_t M1 = BW >= 64 ? 0xffffffffu : ((1u << ((BW - 32) & 31)) - 1u);
                        constexpr uint32_t M2 = BW > 64 ? ((1u << ((BW - 64) & 31)) - 1u) : 0u;
                        uint32_t hi = 0u;
#pragma unroll
                        for (int pq = 0; pq < 16; ++pq) {
                            if (pq < m)
                                continue;
                            if (pq == 0)
                                hi |= ones0 | (ones1 & M1) | (ones2 & M2);
                            else if (pq == 1)
                                hi |= twos0 | (twos1 & M1) | (twos2 & M2);
                            else if (pq == 2)
                                hi |= fours0 | (fours1 & M1) | (fours2 & M2);
                            else
                                hi |= pl[pq][0] | (pl[pq][1] & M1) | (pl[pq][2] & M2);
                        }
                        if (__all_sync(0xffffffffu, hi == 0u)) {
                            all_dead = true;
                            break;
                        }
                    }
                }
            }
            pl[0][0] = ones0;
            pl[0][1] = ones1;
            pl[0][2] = ones2;
            pl[1][0] = twos0;
            pl[1][1] = twos1;
            pl[1][2] = twos2;
            pl[2][0] = fours0;
            pl[2][1] = fours1;
            pl[2][2] = fours2;
            // counts >= emin, bit-serially from the top plane
            uint32_t gt0 = 0u, gt1 = 0u, gt2 = 0u, eq0 = ~0u, eq1 = ~0u, eq2 = ~0u;
#pragma unroll
            for (int pq = 15; pq >= 0; --pq) {
                if ((a.emin >> pq) & 1) {
                    eq0 &= pl[pq][0];
                    eq1 &= pl[pq][1];
                    eq2 &= pl[pq][2];
                } else {
                    gt0 |= eq0 & pl[pq][0];
                    gt1 |= eq1 & pl[pq][1];
                    gt2 |= eq2 & pl[pq][2];
                    eq0 &= ~pl[pq][0];
                    eq1 &= ~pl[pq][1];
                    eq2 &= ~pl[pq][2];
                }
            }
            const uint32_t o0 = all_dead ? 0u : gt0 | eq0;
            const uint32_t o1 =
                all_dead ? 0u : (gt1 | eq1) & (BW >= 64 ? 0xffffffffu : ((1u << ((BW - 32) & 31)) - 1u));
            const uint32_t o2 = (BW > 64 && !all_dead) ? ((gt2 | eq2) & ((1u << ((BW - 64) & 31)) - 1u)) : 0u;
            // the item's whole warp tile is written -inf (coalesced); its
            // surviving RD-row slices go to the queue and are overwritten
            // when they are scored (after this write: the tasks are published
            // behind a fence, the local drain behind a CTA barrier)
            const int seg = (lx * TC) / BW, c0 = lx * TC - seg * BW;
            float *mk = a.map + (size_t)(k - a.k0) * a.H * a.W;
            warp_fill_neg<WTX, WTY>(mk, a.W, a.H, stx0 + (wt % a.sx) * WTX - a.ox, sty0 + (wt / a.sx) * WTY - a.oy,
                                    lane);
            uint32_t nib = 0u;   // surviving slices of this lane's block
#pragma unroll
            for (int sp = 0; sp < SPLIT; ++sp) {
                uint32_t act = 0u;
#pragma unroll
                for (int r = sp * RD; r < (sp + 1) * RD; ++r) {
                    const int src = (ly * TR + r) * LPR + seg;
                    const uint32_t v0 = __shfl_sync(0xffffffffu, o0, src);
                    const uint32_t v1 = __shfl_sync(0xffffffffu, o1, src);
                    const uint32_t v2 = __shfl_sync(0xffffffffu, o2, src);
                    const uint32_t lo = c0 < 32 ? v0 : (c0 < 64 ? v1 : v2);
                    const uint32_t hi = c0 < 32 ? v1 : (c0 < 64 ? v2 : 0u);
                    act |= __funnelshift_r(lo, hi, c0 & 31) & ((1u << TC) - 1u);
                }
                nib |= (act != 0u ? 1u : 0u) << sp;
            }
            // queue order (item, lane, slice): word q of the item's mask holds
            // lanes 8q .. 8q + 7, four slice bits each, so the slices of one
            // block are neighbours in the queue (distinct rows, and with an
            // odd window pitch distinct shared-memory banks)
            uint32_t wq = nib << (4 * (lane & 7));
            wq |= __shfl_xor_sync(0xffffffffu, wq, 1);
            wq |= __shfl_xor_sync(0xffffffffu, wq, 2);
            wq |= __shfl_xor_sync(0xffffffffu, wq, 4);
            if ((lane & 7) == 0)
                s_mask[it][lane >> 3] = wq;
        }
        __syncthreads();
        // one surviving slice per lane, in (item, slice, lane) order
        constexpr int CH = WARPS * 32 < kTaskSlices ? WARPS * 32 : kTaskSlices;   // slices per task
        __shared__ unsigned s_qb, s_tb, s_nt;
        if (warp == 0) {   // queue offsets: exclusive prefix sum of the surviving counts
            int carry = 0;
            for (int b0 = 0; b0 < ni; b0 += 32) {
                const int i = b0 + lane;
                int c = 0;
                if (i < ni)
#pragma unroll
                    for (int q = 0; q < 4; ++q)
                        c += __popc(s_mask[i][q]);
                int v = c;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const int t = __shfl_up_sync(0xffffffffu, v, o);
                    if (lane >= o)
                        v += t;
                }
                if (i < ni)
                    s_off[i] = carry + v - c;
                carry += __shfl_sync(0xffffffffu, v, 31);
            }
            if (lane == 0)
                s_off[ni] = carry;
            // persistent form: the unit's queue run and its tasks, allocated
            // by the same warp (one CTA barrier less)
            if (a.queue && lane == 0) {
                const int tot = carry;
                const unsigned nt = (unsigned)((tot + CH - 1) / CH);
                unsigned qb = ~0u, tb = 0;
                if (tot > 0) {
                    qb = atomicAdd(&a.qctr[0], (unsigned)tot);
                    tb = atomicAdd(&a.qctr[1], nt);
                    if (qb + (unsigned)tot > a.qcap || tb + nt > a.tcap) {
                        atomicExch(a.err, 1);   // capacities cover every slice: cannot happen
                        qb = ~0u;
                    } else {
                        for (unsigned j = 0; j < nt; ++j)
                            a.tasks[tb + j] = make_int4(a.unit, (int)(qb + j * CH), min(CH, tot - (int)(j * CH)), 0);
                    }
                }
                s_qb = qb;
                s_tb = tb;
                s_nt = qb == ~0u ? 0u : nt;
            }
        }
        __syncthreads();
        const int total = s_off[ni];
        if (a.queue) {
            // persistent form: the slices to the global queue and one task
            // per CH of them (a CTA's worth), each published once written
            const unsigned qb = s_qb;
            if (qb != ~0u) {
                for (int it = warp; it < ni; it += WARPS) {
                    const int q = lane >> 3, sh = 4 * (lane & 7);
                    unsigned slot = qb + (unsigned)s_off[it];
                    for (int q2 = 0; q2 < q; ++q2)
                        slot += (unsigned)__popc(s_mask[it][q2]);
                    const uint32_t w = s_mask[it][q];
                    slot += (unsigned)__popc(w & ((1u << sh) - 1u));
                    const uint32_t nb = (w >> sh) & 15u;
#pragma unroll
                    for (int sp = 0; sp < SPLIT; ++sp)
                        if ((nb >> sp) & 1u)
                            a.queue[slot++] = ((uint32_t)(r0 + it) << 7) | ((uint32_t)sp << 5) | (uint32_t)lane;
                }
                __threadfence();   // this thread's entries before the tasks' flags
            }
            __syncthreads();
            if (threadIdx.x == 0 && s_nt) {
                __threadfence();
                for (unsigned j = 0; j < s_nt; ++j)
                    st_release_u32(reinterpret_cast<unsigned *>(&a.tasks[s_tb + j].w), 1u);
            }
        } else {
            for (int e0 = warp * 32; e0 < total; e0 += WARPS * 32) {
                const int e = e0 + lane;
                const bool has = e < total;
                int it = 0, src = 0, part = 0;
                if (has) {
                    int lo = 0, hi = ni - 1;   // last item whose first slot <= e
                    while (lo < hi) {
                        const int mid = (lo + hi + 1) >> 1;
                        if (s_off[mid] <= e)
                            lo = mid;
                        else
                            hi = mid - 1;
                    }
                    it = lo;
                    int rank = e - s_off[it];
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const int c = __popc(s_mask[it][q]);
                        if (rank >= 0 && rank < c) {
                            const int bit = nth_set_bit(s_mask[it][q], rank);
                            src = 8 * q + (bit >> 2);
                            part = bit & 3;
                        }
                        rank -= c;
                    }
                }
                score_slice<E, NB, POL, TC>(win, pp, wx0, wy0, stx0, sty0, k_begin, r0 + it, src, part, has, a,
                                            executed);
            }
        }
        __syncthreads();   // s_mask and s_off are refilled by the next round
    }
    // executed pose-points of this thread's blocks, one atomic per warp
    unsigned long long tot = executed;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
        tot += __shfl_xor_sync(0xffffffffu, tot, o);
    if (lane == 0 && tot)
        atomicAdd(a.exec, tot);
}

// Persistent form for batches of uneven (image, model) pairs: every CTA
// pulls work units (pair, super-tile, angle group) from one atomic counter,
// stages the unit's window with that pair's own 2-D tensor map (box sized for
// the pair), and scores it.  The window buffer and its mbarrier are reused
// unit after unit (the barrier's phase alternates).  Pairs are laid out
// largest first so the dynamic schedule ends with small units.
template <typename E, int NB, bool POL, int WARPS, int TC>
__global__ void __launch_bounds__(WARPS * 32) score_pairs_kernel(const PairScore *__restrict__ pairs, int n_pairs,
                                                                  int total, int sx, int sy, int tg, int early,
                                                                  unsigned *__restrict__ counter, int *err,
                                                                  unsigned long long *exec, unsigned win_bytes) {
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
                atomicExch(err, 1);
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
        t.exec = exec;
        t.emin = P.emin;
        t.byw = P.byw;
        t.bits = reinterpret_cast<uint32_t *>(smem_raw + pad + ((win_bytes + 15u) & ~15u));
        t.err = err;
        t.queue = nullptr;
        t.tasks = nullptr;
        t.qctr = nullptr;
        t.qcap = t.tcap = 0;
        t.unit = 0;
        t.hot_cnt = P.hot_cnt;
        t.hot = P.hot;
        t.hot_cap = P.hot_cap;
        t.hot_thr = P.hot_thr;
        t.img = (unsigned)P.job;
        score_items<E, NB, POL, WARPS, TC>(win, P.bxw / 2, s_unit[4], s_unit[5], s_unit[2], s_unit[3], group * tg,
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
// before the next copy).  With the edge-presence bound (a.alive, written by
// chunk_bound_kernel) poses it proves below min_score are written -inf, a
// warp none of whose poses is alive computes nothing, and a CTA none of whose
// poses is alive stages no window.
template <typename E, int NB, bool POL, int WARPS, int TC>
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
    // poses the edge-presence bound leaves: bit 2j (2j + 1) of keep[r] for
    // pose (x0 + 2j (+ 1), y0 + r); every pose when there is no bound
    uint32_t keep[TR];
#pragma unroll
    for (int r = 0; r < TR; ++r)
        keep[r] = (1u << TC) - 1u;
    if (a.alive) {
        const uint32_t *am = a.alive + ((size_t)img * gridDim.y + kl) * (size_t)a.H * a.alive_w;
        const int mx = x0 - a.ox, wi = mx >> 5, sh = mx & 31;
        bool any = false;
#pragma unroll
        for (int r = 0; r < TR; ++r) {
            const int my = y0 - a.oy + r;
            uint32_t v = 0u;
            if (my < a.H && wi < a.alive_w) {
                const uint32_t *row = am + (size_t)my * a.alive_w;
                v = __funnelshift_r(row[wi], wi + 1 < a.alive_w ? row[wi + 1] : 0u, sh) & ((1u << TC) - 1u);
            }
            keep[r] = v;
            any = any || v != 0u;
        }
        alive = __any_sync(0xffffffffu, any);
    }
    // a CTA none of whose poses survived the bound stages nothing
    const int c_stop = (a.alive && !__syncthreads_or(alive)) ? c_begin : c_end;
    int done = 0;
    uint32_t parity = 0;
    for (int c = c_begin; c < c_stop; ++c) {
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
                atomicExch(a.err, 1);
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
                        point_nb3<E, POL, true, TC>(win, pp, row0, (xs - 1) >> 1, pxx, pyy, part);
                    else
                        point_nb3<E, POL, false, TC>(win, pp, row0, xs >> 1, pxx, pyy, part);
                } else {
                    const int xs = bx + 1 + cur.ox;
                    const int row0 = by + 1 + cur.oy;
                    if (xs & 1)
                        point_nb1<E, POL, true, TC>(win, pp, row0, (xs - 1) >> 1, pxx, pyy, part);
                    else
                        point_nb1<E, POL, false, TC>(win, pp, row0, xs >> 1, pxx, pyy, part);
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
                        low = low && (!((keep[r] >> (2 * j)) & 1u) || acc[r][j].x < lim) &&
                              (!((keep[r] >> (2 * j + 1)) & 1u) || acc[r][j].y < lim);
                if (__all_sync(0xffffffffu, low))
                    alive = false;
            }
        }
        // every warp is done with the window before the next copy; stop when
        // all warps have pruned
        if (!__syncthreads_or(alive))
            break;
    }
    {
        const int vx = max(0, min(TC, a.W - (x0 - a.ox))), vy = max(0, min(TR, a.H - (y0 - a.oy)));
        const unsigned valid = __reduce_add_sync(0xffffffffu, (unsigned)(vx * vy));
        if (lane == 0)
            atomicAdd(a.exec, (unsigned long long)done * valid);
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
            const float v0 = alive && ((keep[r] >> (2 * j)) & 1u) ? acc[r][j].x * a.inv_n : -INFINITY;
            const float v1 = alive && ((keep[r] >> (2 * j + 1)) & 1u) ? acc[r][j].y * a.inv_n : -INFINITY;
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

// Edge-presence bound of the chunked form.  A chunked CTA cannot hold the
// bitmaps of every point's reach (a 512-pixel template reaches ~724 pixels),
// so the bound works from whole-image planes in global memory instead:
//   1. chunk_edge_planes_kernel: plane q of N holds, for every pixel of the
//      field's TMA extent (wp x H) and a one-pixel margin, whether it is an
//      edge pixel that can give a positive vote to a model direction in
//      quadrant q (the rule of build_edge_bits);
//   2. chunk_dilate_kernel: D_q = N_q dilated by 3 x 3;
//   3. chunk_bound_kernel: for each pose of the window, the number of points
//      whose projected centre hits D of their direction's quadrant, counted
//      bit-sliced 32 poses per word, and one alive bit per pose: count >=
//      emin.  A pose with count < emin is below min_score (the argument of
//      edge_count_threshold), so the chunked kernel writes it -inf and skips
//      every CTA none of whose poses is alive.
// Plane layout: [image][q][H + 2][ppw] words, bit c of word w of row r for
// field pixel (32 w + c - 1, r - 1); ppw = (wp + 2 + 31) / 32.
template <typename E, bool POL>
__global__ void __launch_bounds__(256) chunk_edge_planes_kernel(const typename Pairs<E>::Raw *__restrict__ field,
                                                                int wp, int H, size_t img_pairs, int ppw,
                                                                uint32_t *__restrict__ nplanes) {
    constexpr int NQ = POL ? 1 : 4;
    const int wi = blockIdx.x * blockDim.x + threadIdx.x;
    const int r = blockIdx.y, img = blockIdx.z;
    if (wi >= ppw)
        return;
    uint32_t e[NQ];
#pragma unroll
    for (int q = 0; q < NQ; ++q)
        e[q] = 0u;
    const int y = r - 1;
    if (y >= 0 && y < H) {
        const typename Pairs<E>::Raw *row = field + img * img_pairs + (size_t)y * (wp / 2);
        for (int c = 0; c < 32; ++c) {
            const int x = 32 * wi + c - 1;
            if (x < 0 || x >= wp)
                continue;
            const float4 v = Pairs<E>::get(row, x >> 1);   // {x0, x1, y0, y1}
            const float gx = (x & 1) ? v.y : v.x, gy = (x & 1) ? v.w : v.z;
            if (gx != 0.f || gy != 0.f) {
                if (POL) {
                    e[0] |= 1u << c;
                } else {
                    const int opp = (quadrant(gx, gy) + 2) & 3;
#pragma unroll
                    for (int q = 0; q < NQ; ++q)
                        if (q != opp)
                            e[q] |= 1u << c;
                }
            }
        }
    }
    const size_t plane = (size_t)(H + 2) * ppw;
#pragma unroll
    for (int q = 0; q < NQ; ++q)
        nplanes[((size_t)img * NQ + q) * plane + (size_t)r * ppw + wi] = e[q];
}

// D = N dilated by 3 x 3 (grid: words x rows x image-planes).
template <typename E>
__global__ void __launch_bounds__(256) chunk_dilate_kernel(const uint32_t *__restrict__ nplanes, int rows, int ppw,
                                                           uint32_t *__restrict__ dplanes) {
    const int wi = blockIdx.x * blockDim.x + threadIdx.x;
    const int r = blockIdx.y;
    if (wi >= ppw)
        return;
    const uint32_t *pl = nplanes + (size_t)blockIdx.z * rows * ppw;
    uint32_t d = 0u;
    for (int rr = r - 1; rr <= r + 1; ++rr) {
        if (rr < 0 || rr >= rows)
            continue;
        const uint32_t *row = pl + (size_t)rr * ppw;
        const uint32_t c = row[wi];
        const uint32_t lft = wi > 0 ? row[wi - 1] : 0u, rgt = wi + 1 < ppw ? row[wi + 1] : 0u;
        // bit b of the result: pixels b - 1, b, b + 1
        d |= c | (c << 1) | (lft >> 31) | (c >> 1) | (rgt << 31);
    }
    dplanes[(size_t)blockIdx.z * rows * ppw + (size_t)r * ppw + wi] = d;
}

// One warp per (image, angle, 32 / lpr pose rows, lpr words): lane L counts
// for the 32 poses of word (g lpr + L % lpr) of pose row (rb + L / lpr).
// Lanes of one pose row read consecutive words, so the upper word a lane's
// 32-bit window needs is its right neighbour's lower word (a shuffle); the
// last lane of the row loads its own.
template <typename E, bool POL>
__global__ void __launch_bounds__(256) chunk_bound_kernel(const ChunkBoundArgs a) {
    const int lane = threadIdx.x & 31;
    const int rpw = 32 / a.lpr;
    const long long task = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const long long row_tasks = (long long)((a.gh + rpw - 1) / rpw) * a.groups;
    if (task >= row_tasks * a.nk * a.count)
        return;
    const int g = (int)(task % a.groups);
    const int rb = (int)((task / a.groups) % ((a.gh + rpw - 1) / rpw)) * rpw;
    const int kl = (int)((task / row_tasks) % a.nk);
    const int img = (int)(task / (row_tasks * a.nk));
    const int lw = lane % a.lpr;
    const bool last = lw == a.lpr - 1;
    const int wi = g * a.lpr + lw;
    const int y = rb + lane / a.lpr;
    constexpr int NQ = POL ? 1 : 4;
    const int rows = a.H + 2;
    const int plane = rows * a.ppw;   // 4 planes < 2^31 words (checked by the launcher)
    const uint32_t *pl = a.dplanes + (size_t)img * NQ * plane;
    // plane row of this lane's pose row before the point's offset (+1: the
    // planes' margin); the plane column of bit b of its word for a point
    // with column offset ox is (gx0 + 1 + ox) + 32 wi + b
    const int prow = a.gy0 + y + 1;
    const uint32_t *lrow = pl + (size_t)max(prow, 0) * a.ppw;   // only used when the row is inside
    const RotPt *P = a.rot + (size_t)(a.k0 + kl) * a.n;
    uint32_t ones = 0u, twos = 0u, fours = 0u, pl16[16];
#pragma unroll
    for (int q = 0; q < 16; ++q)
        pl16[q] = 0u;
    // per point, computed by the lane that loads it: the plane column of the
    // first pose's centre, the row offset, and the word offset of its
    // quadrant plane and row
    int qc = 0, qoy = 0, qoff = 0;
    const int np8 = (a.n + 7) & ~7;
    for (int i0 = 0; i0 < np8; i0 += 8) {
        if ((i0 & 31) == 0) {
            const int ii = i0 + lane;
            qc = qoy = qoff = 0;
            if (ii < a.n) {
                const RotPt t = P[ii];
                const int q = POL ? 0 : quadrant(t.px, t.py);
                qc = a.gx0 + 1 + t.ox;
                qoy = t.oy;
                qoff = q * plane + t.oy * a.ppw;
            }
        }
        uint32_t mm[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const int c = __shfl_sync(0xffffffffu, qc, (i0 + j) & 31) + 32 * wi;
            const int oy = __shfl_sync(0xffffffffu, qoy, (i0 + j) & 31);
            const int off = __shfl_sync(0xffffffffu, qoff, (i0 + j) & 31);
            const int w0 = c >> 5, sh = c & 31;   // arithmetic shift: floor
            const bool row_in = i0 + j < a.n && (unsigned)(prow + oy) < (unsigned)rows;
            const uint32_t *src = lrow + off + w0;   // plane q, row prow + oy, word w0 (when inside)
            uint32_t lo = 0u;
            if (row_in && (unsigned)w0 < (unsigned)a.ppw)
                lo = *src;
            uint32_t hi = __shfl_down_sync(0xffffffffu, lo, 1);
            if (last)
                hi = row_in && (unsigned)(w0 + 1) < (unsigned)a.ppw ? src[1] : 0u;
            mm[j] = __funnelshift_r(lo, hi, sh);
        }
        auto csa = [](uint32_t &h, uint32_t &l, uint32_t a_, uint32_t b_, uint32_t c_) {
            const uint32_t u = a_ ^ b_;
            h = (a_ & b_) | (u & c_);
            l = u ^ c_;
        };
        uint32_t t1, t2, t3, t4, f1, f2, e8;
        csa(t1, ones, ones, mm[0], mm[1]);
        csa(t2, ones, ones, mm[2], mm[3]);
        csa(f1, twos, twos, t1, t2);
        csa(t3, ones, ones, mm[4], mm[5]);
        csa(t4, ones, ones, mm[6], mm[7]);
        csa(f2, twos, twos, t3, t4);
        csa(e8, fours, fours, f1, f2);
#pragma unroll
        for (int q = 3; q < 16; ++q) {
            if (e8 == 0u)
                break;
            const uint32_t cy = pl16[q] & e8;
            pl16[q] ^= e8;
            e8 = cy;
        }
    }
    pl16[0] = ones;
    pl16[1] = twos;
    pl16[2] = fours;
    uint32_t gt = 0u, eq = ~0u;
#pragma unroll
    for (int q = 15; q >= 0; --q) {
        if ((a.emin >> q) & 1) {
            eq &= pl16[q];
        } else {
            gt |= eq & pl16[q];
            eq &= ~pl16[q];
        }
    }
    if (wi < a.aw && y < a.gh)
        a.alive[(((size_t)img * a.nk + kl) * a.gh + y) * a.aw + wi] = gt | eq;
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------

template <typename E, int NB, bool POL, int WARPS, int TC>
cudaError_t launch_t(const CUtensorMap &tm, const TiledArgs &a, dim3 grid, size_t smem, cudaStream_t st) {
    auto kern = score_tiled_kernel<E, NB, POL, WARPS, TC>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess)
        return e;
    // prefer the largest shared-memory carve-out so window size, not the
    // L1/shared split, limits resident CTAs
    e = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared);
    if (e != cudaSuccess)
        return e;
    if (!a.queue) {
        prof_begin(kStageScoreBound, st);
        kern<<<grid, WARPS * 32, smem, st>>>(tm, a);
        count_launches(1);
        prof_end(kStageScoreBound, st);
        return cudaGetLastError();
    }
    // persistent form: as many CTAs as are resident at once
    auto fk = score_fused_kernel<E, NB, POL, WARPS, TC>;
    e = cudaFuncSetAttribute(fk, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess)
        return e;
    e = cudaFuncSetAttribute(fk, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared);
    if (e != cudaSuccess)
        return e;
    int dev = 0, sms = 0, occ = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess ||
        (e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess ||
        (e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fk, WARPS * 32, smem)) != cudaSuccess)
        return e;
    const unsigned ctas = (unsigned)std::max(1, sms * std::max(occ, 1));
    prof_begin(kStageScoreBound, st);
    fk<<<ctas, WARPS * 32, smem, st>>>(tm, a);
    count_launches(1);
    prof_end(kStageScoreBound, st);
    return cudaGetLastError();
}

template <typename E, int NB, bool POL, int WARPS>
cudaError_t launch_tc(const CUtensorMap &tm, const TiledArgs &a, dim3 grid, size_t smem, int tc, cudaStream_t st) {
    return tc == 10 ? launch_t<E, NB, POL, WARPS, 10>(tm, a, grid, smem, st)
                    : launch_t<E, NB, POL, WARPS, 6>(tm, a, grid, smem, st);
}

template <typename E>
cudaError_t tiled_dispatch(const CUtensorMap &tm, const TiledArgs &a, dim3 grid, size_t smem, int nbhd, bool pol,
                           int warps, int tc, cudaStream_t st) {
    if (warps == 4) {
        if (nbhd == 3)
            return pol ? launch_tc<E, 3, true, 4>(tm, a, grid, smem, tc, st)
                       : launch_tc<E, 3, false, 4>(tm, a, grid, smem, tc, st);
        return pol ? launch_tc<E, 1, true, 4>(tm, a, grid, smem, tc, st)
                   : launch_tc<E, 1, false, 4>(tm, a, grid, smem, tc, st);
    }
    if (nbhd == 3)
        return pol ? launch_tc<E, 3, true, 8>(tm, a, grid, smem, tc, st)
                   : launch_tc<E, 3, false, 8>(tm, a, grid, smem, tc, st);
    return pol ? launch_tc<E, 1, true, 8>(tm, a, grid, smem, tc, st)
               : launch_tc<E, 1, false, 8>(tm, a, grid, smem, tc, st);
}

template <typename E, int NB, bool POL, int WARPS>
cudaError_t launch_c(const CUtensorMap &tm, const ChunkArgs &a, dim3 grid, size_t smem, cudaStream_t st) {
    auto kern = score_chunked_kernel<E, NB, POL, WARPS, kChunkCols>;
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
cudaError_t chunked_dispatch(const CUtensorMap &tm, const ChunkArgs &a, dim3 grid, size_t smem, int nbhd, bool pol,
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

// The three bound kernels of the chunked form (buffers as chunk_bound_kernel).
template <typename E>
cudaError_t chunk_bound_dispatch(const void *field, int wp, int H, size_t img_px, bool pol, uint32_t *nplanes,
                                 const ChunkBoundArgs &b, cudaStream_t st) {
    using Raw = typename Pairs<E>::Raw;
    const int nq = pol ? 1 : 4;
    const dim3 gp((unsigned)((b.ppw + 255) / 256), (unsigned)(H + 2), (unsigned)b.count);
    if (pol)
        chunk_edge_planes_kernel<E, true><<<gp, 256, 0, st>>>(static_cast<const Raw *>(field), wp, H, img_px / 2,
                                                                b.ppw, nplanes);
    else
        chunk_edge_planes_kernel<E, false><<<gp, 256, 0, st>>>(static_cast<const Raw *>(field), wp, H, img_px / 2,
                                                                 b.ppw, nplanes);
    const dim3 gd((unsigned)((b.ppw + 255) / 256), (unsigned)(H + 2), (unsigned)(b.count * nq));
    chunk_dilate_kernel<E><<<gd, 256, 0, st>>>(nplanes, H + 2, b.ppw, const_cast<uint32_t *>(b.dplanes));
    const int rpw = 32 / b.lpr;
    const long long tasks = (long long)((b.gh + rpw - 1) / rpw) * b.groups * b.nk * b.count;
    const unsigned blocks = (unsigned)((tasks + 7) / 8);
    if (pol)
        chunk_bound_kernel<E, true><<<blocks, 256, 0, st>>>(b);
    else
        chunk_bound_kernel<E, false><<<blocks, 256, 0, st>>>(b);
    count_launches(3);
    return cudaGetLastError();
}

template <typename E, int NB, bool POL, int WARPS, int TC>
cudaError_t launch_pairs_t(const PairScore *pairs, int n_pairs, int total, const TileConfig &cfg, int early,
                           size_t smem, size_t win_bytes, unsigned *counter, int *err, unsigned long long *exec,
                           cudaStream_t st) {
    auto kern = score_pairs_kernel<E, NB, POL, WARPS, TC>;
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
    kern<<<grid, WARPS * 32, smem, st>>>(pairs, n_pairs, total, cfg.sx, cfg.sy, cfg.tg, early, counter, err, exec,
                                         (unsigned)win_bytes);
    count_launches(1);
    return cudaGetLastError();
}

template <typename E, int NB, bool POL, int WARPS>
cudaError_t launch_pairs_tc(const PairScore *pairs, int n_pairs, int total, const TileConfig &cfg, int early,
                            size_t smem, size_t win_bytes, unsigned *counter, int *err, unsigned long long *exec,
                            cudaStream_t st) {
    return cfg.tc == 10 ? launch_pairs_t<E, NB, POL, WARPS, 10>(pairs, n_pairs, total, cfg, early, smem, win_bytes,
                                                                counter, err, exec, st)
                        : launch_pairs_t<E, NB, POL, WARPS, 6>(pairs, n_pairs, total, cfg, early, smem, win_bytes,
                                                               counter, err, exec, st);
}

template <typename E>
cudaError_t pairs_dispatch(const PairScore *pairs, int n_pairs, int total, const TileConfig &cfg, int nbhd, bool pol,
                           int early, size_t smem, size_t win_bytes, unsigned *counter, int *err,
                           unsigned long long *exec, cudaStream_t st) {
#define SAM_PAIRS_ARGS pairs, n_pairs, total, cfg, early, smem, win_bytes, counter, err, exec, st
    if (cfg.warps == 4) {
        if (nbhd == 3)
            return pol ? launch_pairs_tc<E, 3, true, 4>(SAM_PAIRS_ARGS) : launch_pairs_tc<E, 3, false, 4>(SAM_PAIRS_ARGS);
        return pol ? launch_pairs_tc<E, 1, true, 4>(SAM_PAIRS_ARGS) : launch_pairs_tc<E, 1, false, 4>(SAM_PAIRS_ARGS);
    }
    if (nbhd == 3)
        return pol ? launch_pairs_tc<E, 3, true, 8>(SAM_PAIRS_ARGS) : launch_pairs_tc<E, 3, false, 8>(SAM_PAIRS_ARGS);
    return pol ? launch_pairs_tc<E, 1, true, 8>(SAM_PAIRS_ARGS) : launch_pairs_tc<E, 1, false, 8>(SAM_PAIRS_ARGS);
#undef SAM_PAIRS_ARGS
}

}  // namespace
}  // namespace sam
