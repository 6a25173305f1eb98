// Fused separable downscaler: two chained repetitive tasks (horizontal then
// vertical 8-tap -> 3-output FIR bank, step 8, no wrap) sharing one array
// (Sec. 5, associatedParts).  Each 8x8 input block maps to a 3x3 output block,
// so the intermediate (the horizontal task's output) lives only in registers:
// the chain reads X once and writes Y once.
//
// Thread mapping.  A work item is 8 rows x 4 columns (one float4 per row) of
// one frame; the two items of an 8x8 block sit in adjacent lanes (even lane:
// columns 0-3, odd lane: columns 4-7).  A warp therefore reads 32 contiguous
// float4 per row: fully coalesced 128-bit loads.  Each lane applies the
// horizontal taps to its 4 columns and the vertical taps to the partial sums;
// the two partial 3x3 blocks are added with one shuffle per output.
//
// Backward (loss gradient g = dL/dY given):
//   dmid[kv][jh] = sum_jv Hv[jv,kv] g[jv][jh]          (transposed vertical tiler)
//   dX[kv][kh]   = sum_jh Hh[jh,kh] dmid[kv][jh]        (transposed horizontal tiler)
//   dHv[jv,kv]  += sum_jh g[jv][jh] mid[kv][jh]
//   dHh[jh,kh]  += sum_kv dmid[kv][jh] X[kv][kh]
// With step == T every input element belongs to exactly one block, so dX is
// written once per element (owner computes; no atomics).  Tap gradients are
// reduced per warp (shuffles), per CTA (shared memory, fixed order) into a
// per-CTA partial, then across CTAs in fixed order by a second kernel:
// deterministic run to run.
#include <cstdlib>
#include <cstring>

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "arol_internal.h"
#include "ptx.h"

namespace arol {
namespace {

constexpr int kThr = 256;
constexpr unsigned kFull = 0xffffffffu;
constexpr int kTapGrads = 48;   // 3x8 horizontal + 3x8 vertical
constexpr int kTapGroups = 8;   // thread groups of the last-CTA tap-gradient reduction

__device__ __forceinline__ float4 ld_stream4(const float* p) {
    float4 v;
    asm("ld.global.nc.L1::no_allocate.v4.f32 {%0,%1,%2,%3}, [%4];"
        : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
        : "l"(p));
    return v;
}

__device__ __forceinline__ void st_stream4(float* p, float4 v) {
    asm volatile("st.global.cs.v4.f32 [%0], {%1,%2,%3,%4};" ::"l"(p), "f"(v.x), "f"(v.y), "f"(v.z),
                 "f"(v.w)
                 : "memory");
}

struct Taps {
    float hh[3][4];   // horizontal taps of this lane's 4 columns: Hh[jh][4*half + t]
    float hv[3][8];   // vertical taps Hv[jv][kv]
};

__device__ __forceinline__ void load_taps(const float* taps, int half, Taps& tp) {
#pragma unroll
    for (int j = 0; j < 3; ++j) {
#pragma unroll
        for (int t = 0; t < 4; ++t) tp.hh[j][t] = __ldg(taps + j * 8 + 4 * half + t);
#pragma unroll
        for (int k = 0; k < 8; ++k) tp.hv[j][k] = __ldg(taps + 24 + j * 8 + k);
    }
}

// Horizontal taps on this lane's 4 columns of one row (a partial sum of mid).
__device__ __forceinline__ void horiz(const Taps& tp, const float4 v, float mh[3]) {
#pragma unroll
    for (int j = 0; j < 3; ++j)
        mh[j] = fmaf(tp.hh[j][3], v.w, fmaf(tp.hh[j][2], v.z, fmaf(tp.hh[j][1], v.y, tp.hh[j][0] * v.x)));
}

struct Item {
    bool valid;
    int half;
    uint32_t f, sy, c4;
};

__device__ __forceinline__ Item decode(uint32_t item, uint32_t items, uint32_t Q, uint32_t HB) {
    Item it;
    it.valid = item < items;
    it.half = (int)(item & 1u);
    const uint32_t s = it.valid ? item / Q : 0u;
    it.c4 = it.valid ? item - s * Q : 0u;
    it.f = s / HB;
    it.sy = s - it.f * HB;
    return it;
}

// Adds the two lanes' partial 3x3 blocks and stores the block: the even lane
// writes output rows 0 and 1, the odd lane row 2.
__device__ __forceinline__ void store_block(const DownscaleDev& p, const Item& it, float y[3][3]) {
#pragma unroll
    for (int j = 0; j < 3; ++j)
#pragma unroll
        for (int i = 0; i < 3; ++i) y[j][i] += __shfl_xor_sync(kFull, y[j][i], 1);
    if (!it.valid) return;
    const int Wo = (p.W >> 3) * 3;
    const int Ho = (p.H >> 3) * 3;
    float* yp = p.y + ((int64_t)it.f * Ho + 3 * it.sy) * (int64_t)Wo + 3 * (it.c4 >> 1);
    if (it.half == 0) {
#pragma unroll
        for (int i = 0; i < 3; ++i) yp[i] = y[0][i];
#pragma unroll
        for (int i = 0; i < 3; ++i) yp[Wo + i] = y[1][i];
    } else {
#pragma unroll
        for (int i = 0; i < 3; ++i) yp[2 * Wo + i] = y[2][i];
    }
}

__global__ void __launch_bounds__(kThr) downscale_fwd_kernel(const DownscaleDev p) {
    const int lane = threadIdx.x & 31;
    Taps tp;
    load_taps(p.taps, threadIdx.x & 1, tp);
    const uint32_t Q = (uint32_t)p.W >> 2, HB = (uint32_t)p.H >> 3;
    const uint32_t items = (uint32_t)p.frames * HB * Q;
    const uint32_t stride = gridDim.x * blockDim.x;
    for (uint32_t base = blockIdx.x * blockDim.x + (threadIdx.x & ~31u); base < items; base += stride) {
        const Item it = decode(base + lane, items, Q, HB);
        const float* xp = p.x + ((int64_t)it.f * p.H + 8 * it.sy) * (int64_t)p.W + 4 * it.c4;
        float4 v[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) v[k] = it.valid ? ld_stream4(xp + (int64_t)k * p.W) : make_float4(0.f, 0.f, 0.f, 0.f);
        float y[3][3];
#pragma unroll
        for (int j = 0; j < 3; ++j)
#pragma unroll
            for (int i = 0; i < 3; ++i) y[j][i] = 0.f;
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            float mh[3];
            horiz(tp, v[k], mh);
#pragma unroll
            for (int j = 0; j < 3; ++j)
#pragma unroll
                for (int i = 0; i < 3; ++i) y[j][i] = fmaf(tp.hv[j][k], mh[i], y[j][i]);
        }
        store_block(p, it, y);
    }
}

template <bool kFwd>
__global__ void __launch_bounds__(kThr) downscale_bwd_kernel(const DownscaleDev p) {
    const int lane = threadIdx.x & 31;
    const int half = threadIdx.x & 1;
    Taps tp;
    load_taps(p.taps, half, tp);
    float dhh[3][4], dhv[3][8];
#pragma unroll
    for (int j = 0; j < 3; ++j) {
#pragma unroll
        for (int t = 0; t < 4; ++t) dhh[j][t] = 0.f;
#pragma unroll
        for (int k = 0; k < 8; ++k) dhv[j][k] = 0.f;
    }
    const uint32_t Q = (uint32_t)p.W >> 2, HB = (uint32_t)p.H >> 3;
    const uint32_t items = (uint32_t)p.frames * HB * Q;
    const int Wo = (p.W >> 3) * 3, Ho = (p.H >> 3) * 3;
    const uint32_t stride = gridDim.x * blockDim.x;
    for (uint32_t base = blockIdx.x * blockDim.x + (threadIdx.x & ~31u); base < items; base += stride) {
        const Item it = decode(base + lane, items, Q, HB);
        const int64_t xoff = ((int64_t)it.f * p.H + 8 * it.sy) * (int64_t)p.W + 4 * it.c4;
        float4 v[8];
#pragma unroll
        for (int k = 0; k < 8; ++k)
            v[k] = it.valid ? ld_stream4(p.x + xoff + (int64_t)k * p.W) : make_float4(0.f, 0.f, 0.f, 0.f);
        float g[3][3];
        const float* gp = p.gy + ((int64_t)it.f * Ho + 3 * it.sy) * (int64_t)Wo + 3 * (it.c4 >> 1);
#pragma unroll
        for (int j = 0; j < 3; ++j)
#pragma unroll
            for (int i = 0; i < 3; ++i) g[j][i] = it.valid ? __ldg(gp + (int64_t)j * Wo + i) : 0.f;
        float y[3][3];
#pragma unroll
        for (int j = 0; j < 3; ++j)
#pragma unroll
            for (int i = 0; i < 3; ++i) y[j][i] = 0.f;
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            float mh[3];
            horiz(tp, v[k], mh);
            float dmid[3];
#pragma unroll
            for (int i = 0; i < 3; ++i) {
                dmid[i] = fmaf(tp.hv[2][k], g[2][i], fmaf(tp.hv[1][k], g[1][i], tp.hv[0][k] * g[0][i]));
#pragma unroll
                for (int j = 0; j < 3; ++j) {
                    dhv[j][k] = fmaf(g[j][i], mh[i], dhv[j][k]);
                    if (kFwd) y[j][i] = fmaf(tp.hv[j][k], mh[i], y[j][i]);
                }
            }
            float dx[4];
            const float vv[4] = {v[k].x, v[k].y, v[k].z, v[k].w};
#pragma unroll
            for (int t = 0; t < 4; ++t) {
                dx[t] = fmaf(tp.hh[2][t], dmid[2], fmaf(tp.hh[1][t], dmid[1], tp.hh[0][t] * dmid[0]));
#pragma unroll
                for (int i = 0; i < 3; ++i) dhh[i][t] = fmaf(dmid[i], vv[t], dhh[i][t]);
            }
            if (it.valid && p.gx) st_stream4(p.gx + xoff + (int64_t)k * p.W, make_float4(dx[0], dx[1], dx[2], dx[3]));
        }
        if (kFwd) store_block(p, it, y);
    }
    // Warp reduction: dHh over lanes of equal parity (same 4 columns), dHv over all lanes.
#pragma unroll
    for (int off = 2; off < 32; off <<= 1)
#pragma unroll
        for (int j = 0; j < 3; ++j)
#pragma unroll
            for (int t = 0; t < 4; ++t) dhh[j][t] += __shfl_xor_sync(kFull, dhh[j][t], off);
#pragma unroll
    for (int off = 1; off < 32; off <<= 1)
#pragma unroll
        for (int j = 0; j < 3; ++j)
#pragma unroll
            for (int k = 0; k < 8; ++k) dhv[j][k] += __shfl_xor_sync(kFull, dhv[j][k], off);
    __shared__ float s_red[kThr / 32][kTapGrads];
    const int w = threadIdx.x >> 5;
    if (lane < 2) {
#pragma unroll
        for (int j = 0; j < 3; ++j)
#pragma unroll
            for (int t = 0; t < 4; ++t) s_red[w][j * 8 + 4 * lane + t] = dhh[j][t];
    }
    if (lane == 0) {
#pragma unroll
        for (int j = 0; j < 3; ++j)
#pragma unroll
            for (int k = 0; k < 8; ++k) s_red[w][24 + j * 8 + k] = dhv[j][k];
    }
    __syncthreads();
    if (threadIdx.x < kTapGrads) {
        float s = 0.f;
        for (int ww = 0; ww < kThr / 32; ++ww) s += s_red[ww][threadIdx.x];
        p.partials[(int64_t)blockIdx.x * kTapGrads + threadIdx.x] = s;
    }
}

// Sums the per-CTA partials in a fixed order: 16 lanes per tap gradient, each
// summing a strided subset, then a fixed shuffle tree over the 16 lanes.
__global__ void __launch_bounds__(kTapGrads * 16) tapgrad_reduce_kernel(const float* __restrict__ partials,
                                                                         int nparts, float* __restrict__ out) {
    const int o = threadIdx.x >> 4, l = threadIdx.x & 15;
    float s = 0.f;
    for (int b = l; b < nparts; b += 16) s += partials[(int64_t)b * kTapGrads + o];
#pragma unroll
    for (int off = 8; off > 0; off >>= 1) s += __shfl_xor_sync(kFull, s, off, 16);
    if (l == 0) out[o] = s;
}

// ---------------------------------------------------------------------------
// Bulk-copy pipelined variants.  A unit of work is one 8-row stripe of one
// frame restricted to a chunk of Wc columns (Wc a multiple of 32, at most
// 1024).  A producer warp streams each unit's 8 row segments (and, for the
// backward, the 3 matching rows of dL/dY) into a kStages-deep shared-memory
// ring with cp.async.bulk, completing on the stage's "full" mbarrier; eight
// consumer warps compute from shared memory and release the stage on its
// "empty" mbarrier.  Bytes in flight no longer live in registers, so a CTA
// keeps up to kStages units (~100 KB) of loads outstanding.
// ---------------------------------------------------------------------------

// Per mode: consumer warps, ring depth, CTAs per SM.  The forward needs ~95
// registers, so two CTAs of 8 consumer warps share an SM (6 stages in
// flight per SM); the backward needs ~170, so one CTA of 11 consumer warps
// owns the SM with a deeper ring.
template <int kMode> struct BulkCfg {
    static constexpr int kCWarps = kMode == 2 ? 11 : 8;      // the backward (mode 1): one warp per stripe row
    static constexpr int kStages = kMode == 2 ? 5 : 3;
    static constexpr int kThreads = (kCWarps + 1) * 32;
    static constexpr int kMinCtas = kMode == 2 ? 1 : 2;
};

__host__ __device__ __forceinline__ int stage_floats(int Wc, bool with_g) { return 8 * Wc + (with_g ? 9 * Wc / 8 : 0); }

__device__ __forceinline__ void flag_error(const DownscaleDev& p, unsigned bit) {
    if (p.err) atomicOr(p.err, bit);
}

// After each CTA's 48 partials are stored: the last CTA to finish (a ticket
// counter) adds all CTAs' partials in block order into grad_taps and resets
// the ticket, so the tap gradients are deterministic and need no second
// launch.  Called by the `nthreads` consumer threads of every CTA.
__device__ __forceinline__ void finish_tap_gradients(const DownscaleDev& p, int nthreads) {
    if (!p.grad_taps) return;
    __shared__ int s_last;
    __threadfence();                                            // partials visible device-wide
    asm volatile("bar.sync 2, %0;" ::"r"(nthreads) : "memory");
    if (threadIdx.x == 0) s_last = atomicAdd(p.ticket, 1u) == gridDim.x - 1 ? 1 : 0;
    asm volatile("bar.sync 2, %0;" ::"r"(nthreads) : "memory");
    if (!s_last) return;
    __threadfence();
    // G groups of 48 threads: group g sums the partials of CTAs g, g + G, ...
    // (four interleaved accumulators), then thread o adds the G group sums in
    // order.  Fixed thread count and grid give a fixed summation order.
    __shared__ float s_grp[kTapGroups][kTapGrads];
    const int G = nthreads / kTapGrads < kTapGroups ? nthreads / kTapGrads : kTapGroups;
    const int grp = threadIdx.x / kTapGrads, o = threadIdx.x - grp * kTapGrads;
    if (grp < G) {
        float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f;
        const float* q = p.partials + o;
        const int n = (int)gridDim.x;
        int b = grp;
        for (; b + 3 * G < n; b += 4 * G) {
            a0 += __ldcg(q + (int64_t)b * kTapGrads);
            a1 += __ldcg(q + (int64_t)(b + G) * kTapGrads);
            a2 += __ldcg(q + (int64_t)(b + 2 * G) * kTapGrads);
            a3 += __ldcg(q + (int64_t)(b + 3 * G) * kTapGrads);
        }
        for (; b < n; b += G) a0 += __ldcg(q + (int64_t)b * kTapGrads);
        s_grp[grp][o] = (a0 + a1) + (a2 + a3);
    }
    asm volatile("bar.sync 2, %0;" ::"r"(nthreads) : "memory");
    if (threadIdx.x < kTapGrads) {
        float acc = 0.f;
        for (int g = 0; g < G; ++g) acc += s_grp[g][threadIdx.x];
        p.grad_taps[threadIdx.x] = acc;
    }
    if (threadIdx.x == 0) *p.ticket = 0u;
}

// Backward consumers, one warp per stripe row k (8 warps) and one lane per
// 8-column block: the thread holds the 24 horizontal taps but only column k
// of the vertical taps, and accumulates dHh (3 x 8) and column k of dHv.
//   mid[j]  = sum_c Hh[j,c] x[k,c]           dmid[j] = sum_i Hv[i,k] g[i,j]
//   dx[c]   = sum_j Hh[j,c] dmid[j]           dHh[j,c] += dmid[j] x[k,c]
//   dHv[i,k] += sum_j g[i,j] mid[j]
__device__ __forceinline__ void backward_rows(const DownscaleDev& p, const float* sm, int sf, uint32_t full0,
                                              uint32_t empty0, int Wc, int nch, uint32_t units, uint32_t HB,
                                              int Wo, int Ho, int gw) {
    constexpr int kStages = BulkCfg<1>::kStages;
    static_assert(BulkCfg<1>::kCWarps == 8, "one consumer warp per stripe row");
    const int k = threadIdx.x >> 5, lane = threadIdx.x & 31;
    float hh[3][8], hvk[3];
#pragma unroll
    for (int j = 0; j < 3; ++j) {
#pragma unroll
        for (int c = 0; c < 8; ++c) hh[j][c] = __ldg(p.taps + j * 8 + c);
        hvk[j] = __ldg(p.taps + 24 + j * 8 + k);
    }
    float dhh[3][8], dhv[3];
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        dhv[j] = 0.f;
#pragma unroll
        for (int c = 0; c < 8; ++c) dhh[j][c] = 0.f;
    }
    (void)Ho;
    uint32_t i = 0;
    for (uint32_t u = blockIdx.x; u < units; u += gridDim.x, ++i) {
        const int st = (int)(i % kStages);
        if (!ptx::mbar_wait(full0 + 8 * st, (i / kStages) & 1u)) {
            flag_error(p, 2u);
            break;
        }
        // units in reverse: a backward that follows the forward finds the last
        // frames that pass read still in L2
        const uint32_t v = units - 1u - u;
        const uint32_t c = v % (uint32_t)nch, stripe = v / (uint32_t)nch;
        const uint32_t f = stripe / HB, sy = stripe - f * HB;
        const int c0 = (int)c * Wc;
        const int nb = min(Wc, p.W - c0) >> 3;
        const float* src = sm + st * sf;
        float* gxrow = p.gx ? p.gx + ((int64_t)f * p.H + 8 * sy + k) * (int64_t)p.W + c0 : nullptr;
        for (int b0 = 0; b0 < nb; b0 += 32) {
            const int b = b0 + lane;
            const bool valid = b < nb;
            const int bb = valid ? b : 0;
            const float4 xa = *reinterpret_cast<const float4*>(src + k * Wc + 8 * bb);
            const float4 xb = *reinterpret_cast<const float4*>(src + k * Wc + 8 * bb + 4);
            float x[8] = {xa.x, xa.y, xa.z, xa.w, xb.x, xb.y, xb.z, xb.w};
            float g[3][3];
            const float* gs = src + 8 * Wc + 3 * bb;
#pragma unroll
            for (int ii = 0; ii < 3; ++ii)
#pragma unroll
                for (int j = 0; j < 3; ++j) g[ii][j] = gs[ii * gw + j];
            if (!valid) {
#pragma unroll
                for (int cc = 0; cc < 8; ++cc) x[cc] = 0.f;
#pragma unroll
                for (int ii = 0; ii < 3; ++ii)
#pragma unroll
                    for (int j = 0; j < 3; ++j) g[ii][j] = 0.f;
            }
            float mid[3], dmid[3];
#pragma unroll
            for (int j = 0; j < 3; ++j) {
                float a = hh[j][0] * x[0];
#pragma unroll
                for (int cc = 1; cc < 8; ++cc) a = fmaf(hh[j][cc], x[cc], a);
                mid[j] = a;
                dmid[j] = fmaf(hvk[2], g[2][j], fmaf(hvk[1], g[1][j], hvk[0] * g[0][j]));
            }
            float dx[8];
#pragma unroll
            for (int cc = 0; cc < 8; ++cc) {
                dx[cc] = fmaf(hh[2][cc], dmid[2], fmaf(hh[1][cc], dmid[1], hh[0][cc] * dmid[0]));
#pragma unroll
                for (int j = 0; j < 3; ++j) dhh[j][cc] = fmaf(dmid[j], x[cc], dhh[j][cc]);
            }
#pragma unroll
            for (int ii = 0; ii < 3; ++ii)
                dhv[ii] = fmaf(g[ii][2], mid[2], fmaf(g[ii][1], mid[1], fmaf(g[ii][0], mid[0], dhv[ii])));
            if (valid && gxrow) {
                st_stream4(gxrow + 8 * b, make_float4(dx[0], dx[1], dx[2], dx[3]));
                st_stream4(gxrow + 8 * b + 4, make_float4(dx[4], dx[5], dx[6], dx[7]));
            }
        }
        __syncwarp();
        if (lane == 0) ptx::mbar_arrive(empty0 + 8 * st);
    }
    // Tap gradients: warp shuffles, then the 8 row warps in fixed order.
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            dhv[j] += __shfl_xor_sync(kFull, dhv[j], off);
#pragma unroll
            for (int cc = 0; cc < 8; ++cc) dhh[j][cc] += __shfl_xor_sync(kFull, dhh[j][cc], off);
        }
    }
    __shared__ float s_red[8][kTapGrads];
    if (lane == 0) {
#pragma unroll
        for (int j = 0; j < 3; ++j) {
#pragma unroll
            for (int cc = 0; cc < 8; ++cc) {
                s_red[k][j * 8 + cc] = dhh[j][cc];
                s_red[k][24 + j * 8 + cc] = cc == k ? dhv[j] : 0.f;
            }
        }
    }
    asm volatile("bar.sync 1, %0;" ::"r"(8 * 32) : "memory");   // the 8 consumer warps
    if (threadIdx.x < kTapGrads) {
        float acc = 0.f;
        for (int w = 0; w < 8; ++w) acc += s_red[w][threadIdx.x];
        p.partials[(int64_t)blockIdx.x * kTapGrads + threadIdx.x] = acc;
    }
    finish_tap_gradients(p, 8 * 32);
}

// kMode: 0 forward, 1 backward, 2 forward + backward.
template <int kMode>
__global__ void __launch_bounds__(BulkCfg<kMode>::kThreads, BulkCfg<kMode>::kMinCtas)
    downscale_bulk_kernel(const DownscaleDev p, int Wc, int nch) {
    constexpr bool kBwd = kMode != 0;
    constexpr bool kFwd = kMode != 1;
    constexpr int kCWarps = BulkCfg<kMode>::kCWarps;
    constexpr int kStages = BulkCfg<kMode>::kStages;
    extern __shared__ __align__(128) float sm[];
    const int sf = stage_floats(Wc, kBwd);
    uint64_t* bars = reinterpret_cast<uint64_t*>(sm + kStages * sf);
    const uint32_t full0 = ptx::smem_addr(bars), empty0 = ptx::smem_addr(bars + kStages);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t HB = (uint32_t)p.H >> 3;
    const uint32_t units = (uint32_t)p.frames * HB * (uint32_t)nch;
    const int Wo = (p.W >> 3) * 3, Ho = (int)HB * 3;
    const int gw = 3 * Wc / 8;   // floats per staged dL/dY row
    if (threadIdx.x == 0) {
        for (int st = 0; st < kStages; ++st) {
            ptx::mbar_init(full0 + 8 * st, 1);
            ptx::mbar_init(empty0 + 8 * st, kCWarps);
        }
        ptx::fence_barrier_init();
    }
    __syncthreads();

    if (warp == kCWarps) {
        // ---------------- producer
        if (lane == 0) {
            int last[kStages];
#pragma unroll
            for (int st = 0; st < kStages; ++st) last[st] = -1;
            uint32_t i = 0;
            for (uint32_t u = blockIdx.x; u < units; u += gridDim.x, ++i) {
                const int st = (int)(i % kStages);
                if (i >= (uint32_t)kStages && !ptx::mbar_wait(empty0 + 8 * st, ((i / kStages) & 1u) ^ 1u)) {
                    flag_error(p, 1u);
                    break;
                }
                const uint32_t v = kMode == 1 ? units - 1u - u : u;   // the backward walks units in reverse
                const uint32_t c = v % (uint32_t)nch, stripe = v / (uint32_t)nch;
                const uint32_t f = stripe / HB, sy = stripe - f * HB;
                const int c0 = (int)c * Wc;
                const int wc = min(Wc, p.W - c0);
                const uint32_t xrow = (uint32_t)wc * 4u, grow = (uint32_t)(3 * wc / 8) * 4u;
                const uint32_t fb = full0 + 8 * st;
                ptx::mbar_expect_tx(fb, 8u * xrow + (kBwd ? 3u * grow : 0u));
                float* dst = sm + st * sf;
                const float* xs = p.x + ((int64_t)f * p.H + 8 * sy) * (int64_t)p.W + c0;
#pragma unroll
                for (int r = 0; r < 8; ++r) ptx::bulk_g2s(ptx::smem_addr(dst + r * Wc), xs + (int64_t)r * p.W, xrow, fb);
                if (kBwd) {
                    const float* gs = p.gy + ((int64_t)f * Ho + 3 * sy) * (int64_t)Wo + 3 * c0 / 8;
#pragma unroll
                    for (int j = 0; j < 3; ++j)
                        ptx::bulk_g2s(ptx::smem_addr(dst + 8 * Wc + j * gw), gs + (int64_t)j * Wo, grow, fb);
                }
                last[st] = (int)i;
            }
            // every issued copy lands before the CTA (and its shared memory) goes away
#pragma unroll
            for (int st = 0; st < kStages; ++st)
                if (last[st] >= 0) ptx::mbar_wait(full0 + 8 * st, ((uint32_t)last[st] / kStages) & 1u);
        }
        return;
    }

    // ---------------- consumers
    if (kMode == 1) {
        backward_rows(p, sm, sf, full0, empty0, Wc, nch, units, HB, Wo, Ho, gw);
        return;
    }
    const int half = lane & 1;
    Taps tp;
    load_taps(p.taps, half, tp);
    float dhh[3][4], dhv[3][8];
#pragma unroll
    for (int j = 0; j < 3; ++j) {
#pragma unroll
        for (int t = 0; t < 4; ++t) dhh[j][t] = 0.f;
#pragma unroll
        for (int k = 0; k < 8; ++k) dhv[j][k] = 0.f;
    }
    uint32_t i = 0;
    for (uint32_t u = blockIdx.x; u < units; u += gridDim.x, ++i) {
        const int st = (int)(i % kStages);
        if (!ptx::mbar_wait(full0 + 8 * st, (i / kStages) & 1u)) {
            flag_error(p, 2u);
            break;
        }
        const uint32_t c = u % (uint32_t)nch, stripe = u / (uint32_t)nch;
        const uint32_t f = stripe / HB, sy = stripe - f * HB;
        const int c0 = (int)c * Wc;
        const int nq = min(Wc, p.W - c0) >> 2;
        const float* src = sm + st * sf;
        for (int qb = warp * 32; qb < nq; qb += kCWarps * 32) {
            const int q = qb + lane;
            Item it;
            it.valid = q < nq;
            it.half = half;
            it.f = f;
            it.sy = sy;
            it.c4 = (uint32_t)(c0 >> 2) + (uint32_t)q;
            // rows are read from shared memory as they are used (lanes past the
            // chunk's end read column 0; their results are discarded)
            const float* row0 = src + 4 * (it.valid ? q : 0);
            float y[3][3];
#pragma unroll
            for (int j = 0; j < 3; ++j)
#pragma unroll
                for (int ii = 0; ii < 3; ++ii) y[j][ii] = 0.f;
            if (!kBwd) {
#pragma unroll
                for (int k = 0; k < 8; ++k) {
                    const float4 vk = *reinterpret_cast<const float4*>(row0 + k * Wc);
                    float mh[3];
                    horiz(tp, vk, mh);
#pragma unroll
                    for (int j = 0; j < 3; ++j)
#pragma unroll
                        for (int ii = 0; ii < 3; ++ii) y[j][ii] = fmaf(tp.hv[j][k], mh[ii], y[j][ii]);
                }
            } else {
                float g[3][3];
                const float* gsrc = src + 8 * Wc + 3 * ((it.valid ? q : 0) >> 1);
#pragma unroll
                for (int j = 0; j < 3; ++j)
#pragma unroll
                    for (int ii = 0; ii < 3; ++ii) g[j][ii] = it.valid ? gsrc[j * gw + ii] : 0.f;
                const int64_t xoff = ((int64_t)f * p.H + 8 * sy) * (int64_t)p.W + c0 + 4 * q;
#pragma unroll
                for (int k = 0; k < 8; ++k) {
                    const float4 vk = *reinterpret_cast<const float4*>(row0 + k * Wc);
                    float mh[3];
                    horiz(tp, vk, mh);
                    float dmid[3];
#pragma unroll
                    for (int ii = 0; ii < 3; ++ii) {
                        dmid[ii] = fmaf(tp.hv[2][k], g[2][ii], fmaf(tp.hv[1][k], g[1][ii], tp.hv[0][k] * g[0][ii]));
#pragma unroll
                        for (int j = 0; j < 3; ++j) {
                            dhv[j][k] = fmaf(g[j][ii], mh[ii], dhv[j][k]);
                            if (kFwd) y[j][ii] = fmaf(tp.hv[j][k], mh[ii], y[j][ii]);
                        }
                    }
                    float dx[4];
                    const float vv[4] = {vk.x, vk.y, vk.z, vk.w};
#pragma unroll
                    for (int t = 0; t < 4; ++t) {
                        dx[t] = fmaf(tp.hh[2][t], dmid[2], fmaf(tp.hh[1][t], dmid[1], tp.hh[0][t] * dmid[0]));
#pragma unroll
                        for (int ii = 0; ii < 3; ++ii) dhh[ii][t] = fmaf(dmid[ii], vv[t], dhh[ii][t]);
                    }
                    if (it.valid && p.gx) st_stream4(p.gx + xoff + (int64_t)k * p.W, make_float4(dx[0], dx[1], dx[2], dx[3]));
                }
            }
            if (kFwd) store_block(p, it, y);
        }
        __syncwarp();
        if (lane == 0) ptx::mbar_arrive(empty0 + 8 * st);
    }
    if (!kBwd) return;
    // Tap gradients: warp shuffles, then the 8 consumer warps in fixed order.
#pragma unroll
    for (int off = 2; off < 32; off <<= 1)
#pragma unroll
        for (int j = 0; j < 3; ++j)
#pragma unroll
            for (int t = 0; t < 4; ++t) dhh[j][t] += __shfl_xor_sync(kFull, dhh[j][t], off);
#pragma unroll
    for (int off = 1; off < 32; off <<= 1)
#pragma unroll
        for (int j = 0; j < 3; ++j)
#pragma unroll
            for (int k = 0; k < 8; ++k) dhv[j][k] += __shfl_xor_sync(kFull, dhv[j][k], off);
    __shared__ float s_red[kCWarps][kTapGrads];
    if (lane < 2) {
#pragma unroll
        for (int j = 0; j < 3; ++j)
#pragma unroll
            for (int t = 0; t < 4; ++t) s_red[warp][j * 8 + 4 * lane + t] = dhh[j][t];
    }
    if (lane == 0) {
#pragma unroll
        for (int j = 0; j < 3; ++j)
#pragma unroll
            for (int k = 0; k < 8; ++k) s_red[warp][24 + j * 8 + k] = dhv[j][k];
    }
    asm volatile("bar.sync 1, %0;" ::"r"(kCWarps * 32) : "memory");   // consumer warps only
    if (threadIdx.x < kTapGrads) {
        float acc = 0.f;
        for (int w = 0; w < kCWarps; ++w) acc += s_red[w][threadIdx.x];
        p.partials[(int64_t)blockIdx.x * kTapGrads + threadIdx.x] = acc;
    }
    finish_tap_gradients(p, kCWarps * 32);
}

// Column chunk of the bulk variants: the fewest chunks of at most 1024
// columns, each a multiple of 32 columns.
int bulk_chunk(int W) {
    const int n = (W + 1023) / 1024;
    int wc = (W + n - 1) / n;
    return (wc + 31) / 32 * 32;
}

template <int kMode>
size_t bulk_smem(int Wc) {
    constexpr int kStages = BulkCfg<kMode>::kStages;
    return (size_t)kStages * stage_floats(Wc, kMode != 0) * 4 + 2 * kStages * 8;
}

template <int kMode>
int bulk_ctas_per_sm(int Wc) {
    const size_t smem = bulk_smem<kMode>(Wc);
    static int last_wc = -1, last = 1;
    if (Wc != last_wc) {
        cudaFuncSetAttribute(downscale_bulk_kernel<kMode>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        int n = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, downscale_bulk_kernel<kMode>, BulkCfg<kMode>::kThreads, smem);
        last = n > 0 ? n : 1;
        last_wc = Wc;
    }
    return last;
}

template <int kMode>
cudaError_t launch_bulk(const DownscaleDev& p, int grid, cudaStream_t s) {
    const int Wc = bulk_chunk(p.W);
    const int nch = (p.W + Wc - 1) / Wc;
    const size_t smem = bulk_smem<kMode>(Wc);
    bulk_ctas_per_sm<kMode>(Wc);   // sets the dynamic shared-memory limit
    downscale_bulk_kernel<kMode><<<grid, BulkCfg<kMode>::kThreads, smem, s>>>(p, Wc, nch);
    return cudaGetLastError();
}

// The backward stages dL/dY rows with bulk copies: their byte offsets and
// sizes (1.5 * columns) are multiples of 16 only when W is a multiple of 32.
bool bulk_backward_ok(int W) { return W % 32 == 0; }

// ---------------------------------------------------------------------------
// Batches of 8 -> 3 chains (Sec. 5 chains inside one batch): the forward
// bulk-copy ring over the units of every member in one launch.  Member c's
// units (frame, stripe, chunk of Wc_c columns) follow member c - 1's; staged
// rows keep the stride Ws of the widest chunk; each consumer warp reloads
// the taps when its unit's member changes.  Inputs are 16-byte aligned (the
// host routes other members elsewhere).
// ---------------------------------------------------------------------------
__device__ __forceinline__ int ds_find(const int* ustart, int n, int u, int c) {
    while (c + 1 < n && __ldg(ustart + c + 1) <= u) ++c;
    return c;
}

__global__ void __launch_bounds__(BulkCfg<0>::kThreads, BulkCfg<0>::kMinCtas)
    downscale_batch_kernel(const DsMember* mem, const int* ustart, int nmem, int units, int Ws, unsigned* err) {
    constexpr int kCWarps = BulkCfg<0>::kCWarps;
    constexpr int kStages = BulkCfg<0>::kStages;
    extern __shared__ __align__(128) float sm[];
    const int sf = 8 * Ws;
    uint64_t* bars = reinterpret_cast<uint64_t*>(sm + kStages * sf);
    const uint32_t full0 = ptx::smem_addr(bars), empty0 = ptx::smem_addr(bars + kStages);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int st = 0; st < kStages; ++st) {
            ptx::mbar_init(full0 + 8 * st, 1);
            ptx::mbar_init(empty0 + 8 * st, kCWarps);
        }
        ptx::fence_barrier_init();
    }
    __syncthreads();

    if (warp == kCWarps) {
        // ---------------- producer
        if (lane == 0) {
            int last[kStages];
#pragma unroll
            for (int st = 0; st < kStages; ++st) last[st] = -1;
            uint32_t i = 0;
            int c = 0;
            for (int u = blockIdx.x; u < units; u += gridDim.x, ++i) {
                const int st = (int)(i % kStages);
                if (i >= (uint32_t)kStages && !ptx::mbar_wait(empty0 + 8 * st, ((i / kStages) & 1u) ^ 1u)) {
                    if (err) atomicOr(err, 1u);
                    break;
                }
                c = ds_find(ustart, nmem, u, c);
                const DsMember m = mem[c];
                const uint32_t v = (uint32_t)(u - __ldg(ustart + c)), HB = (uint32_t)m.H >> 3;
                const uint32_t ch = v % (uint32_t)m.nch, stripe = v / (uint32_t)m.nch;
                const uint32_t f = stripe / HB, sy = stripe - f * HB;
                const int c0 = (int)ch * m.Wc;
                const int wc = min(m.Wc, m.W - c0);
                const uint32_t xrow = (uint32_t)wc * 4u, fb = full0 + 8 * st;
                ptx::mbar_expect_tx(fb, 8u * xrow);
                float* dst = sm + st * sf;
                const float* xs = m.x + ((int64_t)f * m.H + 8 * sy) * (int64_t)m.W + c0;
#pragma unroll
                for (int r = 0; r < 8; ++r) ptx::bulk_g2s(ptx::smem_addr(dst + r * Ws), xs + (int64_t)r * m.W, xrow, fb);
                last[st] = (int)i;
            }
            // every issued copy lands before the CTA (and its shared memory) goes away
#pragma unroll
            for (int st = 0; st < kStages; ++st)
                if (last[st] >= 0) ptx::mbar_wait(full0 + 8 * st, ((uint32_t)last[st] / kStages) & 1u);
        }
        return;
    }

    // ---------------- consumers
    const int half = lane & 1;
    Taps tp;
    uint32_t i = 0;
    int c = 0, cur = -1;
    for (int u = blockIdx.x; u < units; u += gridDim.x, ++i) {
        const int st = (int)(i % kStages);
        if (!ptx::mbar_wait(full0 + 8 * st, (i / kStages) & 1u)) {
            if (err && lane == 0) atomicOr(err, 2u);
            break;
        }
        c = ds_find(ustart, nmem, u, c);
        const DsMember m = mem[c];
        if (c != cur) {
            load_taps(m.taps, half, tp);
            cur = c;
        }
        DownscaleDev p{};
        p.y = m.y;
        p.H = m.H;
        p.W = m.W;
        const uint32_t v = (uint32_t)(u - __ldg(ustart + c)), HB = (uint32_t)m.H >> 3;
        const uint32_t ch = v % (uint32_t)m.nch, stripe = v / (uint32_t)m.nch;
        const uint32_t f = stripe / HB, sy = stripe - f * HB;
        const int c0 = (int)ch * m.Wc;
        const int nq = min(m.Wc, m.W - c0) >> 2;
        const float* src = sm + st * sf;
        for (int qb = warp * 32; qb < nq; qb += kCWarps * 32) {
            const int q = qb + lane;
            Item it;
            it.valid = q < nq;
            it.half = half;
            it.f = f;
            it.sy = sy;
            it.c4 = (uint32_t)(c0 >> 2) + (uint32_t)q;
            // lanes past the chunk's end read column 0; their results are discarded
            const float* row0 = src + 4 * (it.valid ? q : 0);
            float y[3][3];
#pragma unroll
            for (int j = 0; j < 3; ++j)
#pragma unroll
                for (int ii = 0; ii < 3; ++ii) y[j][ii] = 0.f;
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                const float4 vk = *reinterpret_cast<const float4*>(row0 + k * Ws);
                float mh[3];
                horiz(tp, vk, mh);
#pragma unroll
                for (int j = 0; j < 3; ++j)
#pragma unroll
                    for (int ii = 0; ii < 3; ++ii) y[j][ii] = fmaf(tp.hv[j][k], mh[ii], y[j][ii]);
            }
            store_block(p, it, y);
        }
        __syncwarp();
        if (lane == 0) ptx::mbar_arrive(empty0 + 8 * st);
    }
}

size_t ds_batch_smem(int Ws) { return (size_t)BulkCfg<0>::kStages * 8 * Ws * 4 + 2 * BulkCfg<0>::kStages * 8; }

bool use_register_variant() {
    static int v = -1;
    if (v < 0) {
        const char* e = std::getenv("AROL_FUSED_VARIANT");
        v = (e && std::strcmp(e, "regs") == 0) ? 1 : 0;
    }
    return v == 1;
}

// ---------------------------------------------------------------------------
// 16-bit frames, bfloat16 or IEEE half (Sec. 5 typeAllocation): the same
// bulk-copy ring, now with one consumer thread per 8x8 block (one 16-byte
// shared load holds 8 pixels of a row, so no lane pairs and no shuffles).
// The arithmetic is f32; an intermediate declared 16-bit is rounded to
// nearest even exactly where the unfused chain would store it; the output is
// stored as f32 or in the frames' 16-bit type.
// ---------------------------------------------------------------------------
constexpr int kB16Stages = 4;
constexpr int kB16CWarps = 4;
constexpr int kB16Threads = (kB16CWarps + 1) * 32;

// Storage policies: the two halves of a 32-bit word widened exactly to f32,
// rounding to nearest even, and a 16-bit store.
struct Bf16Storage {
    __device__ static float lo(uint32_t w) { return __uint_as_float(w << 16); }
    __device__ static float hi(uint32_t w) { return __uint_as_float(w & 0xffff0000u); }
    __device__ static float round(float v) { return __bfloat162float(__float2bfloat16_rn(v)); }
    __device__ static void store(void* y, int64_t i, float v) { static_cast<__nv_bfloat16*>(y)[i] = __float2bfloat16_rn(v); }
};
struct HalfStorage {
    __device__ static float lo(uint32_t w) { return __half2float(__ushort_as_half((unsigned short)(w & 0xffffu))); }
    __device__ static float hi(uint32_t w) { return __half2float(__ushort_as_half((unsigned short)(w >> 16))); }
    __device__ static float round(float v) { return __half2float(__float2half_rn(v)); }
    __device__ static void store(void* y, int64_t i, float v) { static_cast<__half*>(y)[i] = __float2half_rn(v); }
};

template <class St, bool kRoundMid, bool kOut16>
__device__ __forceinline__ void downscale16(const DownscaleDev& p, int Wc, int nch) {
    extern __shared__ __align__(128) unsigned short smb[];
    const int sf = 8 * Wc;                                   // 16-bit elements per stage
    uint64_t* bars = reinterpret_cast<uint64_t*>(smb + kB16Stages * sf);
    const uint32_t full0 = ptx::smem_addr(bars), empty0 = ptx::smem_addr(bars + kB16Stages);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t HB = (uint32_t)p.H >> 3;
    const uint32_t units = (uint32_t)p.frames * HB * (uint32_t)nch;
    const int Wo = (p.W >> 3) * 3, Ho = (int)HB * 3;
    if (threadIdx.x == 0) {
        for (int st = 0; st < kB16Stages; ++st) {
            ptx::mbar_init(full0 + 8 * st, 1);
            ptx::mbar_init(empty0 + 8 * st, kB16CWarps);
        }
        ptx::fence_barrier_init();
    }
    __syncthreads();
    const unsigned short* x = static_cast<const unsigned short*>(static_cast<const void*>(p.x));
    if (warp == kB16CWarps) {
        if (lane == 0) {
            int last[kB16Stages];
#pragma unroll
            for (int st = 0; st < kB16Stages; ++st) last[st] = -1;
            uint32_t i = 0;
            for (uint32_t u = blockIdx.x; u < units; u += gridDim.x, ++i) {
                const int st = (int)(i % kB16Stages);
                if (i >= (uint32_t)kB16Stages && !ptx::mbar_wait(empty0 + 8 * st, ((i / kB16Stages) & 1u) ^ 1u)) {
                    flag_error(p, 1u);
                    break;
                }
                const uint32_t c = u % (uint32_t)nch, stripe = u / (uint32_t)nch;
                const uint32_t f = stripe / HB, sy = stripe - f * HB;
                const int c0 = (int)c * Wc;
                const uint32_t row_bytes = (uint32_t)min(Wc, p.W - c0) * 2u;
                const uint32_t fb = full0 + 8 * st;
                ptx::mbar_expect_tx(fb, 8u * row_bytes);
                const unsigned short* xs = x + ((int64_t)f * p.H + 8 * sy) * (int64_t)p.W + c0;
#pragma unroll
                for (int r = 0; r < 8; ++r)
                    ptx::bulk_g2s(ptx::smem_addr(smb + st * sf + r * Wc), xs + (int64_t)r * p.W, row_bytes, fb);
                last[st] = (int)i;
            }
#pragma unroll
            for (int st = 0; st < kB16Stages; ++st)
                if (last[st] >= 0) ptx::mbar_wait(full0 + 8 * st, ((uint32_t)last[st] / kB16Stages) & 1u);
        }
        return;
    }
    float hh[3][8], hv[3][8];
#pragma unroll
    for (int j = 0; j < 3; ++j)
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            hh[j][k] = __ldg(p.taps + j * 8 + k);
            hv[j][k] = __ldg(p.taps + 24 + j * 8 + k);
        }
    uint32_t i = 0;
    for (uint32_t u = blockIdx.x; u < units; u += gridDim.x, ++i) {
        const int st = (int)(i % kB16Stages);
        if (!ptx::mbar_wait(full0 + 8 * st, (i / kB16Stages) & 1u)) {
            flag_error(p, 2u);
            break;
        }
        const uint32_t c = u % (uint32_t)nch, stripe = u / (uint32_t)nch;
        const uint32_t f = stripe / HB, sy = stripe - f * HB;
        const int c0 = (int)c * Wc;
        const int nb = min(Wc, p.W - c0) >> 3;
        const unsigned short* src = smb + st * sf;
        for (int bb = warp * 32; bb < nb; bb += kB16CWarps * 32) {
            const int b = bb + lane;
            if (b >= nb) continue;
            float y[3][3];
#pragma unroll
            for (int j = 0; j < 3; ++j)
#pragma unroll
                for (int jj = 0; jj < 3; ++jj) y[j][jj] = 0.f;
#pragma unroll
            for (int r = 0; r < 8; ++r) {
                const uint4 q = *reinterpret_cast<const uint4*>(src + r * Wc + 8 * b);
                const float xr[8] = {St::lo(q.x), St::hi(q.x), St::lo(q.y), St::hi(q.y),
                                     St::lo(q.z), St::hi(q.z), St::lo(q.w), St::hi(q.w)};
#pragma unroll
                for (int j = 0; j < 3; ++j) {
                    float mid = hh[j][0] * xr[0];
#pragma unroll
                    for (int k = 1; k < 8; ++k) mid = fmaf(hh[j][k], xr[k], mid);
                    if (kRoundMid) mid = St::round(mid);
#pragma unroll
                    for (int jv = 0; jv < 3; ++jv) y[jv][j] = fmaf(hv[jv][r], mid, y[jv][j]);
                }
            }
            const int64_t ob = ((int64_t)f * Ho + 3 * sy) * (int64_t)Wo + 3 * ((c0 >> 3) + b);
#pragma unroll
            for (int jv = 0; jv < 3; ++jv)
#pragma unroll
                for (int j = 0; j < 3; ++j) {
                    if (kOut16) St::store(p.y, ob + (int64_t)jv * Wo + j, y[jv][j]);
                    else p.y[ob + (int64_t)jv * Wo + j] = y[jv][j];
                }
        }
        __syncwarp();
        if (lane == 0) ptx::mbar_arrive(empty0 + 8 * st);
    }
}

template <bool kRoundMid, bool kOut16>
__global__ void __launch_bounds__(kB16Threads, 3) downscale_bf16_kernel(const DownscaleDev p, int Wc, int nch) {
    downscale16<Bf16Storage, kRoundMid, kOut16>(p, Wc, nch);
}

template <bool kRoundMid, bool kOut16>
__global__ void __launch_bounds__(kB16Threads, 3) downscale_f16_kernel(const DownscaleDev p, int Wc, int nch) {
    downscale16<HalfStorage, kRoundMid, kOut16>(p, Wc, nch);
}

// Column chunk of the 16-bit variants: at most 1024 columns, a multiple of 64.
int chunk16(int W) {
    const int n = (W + 1023) / 1024;
    const int wc = (W + n - 1) / n;
    return (wc + 63) / 64 * 64;
}

template <bool kHalf, bool kRoundMid, bool kOut16>
cudaError_t launch_16bit_variant(const DownscaleDev& p, cudaStream_t s) {
    void (*kern)(const DownscaleDev, int, int) =
        kHalf ? downscale_f16_kernel<kRoundMid, kOut16> : downscale_bf16_kernel<kRoundMid, kOut16>;
    const int Wc = chunk16(p.W);
    const int nch = (p.W + Wc - 1) / Wc;
    const size_t smem = (size_t)kB16Stages * 8 * Wc * 2 + 2 * kB16Stages * 8;
    static int last_wc = -1, per_sm = 1;
    if (Wc != last_wc) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        int n = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kern, kB16Threads, smem);
        per_sm = n > 0 ? n : 1;
        last_wc = Wc;
    }
    const uint32_t units = (uint32_t)p.frames * ((uint32_t)p.H >> 3) * (uint32_t)nch;
    const uint32_t cap = (uint32_t)(device_sm_count() * per_sm);
    kern<<<(int)(units < cap ? units : cap), kB16Threads, smem, s>>>(p, Wc, nch);
    return cudaGetLastError();
}

template <bool kHalf>
cudaError_t launch_16bit(const DownscaleDev& p, cudaStream_t s) {
    if (p.mid16) return p.out16 ? launch_16bit_variant<kHalf, true, true>(p, s) : launch_16bit_variant<kHalf, true, false>(p, s);
    return p.out16 ? launch_16bit_variant<kHalf, false, true>(p, s) : launch_16bit_variant<kHalf, false, false>(p, s);
}

int fwd_grid(uint32_t items) {
    static int per_sm = 0;
    if (!per_sm) {
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, downscale_fwd_kernel, kThr, 0);
        if (per_sm <= 0) per_sm = 1;
    }
    const int64_t want = ((int64_t)items + kThr - 1) / kThr;
    const int64_t cap = (int64_t)device_sm_count() * per_sm;
    return (int)(want < cap ? (want > 0 ? want : 1) : cap);
}

}  // namespace

// Register-direct backward: CTAs per SM (both modes).
int regs_bwd_per_sm() {
    static int per_sm = 0;
    if (!per_sm) {
        int a = 0, b = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, downscale_bwd_kernel<false>, kThr, 0);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, downscale_bwd_kernel<true>, kThr, 0);
        per_sm = a < b ? a : b;
        if (per_sm <= 0) per_sm = 1;
    }
    return per_sm;
}

// Grid (= tap-gradient partial slots) of one backward launch.
int bwd_grid(int sm_count, int W, bool with_fwd) {
    if (bulk_backward_ok(W) && !use_register_variant()) {
        const int Wc = bulk_chunk(W);
        return sm_count * (with_fwd ? bulk_ctas_per_sm<2>(Wc) : bulk_ctas_per_sm<1>(Wc));
    }
    return sm_count * regs_bwd_per_sm();
}

// Partial slots a caller must provide: enough for either backward mode.
int downscale_bwd_partials(int sm_count, int W) {
    const int a = bwd_grid(sm_count, W, false), b = bwd_grid(sm_count, W, true);
    return a > b ? a : b;
}

cudaError_t launch_downscale_fwd(const DownscaleDev& p, cudaStream_t s) {
    const uint32_t items = (uint32_t)p.frames * ((uint32_t)p.H >> 3) * ((uint32_t)p.W >> 2);
    if (items == 0) return cudaSuccess;
    if (p.in16) return p.half16 ? launch_16bit<true>(p, s) : launch_16bit<false>(p, s);
    if (!use_register_variant()) {
        const int Wc = bulk_chunk(p.W);
        const uint32_t units = (uint32_t)p.frames * ((uint32_t)p.H >> 3) * (uint32_t)((p.W + Wc - 1) / Wc);
        const uint32_t cap = (uint32_t)(device_sm_count() * bulk_ctas_per_sm<0>(Wc));
        return launch_bulk<0>(p, (int)(units < cap ? units : cap), s);
    }
    downscale_fwd_kernel<<<fwd_grid(items), kThr, 0, s>>>(p);
    return cudaGetLastError();
}

int downscale_chunk(int W) { return bulk_chunk(W); }

cudaError_t launch_downscale_batch(const DsMember* mem, const int* ustart, int nmem, int units, int Ws, unsigned* err,
                                   cudaStream_t s) {
    if (units <= 0) return cudaSuccess;
    const size_t smem = ds_batch_smem(Ws);
    static size_t attr = 0;
    if (smem > attr) {
        cudaError_t e =
            cudaFuncSetAttribute(downscale_batch_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        attr = smem;
    }
    int occ = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, downscale_batch_kernel, BulkCfg<0>::kThreads, smem);
    const int cap = device_sm_count() * (occ > 0 ? occ : 1);
    downscale_batch_kernel<<<units < cap ? units : cap, BulkCfg<0>::kThreads, smem, s>>>(mem, ustart, nmem, units, Ws,
                                                                                         err);
    return cudaGetLastError();
}

cudaError_t launch_downscale_bwd(const DownscaleDev& p, float* grad_taps, int capacity, bool with_fwd,
                                 cudaStream_t s) {
    cudaError_t e;
    int nparts = bwd_grid(device_sm_count(), p.W, with_fwd);
    if (nparts > capacity) nparts = capacity;   // grid-stride kernels: fewer CTAs still cover the work
    if (bulk_backward_ok(p.W) && !use_register_variant()) {
        // the last CTA reduces the tap gradients itself
        DownscaleDev q = p;
        q.grad_taps = grad_taps;
        return with_fwd ? launch_bulk<2>(q, nparts, s) : launch_bulk<1>(q, nparts, s);
    }
    if (with_fwd) downscale_bwd_kernel<true><<<nparts, kThr, 0, s>>>(p);
    else downscale_bwd_kernel<false><<<nparts, kThr, 0, s>>>(p);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (grad_taps) {
        tapgrad_reduce_kernel<<<1, kTapGrads * 16, 0, s>>>(p.partials, nparts, grad_taps);
        e = cudaGetLastError();
    }
    return e;
}

}  // namespace arol

// ---------------------------------------------------------------------------
// Backward of the fused downscaler without any device allocation.
//
// Some callers cannot call cudaMalloc: code that runs while a CUDA stream is
// being captured into a graph (an allocation there breaks or invalidates the
// capture), real-time or embedded hosts that fix their device-memory budget
// at start-up and forbid allocation afterwards, and programs whose memory is
// owned by an allocator that must not be bypassed.  For them this entry point
// takes every buffer from the caller and keeps its only scratch — one
// 48-float tap-gradient partial per CTA — in the file-scope array below,
// which every GPU that loads the library holds until the process exits.
// ---------------------------------------------------------------------------

#include <mutex>

#include "arol.h"

namespace arol {
namespace {

constexpr int kNoAllocMaxParts = 1024;   // CTA partials the array holds: 1024 x 48 floats = 192 KiB
constexpr int kNoAllocTicket = kNoAllocMaxParts * kTapGrads;   // word: CTAs done (each launch leaves it at 0)
constexpr int kNoAllocErr = kNoAllocTicket + 1;                 // word: bounded waits that gave up (sticky)
// the 48-float partial of each CTA, then the ticket of the last-CTA reduction
// and the error word (both zero at load)
static __device__ __align__(256) float g_noalloc_partials[kNoAllocMaxParts * kTapGrads + 4];

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
float* g_noalloc_ptr[kMaxDevices] = {};

// The device address of the static array on the current device, looked up
// once per device with that device current (host code only knows a host-side
// stand-in for the array; the device address comes from the runtime).
arol_status noalloc_scratch(float** out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return AROL_ERR_CUDA;
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_partials) != cudaSuccess || !p) return AROL_ERR_CUDA;
        g_noalloc_ptr[dev] = static_cast<float*>(p);
    }
    *out = g_noalloc_ptr[dev];
    return AROL_OK;
}

}  // namespace

}  // namespace arol

extern "C" arol_status arol_downscale_backward_noalloc(const float* x, const float* grad_out, const float* taps,
                                                       int64_t frames, int32_t height, int32_t width,
                                                       float* grad_in, float* grad_taps, void* stream) {
    using namespace arol;
    if (!x || !grad_out || !taps) return AROL_ERR_INVALID;
    if (frames < 0 || height < 0 || width < 0 || height % 8 || width % 8) return AROL_ERR_INVALID;
    if ((double)frames * (height / 8) * (width / 4) >= 2147483647.0) return AROL_ERR_UNSUPPORTED;
    if ((reinterpret_cast<uintptr_t>(x) | reinterpret_cast<uintptr_t>(grad_in) | reinterpret_cast<uintptr_t>(grad_out)) & 15u)
        return AROL_ERR_INVALID;
    float* scratch = nullptr;
    const arol_status st = noalloc_scratch(&scratch);
    if (st != AROL_OK) return st;
    if (frames == 0 || height == 0 || width == 0) {
        cudaStream_t s = static_cast<cudaStream_t>(stream);
        if (grad_taps && cudaMemsetAsync(grad_taps, 0, kTapGrads * sizeof(float), s) != cudaSuccess) return AROL_ERR_CUDA;
        return AROL_OK;
    }
    DownscaleDev p{};
    p.x = x;
    p.taps = taps;
    p.gy = grad_out;
    p.gx = grad_in;
    p.err = reinterpret_cast<unsigned*>(scratch + kNoAllocErr);
    p.partials = scratch;   // every CTA overwrites its own 48 slots before the reduction reads them
    p.ticket = reinterpret_cast<unsigned*>(scratch + kNoAllocTicket);
    p.frames = frames;
    p.H = height;
    p.W = width;
    // at most kNoAllocMaxParts CTAs: the kernels stride over the work, so a
    // smaller grid than the device could hold still covers it
    if (launch_downscale_bwd(p, grad_taps, kNoAllocMaxParts, false, static_cast<cudaStream_t>(stream)) != cudaSuccess)
        return AROL_ERR_CUDA;
    return AROL_OK;
}

extern "C" arol_status arol_downscale_backward_noalloc_status(void* stream) {
    using namespace arol;
    float* scratch = nullptr;
    arol_status st = noalloc_scratch(&scratch);
    if (st != AROL_OK) return st;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    unsigned word = 0;
    if (cudaMemcpyAsync(&word, scratch + kNoAllocErr, sizeof word, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return AROL_ERR_CUDA;
    if (!word) return AROL_OK;
    if (cudaMemsetAsync(scratch + kNoAllocErr, 0, sizeof word, s) != cudaSuccess || cudaStreamSynchronize(s) != cudaSuccess)
        return AROL_ERR_CUDA;
    return AROL_ERR_TIMEOUT;
}
