// Backward of one separable FIR pass in a single sweep over its data (Sec. 5
// chains, differentiated): the adjoint dX (the pass's transposed tiler) and
// the tap gradients dH[j, k] = sum_r dY[m r + j] X[(o + S r + k) mod n_in]
// share every read of dY.  Both forms need repetitions that tile the axis
// exactly (S R = n_in): input position (o + S r + d) mod n_in, d < S, is then
// the "home" of repetition r, and the windows that reach it are those of
// repetitions (r - q) mod R with tap index d + S q < T, q < Q = ceil(T / S).
//
//  * Row pass, 16-word regions (steps 2, 4, 8; rows and origin multiples of
//    16; X in f32): rows staged swizzled (region.h), each thread owning the
//    16 home words of 16 / S repetitions with every index a compile-time
//    offset: 16-byte shared loads and stores, taps in registers.
//  * Row pass, staged rows (the other shapes): one block per input row at a
//    time.  The row of dY and the row of X are staged in shared memory (one
//    padding word per 32, so lanes reading at a stride of S words spread over
//    the banks; 4-byte cp.async copies a few rows ahead when X is f32); each
//    thread takes repetitions, writes their S home elements of dX into a
//    staged row and adds its m x T tap products in registers; the staged dX
//    row leaves by 16-byte stores.
//  * Column pass: one thread per (frame, repetition, 4 columns): Q m rows of
//    dY and T rows of X as 16-byte loads (the X window before any dX store),
//    S rows of dX as 16-byte stores.
//
// Tap gradients: every thread keeps its m x T sums in registers; the block
// adds them in a fixed order into its partials (one row of m T floats per
// block), which launch_tap_reduce sums in a fixed order.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include "arol_internal.h"
#include "ptx.h"
#include "region.h"
#include "sepchain.h"

namespace arol {
namespace {

#ifndef AROL_BWD_THREADS
#define AROL_BWD_THREADS 256
#endif
constexpr int kBwThreads = AROL_BWD_THREADS;
constexpr int kBwTaps = 64;            // shared taps area (m T <= 64)

// Shared index of word c of a staged row: one padding word after every 32.
__device__ __forceinline__ int spad(int c) { return c + (c >> 5); }
constexpr int spad_len(int n) { return n + (n >> 5) + 1; }

__device__ __forceinline__ float widen16(uint32_t b, int dt) {
    return dt == 1 ? __uint_as_float(b << 16) : __half2float(__ushort_as_half((unsigned short)b));
}

// Element i of an input in its storage (0 f32, 1 bfloat16, 2 IEEE half), widened.
__device__ __forceinline__ float ld1(const void* x, int64_t i, int dt) {
    if (dt == 0) return __ldg(static_cast<const float*>(x) + i);
    return widen16(__ldg(static_cast<const unsigned short*>(x) + i), dt);
}

// Elements i .. i + 3 (aligned: 16 bytes for f32, 8 for 16-bit), widened.
__device__ __forceinline__ float4 ld4(const void* x, int64_t i, int dt) {
    if (dt == 0) return __ldg(reinterpret_cast<const float4*>(static_cast<const float*>(x) + i));
    const uint2 u = __ldg(reinterpret_cast<const uint2*>(static_cast<const unsigned short*>(x) + i));
    return make_float4(widen16(u.x & 0xffffu, dt), widen16(u.x >> 16, dt), widen16(u.y & 0xffffu, dt),
                       widen16(u.y >> 16, dt));
}

// Stages n elements starting at element i0 of x (storage dt) into dst
// (padded), 4 at a time when aligned.
__device__ __forceinline__ void stage_row(float* dst, const void* x, int64_t i0, int n, int dt) {
    const int esz = dt == 0 ? 4 : 2;
    const uintptr_t a = reinterpret_cast<uintptr_t>(x) + (uintptr_t)i0 * esz;
    int c0 = 0;
    if ((a & (uintptr_t)(4 * esz - 1)) == 0) {
        const int n4 = n >> 2;
#pragma unroll 4
        for (int e = threadIdx.x; e < n4; e += blockDim.x) {
            const float4 v = ld4(x, i0 + 4 * e, dt);
            float* d = dst + spad(4 * e);
            d[0] = v.x;
            d[1] = v.y;
            d[2] = v.z;
            d[3] = v.w;
        }
        c0 = 4 * n4;
    }
    for (int c = c0 + threadIdx.x; c < n; c += blockDim.x) dst[spad(c)] = ld1(x, i0 + c, dt);
}

// Writes the staged row src (padded) to dst[0 .. n), 4 at a time when aligned.
__device__ __forceinline__ void unstage_row(float* dst, const float* src, int n) {
    int c0 = 0;
    if ((reinterpret_cast<uintptr_t>(dst) & 15u) == 0) {
        const int n4 = n >> 2;
#pragma unroll 4
        for (int e = threadIdx.x; e < n4; e += blockDim.x) {
            const float* s = src + spad(4 * e);
            reinterpret_cast<float4*>(dst)[e] = make_float4(s[0], s[1], s[2], s[3]);
        }
        c0 = 4 * n4;
    }
    for (int c = c0 + threadIdx.x; c < n; c += blockDim.x) dst[c] = src[spad(c)];
}

// The block's m x T tap sums into its row of partials, in a fixed order
// (lanes by shuffles, then warps in order).
template <int MM, int TT, int NT = kBwThreads>
__device__ __forceinline__ void block_taps(const float (&acc)[MM][TT], int m, int T, float* partials) {
    static_assert(NT % 32 == 0, "whole warps");
    __shared__ float red[NT / 32][MM * TT];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __syncthreads();
#pragma unroll
    for (int j = 0; j < MM; ++j)
#pragma unroll
        for (int k = 0; k < TT; ++k) {
            float v = acc[j][k];
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
            if (lane == 0) red[warp][j * TT + k] = v;
        }
    __syncthreads();
    for (int pp = threadIdx.x; pp < m * T; pp += blockDim.x) {
        const int j = pp / T, k = pp - j * T;
        float v = 0.f;
        for (int w = 0; w < NT / 32; ++w) v += red[w][j * TT + k];
        partials[(int64_t)blockIdx.x * (m * T) + pp] = v;
    }
}

// Asynchronous staging of one row of f32 words into dst (padded): 4-byte
// copies, completed by the caller's wait on the thread's copy groups.
__device__ __forceinline__ void stage_row_async(float* dst, const float* src, int n) {
#pragma unroll 4
    for (int c = threadIdx.x; c < n; c += blockDim.x) ptx::cp_async4(dst + spad(c), src + c);
}

// Row pass: rows (frame, row) of X (n_in = S R words each) and of dY
// (n_out = m R words).  gx or partials may be null (that output skipped).
// ASYNC (X in f32, or no tap gradients): a ring of kBwStages staged row
// pairs, the copies of the block's next kBwStages - 1 rows in flight while
// this row is computed.  SS > 0: the step is SS (its loops unrolled, the
// taps in registers); SS = 0: the step is p.S.
#ifndef AROL_BWD_STAGES
#define AROL_BWD_STAGES 3
#endif
constexpr int kBwStages = AROL_BWD_STAGES;
static_assert(kBwStages >= 2, "the ring holds this row and the next");
template <int QQ, int MM, int TT, bool ASYNC, int SS>
__global__ void __launch_bounds__(kBwThreads) sep_row_bwd_kernel(const SepPassDev p, int64_t rows,
                                                                 const float* __restrict__ taps,
                                                                 const void* __restrict__ x, int x_dt,
                                                                 const float* __restrict__ gy, float* __restrict__ gx,
                                                                 float* __restrict__ partials) {
    extern __shared__ float bsm[];
    const int m = p.m, T = p.T, S = SS > 0 ? SS : p.S, R = p.R, Win = p.n_in, Wout = p.n_out;
    const int Q = (T + S - 1) / S;
    float* hs = bsm;                               // taps, m x T
    // staged pairs: the row of dY, then the row of X (kBwStages pairs when ASYNC)
    float* const gs0 = hs + kBwTaps;
    const int pair = spad_len(Wout) + spad_len(Win);
    float* const ds = gs0 + (ASYNC ? kBwStages : 1) * pair;   // the row of dX
    const float* xf = static_cast<const float*>(x);
    for (int i = threadIdx.x; i < m * T; i += blockDim.x) hs[i] = __ldg(taps + i);
    float acc[MM][TT];
#pragma unroll
    for (int j = 0; j < MM; ++j)
#pragma unroll
        for (int k = 0; k < TT; ++k) acc[j][k] = 0.f;
    float hr[MM][TT];   // the taps in registers (SS > 0; zero past m and T)
    if constexpr (SS > 0) {
        __syncthreads();
#pragma unroll
        for (int j = 0; j < MM; ++j)
#pragma unroll
            for (int k = 0; k < TT; ++k) hr[j][k] = j < m && k < T ? hs[j * T + k] : 0.f;
    }
    // the block's rows: blockIdx.x + i gridDim.x, i = 0, 1, ...; row i sits
    // in pair i mod kBwStages; one copy group per row (empty past the end)
    const int64_t G = gridDim.x;
    if (ASYNC) {
        for (int i = 0; i < kBwStages - 1; ++i) {
            const int64_t rr = blockIdx.x + i * G;
            if (rr < rows) {
                float* g0 = gs0 + i * pair;
                stage_row_async(g0, gy + rr * Wout, Wout);
                if (partials) stage_row_async(g0 + spad_len(Wout), xf + rr * Win, Win);
            }
            ptx::cp_async_commit();
        }
    }
    int b = 0;
    for (int64_t row = blockIdx.x; row < rows; row += G) {
        if (ASYNC) {
            // pair (b - 1) mod kBwStages was last read before the previous
            // row's second barrier: fill it with the row kBwStages - 1
            // ahead, then wait for this row's group
            const int64_t ahead = row + (kBwStages - 1) * G;
            if (ahead < rows) {
                float* g0 = gs0 + (b == 0 ? kBwStages - 1 : b - 1) * pair;
                stage_row_async(g0, gy + ahead * Wout, Wout);
                if (partials) stage_row_async(g0 + spad_len(Wout), xf + ahead * Win, Win);
            }
            ptx::cp_async_commit();
            ptx::cp_async_wait_group<kBwStages - 1>();
        } else {
            stage_row(gs0, gy, row * Wout, Wout, 0);
            if (partials) stage_row(gs0 + spad_len(Wout), x, row * Win, Win, x_dt);
        }
        __syncthreads();
        const float* gs = gs0 + (ASYNC ? b : 0) * pair;
        const float* xs = gs + spad_len(Wout);
        if (++b == kBwStages) b = 0;
        for (int r = threadIdx.x; r < R; r += blockDim.x) {
            float g[QQ][MM];
#pragma unroll
            for (int q = 0; q < QQ; ++q) {
                int rq = r - q;
                while (rq < 0) rq += R;
#pragma unroll
                for (int j = 0; j < MM; ++j) g[q][j] = q < Q && j < m ? gs[spad(m * rq + j)] : 0.f;
            }
            int pos = p.o + S * r;   // o < n_in and S r < n_in
            if (pos >= Win) pos -= Win;
            if (SS > 0 && gx) {
                // home element pos + d: taps d + SS q < T (zero past T
                // terms skipped, so non-finite gradients stay exact)
                const bool wraps = pos + SS > Win;
#pragma unroll
                for (int d = 0; d < SS; ++d) {
                    float a = 0.f;
#pragma unroll
                    for (int q = 0; q < QQ; ++q) {
                        const int k = d + SS * q;
                        if (k < TT && k < T) {
#pragma unroll
                            for (int j = 0; j < MM; ++j)
                                if (j < m) a = fmaf(hr[j][k < TT ? k : 0], g[q][j], a);
                        }
                    }
                    int pp = pos + d;
                    if (wraps && pp >= Win) pp -= Win;
                    ds[spad(pp)] = a;
                }
            } else if (gx) {
                int pp = pos;
                for (int d = 0; d < S; ++d) {
                    float a = 0.f;
#pragma unroll
                    for (int q = 0; q < QQ; ++q) {
                        const int k = d + S * q;
                        if (q < Q && k < T) {
#pragma unroll
                            for (int j = 0; j < MM; ++j)
                                if (j < m) a = fmaf(hs[j * T + k], g[q][j], a);
                        }
                    }
                    ds[spad(pp)] = a;
                    if (++pp == Win) pp = 0;
                }
            }
            if (partials) {
                float xv[TT];
                if (pos + TT <= Win) {
#pragma unroll
                    for (int k = 0; k < TT; ++k) xv[k] = k < T ? xs[spad(pos + k)] : 0.f;
                } else {
                    int c = pos;
#pragma unroll
                    for (int k = 0; k < TT; ++k) {
                        xv[k] = k < T ? xs[spad(c)] : 0.f;
                        if (++c == Win) c = 0;
                    }
                }
#pragma unroll
                for (int j = 0; j < MM; ++j)
#pragma unroll
                    for (int k = 0; k < TT; ++k) acc[j][k] = fmaf(g[0][j], xv[k], acc[j][k]);
            }
        }
        // the staged rows are consumed and dX is complete
        __syncthreads();
        if (gx) unstage_row(gx + row * Win, ds, Win);
    }
    if (ASYNC) ptx::cp_async_wait_all();
    if (partials) block_taps<MM, TT>(acc, m, T, partials);
}

// Row pass in 16-word regions: step SS in {2, 4, 8}, rows of n_in = 16 k
// words, origin o = 16 k', X in f32, dY rows 16-byte aligned.  Thread t of a
// row takes the home region of words h0 .. h0 + 15, h0 = (o + 16 t) mod n_in:
// repetitions NR t .. NR t + NR - 1 (NR = 16 / SS), their windows (XW words
// from h0) and their dY words (plus those of the QQ - 1 repetitions before,
// whose windows also reach the region).  Every index below a region's start
// is a compile-time constant: the window and the 16 dX words move as 16-byte
// shared loads and stores, the taps sit in registers.
//
// Staged X and dX rows take the swizzled layout of region.h (X with its 16
// halo words for the windows that run past the row's end).  The dY row is
// stored plainly after 16 halo words holding the row's last m (Q - 1) words
// (the windows of repetitions 0 .. Q - 2 that wrap to the row's end).
constexpr int kVecThreads = kRegionThreads;

template <int SS, int MM, int TT>
__global__ void __launch_bounds__(kVecThreads) sep_row_bwd_vec_kernel(const SepPassDev p, int64_t rows,
                                                                      const float* __restrict__ taps,
                                                                      const float* __restrict__ x,
                                                                      const float* __restrict__ gy,
                                                                      float* __restrict__ gx,
                                                                      float* __restrict__ partials) {
    constexpr int NR = 16 / SS;                     // repetitions per region
    constexpr int QQ = (TT + SS - 1) / SS;          // repetitions whose windows reach a word, at most
    constexpr int NG = NR + QQ - 1;                 // repetitions whose dY a region reads
    constexpr int XW = (16 - SS + TT + 3) & ~3;     // window words of a region
    static_assert(XW <= 32 && MM * (QQ - 1) <= 16, "a window within two regions, the dY halo within 16 words");
    extern __shared__ __align__(16) float vsm[];
    const int m = p.m, T = p.T, Win = p.n_in, Wout = p.n_out;
    const int Q = (T + SS - 1) / SS;
    const int nreg = Win >> 4, W4 = Win >> 2, Wo4 = Wout >> 2;
    const int halo = m * (Q - 1);                   // dY words before the row
    float* hs = vsm;                                // taps, m x T
    const int gsz = 16 + Wout, stage = gsz + Win + 16;
    float* const st0 = hs + kBwTaps;                // kBwStages stages: [16 | dY row] [X row | 16]
    float* const ds = st0 + kBwStages * stage;      // the dX row
    for (int i = threadIdx.x; i < m * T; i += blockDim.x) hs[i] = __ldg(taps + i);
    float acc[MM][TT];
#pragma unroll
    for (int j = 0; j < MM; ++j)
#pragma unroll
        for (int k = 0; k < TT; ++k) acc[j][k] = 0.f;
    const int64_t G = gridDim.x;
    auto stage_rows = [&](int64_t rr, float* st) {
        const float* gr = gy + rr * Wout;
        float* gs = st + 16;
        for (int f = threadIdx.x; f < Wo4; f += blockDim.x) ptx::cp_async16(gs + 4 * f, gr + 4 * f);
        for (int e = threadIdx.x; e < halo; e += blockDim.x) ptx::cp_async4(gs - halo + e, gr + Wout - halo + e);
        if (partials) stage_region_row(st + gsz, x + rr * Win, Win);
    };
    for (int i = 0; i < kBwStages - 1; ++i) {
        const int64_t rr = blockIdx.x + i * G;
        if (rr < rows) stage_rows(rr, st0 + i * stage);
        ptx::cp_async_commit();
    }
    __syncthreads();   // the taps
    float hr[MM][TT];  // zero past m and T
#pragma unroll
    for (int j = 0; j < MM; ++j)
#pragma unroll
        for (int k = 0; k < TT; ++k) hr[j][k] = j < m && k < T ? hs[j * T + k] : 0.f;
    int b = 0;
    for (int64_t row = blockIdx.x; row < rows; row += G) {
        const int64_t ahead = row + (kBwStages - 1) * G;
        if (ahead < rows) stage_rows(ahead, st0 + (b == 0 ? kBwStages - 1 : b - 1) * stage);
        ptx::cp_async_commit();
        ptx::cp_async_wait_group<kBwStages - 1>();
        __syncthreads();
        const float* gs = st0 + b * stage + 16;
        const float* xs = st0 + b * stage + gsz;
        if (++b == kBwStages) b = 0;
        for (int t = threadIdx.x; t < nreg; t += blockDim.x) {
            int h0 = p.o + 16 * t;
            if (h0 >= Win) h0 -= Win;
            const int u0 = h0 >> 2;                 // the region's first 16-byte unit
            // dY of repetitions NR t - (QQ - 1) + i (below -(Q - 1): unused, zero)
            float g[NG][MM];
            const float* gb = gs + m * (NR * t - (QQ - 1));
#pragma unroll
            for (int i = 0; i < NG; ++i)
#pragma unroll
                for (int j = 0; j < MM; ++j) g[i][j] = j < m && i >= QQ - Q ? gb[m * i + j] : 0.f;
            if (gx) {
                // home word w = SS i + d gets taps k = d + SS q < T against
                // the dY of repetition i - q
                float o4[16];
#pragma unroll
                for (int i = 0; i < NR; ++i)
#pragma unroll
                    for (int d = 0; d < SS; ++d) {
                        float a = 0.f;
#pragma unroll
                        for (int q = 0; q < QQ; ++q) {
                            const int k = d + SS * q;
                            if (k < TT && k < T) {
#pragma unroll
                                for (int j = 0; j < MM; ++j) a = fmaf(hr[j][k < TT ? k : 0], g[i + QQ - 1 - q][j], a);
                            }
                        }
                        o4[SS * i + d] = a;
                    }
#pragma unroll
                for (int v = 0; v < 4; ++v)
                    *reinterpret_cast<float4*>(ds + 4 * region_unit(u0 + v)) =
                        make_float4(o4[4 * v], o4[4 * v + 1], o4[4 * v + 2], o4[4 * v + 3]);
            }
            if (partials) {
                float xw[XW];
#pragma unroll
                for (int v = 0; v < XW / 4; ++v) {
                    const float4 q4 = *reinterpret_cast<const float4*>(xs + 4 * region_unit(u0 + v));
                    xw[4 * v] = q4.x;
                    xw[4 * v + 1] = q4.y;
                    xw[4 * v + 2] = q4.z;
                    xw[4 * v + 3] = q4.w;
                }
#pragma unroll
                for (int i = 0; i < NR; ++i)
#pragma unroll
                    for (int j = 0; j < MM; ++j)
#pragma unroll
                        for (int k = 0; k < TT; ++k) acc[j][k] = fmaf(g[i + QQ - 1][j], xw[SS * i + k], acc[j][k]);
            }
        }
        __syncthreads();
        if (gx) {
            float4* dst = reinterpret_cast<float4*>(gx + row * Win);
            for (int f = threadIdx.x; f < W4; f += blockDim.x) dst[f] = *reinterpret_cast<const float4*>(ds + 4 * region_unit(f));
        }
    }
    ptx::cp_async_wait_all();
    if (partials) block_taps<MM, TT, kVecThreads>(acc, m, T, partials);
}

// Division by d of values below 2^31 by multiply and shift.
struct BDiv {
    uint64_t mul;
    uint32_t sh;
};
BDiv bdiv_of(uint32_t d) {
    uint32_t l = 0;
    while ((1ull << l) < d) ++l;
    BDiv f;
    f.sh = 31 + l;
    f.mul = ((1ull << f.sh) + d - 1) / d;
    return f;
}
__device__ __forceinline__ uint32_t bdiv(uint32_t v, const BDiv& f) { return (uint32_t)(((uint64_t)v * f.mul) >> f.sh); }

__device__ __forceinline__ float4 fma4(float h, const float4& g, const float4& a) {
    return make_float4(fmaf(h, g.x, a.x), fmaf(h, g.y, a.y), fmaf(h, g.z, a.z), fmaf(h, g.w, a.w));
}

// Column pass: items (frame, repetition, group of 4 columns), W4 = n
// columns / 4 groups per row, below 2^31 items.  dY and dX rows are n
// columns wide; X row (f, c) starts at element (f n_in + c) n.
#ifndef AROL_BWD_COL_MINB
#define AROL_BWD_COL_MINB 1
#endif
template <int QQ, int MM, int TT>
__global__ void __launch_bounds__(kBwThreads, AROL_BWD_COL_MINB) sep_col_bwd_kernel(const SepPassDev p, uint32_t items, int W,
                                                                 BDiv dw4, BDiv dr, const float* __restrict__ taps,
                                                                 const void* __restrict__ x, int x_dt,
                                                                 const float* __restrict__ gy, float* __restrict__ gx,
                                                                 float* __restrict__ partials) {
    __shared__ float hs[kBwTaps];
    const int m = p.m, T = p.T, S = p.S, R = p.R, Hin = p.n_in, Hout = p.n_out;
    const int Q = (T + S - 1) / S;
    const int W4 = W >> 2;
    for (int i = threadIdx.x; i < m * T; i += blockDim.x) hs[i] = __ldg(taps + i);
    __syncthreads();
    float acc[MM][TT];
#pragma unroll
    for (int j = 0; j < MM; ++j)
#pragma unroll
        for (int k = 0; k < TT; ++k) acc[j][k] = 0.f;
    for (uint32_t it = blockIdx.x * blockDim.x + threadIdx.x; it < items; it += gridDim.x * blockDim.x) {
        const uint32_t line = bdiv(it, dw4);
        const int cg = (int)(it - line * (uint32_t)W4);
        const uint32_t f = bdiv(line, dr);
        const int r = (int)(line - f * (uint32_t)R);
        const float* gb = gy + (int64_t)f * Hout * W + 4 * cg;
        float4 g[QQ][MM];
#pragma unroll
        for (int q = 0; q < QQ; ++q) {
            int rq = r - q;
            while (rq < 0) rq += R;
#pragma unroll
            for (int j = 0; j < MM; ++j)
                g[q][j] = q < Q && j < m ? __ldg(reinterpret_cast<const float4*>(gb + (int64_t)(m * rq + j) * W))
                                         : make_float4(0.f, 0.f, 0.f, 0.f);
        }
        int pos = p.o + S * r;
        if (pos >= Hin) pos -= Hin;
        // the window of X in registers before any store of dX (loads issued
        // ahead of the stores: 30 against 41 us on the 5 -> 2 chain's pass)
        float4 xw[TT];
        if (partials) {
            const int64_t xf = (int64_t)f * Hin * W + 4 * cg;
            int c = pos;
#pragma unroll
            for (int k = 0; k < TT; ++k) {
                xw[k] = k < T ? ld4(x, xf + (int64_t)c * W, x_dt) : make_float4(0.f, 0.f, 0.f, 0.f);
                if (++c == Hin) c = 0;
            }
        }
        if (gx) {
            float* xb = gx + (int64_t)f * Hin * W + 4 * cg;
            int pp = pos;
            for (int d = 0; d < S; ++d) {
                float4 a = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
                for (int q = 0; q < QQ; ++q) {
                    const int k = d + S * q;
                    if (q < Q && k < T) {
#pragma unroll
                        for (int j = 0; j < MM; ++j)
                            if (j < m) a = fma4(hs[j * T + k], g[q][j], a);
                    }
                }
                *reinterpret_cast<float4*>(xb + (int64_t)pp * W) = a;
                if (++pp == Hin) pp = 0;
            }
        }
        if (partials) {
#pragma unroll
            for (int k = 0; k < TT; ++k) {
                if (k < T) {
                    const float4 xv = xw[k];
#pragma unroll
                    for (int j = 0; j < MM; ++j) {
                        float a = acc[j][k];
                        a = fmaf(g[0][j].x, xv.x, a);
                        a = fmaf(g[0][j].y, xv.y, a);
                        a = fmaf(g[0][j].z, xv.z, a);
                        a = fmaf(g[0][j].w, xv.w, a);
                        acc[j][k] = a;
                    }
                }
            }
        }
    }
    if (partials) block_taps<MM, TT>(acc, m, T, partials);
}

// The (QQ, MM, TT) bins: 0 (2, 2, 8), 1 (2, 4, 8), 2 (4, 4, 16); -1 none.
int bwd_bin(const SepPassDev& p, bool col) {
    const int Q = (p.T + p.S - 1) / p.S;
    if (p.m * p.T > kBwTaps) return -1;
    if (Q <= 2 && p.T <= 8 && p.m <= 2) return 0;
    if (Q <= 2 && p.T <= 8 && p.m <= 4) return 1;
    if (!col && Q <= 4 && p.T <= 16 && p.m <= 4) return 2;
    return -1;
}

// Row-pass form: asynchronous staging needs X in f32 (or no tap gradients).
bool row_async(int x_dt, bool want_taps) { return x_dt == 0 || !want_taps; }

size_t row_smem(const SepPassDev& p, bool async) {
    const size_t pair = spad_len(p.n_out) + (size_t)spad_len(p.n_in);
    return sizeof(float) * ((size_t)kBwTaps + (async ? kBwStages : 1) * pair + spad_len(p.n_in));
}

size_t vec_smem(const SepPassDev& p) {
    return sizeof(float) * ((size_t)kBwTaps + (size_t)kBwStages * (32 + p.n_out + p.n_in) + p.n_in);
}

template <typename K>
int blocks_of(K kernel, int threads, size_t smem) {
    int n = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kernel, threads, smem);
    return device_sm_count() * (n > 0 ? n : 1);
}

using RowKernel = void (*)(const SepPassDev, int64_t, const float*, const void*, int, const float*, float*, float*);
using VecKernel = void (*)(const SepPassDev, int64_t, const float*, const float*, const float*, float*, float*);
using ColKernel = void (*)(const SepPassDev, uint32_t, int, BDiv, BDiv, const float*, const void*, int, const float*,
                           float*, float*);

// Step-specialised forms: steps 2, 4 and 8 of the asynchronous QQ = 2 bins.
int row_step(int bin, bool async, int S) {
    return async && bin < 2 && (S == 2 || S == 4 || S == 8) ? S : 0;
}

template <int QQ, int MM, int TT>
RowKernel row_kernel_async(int ss) {
    return ss == 2 ? sep_row_bwd_kernel<QQ, MM, TT, true, 2>
                   : ss == 4 ? sep_row_bwd_kernel<QQ, MM, TT, true, 4>
                             : ss == 8 ? sep_row_bwd_kernel<QQ, MM, TT, true, 8> : sep_row_bwd_kernel<QQ, MM, TT, true, 0>;
}

RowKernel row_kernel(int bin, bool async, int ss) {
    if (async)
        return bin == 0 ? row_kernel_async<2, 2, 8>(ss)
                        : bin == 1 ? row_kernel_async<2, 4, 8>(ss) : sep_row_bwd_kernel<4, 4, 16, true, 0>;
    return bin == 0 ? sep_row_bwd_kernel<2, 2, 8, false, 0>
                    : bin == 1 ? sep_row_bwd_kernel<2, 4, 8, false, 0> : sep_row_bwd_kernel<4, 4, 16, false, 0>;
}

// The 16-word-region forms: (step, bank) = (2, m <= 2), (4 or 8, m <= 4), T <= 8.
VecKernel vec_kernel(int ss, int mm) {
    if (ss == 2) return sep_row_bwd_vec_kernel<2, 2, 8>;
    if (ss == 4) return mm == 2 ? sep_row_bwd_vec_kernel<4, 2, 8> : sep_row_bwd_vec_kernel<4, 4, 8>;
    return mm == 2 ? sep_row_bwd_vec_kernel<8, 2, 8> : sep_row_bwd_vec_kernel<8, 4, 8>;
}
ColKernel col_kernel(int bin) { return bin == 0 ? sep_col_bwd_kernel<2, 2, 8> : sep_col_bwd_kernel<2, 4, 8>; }

constexpr size_t kRowSmemMax = 96 * 1024;

bool aligned16(const void* q) { return (reinterpret_cast<uintptr_t>(q) & 15) == 0; }

void opt_in_smem() {
    static bool done = false;
    if (done) return;
    for (int b = 0; b < 3; ++b)
        for (int a = 0; a < 2; ++a)
            for (int ss : {0, 2, 4, 8})
                cudaFuncSetAttribute(row_kernel(b, a == 1, ss), cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)kRowSmemMax);
    for (int ss : {2, 4, 8})
        for (int mm : {2, 4})
            cudaFuncSetAttribute(vec_kernel(ss, mm), cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kRowSmemMax);
    done = true;
}

}  // namespace

bool sep_bwd_plan(const SepPassDev& p, int64_t F, int Hin, int Win, int x_dt, const void* x, const float* gy,
                  const float* gx, bool want_taps, SepBwdPlan* plan) {
    if ((int64_t)p.S * p.R != p.n_in || F < 1) return false;
    const int bin = bwd_bin(p, p.axis == 0);
    if (bin < 0) return false;
    SepBwdPlan pl{};
    pl.bin = bin;
    if (p.axis == 1) {
        opt_in_smem();
        const bool vec = (p.S == 2 ? p.m <= 2 : (p.S == 4 || p.S == 8) && p.m <= 4) && p.T <= 8 && p.n_in % 16 == 0 &&
                         p.o % 16 == 0 && p.n_out % 4 == 0 && (x_dt == 0 || !want_taps) && aligned16(gy) &&
                         aligned16(gx) && (!want_taps || aligned16(x)) && vec_smem(p) <= kRowSmemMax;
        if (vec) {
            pl.form = 2;
            pl.ss = p.S;
            pl.mm = p.m <= 2 ? 2 : 4;
            pl.smem = vec_smem(p);
            pl.threads = kVecThreads;
            static int cache[9][5] = {};
            static size_t cache_smem[9][5] = {};
            int& c = cache[pl.ss][pl.mm];
            if (!c || cache_smem[pl.ss][pl.mm] != pl.smem) {
                c = blocks_of(vec_kernel(pl.ss, pl.mm), kVecThreads, pl.smem);
                cache_smem[pl.ss][pl.mm] = pl.smem;
            }
            pl.blocks = c;
        } else {
            pl.form = 1;
            pl.async = row_async(x_dt, want_taps);
            pl.ss = row_step(bin, pl.async, p.S);
            pl.smem = row_smem(p, pl.async);
            if (pl.smem > kRowSmemMax) return false;
            pl.threads = kBwThreads;
            static int cache[3][2][9] = {};
            static size_t cache_smem[3][2][9] = {};
            int& c = cache[bin][pl.async][pl.ss];
            if (!c || cache_smem[bin][pl.async][pl.ss] != pl.smem) {
                c = blocks_of(row_kernel(bin, pl.async, pl.ss), kBwThreads, pl.smem);
                cache_smem[bin][pl.async][pl.ss] = pl.smem;
            }
            pl.blocks = c;
        }
        *plan = pl;
        return true;
    }
    // column pass: 16-byte rows of 4-column groups
    const uintptr_t xa = x_dt == 0 ? 15 : 7;
    if (Win % 4 || !aligned16(gy) || !aligned16(gx) || (want_taps && (reinterpret_cast<uintptr_t>(x) & xa)))
        return false;
    if (F * p.R * (Win / 4) >= (int64_t)1 << 31 || F * (int64_t)Hin * Win >= (int64_t)1 << 40) return false;
    pl.form = 0;
    pl.threads = kBwThreads;
    static int ccache[2] = {0, 0};
    if (!ccache[bin]) ccache[bin] = blocks_of(col_kernel(bin), kBwThreads, 0);
    pl.blocks = ccache[bin];
    *plan = pl;
    return true;
}

cudaError_t launch_sep_bwd(const SepBwdPlan& pl, const SepPassDev& p, int64_t F, int Hin, int Win, const float* taps,
                           const void* x, int x_dt, const float* gy, float* gx, float* partials, float* grad_taps,
                           cudaStream_t s) {
    if (pl.blocks < 1) return cudaErrorInvalidValue;
    float* part = grad_taps ? partials : nullptr;
    if (pl.form == 2) {
        vec_kernel(pl.ss, pl.mm)<<<pl.blocks, kVecThreads, pl.smem, s>>>(p, F * Hin, taps,
                                                                         static_cast<const float*>(x), gy, gx, part);
    } else if (pl.form == 1) {
        row_kernel(pl.bin, pl.async, pl.ss)<<<pl.blocks, kBwThreads, pl.smem, s>>>(p, F * Hin, taps, x, x_dt, gy, gx,
                                                                                   part);
    } else {
        const uint32_t W4 = (uint32_t)(Win / 4);
        const uint32_t items = (uint32_t)(F * p.R * (int64_t)W4);
        col_kernel(pl.bin)<<<pl.blocks, kBwThreads, 0, s>>>(p, items, Win, bdiv_of(W4), bdiv_of((uint32_t)p.R), taps,
                                                            x, x_dt, gy, gx, part);
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess || !grad_taps) return e;
    return launch_tap_reduce(partials, pl.blocks, p.m * p.T, grad_taps, s);
}

}  // namespace arol
