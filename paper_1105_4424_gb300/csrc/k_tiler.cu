// Generic Array-OL tiler kernel (gather -> copy/FIR -> scatter) and the
// persistent batched kernel that runs many such tasks from one work list.
//
// Address generation (the tiler of the MARTE RSM package, Sec. 3; repetitive
// tasks, Sec. 7): for repetition r and pattern index i an array element is
// e(r, i) = (o + P r + F i) mod s.  The host reduces o, P and F into [0, s)
// so the device computes the base (o + P r) mod s once per repetition and then
// walks the pattern by adding fitting columns with one conditional subtract
// per dimension (strength-reduced modulo), all in 32-bit registers.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "arol_internal.h"
#include "ptx.h"
#include "tiler_dev.h"


namespace arol {
namespace {

template <int MAXM>
__device__ __forceinline__ void process_rep(const TaskDev& t, int64_t lr) {
    const bool wide = t.wide != 0;
    uint32_t r[4], b[4], bo[4];
    decode_rep(t, lr, wide, r);
    base_index(t.in, r, wide, b);
    base_index(t.out, r, wide, bo);
    process_rep_at<MAXM>(t, b, bo);
}

template <int MAXM>
__global__ void __launch_bounds__(kThreads) tiler_generic_kernel(const TaskDev t) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t lr = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; lr < t.nreps; lr += stride)
        process_rep<MAXM>(t, lr);
}


// ---------------------------------------------------------------------------
// Column FIR tile (repetitions start .. start + count - 1 of a column-FIR
// task, column fastest, frames outermost): repetition (f, r0, c) reads rows
// (o0 + step*r0 + k) mod H of column (o1 + c) mod W of frame f and writes m
// consecutive output rows of one column of frame f (a task without frames
// has one).  Consecutive threads take consecutive columns, so the loads of a
// warp and its stores are contiguous; the input is read straight from global
// memory (each element once when T <= step), the transposed taps from shared
// memory.  Two repetitions per thread share every tap load.
// ---------------------------------------------------------------------------
template <int M>
__device__ __forceinline__ void col_fir_compute(const TaskDev& t, const float* ht, int64_t start, int count) {
    constexpr int kHt = 16;
    const int T = t.T;
    const uint32_t S = (uint32_t)t.step, C = (uint32_t)t.rep[3];
    const uint32_t hin = (uint32_t)t.in.shape[0], win = (uint32_t)t.in.shape[1];
    const uint32_t hout = (uint32_t)t.out.shape[0], wout = (uint32_t)t.out.shape[1];
    const float* x = static_cast<const float*>(t.x);
    float* y = static_cast<float*>(t.y);
    const int B = blockDim.x;
    for (int base = 0; base < count; base += 2 * B) {
        // repetition pairs as in the row FIR: (t, t + B), the last chunk (t, t + ceil(rem / 2))
        const int rem = count - base, half = rem >= 2 * B ? B : (rem + 1) >> 1;
        if ((int)threadIdx.x >= half) break;
        const int i0 = base + (int)threadIdx.x;
        const int i1 = i0 + half < count ? i0 + half : i0;
        uint32_t r0[2], col[2], row[2], fr[2];
        const uint32_t lr[2] = {(uint32_t)(start + i0), (uint32_t)(start + i1)};   // < 2^31: not wide
#pragma unroll
        for (int a = 0; a < 2; ++a) {
            // repetition (frame, r0, c): c fastest, frames outermost
            const uint32_t q = fast_div(lr[a], t.rep_div[3]);
            const uint32_t c = lr[a] - q * C;
            fr[a] = fast_div(q, t.rep_div[2]);
            r0[a] = q - fr[a] * (uint32_t)t.rep[2];
            const uint32_t vr = t.in.origin[0] + S * r0[a];              // < 2^31: checked on the host
            row[a] = vr - fast_div(vr, t.in.shape_div[0]) * hin;
            const uint32_t vc = t.in.origin[1] + c;
            col[a] = vc - fast_div(vc, t.in.shape_div[1]) * win;
        }
        float acc0[M], acc1[M];
#pragma unroll
        for (int j = 0; j < M; ++j) acc0[j] = acc1[j] = 0.f;
        // unrolled by 4: the taps' global loads are independent of the FMAs,
        // so more of them are in flight per thread
        const float* x0 = x + (int64_t)fr[0] * t.cf_in_frame;
        const float* x1 = x + (int64_t)fr[1] * t.cf_in_frame;
#pragma unroll 4
        for (int kk = 0; kk < T; ++kk) {
            const float p0 = __ldg(x0 + (int64_t)row[0] * win + col[0]);
            const float p1 = __ldg(x1 + (int64_t)row[1] * win + col[1]);
            row[0] = row[0] + 1u == hin ? 0u : row[0] + 1u;
            row[1] = row[1] + 1u == hin ? 0u : row[1] + 1u;
            float h[M];
            load_taps<M>(ht + kk * kHt, h);
#pragma unroll
            for (int j = 0; j < M; ++j) {
                acc0[j] = fmaf(h[j], p0, acc0[j]);
                acc1[j] = fmaf(h[j], p1, acc1[j]);
            }
        }
#pragma unroll
        for (int a = 0; a < 2; ++a) {
            if (a == 1 && i1 == i0) break;
            const uint32_t c = lr[a] - fast_div(lr[a], t.rep_div[3]) * C;
            float* ya = y + (int64_t)fr[a] * t.cf_out_frame;
            const uint32_t vr = t.out.origin[0] + (uint32_t)M * r0[a];   // < 2^31: checked on the host
            uint32_t orow = vr - fast_div(vr, t.out.shape_div[0]) * hout;
            const uint32_t vc = t.out.origin[1] + c;
            const uint32_t ocol = vc - fast_div(vc, t.out.shape_div[1]) * wout;
#pragma unroll
            for (int j = 0; j < M; ++j) {
                ya[(int64_t)orow * wout + ocol] = a == 0 ? acc0[j] : acc1[j];
                orow = orow + 1u == hout ? 0u : orow + 1u;
            }
        }
    }
}

__device__ __forceinline__ void col_fir_dispatch(const TaskDev& t, const float* ht, int64_t start, int count) {
#define AROL_COL_FIR_CASE(M) \
    case M: col_fir_compute<M>(t, ht, start, count); break;
    switch (t.m) {
        AROL_COL_FIR_CASE(1) AROL_COL_FIR_CASE(2) AROL_COL_FIR_CASE(3) AROL_COL_FIR_CASE(4)
        AROL_COL_FIR_CASE(5) AROL_COL_FIR_CASE(6) AROL_COL_FIR_CASE(7) AROL_COL_FIR_CASE(8)
        AROL_COL_FIR_CASE(9) AROL_COL_FIR_CASE(10) AROL_COL_FIR_CASE(11) AROL_COL_FIR_CASE(12)
        AROL_COL_FIR_CASE(13) AROL_COL_FIR_CASE(14) AROL_COL_FIR_CASE(15)
        default: col_fir_compute<16>(t, ht, start, count); break;
    }
#undef AROL_COL_FIR_CASE
}

// ---------------------------------------------------------------------------
// FIR on a 2-D pattern (a stencil when m = 1): repetition (r0, r1) reads the
// p0 x p1 block of rows o0 + s0*r0 + a and columns o1 + s1*r1 + b (mod the
// array shape) and writes m consecutive elements of output row (oo0 + r0)
// from column oo1 + m*r1.  A CTA takes a bh x bw block of repetitions: it
// stages the (s0*(bh-1) + p0) x (s1*(bw-1) + p1) input window (wrapped) and
// the transposed taps in shared memory, then each thread computes
// repetitions of one column of the block, reading the window with
// consecutive columns in consecutive lanes.
// ---------------------------------------------------------------------------
constexpr int kFir2dThreads = 256;
constexpr int kFir2dWin = 8192;   // window floats (host-checked)

template <int M>
__device__ __forceinline__ void fir2d_compute(const TaskDev& t, const float* win, int ww, const float* ht,
                                              uint32_t r0a, uint32_t r1a) {
    constexpr int kHt = 16;
    // thread: column lr1 of the block and rows g, g + rs, g + 2 rs, g + 3 rs
    // (bh = 4 rs, rs = blockDim.x / bw); the four share every tap load
    const int bw = t.bw, rs = (int)blockDim.x / bw;
    const int lr1 = (int)threadIdx.x % bw, g = (int)threadIdx.x / bw;
    const int s0 = t.s0, s1 = t.s1, p0 = t.p0, p1 = t.p1;
    const uint32_t R0 = (uint32_t)t.rep[2], R1 = (uint32_t)t.rep[3];
    const uint32_t r1 = r1a + (uint32_t)lr1;
    if (r1 >= R1) return;
    float acc[4][M];
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int j = 0; j < M; ++j) acc[u][j] = 0.f;
    const float* w0 = win + (s0 * g) * ww + s1 * lr1;
    const int du = s0 * rs * ww;   // window offset between the thread's rows
    int k = 0;
    for (int a = 0; a < p0; ++a) {
        const float* wr = w0 + a * ww;
        for (int b = 0; b < p1; ++b, ++k) {
            float h[M];
            load_taps<M>(ht + k * kHt, h);
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const float v = wr[u * du + b];
#pragma unroll
                for (int j = 0; j < M; ++j) acc[u][j] = fmaf(h[j], v, acc[u][j]);
            }
        }
    }
    const uint32_t hout = (uint32_t)t.out.shape[0], wout = (uint32_t)t.out.shape[1];
    float* y = static_cast<float*>(t.y);
    const uint64_t vc = (uint64_t)t.out.origin[1] + (uint64_t)M * r1;
    const uint32_t c0 = vc < 0x7fffffffull ? (uint32_t)vc - fast_div((uint32_t)vc, t.out.shape_div[1]) * wout
                                           : (uint32_t)(vc % wout);
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        const uint32_t r0 = r0a + (uint32_t)(g + u * rs);
        if (r0 >= R0) break;
        const uint32_t vr = t.out.origin[0] + r0;                      // < 2^31: checked on the host
        const uint32_t orow = vr - fast_div(vr, t.out.shape_div[0]) * hout;
        float* yrow = y + (int64_t)orow * wout;
        uint32_t c = c0;
#pragma unroll
        for (int j = 0; j < M; ++j) {
            yrow[c] = acc[u][j];
            c = (c + 1u == wout) ? 0u : c + 1u;
        }
    }
}

// Issues (cp.async, no wait) the copies of tile `tile`'s input window:
// rows (o0 + s0*r0a + i) mod H, columns (o1 + s1*r1a + j) mod W.
__device__ __forceinline__ void fir2d_stage(const TaskDev& t, uint32_t r0a, uint32_t r1a, int wh, int ww, float* win) {
    const uint32_t hin = (uint32_t)t.in.shape[0], wi = (uint32_t)t.in.shape[1];
    const uint32_t vr = t.in.origin[0] + (uint32_t)t.s0 * r0a;      // < 2^31: checked on the host
    const uint32_t rb = vr - fast_div(vr, t.in.shape_div[0]) * hin;
    const uint32_t vc = t.in.origin[1] + (uint32_t)t.s1 * r1a;
    const uint32_t cb = vc - fast_div(vc, t.in.shape_div[1]) * wi;
    const float* x = static_cast<const float*>(t.x);
    // element e = i * ww + j of the window, walked with an incremental (i, j)
    const int B = (int)blockDim.x, di = B / ww, dj = B - di * ww;
    int i = (int)threadIdx.x / ww, j = (int)threadIdx.x - i * ww;
    if ((uint32_t)wh <= hin && (uint32_t)ww <= wi) {
        // the window wraps at most once in each dimension
        for (int e = threadIdx.x; e < wh * ww; e += B) {
            uint32_t row = rb + (uint32_t)i, col = cb + (uint32_t)j;
            row = row >= hin ? row - hin : row;
            col = col >= wi ? col - wi : col;
            ptx::cp_async4(win + e, x + (int64_t)row * wi + col);
            i += di;
            j += dj;
            if (j >= ww) {
                j -= ww;
                ++i;
            }
        }
        return;
    }
    for (int e = threadIdx.x; e < wh * ww; e += B) {
        uint32_t row = rb + (uint32_t)i, col = cb + (uint32_t)j;
        row -= fast_div(row, t.in.shape_div[0]) * hin;
        col -= fast_div(col, t.in.shape_div[1]) * wi;
        ptx::cp_async4(win + e, x + (int64_t)row * wi + col);
        i += di;
        j += dj;
        if (j >= ww) {
            j -= ww;
            ++i;
        }
    }
}

// One CTA per tile (tile = ty * tiles_x + tx covers repetitions r0 in
// [ty*bh, +bh), r1 in [tx*bw, +bw)); CTAs of different tiles overlap their
// copies and compute on an SM.  kMaxM: the largest output count the
// instantiation handles; the one for m <= 4 keeps to 64 registers so that
// four CTAs share an SM.
template <int kMaxM>
__global__ void __launch_bounds__(kFir2dThreads, kMaxM <= 4 ? 4 : 2) fir2d_kernel(const TaskDev t, int tiles_x) {
    extern __shared__ __align__(16) float f2[];
    const int ww = t.s1 * (t.bw - 1) + t.p1, wh = t.s0 * (t.bh - 1) + t.p0;
    float* win = f2;
    float* ht = f2 + ((wh * ww + 3) & ~3);
    const int tile = blockIdx.x, ty = tile / tiles_x, tx = tile - ty * tiles_x;
    const uint32_t r0a = (uint32_t)(ty * t.bh), r1a = (uint32_t)(tx * t.bw);
    fir2d_stage(t, r0a, r1a, wh, ww, win);
    // taps transposed: ht[k * 16 + j] = H[j, k]
    const int T = t.T, m = t.m;
    for (int e = threadIdx.x; e < T * 16; e += blockDim.x) {
        const int k = e >> 4, j = e & 15;
        ht[e] = j < m ? __ldg(t.taps + j * T + k) : 0.f;
    }
    ptx::cp_async_wait_all();
    __syncthreads();
#define AROL_FIR2D_CASE(M) \
    case M: fir2d_compute<(M <= kMaxM ? M : kMaxM)>(t, win, ww, ht, r0a, r1a); break;
    switch (m) {
        AROL_FIR2D_CASE(1) AROL_FIR2D_CASE(2) AROL_FIR2D_CASE(3) AROL_FIR2D_CASE(4)
        AROL_FIR2D_CASE(5) AROL_FIR2D_CASE(6) AROL_FIR2D_CASE(7) AROL_FIR2D_CASE(8)
        AROL_FIR2D_CASE(9) AROL_FIR2D_CASE(10) AROL_FIR2D_CASE(11) AROL_FIR2D_CASE(12)
        AROL_FIR2D_CASE(13) AROL_FIR2D_CASE(14) AROL_FIR2D_CASE(15)
        default: fir2d_compute<kMaxM>(t, win, ww, ht, r0a, r1a); break;
    }
#undef AROL_FIR2D_CASE
}

// Stencil specialisation (steps 1, one output, a P0 x P1 pattern): a tile
// is 32 x 128 repetitions; thread (column c, strip g) computes the 16
// consecutive output rows 16 g .. 16 g + 15 of column c.  It walks the window
// down one row at a time, holding that row's P1 values and the taps in
// registers, and adds the row into every output it belongs to, so each
// window value is read from shared memory once per thread.
constexpr int kStencilBh = 32, kStencilBw = 128, kStencilRows = 16;

// Copies rows (rb + i) mod H, i < wh, columns c0 .. c0 + 4 nq - 1 (c0 a
// multiple of 4, W a multiple of 4, so no 16-byte chunk straddles the wrap)
// of x into win (row stride 4 nq) with 16-byte cp.async.
__device__ __forceinline__ void stage_rows16(const float* x, uint32_t hin, uint32_t wi, uint32_t rb, uint32_t c0,
                                             int wh, int nq, float* win) {
    const int B = (int)blockDim.x, di = B / nq, dj = B - di * nq;
    int i = (int)threadIdx.x / nq, j = (int)threadIdx.x - i * nq;
    for (int e = threadIdx.x; e < wh * nq; e += B) {
        uint32_t row = rb + (uint32_t)i, col = c0 + 4u * (uint32_t)j;
        row = row >= hin ? row - hin : row;
        col = col >= wi ? col - wi : col;
        ptx::cp_async16(win + 4 * e, x + (int64_t)row * wi + col);
        i += di;
        j += dj;
        if (j >= nq) {
            j -= nq;
            ++i;
        }
    }
}

// Stages the window of stencil tile (ty, tx) (repetitions r0 in
// [kStencilBh ty, +kStencilBh), r1 in [kStencilBw tx, +kStencilBw)) into win
// and returns the window's first column within a staged row.  fast: 16-byte
// copies of 4-aligned row pieces (row stride 4 nq); otherwise element copies
// (row stride ww).
template <int P0, int P1>
__device__ __forceinline__ int stencil_stage(const TaskDev& t, bool fast, uint32_t ty, uint32_t tx, float* win) {
    constexpr int ww = kStencilBw + P1 - 1, wh = kStencilBh + P0 - 1;
    constexpr int nq = (ww + 3 + 3) / 4;
    const uint32_t r0a = ty * (uint32_t)kStencilBh, r1a = tx * (uint32_t)kStencilBw;
    if (!fast) {
        fir2d_stage(t, r0a, r1a, wh, ww, win);
        return 0;
    }
    const uint32_t hin = (uint32_t)t.in.shape[0], wi = (uint32_t)t.in.shape[1];
    const uint32_t vr = t.in.origin[0] + r0a;                        // < 2^31: checked on the host
    const uint32_t rb = vr - fast_div(vr, t.in.shape_div[0]) * hin;
    const uint32_t vc = t.in.origin[1] + r1a;
    const uint32_t cb = vc - fast_div(vc, t.in.shape_div[1]) * wi;
    stage_rows16(static_cast<const float*>(t.x), hin, wi, rb, cb & ~3u, wh, nq, win);
    return (int)(cb & 3u);
}

// Computes and stores stencil tile (ty, tx) from its staged window.
template <int P0, int P1>
__device__ __forceinline__ void stencil_tile(const TaskDev& t, const float* win, int rs, int delta, uint32_t ty,
                                             uint32_t tx, const float (&h)[P0][P1]) {
    const int c = (int)threadIdx.x % kStencilBw, g = (int)threadIdx.x / kStencilBw;
    const uint32_t R0 = (uint32_t)t.rep[2], R1 = (uint32_t)t.rep[3];
    const uint32_t r1 = tx * (uint32_t)kStencilBw + (uint32_t)c;
    if (r1 >= R1) return;
    float acc[kStencilRows];
#pragma unroll
    for (int r = 0; r < kStencilRows; ++r) acc[r] = 0.f;
    const float* w0 = win + (g * kStencilRows) * rs + delta + c;
#pragma unroll
    for (int i = 0; i < kStencilRows + P0 - 1; ++i) {
        float v[P1];
#pragma unroll
        for (int b = 0; b < P1; ++b) v[b] = w0[b];
        w0 += rs;
        // window row i feeds output rows r = i - a for pattern rows a, in a order per output
#pragma unroll
        for (int a = 0; a < P0; ++a) {
            const int r = i - a;
            if (r >= 0 && r < kStencilRows) {
#pragma unroll
                for (int b = 0; b < P1; ++b) acc[r] = fmaf(h[a][b], v[b], acc[r]);
            }
        }
    }
    const uint32_t hout = (uint32_t)t.out.shape[0], wout = (uint32_t)t.out.shape[1];
    const uint32_t vc = t.out.origin[1] + r1;                           // < 2^31: checked on the host
    const uint32_t ocol = vc - fast_div(vc, t.out.shape_div[1]) * wout;
    const uint32_t r00 = ty * (uint32_t)kStencilBh + (uint32_t)(g * kStencilRows);
    const uint32_t vr = t.out.origin[0] + r00;
    uint32_t orow = vr - fast_div(vr, t.out.shape_div[0]) * hout;
    float* yp = static_cast<float*>(t.y) + (int64_t)orow * wout + ocol;
    if (orow + (uint32_t)kStencilRows <= hout && r00 + (uint32_t)kStencilRows <= R0) {
        // the strip neither wraps nor runs past the last repetition row
#pragma unroll
        for (int r = 0; r < kStencilRows; ++r) {
            *yp = acc[r];
            yp += wout;
        }
        return;
    }
    float* y = static_cast<float*>(t.y);
#pragma unroll
    for (int r = 0; r < kStencilRows; ++r) {
        if (r00 + (uint32_t)r >= R0) break;
        y[(int64_t)orow * wout + ocol] = acc[r];
        orow = orow + 1u == hout ? 0u : orow + 1u;
    }
}

// Window floats of one stencil tile buffer (rows of 4 nq floats).
template <int P0, int P1>
constexpr int stencil_buf_floats() {
    return (kStencilBh + P0 - 1) * ((kStencilBw + P1 - 1 + 3 + 3) / 4) * 4;
}

// Persistent over tiles (static schedule: CTA b takes tiles b, b + grid, ...,
// grid <= ntiles; tile = ty * tiles_x + tx), with three window buffers in
// dynamic shared memory: while a CTA computes tile k, the copies of tiles
// k + 1 and k + 2 are in flight.  One barrier per tile suffices: the buffer
// refilled after it was last read by the previous tile, which every thread
// finished before the barrier.
template <int P0, int P1>
__global__ void __launch_bounds__(kFir2dThreads, 4) stencil_kernel(const TaskDev t, uint32_t tiles_x, uint32_t ntiles) {
    constexpr int ww = kStencilBw + P1 - 1, wh = kStencilBh + P0 - 1;
    constexpr int nq = (ww + 3 + 3) / 4;   // 16-byte chunks per row when the start is rounded down to 4
    constexpr int kBuf = stencil_buf_floats<P0, P1>();
    extern __shared__ __align__(16) float swin[];
    const uint32_t hin = (uint32_t)t.in.shape[0], wi = (uint32_t)t.in.shape[1];
    const bool fast = (wi & 3u) == 0u && ((uintptr_t)t.x & 15u) == 0u && (uint32_t)wh <= hin && (uint32_t)(4 * nq) <= wi;
    const int rs = fast ? 4 * nq : ww;   // staged row stride
    float h[P0][P1];
#pragma unroll
    for (int a = 0; a < P0; ++a)
#pragma unroll
        for (int b = 0; b < P1; ++b) h[a][b] = __ldg(t.taps + a * P1 + b);
    // tile coordinates advance by the grid: (gq, gr) = divmod(grid, tiles_x)
    const uint32_t gq = gridDim.x / tiles_x, gr = gridDim.x - gq * tiles_x;
    // the tile a CTA computes now (0), and the next two (1, 2); indices are
    // 64-bit so that tile + 2 grid cannot wrap
    uint64_t t0 = blockIdx.x, t1 = t0 + gridDim.x;
    uint32_t y0 = (uint32_t)t0 / tiles_x, x0 = (uint32_t)t0 - y0 * tiles_x;
    uint32_t y1 = y0 + gq, x1 = x0 + gr;
    if (x1 >= tiles_x) {
        x1 -= tiles_x;
        ++y1;
    }
    int b0 = 0, b1 = 1, b2 = 2;   // buffers of tiles 0, 1, 2
    int d0 = stencil_stage<P0, P1>(t, fast, y0, x0, swin);
    ptx::cp_async_commit();
    int d1 = 0;
    if (t1 < ntiles) d1 = stencil_stage<P0, P1>(t, fast, y1, x1, swin + kBuf);
    ptx::cp_async_commit();
    while (t0 < ntiles) {
        ptx::cp_async_wait_group<1>();   // tile 0's copies have landed (tile 1's may be in flight)
        __syncthreads();
        const uint64_t t2 = t1 + gridDim.x;
        uint32_t y2 = y1 + gq, x2 = x1 + gr;
        if (x2 >= tiles_x) {
            x2 -= tiles_x;
            ++y2;
        }
        int d2 = 0;
        if (t2 < ntiles) d2 = stencil_stage<P0, P1>(t, fast, y2, x2, swin + b2 * kBuf);
        ptx::cp_async_commit();
        stencil_tile<P0, P1>(t, swin + b0 * kBuf, rs, d0, y0, x0, h);
        const int bf = b0;
        t0 = t1; y0 = y1; x0 = x1; d0 = d1; b0 = b1;
        t1 = t2; y1 = y2; x1 = x2; d1 = d2; b1 = b2;
        b2 = bf;
    }
    ptx::cp_async_wait_all();
}

// Shared memory of the batch kernel: a ring of three task records (the
// TaskDev of the tile being computed, of the next tile, and of the one after,
// being copied), then two slots for the transposed, zero-padded taps of a
// column-FIR tile's task (ht[k * 16 + j] = H[j, k], k < 32).
constexpr int kTaskFloats = (int)((sizeof(TaskDev) + 15) / 16 * 4);
constexpr int kMetaSlots = 3;
constexpr int kSlotFloats = 32 * 16;
static_assert(sizeof(TaskDev) % 4 == 0, "TaskDev is copied in 4-byte words");

// Issues (cp.async, no wait) the copies of a task's transposed taps into a data slot.
__device__ __forceinline__ void stage_taps(const TaskDev& t, float* slot) {
    for (int i = threadIdx.x; i < t.T * 16; i += blockDim.x) ptx::cp_async4(slot + i, t.taps_t + i);
}

// Copies (cp.async, no wait) task record `t` into a meta slot.
__device__ __forceinline__ void stage_meta(const TaskDev& t, float* meta) {
    const float* src = reinterpret_cast<const float*>(&t);
    for (int w = threadIdx.x; w < (int)(sizeof(TaskDev) / 4); w += blockDim.x) ptx::cp_async4(meta + w, src + w);
}

// Persistent batched kernel for the tiles that are not row-FIR tiles (those
// run on the row-FIR kernel).  CTA b takes tiles b, b + gridDim.x, ... (the
// host orders tiles by cost).  The task record of tile i + 2 is copied into
// shared memory while tile i is computed, and the taps of tile i + 1 (a
// column-FIR tile), whose address comes from its record already in shared
// memory, fill the other data slot, so no global load stands between a
// barrier and the compute.  Column-FIR tiles read their columns from global
// memory; other tiles run the generic per-repetition path.  No CTA ever waits
// on another.
template <int MAXM>
__global__ void __launch_bounds__(kBatchThreads, 4) batch_persistent_kernel(const TaskDev* __restrict__ tasks,
                                                                  const TileDev* __restrict__ tiles, int ntiles) {
    constexpr bool kCols = MAXM <= 16;
    extern __shared__ __align__(16) float dsm[];
    float* meta = dsm;                                  // kMetaSlots task records
    float* data = dsm + kMetaSlots * kTaskFloats;       // two tap slots
    const int G = gridDim.x;
    int slot_task[2] = {-1, -1};   // task whose taps each data slot holds (the same in every thread)
    // records of tiles i, i + 1, i + 2 (registers), valid when the index < ntiles
    const int t0 = blockIdx.x;
    TileDev tl0{}, tl1{}, tl2{};
    if (t0 < ntiles) tl0 = tiles[t0];
    if (t0 + G < ntiles) tl1 = tiles[t0 + G];
    if (t0 + 2 * G < ntiles) tl2 = tiles[t0 + 2 * G];
    if (kCols) {
        if (t0 < ntiles) stage_meta(tasks[tl0.task], meta);
        if (t0 + G < ntiles) stage_meta(tasks[tl1.task], meta + kTaskFloats);
        ptx::cp_async_commit();
        ptx::cp_async_wait_group<0>();
        __syncthreads();
        if (t0 < ntiles) {
            const TaskDev& m0 = *reinterpret_cast<const TaskDev*>(meta);
            if (m0.colfir) {
                stage_taps(m0, data);
                slot_task[0] = tl0.task;
            }
        }
        ptx::cp_async_commit();
    }
    for (int i = 0, ti = t0; ti < ntiles; ++i, ti += G) {
        const int cur = i & 1, nxt = cur ^ 1;
        if (kCols) {
            // taps of tile i and the record of tile i + 1 have landed; every
            // thread is done with tile i - 1 (its data slot and its record)
            ptx::cp_async_wait_group<0>();
            __syncthreads();
            if (ti + G < ntiles) {
                const TaskDev& m1 = *reinterpret_cast<const TaskDev*>(meta + ((i + 1) % kMetaSlots) * kTaskFloats);
                if (m1.colfir) {
                    if (slot_task[nxt] != tl1.task) stage_taps(m1, data + nxt * kSlotFloats);
                    slot_task[nxt] = tl1.task;
                }
            }
            if (ti + 2 * G < ntiles) stage_meta(tasks[tl2.task], meta + ((i + 2) % kMetaSlots) * kTaskFloats);
            ptx::cp_async_commit();
        }
        const TileDev tile = tl0;
        tl0 = tl1;
        tl1 = tl2;
        if (ti + 3 * G < ntiles) tl2 = tiles[ti + 3 * G];   // used at the next iteration
        const TaskDev* mcur = reinterpret_cast<const TaskDev*>(meta + (i % kMetaSlots) * kTaskFloats);
        if (kCols && mcur->colfir) {
            col_fir_dispatch(*mcur, data + cur * kSlotFloats, tile.start, tile.count);
            continue;
        }
        const TaskDev& t = tasks[tile.task];
        const int64_t end = tile.start + tile.count;
        for (int64_t lr = tile.start + threadIdx.x; lr < end; lr += blockDim.x) process_rep<MAXM>(t, lr);
    }
    ptx::cp_async_wait_all();
}

// Element of port p at flat pattern index j of the repetition whose base is b
// (pattern dim 1 fastest); direct form, used by the backward kernels.
__device__ __forceinline__ int64_t pattern_offset(const PortDev& p, const uint32_t b[4], int j) {
    const uint32_t i0 = (uint32_t)j / (uint32_t)p.pattern[1];
    const uint32_t i1 = (uint32_t)j - i0 * (uint32_t)p.pattern[1];
    int64_t off = 0;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const uint64_t v = (uint64_t)b[k] + (uint64_t)p.fitting[k][0] * i0 + (uint64_t)p.fitting[k][1] * i1;
        off += (int64_t)(v % (uint64_t)(uint32_t)p.shape[k]) * p.stride[k];
    }
    return off;
}

// The same offset when the pattern cannot wrap (pattern_fits; `base` its
// first element's offset): the linear walk, no modulo.
__device__ __forceinline__ int64_t pattern_off(const PortDev& p, const uint32_t b[4], bool fits, int64_t base, int j) {
    if (!fits) return pattern_offset(p, b, j);
    const uint32_t i0 = (uint32_t)j / (uint32_t)p.pattern[1];
    const uint32_t i1 = (uint32_t)j - i0 * (uint32_t)p.pattern[1];
    return base + (int64_t)i0 * p.lin[0] + (int64_t)i1 * p.lin[1];
}

// dL/dX by owner computes: input element e sums, over the (r, k) pairs whose
// gather visited it (inverse map, increasing order), sum_j H[j,k] g[e_out(r,j)]
// (fir) or g[e_out(r,k)] (copy).  Each element is written once: no atomics.
__global__ void __launch_bounds__(kThreads) tiler_bwd_dx_kernel(const TaskDev t, const int64_t* __restrict__ start,
                                                                const int32_t* __restrict__ list, float* __restrict__ gx,
                                                                const float* __restrict__ gy, int64_t n) {
    const bool wide = t.wide != 0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += stride) {
        float acc = 0.f;
        const int64_t a = start[e], z = start[e + 1];
        for (int64_t idx = a; idx < z; ++idx) {
            // r * T + k < 2^31 (the host checks): 32-bit division
            const uint32_t rk = (uint32_t)list[idx];
            const uint32_t lr = rk / (uint32_t)t.T;
            const int k = (int)(rk - lr * (uint32_t)t.T);
            uint32_t r[4], b[4];
            decode_rep(t, lr, wide, r);
            base_index(t.out, r, wide, b);
            const bool fo = pattern_fits(t.out, b);
            const int64_t bo = fo ? offset_of(t.out, b) : 0;
            if (t.elem == ELEM_FIR) {
                for (int j = 0; j < t.m; ++j)
                    acc = fmaf(__ldg(t.taps + (int64_t)j * t.T + k), __ldg(gy + pattern_off(t.out, b, fo, bo, j)), acc);
            } else {
                acc += __ldg(gy + pattern_off(t.out, b, fo, bo, k));
            }
        }
        gx[e] = acc;
    }
}

// Per-block partial tap gradients: block b covers repetitions
// [b*chunk, (b+1)*chunk); thread p owns the pair (j, k) = (p / T, p % T) and
// sums g[e_out(r,j)] * x[e_in(r,k)] over them in order.
__global__ void __launch_bounds__(kThreads) tiler_bwd_dh_kernel(const TaskDev t, const float* __restrict__ gy,
                                                                float* __restrict__ partials, int64_t chunk) {
    const bool wide = t.wide != 0;
    const int64_t r0 = (int64_t)blockIdx.x * chunk;
    const int64_t r1 = r0 + chunk < t.nreps ? r0 + chunk : t.nreps;
    const int npairs = t.m * t.T;
    for (int p = threadIdx.x; p < npairs; p += blockDim.x) {
        const int j = p / t.T, k = p - (p / t.T) * t.T;
        float acc = 0.f;
        for (int64_t lr = r0; lr < r1; ++lr) {
            uint32_t r[4], bi[4], bo[4];
            decode_rep(t, lr, wide, r);
            base_index(t.in, r, wide, bi);
            base_index(t.out, r, wide, bo);
            acc = fmaf(__ldg(gy + pattern_offset(t.out, bo, j)), load_value(t, pattern_offset(t.in, bi, k)), acc);
        }
        partials[(int64_t)blockIdx.x * npairs + p] = acc;
    }
}

// The same partials with every thread of the block at work: thread t takes
// repetitions r0 + t, r0 + t + blockDim, ... and keeps all m x T pair sums
// in registers (m <= MM, T <= TT), then the block adds them in a fixed order
// (warp shuffles, then warps in order), so the result is the same every run.
template <int MM, int TT>
__global__ void __launch_bounds__(kThreads) tiler_bwd_dh_regs_kernel(const TaskDev t, const float* __restrict__ gy,
                                                                     float* __restrict__ partials, int64_t chunk) {
    const bool wide = t.wide != 0;
    const int64_t r0 = (int64_t)blockIdx.x * chunk;
    const int64_t r1 = r0 + chunk < t.nreps ? r0 + chunk : t.nreps;
    const int m = t.m, T = t.T;
    float acc[MM][TT];
#pragma unroll
    for (int j = 0; j < MM; ++j)
#pragma unroll
        for (int k = 0; k < TT; ++k) acc[j][k] = 0.f;
    for (int64_t lr = r0 + threadIdx.x; lr < r1; lr += blockDim.x) {
        uint32_t r[4], bi[4], bo[4];
        decode_rep(t, lr, wide, r);
        base_index(t.in, r, wide, bi);
        base_index(t.out, r, wide, bo);
        const bool fi = pattern_fits(t.in, bi), fo = pattern_fits(t.out, bo);
        const int64_t oi = fi ? offset_of(t.in, bi) : 0, oo = fo ? offset_of(t.out, bo) : 0;
        float xv[TT], gv[MM];
#pragma unroll
        for (int k = 0; k < TT; ++k) xv[k] = k < T ? load_value(t, pattern_off(t.in, bi, fi, oi, k)) : 0.f;
#pragma unroll
        for (int j = 0; j < MM; ++j) gv[j] = j < m ? __ldg(gy + pattern_off(t.out, bo, fo, oo, j)) : 0.f;
#pragma unroll
        for (int j = 0; j < MM; ++j)
#pragma unroll
            for (int k = 0; k < TT; ++k) acc[j][k] = fmaf(gv[j], xv[k], acc[j][k]);
    }
    __shared__ float red[kThreads / 32][MM * TT];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
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
    const int npairs = m * T, nw = (int)(blockDim.x >> 5);
    for (int p = threadIdx.x; p < npairs; p += blockDim.x) {
        const int j = p / T, k = p - j * T;
        float v = 0.f;
        for (int w = 0; w < nw; ++w) v += red[w][j * TT + k];
        partials[(int64_t)blockIdx.x * npairs + p] = v;
    }
}

// One warp per tap pair: lane l adds the partials of blocks l, l + 32, ...
// in order, then the lanes' sums meet in a fixed shuffle tree.
__global__ void __launch_bounds__(kThreads) tiler_bwd_reduce_kernel(const float* __restrict__ partials, int nblocks,
                                                                    int npairs, float* __restrict__ out) {
    const int p = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
    if (p >= npairs) return;
    float s = 0.f;
    for (int b = lane; b < nblocks; b += 32) s += partials[(int64_t)b * npairs + p];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
    if (lane == 0) out[p] = s;
}

int grid_for(int64_t work, int threads) {
    const int64_t blocks = (work + threads - 1) / threads;
    const int64_t cap = (int64_t)device_sm_count() * 16;
    return (int)(blocks < cap ? (blocks > 0 ? blocks : 1) : cap);
}

}  // namespace

int device_sm_count() {
    static int sms = 0;
    if (!sms) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (sms <= 0) sms = 1;
    }
    return sms;
}

// Self-test of the bounded waits the pipelined kernels use: thread 0 waits
// on an mbarrier that nothing ever completes; the wait gives up after its
// limit and the kernel records it in *err and returns.
__global__ void wait_selftest_kernel(unsigned* err) {
    __shared__ __align__(8) uint64_t bar;
    const uint32_t a = ptx::smem_addr(&bar);
    if (threadIdx.x == 0) {
        ptx::mbar_init(a, 1);
        ptx::fence_barrier_init();
    }
    __syncthreads();
    if (threadIdx.x == 0 && !ptx::mbar_wait(a, 0)) atomicOr(err, 1u);
}

cudaError_t launch_wait_selftest(unsigned* err, cudaStream_t s) {
    wait_selftest_kernel<<<1, 32, 0, s>>>(err);
    return cudaGetLastError();
}

bool fir2d_uses_stencil(const TaskDev& t) {
    return t.fir2d && t.m == 1 && t.s0 == 1 && t.s1 == 1 && t.p0 == t.p1 && (t.p0 == 3 || t.p0 == 5);
}

cudaError_t launch_fir2d(const TaskDev& t, cudaStream_t s) {
    static bool attr = false;
    const int ww = t.s1 * (t.bw - 1) + t.p1, wh = t.s0 * (t.bh - 1) + t.p0;
    const size_t smem = (size_t)(((wh * ww + 3) & ~3) + t.T * 16) * sizeof(float);
    if (!attr) {
        const int most = (int)((kFir2dWin + 64 * 16) * sizeof(float));
        cudaError_t e = cudaFuncSetAttribute(fir2d_kernel<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, most);
        if (e == cudaSuccess) e = cudaFuncSetAttribute(fir2d_kernel<16>, cudaFuncAttributeMaxDynamicSharedMemorySize, most);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    if (fir2d_uses_stencil(t)) {
        const int64_t sx = (t.rep[3] + kStencilBw - 1) / kStencilBw, sy = (t.rep[2] + kStencilBh - 1) / kStencilBh;
        const uint32_t ntiles = (uint32_t)(sx * sy);   // fewer tiles than the general tiling: < 2^31
        static int occ3 = 0, occ5 = 0;
        int& occ = t.p0 == 3 ? occ3 : occ5;
        void (*kern)(const TaskDev, uint32_t, uint32_t) = t.p0 == 3 ? stencil_kernel<3, 3> : stencil_kernel<5, 5>;
        const size_t ssmem = 3 * sizeof(float) * (size_t)(t.p0 == 3 ? stencil_buf_floats<3, 3>() : stencil_buf_floats<5, 5>());
        if (occ == 0) {
            cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ssmem);
            int n = 0;
            if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kern, kFir2dThreads, ssmem);
            if (e != cudaSuccess) return e;
            occ = n > 0 ? n : 1;
        }
        const uint32_t grid = (uint32_t)std::min<int64_t>((int64_t)device_sm_count() * occ, ntiles);
        kern<<<grid, kFir2dThreads, ssmem, s>>>(t, (uint32_t)sx, ntiles);
        return cudaGetLastError();
    }
    const int64_t tiles_x = (t.rep[3] + t.bw - 1) / t.bw, tiles_y = (t.rep[2] + t.bh - 1) / t.bh;
    const unsigned grid = (unsigned)(tiles_x * tiles_y);   // < 2^31: checked on the host
    if (t.m <= 4) fir2d_kernel<4><<<grid, kFir2dThreads, smem, s>>>(t, (int)tiles_x);
    else fir2d_kernel<16><<<grid, kFir2dThreads, smem, s>>>(t, (int)tiles_x);
    return cudaGetLastError();
}

cudaError_t launch_tiler_generic(const TaskDev& t, int max_m, cudaStream_t s) {
    if (t.nreps == 0) return cudaSuccess;
    const int grid = grid_for(t.nreps, kThreads);
    if (max_m <= 4) tiler_generic_kernel<4><<<grid, kThreads, 0, s>>>(t);
    else if (max_m <= 8) tiler_generic_kernel<8><<<grid, kThreads, 0, s>>>(t);
    else if (max_m <= 16) tiler_generic_kernel<16><<<grid, kThreads, 0, s>>>(t);
    else tiler_generic_kernel<32><<<grid, kThreads, 0, s>>>(t);
    return cudaGetLastError();
}

size_t batch_smem(int max_m) {
    return max_m <= 16 ? ((size_t)kMetaSlots * kTaskFloats + 2 * (size_t)kSlotFloats) * sizeof(float) : 0;
}

template <int MAXM>
cudaError_t launch_batch_m(const TaskDev* tasks, const TileDev* tiles, int ntiles, int grid, int threads,
                           cudaStream_t s) {
    static bool attr = false;
    static int occ_threads = 0, occ = 1;
    const size_t smem = batch_smem(MAXM);
    if (!attr && smem > 0) {
        cudaError_t e = cudaFuncSetAttribute(batch_persistent_kernel<MAXM>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    if (occ_threads != threads) {
        int n = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, batch_persistent_kernel<MAXM>, threads, smem);
        occ = n > 0 ? n : 1;
        occ_threads = threads;
    }
    // static schedule: every CTA must be resident, or late CTAs stretch the tail
    const int cap = device_sm_count() * occ;
    if (grid > cap) grid = cap;
    batch_persistent_kernel<MAXM><<<grid, threads, smem, s>>>(tasks, tiles, ntiles);
    return cudaGetLastError();
}

cudaError_t launch_batch_persistent(const TaskDev* tasks, const TileDev* tiles, int ntiles, unsigned* counter,
                                    int grid, int threads, int max_m, cudaStream_t s) {
    (void)counter;   // the schedule is static: CTA b takes tiles b, b + grid, ...
    if (ntiles == 0) return cudaSuccess;
    if (grid > ntiles) grid = ntiles;
    threads = kBatchThreads;   // the kernel's launch bound
    if (max_m <= 4) return launch_batch_m<4>(tasks, tiles, ntiles, grid, threads, s);
    if (max_m <= 8) return launch_batch_m<8>(tasks, tiles, ntiles, grid, threads, s);
    if (max_m <= 16) return launch_batch_m<16>(tasks, tiles, ntiles, grid, threads, s);
    return launch_batch_m<32>(tasks, tiles, ntiles, grid, threads, s);
}

cudaError_t launch_tap_reduce(const float* partials, int nblocks, int npairs, float* out, cudaStream_t s) {
    tiler_bwd_reduce_kernel<<<(npairs * 32 + kThreads - 1) / kThreads, kThreads, 0, s>>>(partials, nblocks, npairs, out);
    return cudaGetLastError();
}

int tiler_bwd_blocks(int64_t nreps, int m, int T, int64_t* chunk) {
    // the register kernel keeps every thread busy: two blocks per SM; the
    // per-pair kernel runs one thread per pair, so it wants more blocks
    const bool regs = (m <= 4 && T <= 16) || (m <= 8 && T <= 16);
    int64_t nb = regs ? (nreps + 255) / 256 : (nreps + 63) / 64;
    const int64_t cap = (int64_t)device_sm_count() * (regs ? 2 : 8);
    if (nb > cap) nb = cap;
    if (nb < 1) nb = 1;
    *chunk = (nreps + nb - 1) / nb;
    if (*chunk < 1) *chunk = 1;
    return (int)nb;
}

cudaError_t launch_tiler_bwd(const TaskDev& t, const int64_t* inv_start, const int32_t* inv_list, float* gx,
                             const float* gy, float* grad_taps, float* partials, int nblocks, int64_t chunk,
                             cudaStream_t s) {
    if (gx) {
        int64_t n = 1;
        for (int k = 0; k < 4; ++k) n *= t.in.shape[k];
        tiler_bwd_dx_kernel<<<grid_for(n, kThreads), kThreads, 0, s>>>(t, inv_start, inv_list, gx, gy, n);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    if (grad_taps) {
        const int npairs = t.m * t.T;
        if (t.m <= 4 && t.T <= 8) tiler_bwd_dh_regs_kernel<4, 8><<<nblocks, kThreads, 0, s>>>(t, gy, partials, chunk);
        else if (t.m <= 4 && t.T <= 16) tiler_bwd_dh_regs_kernel<4, 16><<<nblocks, kThreads, 0, s>>>(t, gy, partials, chunk);
        else if (t.m <= 8 && t.T <= 16) tiler_bwd_dh_regs_kernel<8, 16><<<nblocks, kThreads, 0, s>>>(t, gy, partials, chunk);
        else tiler_bwd_dh_kernel<<<nblocks, kThreads, 0, s>>>(t, gy, partials, chunk);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        tiler_bwd_reduce_kernel<<<(npairs * 32 + kThreads - 1) / kThreads, kThreads, 0, s>>>(partials, nblocks, npairs,
                                                                                             grad_taps);
        return cudaGetLastError();
    }
    return cudaSuccess;
}

}  // namespace arol
