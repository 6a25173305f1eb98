// Fused chains of separable FIR passes (row and column passes, any taps,
// outputs, step and origin, wrap included): the general form of the chained
// downscaler (Sec. 5 associatedParts; repetitive tasks on the GPU, Sec. 7).
//
// One CTA per tile of the last stage.  It loads the tile's stage-0 window
// (rows and columns from sep_regions, tabulated by the host per tile row and
// per tile column, wrapped at the array edges) into shared
// memory, then runs the passes in order between two shared buffers; the last
// pass writes the tile to global memory.  The intermediate arrays never
// reach HBM: only halos (the T - S overlap of neighbouring tiles' windows)
// are read twice, mostly from L2.
//
// In a pass, a warp takes one repetition at a time (its index arithmetic is
// the same for every lane) and its lanes take the region's rows (row pass)
// or columns (column pass); a thread computes the m outputs of its row or
// column, the m accumulators in registers (m is a template parameter), the
// taps transposed in shared memory (one broadcast load feeds m FMAs).  Region rows have an odd stride,
// so both kinds of pass read shared memory without bank conflicts; column
// passes store consecutive columns from consecutive lanes.
#include <algorithm>

#include <cuda_fp16.h>

#include "arol_internal.h"
#include "ptx.h"
#include "sepchain.h"

namespace arol {
namespace {

constexpr int kSepThreads = 256;

// Row stride (floats) of a region of `cols` columns in shared memory: odd,
// so lanes that walk down a column of the region hit distinct banks.
__device__ __forceinline__ int ld_of(int cols) { return cols | 1; }

// Walks the repetitions ra + w, ra + w + nw, ... of a pass (w: this warp,
// nw: the warps of the CTA) and keeps, for the current one, where it reads
// the input region (`base`, a local index) and where its m outputs start in
// the output region (`first`; some may fall outside).  Each step adds nw
// repetitions with one conditional subtract; only a step past repetition
// R - 1 recomputes from the definition.  Warp-uniform.
struct RepWalk {
    int ur, r, base, first;
    int step_base, step_first;
    __device__ __forceinline__ void set(const SepPassDev& p, SepRange in, SepRange out) {
        r = ur % p.R;
        // o + S r - start fits 32 bits: the host keeps S R and the extents below 2^30
        const int b = (p.o + p.S * r - in.start) % p.n_in;
        base = b < 0 ? b + p.n_in : b;
        first = sep_upos(p, ur) - out.start;
    }
    __device__ __forceinline__ void start(const SepPassDev& p, int ur0, int nw, SepRange in, SepRange out) {
        ur = ur0;
        step_base = (p.S * nw) % p.n_in;
        step_first = p.m * nw;
        set(p, in, out);
    }
    __device__ __forceinline__ void next(const SepPassDev& p, int nw, SepRange in, SepRange out) {
        ur += nw;
        if (r + nw >= p.R) {
            set(p, in, out);
            return;
        }
        r += nw;
        base += step_base;
        if (base >= p.n_in) base -= p.n_in;
        first += step_first;
    }
};

// Row pass: warps take repetitions, lanes take the region's rows (all rows
// of a row pass share the repetition's columns).  Input rows of stride
// ld_of(ci.len), output rows of stride ldo; ht: the pass's taps transposed,
// ht[kk * G + j] = H[j, kk] (G: the kernel's tap row, >= m).
template <int M, int G>
__device__ void row_pass(const SepPassDev& p, const float* ht, const float* in, SepRange ri, SepRange ci, SepRange co,
                         float* out, int64_t ldo) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarps = blockDim.x >> 5;
    const int ra = co.start / M;   // the first output position is < n_out
    const int nrep = sep_urep(p, co.start + co.len - 1) - ra + 1;
    const int ldi = ld_of(ci.len), T = p.T;
    RepWalk w;
    w.start(p, ra + warp, nwarps, ci, co);
    for (int rr = warp; rr < nrep; rr += nwarps, w.next(p, nwarps, ci, co)) {
        for (int i = lane; i < ri.len; i += 32) {
            const float* src = in + i * ldi + w.base;
            float acc[M];
#pragma unroll
            for (int j = 0; j < M; ++j) acc[j] = 0.f;
#pragma unroll 4
            for (int kk = 0; kk < T; ++kk) {
                const float v = src[kk];
                const float* h = ht + kk * G;
#pragma unroll
                for (int j = 0; j < M; ++j) acc[j] = fmaf(h[j], v, acc[j]);
            }
            float* o = out + (int64_t)i * ldo + w.first;
#pragma unroll
            for (int j = 0; j < M; ++j)
                if (w.first + j >= 0 && w.first + j < co.len) o[j] = acc[j];
        }
    }
}

// Column pass: warps take repetitions, lanes take the region's columns.
template <int M, int G>
__device__ void col_pass(const SepPassDev& p, const float* ht, const float* in, SepRange ri, SepRange ci, SepRange ro,
                         float* out, int64_t ldo) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarps = blockDim.x >> 5;
    const int ra = ro.start / M;
    const int nrep = sep_urep(p, ro.start + ro.len - 1) - ra + 1;
    const int ldi = ld_of(ci.len), T = p.T;
    RepWalk w;
    w.start(p, ra + warp, nwarps, ri, ro);
    for (int rr = warp; rr < nrep; rr += nwarps, w.next(p, nwarps, ri, ro)) {
        for (int c = lane; c < ci.len; c += 32) {
            const float* src = in + w.base * ldi + c;
            float acc[M];
#pragma unroll
            for (int j = 0; j < M; ++j) acc[j] = 0.f;
#pragma unroll 4
            for (int kk = 0; kk < T; ++kk) {
                const float v = src[kk * ldi];
                const float* h = ht + kk * G;
#pragma unroll
                for (int j = 0; j < M; ++j) acc[j] = fmaf(h[j], v, acc[j]);
            }
#pragma unroll
            for (int j = 0; j < M; ++j) {
                const int i = w.first + j;
                if (i >= 0 && i < ro.len) out[(int64_t)i * ldo + c] = acc[j];
            }
        }
    }
}

template <bool kRow, int kMaxM>
__device__ void run_pass(const SepPassDev& p, const float* hk, const float* in, SepRange ri, SepRange ci, SepRange ro,
                         SepRange co, float* out, int64_t ldo) {
    constexpr int G = kMaxM <= 4 ? 4 : 16;   // the kernel's transposed-tap row (kMaxM >= every m)
#define AROL_SEP_CASE(M)                                                                          \
    case M:                                                                                       \
        if (kRow) row_pass<(M <= kMaxM ? M : kMaxM), G>(p, hk, in, ri, ci, co, out, ldo);       \
        else col_pass<(M <= kMaxM ? M : kMaxM), G>(p, hk, in, ri, ci, ro, out, ldo);            \
        break;
    switch (p.m) {
        AROL_SEP_CASE(1) AROL_SEP_CASE(2) AROL_SEP_CASE(3) AROL_SEP_CASE(4)
        AROL_SEP_CASE(5) AROL_SEP_CASE(6) AROL_SEP_CASE(7) AROL_SEP_CASE(8)
        AROL_SEP_CASE(9) AROL_SEP_CASE(10) AROL_SEP_CASE(11) AROL_SEP_CASE(12)
        AROL_SEP_CASE(13) AROL_SEP_CASE(14) AROL_SEP_CASE(15) AROL_SEP_CASE(16)
        default: break;
    }
#undef AROL_SEP_CASE
}

// Stage-0 window: rows (rs + i) mod H0, columns (cs + q) mod W0, one warp per
// row, lanes along it with 4-byte asynchronous copies (each row a run of at
// most a few contiguous pieces, split where it wraps).
__device__ void stage_window(const float* xf, int H0, int W0, SepRange rows, SepRange cols, float* dst) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarps = blockDim.x >> 5;
    const int ld = ld_of(cols.len);
    for (int i = warp; i < rows.len; i += nwarps) {
        int gr = rows.start + i;
        while (gr >= H0) gr -= H0;
        const float* src = xf + (int64_t)gr * W0;
        float* d = dst + i * ld;
        // pieces [q0, q1) of the window that are contiguous in the row
        int q0 = 0, c = cols.start;
        while (q0 < cols.len) {
            while (c >= W0) c -= W0;
            const int q1 = min(cols.len, q0 + (W0 - c));
            for (int q = q0 + lane; q < q1; q += 32) ptx::cp_async4(d + q, src + c + (q - q0));
            c += q1 - q0;
            q0 = q1;
        }
    }
    ptx::cp_async_wait_all();
}

// kMaxM: the largest m of the chain's passes the instantiation handles (the
// one for m <= 4 keeps to 64 registers, four CTAs per SM).
template <int kMaxM>
__global__ void __launch_bounds__(kSepThreads, kMaxM <= 4 ? 4 : 2) sepchain_kernel(const SepChainDev d) {
    extern __shared__ __align__(16) float ssm[];
    // each pass's taps transposed: ht_k[kk * G + j] = H_k[j, kk], G = 4 (m <= 4) or 16
    constexpr int G = kMaxM <= 4 ? 4 : 16;
    float* taps = ssm;
    float* buf[2] = {ssm + kSepMaxPasses * 32 * G, ssm + kSepMaxPasses * 32 * G + d.buf};
    for (int k = 0; k < d.K; ++k)
        for (int e = threadIdx.x; e < 32 * G; e += blockDim.x) {
            const int kk = e / G, j = e - kk * G;
            taps[k * 32 * G + e] = (kk < d.p[k].T && j < d.p[k].m) ? __ldg(d.taps + d.p[k].tap_off + j * d.p[k].T + kk) : 0.f;
        }
    const int K = d.K;
    const uint32_t ntile = (uint32_t)d.tiles_y * (uint32_t)d.tiles_x;   // F * ntile < 2^31 (host)
    const uint32_t total = (uint32_t)d.F * ntile;
    for (uint32_t t = blockIdx.x; t < total; t += gridDim.x) {
        const uint32_t f = t / ntile;
        const uint32_t tt = t - f * ntile;
        const int ty = (int)(tt / (uint32_t)d.tiles_x), tx = (int)(tt - (uint32_t)ty * (uint32_t)d.tiles_x);
        SepRange rows[kSepMaxPasses + 1], cols[kSepMaxPasses + 1];
        const int2* rt = reinterpret_cast<const int2*>(d.row_tab) + ty * (K + 1);
        const int2* ct = reinterpret_cast<const int2*>(d.col_tab) + tx * (K + 1);
        for (int k = 0; k <= K; ++k) {
            const int2 a = __ldg(rt + k), b = __ldg(ct + k);
            rows[k].start = a.x;
            rows[k].len = a.y;
            cols[k].start = b.x;
            cols[k].len = b.y;
        }
        __syncthreads();   // the previous tile's last pass is done with the buffers
        stage_window(d.x + (int64_t)f * d.H[0] * d.W[0], d.H[0], d.W[0], rows[0], cols[0], buf[0]);
        __syncthreads();
        for (int k = 0; k < K; ++k) {
            const SepPassDev& p = d.p[k];
            const float* in = buf[k & 1];
            float* out;
            int64_t ldo;
            if (k + 1 == K) {
                out = d.y + ((int64_t)f * d.H[K] + rows[K].start) * (int64_t)d.W[K] + cols[K].start;
                ldo = d.W[K];
            } else {
                out = buf[(k + 1) & 1];
                ldo = ld_of(cols[k + 1].len);
            }
            const float* ht = taps + k * 32 * G;
            if (p.axis == 1) run_pass<true, kMaxM>(p, ht, in, rows[k], cols[k], rows[k + 1], cols[k + 1], out, ldo);
            else run_pass<false, kMaxM>(p, ht, in, rows[k], cols[k], rows[k + 1], cols[k + 1], out, ldo);
            __syncthreads();
        }
    }
}

}  // namespace

size_t sepchain_smem(const SepChainDev& d) {
    int max_m = 1;
    for (int k = 0; k < d.K; ++k) max_m = std::max(max_m, (int)d.p[k].m);
    return ((size_t)kSepMaxPasses * 32 * (max_m <= 4 ? 4 : 16) + (size_t)d.buf + (size_t)d.buf1) * sizeof(float);
}

template <int kMaxM>
cudaError_t launch_sepchain_m(const SepChainDev& d, int64_t work, cudaStream_t s) {
    const size_t smem = sepchain_smem(d);
    static size_t attr = 0;
    static int occ = 0;
    if (smem > attr || occ == 0) {
        cudaError_t e = cudaFuncSetAttribute(sepchain_kernel<kMaxM>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)std::max(smem, attr));
        if (e != cudaSuccess) return e;
        attr = std::max(smem, attr);
    }
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, sepchain_kernel<kMaxM>, kSepThreads, smem);
    const int64_t cap = (int64_t)device_sm_count() * (occ > 0 ? occ : 1);
    sepchain_kernel<kMaxM><<<(int)(work < cap ? work : cap), kSepThreads, smem, s>>>(d);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Adjoint of one pass of a separable chain with respect to its input (Sec. 5
// chains, differentiated: the transposed tiler), as a gather: input position
// c along the pass's axis receives, for every repetition r whose window
// (o + S r + k) mod n_in, k < T, covers it, sum_j H[j, k] dY[m r + j].  With
// u = (c - o) mod n_in, the windows that reach c start at S r <= u + q n_in
// < S r + T for q = 0, 1, ... (windows that wrap once or more); no inverse
// map is needed.  One thread per input element, the non-axis index fastest
// for a column pass and the axis index for a row pass: coalesced loads and
// stores either way.
// ---------------------------------------------------------------------------
namespace {

// Division by S of values below 2^31: multiply by ceil(2^(31 + l) / S),
// l = ceil(log2 S), and shift (the multiply-shift division the host uses for
// the tilers, set up once per thread here).
struct SDiv {
    uint64_t m;
    uint32_t s;
};
__device__ __forceinline__ SDiv sdiv_of(uint32_t d) {
    uint32_t l = 0;
    while ((1ull << l) < d) ++l;
    SDiv f;
    f.s = 31 + l;
    f.m = ((1ull << f.s) + d - 1) / d;
    return f;
}
__device__ __forceinline__ int sdiv(int v, const SDiv& f) { return (int)(((uint64_t)(uint32_t)v * f.m) >> f.s); }

// Rows of the input (frame, row) go to blocks, columns to threads; the
// windows that reach a position depend only on that position.
__device__ __forceinline__ float sep_adjoint_sum(const SepPassDev& p, const SDiv& ds, int pos,
                                                 const float* __restrict__ h, const float* __restrict__ gy, int64_t o0,
                                                 int64_t ostep) {
    int u = pos - p.o;
    if (u < 0) u += p.n_in;
    float acc = 0.f;
    // S R + T + n_in < 2^31 (host-checked), so v stays in 32 bits
    for (int v = u;; v += p.n_in) {
        const int lo = v - p.T + 1;
        const int rlo = lo <= 0 ? 0 : sdiv(lo + p.S - 1, ds);
        if (rlo >= p.R) break;
        int rhi = sdiv(v, ds);
        if (rhi >= p.R) rhi = p.R - 1;
        for (int r = rlo; r <= rhi; ++r) {
            const int k = v - p.S * r;
            const float* g = gy + o0 + ((int64_t)p.m * r) * ostep;
            for (int j = 0; j < p.m; ++j) acc = fmaf(__ldg(h + j * p.T + k), __ldg(g + (int64_t)j * ostep), acc);
        }
    }
    return acc;
}

__global__ void __launch_bounds__(256) sep_adjoint_kernel(const SepPassDev p, int64_t F, int Hin, int Win, int Hout,
                                                          int Wout, const float* __restrict__ h,
                                                          const float* __restrict__ gy, float* __restrict__ gx) {
    const int64_t rows = F * Hin;
    const SDiv ds = sdiv_of((uint32_t)p.S);
    for (int64_t row = blockIdx.x; row < rows; row += gridDim.x) {
        const int64_t f = row / Hin;
        const int i = (int)(row - f * Hin);
        float* gxr = gx + row * Win;
        if (p.axis == 1) {
            // row pass: position c along the row; dY row (f, i), column m r + j
            const int64_t o0 = (f * Hout + i) * (int64_t)Wout;
            for (int c = threadIdx.x; c < Win; c += blockDim.x) gxr[c] = sep_adjoint_sum(p, ds, c, h, gy, o0, 1);
        } else {
            // column pass: position i down the column; dY rows m r + j, column c
            const int64_t o0 = f * Hout * (int64_t)Wout;
            for (int c = threadIdx.x; c < Win; c += blockDim.x) gxr[c] = sep_adjoint_sum(p, ds, i, h, gy, o0 + c, Wout);
        }
    }
}

// Tap gradients of one pass: dH[j, k] = sum over repetitions of
// dY[m r + j] X[(o + S r + k) mod n_in] (the other indices passing through).
// Row pass: blocks take input rows, threads the repetitions along them;
// column pass: blocks take (frame, repetition) lines, threads the columns.
// Every thread keeps all m x T sums in registers; the block adds them in a
// fixed order (warp shuffles, then warps in order) into its partials.
#ifndef AROL_DH_BLOCKS
#define AROL_DH_BLOCKS 4
#endif
constexpr int kDhBlocksPerSm = AROL_DH_BLOCKS;

// An input element in its storage (0 f32, 1 bfloat16, 2 IEEE half), widened.
__device__ __forceinline__ float ld_x(const void* x, int64_t i, int dt) {
    if (dt == 1) return __uint_as_float((uint32_t)__ldg(static_cast<const unsigned short*>(x) + i) << 16);
    if (dt == 2) return __half2float(__ushort_as_half(__ldg(static_cast<const unsigned short*>(x) + i)));
    return __ldg(static_cast<const float*>(x) + i);
}

template <int MM, int TT>
__global__ void __launch_bounds__(256) sep_dh_kernel(const SepPassDev p, int64_t F, int Hin, int Win, int Hout, int Wout,
                                                     const void* __restrict__ x, int x_dt, const float* __restrict__ gy,
                                                     float* __restrict__ partials) {
    const int m = p.m, T = p.T;
    float acc[MM][TT];
#pragma unroll
    for (int j = 0; j < MM; ++j)
#pragma unroll
        for (int k = 0; k < TT; ++k) acc[j][k] = 0.f;
    const int64_t lines = p.axis == 1 ? F * Hin : F * p.R;
    const int width = p.axis == 1 ? p.R : Win;
    for (int64_t line = blockIdx.x; line < lines; line += gridDim.x) {
#pragma unroll 2
        for (int q = threadIdx.x; q < width; q += blockDim.x) {
            float xv[TT], gv[MM];
            if (p.axis == 1) {
                // row (f, i) = line, repetition r = q
                const int64_t f = line / Hin, i = line - f * Hin;
                const int64_t xr = line * Win;
                const float* gr = gy + (f * Hout + i) * (int64_t)Wout + (int64_t)m * q;
                int col = (int)(((int64_t)p.o + (int64_t)p.S * q) % p.n_in);
#pragma unroll
                for (int k = 0; k < TT; ++k) {
                    xv[k] = k < T ? ld_x(x, xr + col, x_dt) : 0.f;
                    if (++col == p.n_in) col = 0;
                }
#pragma unroll
                for (int j = 0; j < MM; ++j) gv[j] = j < m ? __ldg(gr + j) : 0.f;
            } else {
                // (f, r) = line, column c = q
                const int64_t f = line / p.R;
                const int r = (int)(line - f * p.R);
                const int64_t xf = f * Hin * (int64_t)Win + q;
                const float* gf = gy + (f * Hout + (int64_t)m * r) * (int64_t)Wout + q;
                int row = (int)(((int64_t)p.o + (int64_t)p.S * r) % p.n_in);
#pragma unroll
                for (int k = 0; k < TT; ++k) {
                    xv[k] = k < T ? ld_x(x, xf + (int64_t)row * Win, x_dt) : 0.f;
                    if (++row == p.n_in) row = 0;
                }
#pragma unroll
                for (int j = 0; j < MM; ++j) gv[j] = j < m ? __ldg(gf + (int64_t)j * Wout) : 0.f;
            }
#pragma unroll
            for (int j = 0; j < MM; ++j)
#pragma unroll
                for (int k = 0; k < TT; ++k) acc[j][k] = fmaf(gv[j], xv[k], acc[j][k]);
        }
    }
    __shared__ float red[8][MM * TT];
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
    const int npairs = m * T;
    for (int pp = threadIdx.x; pp < npairs; pp += blockDim.x) {
        const int j = pp / T, k = pp - j * T;
        float v = 0.f;
        for (int w = 0; w < 8; ++w) v += red[w][j * TT + k];
        partials[(int64_t)blockIdx.x * npairs + pp] = v;
    }
}

// The adjoint when the repetitions tile the axis exactly (S R = n_in):
// input position (o + S r + d) mod n_in, d < S, is the "home" of repetition
// r, and the windows that reach it are those of repetitions (r - q) mod R
// with tap index d + S q < T.  One thread per (line, r) keeps the Q x m
// gradients dY[m ((r - q) mod R) + j] in registers (Q = ceil(T / S) <= QQ,
// m <= MM) and writes its S home elements: no division per element.
template <int QQ, int MM>
__global__ void __launch_bounds__(256) sep_adjoint_poly_kernel(const SepPassDev p, int64_t F, int Hin, int Win,
                                                               int Hout, int Wout, const float* __restrict__ taps,
                                                               const float* __restrict__ gy, float* __restrict__ gx) {
    __shared__ float h[32 * 16];
    const int m = p.m, T = p.T, S = p.S, R = p.R;
    for (int i = threadIdx.x; i < m * T; i += blockDim.x) h[i] = __ldg(taps + i);
    __syncthreads();
    const int Q = (T + S - 1) / S;
    const int64_t lines = p.axis == 1 ? F * Hin : F * R;
    const int width = p.axis == 1 ? R : Win;
    for (int64_t line = blockIdx.x; line < lines; line += gridDim.x) {
        for (int q0 = threadIdx.x; q0 < width; q0 += blockDim.x) {
            int r;
            const float* gb;       // dY of repetition 0 for this thread's line or column
            int64_t gs;            // dY step between outputs j (and, times m, between repetitions)
            float* xb;             // dX of position 0
            int64_t xs;            // dX step between positions
            if (p.axis == 1) {
                const int64_t f = line / Hin, i = line - f * Hin;
                r = q0;
                gb = gy + (f * Hout + i) * (int64_t)Wout;
                gs = 1;
                xb = gx + line * Win;
                xs = 1;
            } else {
                const int64_t f = line / R;
                r = (int)(line - f * R);
                gb = gy + f * Hout * (int64_t)Wout + q0;
                gs = Wout;
                xb = gx + f * Hin * (int64_t)Win + q0;
                xs = Win;
            }
            float g[QQ][MM];
#pragma unroll
            for (int q = 0; q < QQ; ++q) {
                int rq = r - q;
                while (rq < 0) rq += R;
#pragma unroll
                for (int j = 0; j < MM; ++j)
                    g[q][j] = q < Q && j < m ? __ldg(gb + ((int64_t)m * rq + j) * gs) : 0.f;
            }
            int pos = (int)(((int64_t)p.o + (int64_t)S * r) % p.n_in);
            for (int d = 0; d < S; ++d) {
                float acc = 0.f;
#pragma unroll
                for (int q = 0; q < QQ; ++q) {
                    const int k = d + S * q;
                    if (q < Q && k < T) {
#pragma unroll
                        for (int j = 0; j < MM; ++j)
                            if (j < m) acc = fmaf(h[j * T + k], g[q][j], acc);
                    }
                }
                xb[(int64_t)pos * xs] = acc;
                if (++pos == p.n_in) pos = 0;
            }
        }
    }
}

}  // namespace

int sep_dh_blocks() { return device_sm_count() * kDhBlocksPerSm; }

bool sep_dh_supported(const SepPassDev& p) { return p.m <= 8 && p.T <= 16; }

cudaError_t launch_sep_dh(const SepPassDev& p, int64_t F, int Hin, int Win, int Hout, int Wout, const void* x, int x_dt,
                          const float* gy, float* partials, float* grad_taps, cudaStream_t s) {
    const int nb = sep_dh_blocks();
    if (p.m <= 4 && p.T <= 8)
        sep_dh_kernel<4, 8><<<nb, 256, 0, s>>>(p, F, Hin, Win, Hout, Wout, x, x_dt, gy, partials);
    else if (p.m <= 4 && p.T <= 16)
        sep_dh_kernel<4, 16><<<nb, 256, 0, s>>>(p, F, Hin, Win, Hout, Wout, x, x_dt, gy, partials);
    else if (p.m <= 8 && p.T <= 16)
        sep_dh_kernel<8, 16><<<nb, 256, 0, s>>>(p, F, Hin, Win, Hout, Wout, x, x_dt, gy, partials);
    else return cudaErrorInvalidValue;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return launch_tap_reduce(partials, nb, p.m * p.T, grad_taps, s);
}

cudaError_t launch_sep_adjoint(const SepPassDev& p, int64_t F, int Hin, int Win, int Hout, int Wout, const float* taps,
                               const float* gy, float* gx, cudaStream_t s) {
    const int64_t n = F * Hin * (int64_t)Win;
    if (n <= 0) return cudaSuccess;
    // repetitions that tile the axis exactly: the per-repetition form
    const int Q = (p.T + p.S - 1) / p.S;
    if ((int64_t)p.S * p.R == p.n_in && p.m * p.T <= 32 * 16 && Q <= 4 && p.m <= 8) {
        const int64_t lines = p.axis == 1 ? F * Hin : F * p.R;
        const int64_t blocks = std::min<int64_t>(lines, (int64_t)device_sm_count() * 16);
        if (Q <= 2 && p.m <= 4)
            sep_adjoint_poly_kernel<2, 4><<<(int)blocks, 256, 0, s>>>(p, F, Hin, Win, Hout, Wout, taps, gy, gx);
        else
            sep_adjoint_poly_kernel<4, 8><<<(int)blocks, 256, 0, s>>>(p, F, Hin, Win, Hout, Wout, taps, gy, gx);
        return cudaGetLastError();
    }
    const int64_t blocks = std::min<int64_t>(F * Hin, (int64_t)device_sm_count() * 16);
    sep_adjoint_kernel<<<(int)blocks, 256, 0, s>>>(p, F, Hin, Win, Hout, Wout, taps, gy, gx);
    return cudaGetLastError();
}

cudaError_t launch_sepchain(const SepChainDev& d, cudaStream_t s) {
    const int64_t work = d.F * (int64_t)d.tiles_y * d.tiles_x;
    if (work <= 0) return cudaSuccess;
    if (!d.row_tab || !d.col_tab) return cudaErrorInvalidValue;
    int max_m = 1;
    for (int k = 0; k < d.K; ++k) max_m = std::max(max_m, (int)d.p[k].m);
    return max_m <= 4 ? launch_sepchain_m<4>(d, work, s) : launch_sepchain_m<16>(d, work, s);
}

}  // namespace arol
