// Generic walk of any tiler, block-tiled (Sec. 3 tilers; repetitive tasks on
// the GPU, Sec. 7): the kernel behind tasks no specialised path takes.
#include <algorithm>

#include "arol_internal.h"
#include "tiler_dev.h"

#ifndef AROL_GEN_UNROLL
#define AROL_GEN_UNROLL 2
#endif
#ifndef AROL_GEN_MINB
#define AROL_GEN_MINB 3
#endif
#ifndef AROL_GEN_R
#define AROL_GEN_R 4
#endif

namespace arol {
namespace {

constexpr int kGenUnroll = AROL_GEN_UNROLL;   // tap indices of the block-tiled walk in flight together

// ---------------------------------------------------------------------------
// Generic walk, block-tiled.  A pattern whose base coordinates b satisfy
// b + ext < shape on every array dimension never wraps (fittings are reduced
// into [0, shape)), so its elements sit at offset(b) + i0 lin[0] + i1
// lin[1]: one add per element instead of a wrap test per dimension.  Other
// patterns take the wrapping walk.  FIR taps are staged once per block in
// shared memory, transposed (T x MAXM) for 16-byte loads of a tap index's
// MAXM taps.
// ---------------------------------------------------------------------------

// Up to R repetitions of one thread along the lane dimension db, 2^lb
// apart, their base coordinates stepped by g.istep / g.ostep (reduced).  Repetitions whose input and output patterns
// both stay inside their arrays run the linear walk together (one load of a
// tap index's taps for all of them, one add per element and repetition);
// the others take the wrapping walk one by one.
__device__ __forceinline__ void step_base(const PortDev& p, const uint32_t st[4], uint32_t b[4]) {
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const uint32_t v = b[k] + st[k];
        b[k] = v >= (uint32_t)p.shape[k] ? v - (uint32_t)p.shape[k] : v;
    }
}

template <int MAXM, int R, bool F32>
__device__ __forceinline__ void tiled_reps(const TaskDev& t, const GenGeom& g, const uint32_t r[4], int nr,
                                           const float* ht) {
    uint32_t b[4], bo[4];
    base_index(t.in, r, false, b);
    base_index(t.out, r, false, bo);
    int64_t oi[R], oo[R];
    bool lin[R];
    // The common case: no base of the thread's repetitions and no pattern
    // wraps, so their offsets step by a constant.
    bool all = t.in.linear && t.out.linear;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const uint64_t span = (uint64_t)(nr - 1);
        all = all && (uint64_t)b[k] + span * g.istep[k] + t.in.ext[k] < (uint64_t)(uint32_t)t.in.shape[k];
        all = all && (uint64_t)bo[k] + span * g.ostep[k] + t.out.ext[k] < (uint64_t)(uint32_t)t.out.shape[k];
    }
    if (all) {
        const int64_t i0 = offset_of(t.in, b), o0 = offset_of(t.out, bo);
#pragma unroll
        for (int q = 0; q < R; ++q) {
            lin[q] = q < nr;
            oi[q] = i0 + q * g.idelta;
            oo[q] = o0 + q * g.odelta;
        }
    }
#pragma unroll
    for (int q = 0; q < R; ++q) {
        if (all) break;
        lin[q] = false;
        oi[q] = oo[q] = 0;
        if (q < nr) {
            if (pattern_fits(t.in, b) && pattern_fits(t.out, bo)) {
                lin[q] = true;
                oi[q] = offset_of(t.in, b);
                oo[q] = offset_of(t.out, bo);
            } else {
                process_rep_at<MAXM>(t, b, bo);
            }
            step_base(t.in, g.istep, b);
            step_base(t.out, g.ostep, bo);
        }
    }
    const int n = t.T;
    // every repetition's walk takes the same steps: lin[1] within a pattern
    // row, lin[0] - (pattern[1] - 1) lin[1] from a row's end to the next
    const int pi1 = t.in.pattern[1], po1 = t.out.pattern[1];
    const int64_t si1 = t.in.lin[1], si0 = t.in.lin[0] - (int64_t)(pi1 - 1) * si1;
    const int64_t so1 = t.out.lin[1], so0 = t.out.lin[0] - (int64_t)(po1 - 1) * so1;
    if (t.elem == ELEM_COPY) {
        int ii = 0, io = 0;
#pragma unroll 4
        for (int k = 0; k < n; ++k) {
#pragma unroll
            for (int q = 0; q < R; ++q) {
                if (lin[q] && in_ok(t, oi[q]) && out_ok(t, oo[q])) {
                    if (t.esize == 4) static_cast<uint32_t*>(t.y)[oo[q]] = __ldg(static_cast<const uint32_t*>(t.x) + oi[q]);
                    else static_cast<uint16_t*>(t.y)[oo[q]] = __ldg(static_cast<const uint16_t*>(t.x) + oi[q]);
                }
            }
            const bool wi = ++ii == pi1, wo = ++io == po1;
            const int64_t di = wi ? si0 : si1, dout = wo ? so0 : so1;
            if (wi) ii = 0;
            if (wo) io = 0;
#pragma unroll
            for (int q = 0; q < R; ++q) oi[q] += di, oo[q] += dout;
        }
        return;
    }
    // FIR bank: y[j] = sum_k H[j,k] p[k], accumulated in k order with fma
    const int m = t.m;
    float acc[R][MAXM];
#pragma unroll
    for (int q = 0; q < R; ++q)
#pragma unroll
        for (int j = 0; j < MAXM; ++j) acc[q][j] = 0.f;
    const float* xf = static_cast<const float*>(t.x);
    int ii = 0;
    // unrolled: the loads of several tap indices are in flight together
#pragma unroll kGenUnroll
    for (int k = 0; k < n; ++k) {
        float h[MAXM];
        if (ht) {
            load_taps<MAXM>(ht + k * ((MAXM + 3) & ~3), h);
        } else {
#pragma unroll
            for (int j = 0; j < MAXM; ++j) h[j] = j < m ? __ldg(t.taps + (int64_t)j * n + k) : 0.f;
        }
        float p[R];
#pragma unroll
        for (int q = 0; q < R; ++q) {
            if (F32) p[q] = lin[q] && in_ok(t, oi[q]) ? __ldg(xf + oi[q]) : 0.f;
            else p[q] = lin[q] && in_ok(t, oi[q]) ? load_value(t, oi[q]) : 0.f;
        }
#pragma unroll
        for (int q = 0; q < R; ++q)
#pragma unroll
            for (int j = 0; j < MAXM; ++j)
                if (j < m) acc[q][j] = fmaf(h[j], p[q], acc[q][j]);
        const bool wi = ++ii == pi1;
        if (wi) ii = 0;
        const int64_t di = wi ? si0 : si1;
#pragma unroll
        for (int q = 0; q < R; ++q) oi[q] += di;
    }
    float* yf = static_cast<float*>(t.y);
#pragma unroll
    for (int q = 0; q < R; ++q) {
        if (!lin[q]) continue;
        int64_t cur = oo[q];
        int io = 0;
#pragma unroll
        for (int j = 0; j < MAXM; ++j) {
            if (j < m) {
                if (out_ok(t, cur)) {
                    if (F32) yf[cur] = acc[q][j];
                    else store_value(t, cur, acc[q][j]);
                }
                const bool wo = ++io == po1;
                if (wo) io = 0;
                cur += wo ? so0 : so1;
            }
        }
    }
}

// Blocks per SM the launch bound asks for: larger banks need more registers.
constexpr int gen_min_blocks(int maxm) { return maxm <= 4 ? AROL_GEN_MINB : maxm <= 8 ? 2 : 1; }

template <int MAXM, int R, bool F32>
__global__ void __launch_bounds__(kThreads, gen_min_blocks(MAXM)) tiler_tiled_kernel(const TaskDev t, const GenGeom g) {
    extern __shared__ __align__(16) float ht[];
    if (g.tap_floats) {
        const int n = t.T, m = t.m;
        for (int i = threadIdx.x; i < g.tap_floats; i += blockDim.x) {
            constexpr int kHs = (MAXM + 3) & ~3;   // 16-byte rows of taps
            const int k = i / kHs, j = i - k * kHs;
            ht[i] = j < m ? __ldg(t.taps + (int64_t)j * n + k) : 0.f;
        }
        __syncthreads();
    }
    const float* hts = g.tap_floats ? ht : nullptr;
    const uint32_t tb = 1u << g.lb;
    const uint32_t tx = threadIdx.x & (tb - 1u), ty = threadIdx.x >> g.lb;
    const uint32_t RA = g.da >= 0 ? (uint32_t)t.rep[g.da] : 1u, RB = (uint32_t)t.rep[g.db];
    const int qlim = g.da >= 0 ? g.da : g.db;   // dims below qlim come from the outer index
    for (uint32_t tile = blockIdx.x; tile < g.ntiles; tile += gridDim.x) {
        const uint32_t q1 = fast_div(tile, g.nb_div), ib = tile - q1 * g.nb;
        const uint32_t o = fast_div(q1, g.na_div), ia = q1 - o * g.na;
        // a tile covers R * tb repetitions along db: this thread's are bb, bb + tb, ...
        const uint32_t a = ia * (uint32_t)g.ta + ty, bb = ib * (uint32_t)R * tb + tx;
        if (a >= RA || bb >= RB) continue;
        const int nr = (int)min((uint32_t)R, (RB - bb + tb - 1u) >> g.lb);
        uint32_t r[4];
        uint32_t l = o;
#pragma unroll
        for (int q = 3; q >= 0; --q) {
            if (q == g.db) {
                r[q] = bb;
            } else if (q == g.da) {
                r[q] = a;
            } else if (q < qlim) {
                const uint32_t qq = fast_div(l, t.rep_div[q]);
                r[q] = l - qq * (uint32_t)t.rep[q];
                l = qq;
            } else {
                r[q] = 0;
            }
        }
        tiled_reps<MAXM, R, F32>(t, g, r, nr, hts);
    }
}

}  // namespace

int tiler_tiled_maxm(int max_m) {
    return max_m <= 3 ? (max_m < 1 ? 1 : max_m) : max_m <= 4 ? 4 : max_m <= 8 ? 8 : max_m <= 16 ? 16 : 32;
}
int tiler_tiled_reps(int max_m) { return max_m <= 8 ? AROL_GEN_R : max_m <= 16 ? 2 : 1; }

template <int MAXM, bool F32>
static cudaError_t launch_tiled_m(const TaskDev& t, const GenGeom& g, cudaStream_t s) {
    constexpr int R = MAXM <= 8 ? AROL_GEN_R : MAXM <= 16 ? 2 : 1;
    const size_t smem = (size_t)g.tap_floats * sizeof(float);
    static size_t attr = 0;
    if (smem > 48 * 1024 && smem > attr) {
        cudaError_t e = cudaFuncSetAttribute(tiler_tiled_kernel<MAXM, R, F32>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        attr = smem;
    }
    const int threads = g.ta << g.lb;
    int occ = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, tiler_tiled_kernel<MAXM, R, F32>, threads, smem);
    const int64_t cap = (int64_t)device_sm_count() * (occ > 0 ? occ : 1);
    const int grid = (int)std::min<int64_t>(g.ntiles, cap);
    tiler_tiled_kernel<MAXM, R, F32><<<grid, threads, smem, s>>>(t, g);
    return cudaGetLastError();
}

template <int MAXM>
static cudaError_t launch_tiled_dt(const TaskDev& t, const GenGeom& g, cudaStream_t s) {
    // f32 storage on both sides (or a copy): plain loads and stores
    if (t.elem == ELEM_COPY || (t.in_dt == kStF32 && t.out_dt == kStF32)) return launch_tiled_m<MAXM, true>(t, g, s);
    return launch_tiled_m<MAXM, false>(t, g, s);
}

cudaError_t launch_tiler_tiled(const TaskDev& t, const GenGeom& g, int max_m, cudaStream_t s) {
    if (t.nreps == 0 || g.ntiles == 0) return cudaSuccess;
    switch (tiler_tiled_maxm(max_m)) {
        case 1: return launch_tiled_dt<1>(t, g, s);
        case 2: return launch_tiled_dt<2>(t, g, s);
        case 3: return launch_tiled_dt<3>(t, g, s);
        case 4: return launch_tiled_dt<4>(t, g, s);
        case 8: return launch_tiled_dt<8>(t, g, s);
        case 16: return launch_tiled_dt<16>(t, g, s);
        default: return launch_tiled_dt<32>(t, g, s);
    }
}

}  // namespace arol
