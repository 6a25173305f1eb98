// Fused chains of separable FIR passes (row and column passes, any taps,
// outputs, step and origin, wrap included): the general form of the chained
// downscaler (Sec. 5 associatedParts; repetitive tasks on the GPU, Sec. 7).
//
// One CTA per tile of the last stage.  It loads the tile's stage-0 window
// (rows and columns from sep_regions, wrapped at the array edges) into shared
// memory, then runs the passes in order between two shared buffers; the last
// pass writes the tile to global memory.  The intermediate arrays never
// reach HBM: only halos (the T - S overlap of neighbouring tiles' windows)
// are read twice, mostly from L2.
//
// A pass's thread computes all m outputs of one repetition (one row of a row
// pass, one column of a column pass), the m accumulators in registers (m is a
// template parameter), the taps in shared memory (one broadcast load per tap
// and output).  Column passes give consecutive threads consecutive columns:
// conflict-free shared loads and coalesced global stores.
#include "arol_internal.h"
#include "sepchain.h"

namespace arol {
namespace {

constexpr int kSepThreads = 256;

__device__ __forceinline__ int wrap_pos(int v, int n) {
    while (v >= n) v -= n;
    return v;
}

// Row pass k: input region (rows ri, cols ci) in `in` (row stride ci.len),
// output region (rows ri, cols co) to `out` (row stride ldo; a global tile
// when `global`).
template <int M>
__device__ void row_pass(const SepPassDev& p, const float* hk, const float* in, SepRange ri, SepRange ci,
                         SepRange co, float* out, int64_t ldo) {
    const int ra = co.start / M;   // the first output position is < n_out
    const int nrep = sep_urep(p, co.start + co.len - 1) - ra + 1;
    const int n = ri.len * nrep;
    for (int e = threadIdx.x; e < n; e += blockDim.x) {
        const int i = e / nrep, ur = ra + (e - i * nrep);
        const int r = ur % p.R;
        int base = (int)(((int64_t)p.o + (int64_t)p.S * r - ci.start) % p.n_in);
        if (base < 0) base += p.n_in;
        const float* src = in + (int64_t)i * ci.len + base;
        float acc[M];
#pragma unroll
        for (int j = 0; j < M; ++j) acc[j] = 0.f;
        for (int kk = 0; kk < p.T; ++kk) {
            const float v = src[kk];
#pragma unroll
            for (int j = 0; j < M; ++j) acc[j] = fmaf(hk[j * p.T + kk], v, acc[j]);
        }
        const int q0 = sep_upos(p, ur) - co.start;
#pragma unroll
        for (int j = 0; j < M; ++j) {
            const int q = q0 + j;
            if (q >= 0 && q < co.len) out[(int64_t)i * ldo + q] = acc[j];
        }
    }
}

// Column pass k: input region (rows ri, cols ci), output region (rows ro,
// cols ci).
template <int M>
__device__ void col_pass(const SepPassDev& p, const float* hk, const float* in, SepRange ri, SepRange ci,
                         SepRange ro, float* out, int64_t ldo) {
    const int ra = ro.start / M;
    const int nrep = sep_urep(p, ro.start + ro.len - 1) - ra + 1;
    const int n = nrep * ci.len;
    for (int e = threadIdx.x; e < n; e += blockDim.x) {
        const int rr = e / ci.len, q = e - rr * ci.len;
        const int ur = ra + rr;
        const int r = ur % p.R;
        int base = (int)(((int64_t)p.o + (int64_t)p.S * r - ri.start) % p.n_in);
        if (base < 0) base += p.n_in;
        const float* src = in + (int64_t)base * ci.len + q;
        float acc[M];
#pragma unroll
        for (int j = 0; j < M; ++j) acc[j] = 0.f;
        for (int kk = 0; kk < p.T; ++kk) {
            const float v = src[(int64_t)kk * ci.len];
#pragma unroll
            for (int j = 0; j < M; ++j) acc[j] = fmaf(hk[j * p.T + kk], v, acc[j]);
        }
        const int i0 = sep_upos(p, ur) - ro.start;
#pragma unroll
        for (int j = 0; j < M; ++j) {
            const int i = i0 + j;
            if (i >= 0 && i < ro.len) out[(int64_t)i * ldo + q] = acc[j];
        }
    }
}

template <bool kRow>
__device__ void run_pass(const SepPassDev& p, const float* hk, const float* in, SepRange ri, SepRange ci, SepRange ro,
                         SepRange co, float* out, int64_t ldo) {
#define AROL_SEP_CASE(M)                                              \
    case M:                                                           \
        if (kRow) row_pass<M>(p, hk, in, ri, ci, co, out, ldo);      \
        else col_pass<M>(p, hk, in, ri, ci, ro, out, ldo);           \
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

__global__ void __launch_bounds__(kSepThreads) sepchain_kernel(const SepChainDev d) {
    extern __shared__ __align__(16) float ssm[];
    float* taps = ssm;
    float* buf[2] = {ssm + ((d.ntaps + 3) & ~3), ssm + ((d.ntaps + 3) & ~3) + d.buf};
    for (int i = threadIdx.x; i < d.ntaps; i += blockDim.x) taps[i] = __ldg(d.taps + i);
    const int K = d.K;
    const int64_t ntile = (int64_t)d.tiles_y * d.tiles_x;
    for (int64_t t = blockIdx.x; t < d.F * ntile; t += gridDim.x) {
        const int64_t f = t / ntile;
        const int tt = (int)(t - f * ntile);
        const int ty = tt / d.tiles_x, tx = tt - ty * d.tiles_x;
        SepRange rows[kSepMaxPasses + 1], cols[kSepMaxPasses + 1];
        sep_regions(d, ty, tx, rows, cols);
        // stage 0 window: rows (rs + i) mod H0, columns (cs + q) mod W0
        {
            const float* xf = d.x + f * (int64_t)d.H[0] * d.W[0];
            const int nr = rows[0].len, nc = cols[0].len;
            float* dst = buf[0];
            for (int e = threadIdx.x; e < nr * nc; e += blockDim.x) {
                const int i = e / nc, q = e - i * nc;
                const int gr = wrap_pos(rows[0].start + i, d.H[0]), gc = wrap_pos(cols[0].start + q, d.W[0]);
                dst[e] = __ldg(xf + (int64_t)gr * d.W[0] + gc);
            }
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < kSepMaxPasses; ++k) {
            if (k >= K) break;
            const SepPassDev& p = d.p[k];
            const float* in = buf[k & 1];
            float* out;
            int64_t ldo;
            if (k + 1 == K) {
                out = d.y + (f * d.H[K] + rows[K].start) * (int64_t)d.W[K] + cols[K].start;
                ldo = d.W[K];
            } else {
                out = buf[(k + 1) & 1];
                ldo = cols[k + 1].len;
            }
            if (p.axis == 1) run_pass<true>(p, taps + p.tap_off, in, rows[k], cols[k], rows[k + 1], cols[k + 1], out, ldo);
            else run_pass<false>(p, taps + p.tap_off, in, rows[k], cols[k], rows[k + 1], cols[k + 1], out, ldo);
            __syncthreads();
        }
    }
}

}  // namespace

size_t sepchain_smem(const SepChainDev& d) {
    return ((size_t)((d.ntaps + 3) & ~3) + 2 * (size_t)d.buf) * sizeof(float);
}

cudaError_t launch_sepchain(const SepChainDev& d, cudaStream_t s) {
    const int64_t work = d.F * (int64_t)d.tiles_y * d.tiles_x;
    if (work <= 0) return cudaSuccess;
    const size_t smem = sepchain_smem(d);
    static size_t attr = 0;
    if (smem > attr) {
        cudaError_t e = cudaFuncSetAttribute(sepchain_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        attr = smem;
    }
    int occ = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, sepchain_kernel, kSepThreads, smem);
    if (occ < 1) occ = 1;
    const int64_t cap = (int64_t)device_sm_count() * occ;
    sepchain_kernel<<<(int)(work < cap ? work : cap), kSepThreads, smem, s>>>(d);
    return cudaGetLastError();
}

}  // namespace arol
