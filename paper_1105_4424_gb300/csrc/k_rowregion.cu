// Row FIR in 16-word regions (Sec. 3 RSM tilers; a repetitive task mapped
// onto the GPU, Sec. 7): the row-FIR task
//
//     y[i, M r + j] = sum_{k < T} H[j, k] x[i, (o + S r + k) mod W]
//
// whose repetitions tile each row exactly (S R = W), with step S in {2, 4, 8},
// T <= 8, rows of a multiple of 16 words, origin o a multiple of 16, output
// rows of M R words starting at column 0, one output row per input row.
//
// One block of kRrThreads threads takes a row at a time; the rows reach
// shared memory by 16-byte cp.async copies in a ring of kRrStages stages
// (swizzled, with the 16-word halo of region.h), each stage with a "full"
// mbarrier (every thread's copies landed) and an "empty" one (every thread
// has computed the row), so warps run apart instead of meeting at block
// barriers twice per row (0.143 against 0.163 ms on 64 x 1080 x 1920); every
// wait is bounded and a wait that gives up sets the error word.  Thread t owns the home
// region h0 = (o + 16 t) mod W: the windows of repetitions NR t .. NR t + NR -
// 1 (NR = 16 / S) start there, so every window word is a compile-time offset
// from h0 and moves in 16-byte shared loads; the taps sit in registers; the
// NR M outputs are contiguous and leave as 16-byte (8-byte when NR M is not a
// multiple of 4) global stores.
#include <cuda_runtime.h>

#include "arol_internal.h"
#include "ptx.h"
#include "region.h"

namespace arol {
namespace {

#ifndef AROL_RR_STAGES
#define AROL_RR_STAGES 4
#endif
#ifndef AROL_RR_THREADS
#define AROL_RR_THREADS kRegionThreads
#endif
constexpr int kRrStages = AROL_RR_STAGES;
constexpr int kRrThreads = AROL_RR_THREADS;
constexpr int kRrTaps = 64;

template <int SS, int M>
__global__ void __launch_bounds__(kRrThreads) rowfir_region_kernel(int64_t rows, int W, int o, int T,
                                                                       const float* __restrict__ taps,
                                                                       const float* __restrict__ x,
                                                                       float* __restrict__ y, unsigned* err) {
    constexpr int TT = 8;
    constexpr int NR = 16 / SS;                     // repetitions per region
    constexpr int XW = (16 - SS + TT + 3) & ~3;     // window words of a region
    constexpr int NO = NR * M;                      // outputs of a region
    static_assert(XW <= 32 && NO % 2 == 0, "a window within two regions; outputs in pairs");
    extern __shared__ __align__(16) float rsm[];
    __shared__ __align__(8) uint64_t bars[2 * kRrStages];   // full, then empty, per stage
    const int nreg = W >> 4, Wout = M * (W / SS), stage = W + 16;
    float* const hs = rsm;
    float* const st0 = rsm + kRrTaps;
    const uint32_t full0 = ptx::smem_addr(bars), empty0 = ptx::smem_addr(bars + kRrStages);
    for (int i = threadIdx.x; i < M * T; i += blockDim.x) hs[i] = __ldg(taps + i);
    if (threadIdx.x == 0) {
        for (int q = 0; q < 2 * kRrStages; ++q) ptx::mbar_init(full0 + 8 * q, blockDim.x);
        ptx::fence_barrier_init();
    }
    __syncthreads();   // the taps and the barriers
    // stage q's "full" phase k completes when every thread's copies of the
    // block's row q + k kRrStages have landed (one cp.async arrival per
    // thread); its "empty" phase k when every thread has computed that row
    const int64_t G = gridDim.x;
    for (int i = 0; i < kRrStages - 1; ++i) {
        const int64_t rr = blockIdx.x + i * G;
        if (rr < rows) {
            stage_region_row(st0 + i * stage, x + rr * W, W);
            asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];" ::"r"(full0 + 8 * i) : "memory");
        }
    }
    float h[M][TT];    // zero past T (those terms are skipped below)
#pragma unroll
    for (int j = 0; j < M; ++j)
#pragma unroll
        for (int k = 0; k < TT; ++k) h[j][k] = k < T ? hs[j * T + k] : 0.f;
    int b = 0;
    uint32_t it = 0;
    for (int64_t row = blockIdx.x; row < rows; row += G, ++it) {
        // refill the stage of the previous row with the row kRrStages - 1
        // ahead, once every thread has computed that previous row
        const int64_t ahead = row + (kRrStages - 1) * G;
        if (ahead < rows) {
            const int sf = b == 0 ? kRrStages - 1 : b - 1;
            if (it >= 1 && !ptx::mbar_wait(empty0 + 8 * sf, ((it - 1) / kRrStages) & 1u)) {
                if (err) atomicOr(err, 1u);
                break;
            }
            stage_region_row(st0 + sf * stage, x + ahead * W, W);
            asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];" ::"r"(full0 + 8 * sf) : "memory");
        }
        if (!ptx::mbar_wait(full0 + 8 * b, (it / kRrStages) & 1u)) {
            if (err) atomicOr(err, 2u);
            break;
        }
        const float* xs = st0 + b * stage;
        float* yr = y + row * Wout;
        for (int t = threadIdx.x; t < nreg; t += blockDim.x) {
            int h0 = o + 16 * t;
            if (h0 >= W) h0 -= W;
            const int u0 = h0 >> 2;
            float xw[XW];
#pragma unroll
            for (int v = 0; v < XW / 4; ++v) {
                const float4 q = *reinterpret_cast<const float4*>(xs + 4 * region_unit(u0 + v));
                xw[4 * v] = q.x;
                xw[4 * v + 1] = q.y;
                xw[4 * v + 2] = q.z;
                xw[4 * v + 3] = q.w;
            }
            float out[NO];
#pragma unroll
            for (int i = 0; i < NR; ++i)
#pragma unroll
                for (int j = 0; j < M; ++j) {
                    float a = 0.f;
#pragma unroll
                    for (int k = 0; k < TT; ++k)
                        if (k < T) a = fmaf(h[j][k], xw[SS * i + k], a);
                    out[M * i + j] = a;
                }
            float* yo = yr + NO * t;
            if constexpr (NO % 4 == 0) {
#pragma unroll
                for (int v = 0; v < NO / 4; ++v)
                    reinterpret_cast<float4*>(yo)[v] = make_float4(out[4 * v], out[4 * v + 1], out[4 * v + 2], out[4 * v + 3]);
            } else {
#pragma unroll
                for (int v = 0; v < NO / 2; ++v) reinterpret_cast<float2*>(yo)[v] = make_float2(out[2 * v], out[2 * v + 1]);
            }
        }
        ptx::mbar_arrive(empty0 + 8 * b);
        if (++b == kRrStages) b = 0;
    }
    ptx::cp_async_wait_all();
}

using RegionKernel = void (*)(int64_t, int, int, int, const float*, const float*, float*, unsigned*);

RegionKernel region_kernel(int S, int M) {
    if (S == 2) return M == 1 ? rowfir_region_kernel<2, 1> : rowfir_region_kernel<2, 2>;
    if (S == 4)
        return M == 1 ? rowfir_region_kernel<4, 1>
                      : M == 2 ? rowfir_region_kernel<4, 2> : M == 3 ? rowfir_region_kernel<4, 3> : rowfir_region_kernel<4, 4>;
    return M == 1 ? rowfir_region_kernel<8, 1>
                  : M == 2 ? rowfir_region_kernel<8, 2> : M == 3 ? rowfir_region_kernel<8, 3> : rowfir_region_kernel<8, 4>;
}

size_t region_smem(int W) { return sizeof(float) * ((size_t)kRrTaps + (size_t)kRrStages * (W + 16)); }

constexpr size_t kRegionSmemMax = 96 * 1024;

}  // namespace

bool rowfir_region_supported(int S, int T, int M, int64_t W, int64_t Wout, int64_t o, int64_t rows) {
    if (!(S == 2 || S == 4 || S == 8) || T < 1 || T > 8 || M < 1 || M > (S == 2 ? 2 : 4)) return false;
    if (W % 16 || W < 16 || o % 16 || o < 0 || o >= W || Wout != M * (W / S) || rows < 1) return false;
    return W < (1 << 24) && region_smem((int)W) <= kRegionSmemMax;
}

cudaError_t launch_rowfir_region(int S, int T, int M, int64_t rows, int W, int o, const float* taps, const float* x,
                                 float* y, unsigned* err, cudaStream_t s) {
    static bool opted = false;
    if (!opted) {
        for (int ss : {2, 4, 8})
            for (int mm = 1; mm <= (ss == 2 ? 2 : 4); ++mm)
                cudaFuncSetAttribute(region_kernel(ss, mm), cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kRegionSmemMax);
        opted = true;
    }
    const size_t smem = region_smem(W);
    const RegionKernel k = region_kernel(S, M);
    int n = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k, kRrThreads, smem);
    const int64_t cap = (int64_t)device_sm_count() * (n > 0 ? n : 1);
    const int grid = (int)(rows < cap ? rows : cap);
    k<<<grid, kRrThreads, smem, s>>>(rows, W, o, T, taps, x, y, err);
    return cudaGetLastError();
}

}  // namespace arol
