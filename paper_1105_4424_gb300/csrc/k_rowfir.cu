// Row-FIR tiles of a batch: the repetitive task whose input tiler walks one
// row per repetition row r0 with step S along it (paving [[1,0],[0,S]],
// fitting [[0],[1]], a T-element pattern that wraps at the row's end) and
// whose output tiler writes M consecutive elements per repetition (Sec. 3
// RSM tilers; repetitive tasks mapped onto the GPU, Sec. 7):
//
//     y[r0, M r1 + j] = sum_{k < T} H[j, k] x[r0, (o1 + S r1 + k) mod W]
//
// A tile is `nrows` consecutive rows times `cnt` consecutive repetitions of
// each row.  Its input is the window of S (cnt - 1) + T words of every row,
// wrap included.
//
// One producer warp streams tiles into a ring of shared-memory stages: each
// row's contiguous part by one cp.async.bulk (16-byte aligned interior), the
// few words that wrap around the row's end or straddle a 16-byte boundary by
// 4-byte cp.async tracked on the same mbarrier, the task's transposed taps by
// one more bulk copy.  Consumer warps compute from shared memory and write
// their outputs straight from registers; a warp gives its stage back on the
// stage's "empty" mbarrier.
//
// Bank spreading.  A bulk copy keeps an element's address modulo 16 bytes,
// so the low two bits of a word's shared index are its global ones.  Row
// slot k starts at a shared index congruent to 4 ((k >> 2) & 7) modulo 32,
// and a warp covers a rows x 32/a consecutive repetitions: lanes at stride S
// within a row fill one coset of gcd(S, 32), the rows the others (the host
// picks a).  In the tap loop every lane then reads word `kk` past its own
// base: immediate offsets, no per-tap address arithmetic.
#include "arol_internal.h"
#include "ptx.h"

namespace arol {
namespace {

constexpr int kRfCWarps = 4;                        // consumer warps
constexpr int kRfThreads = (kRfCWarps + 1) * 32;   // + one producer warp
constexpr int kRfStages = 4;
constexpr int kRfHdrFloats = 32;                    // the tile record (96 bytes), padded
constexpr int kRfTapFloats = 32 * 16;               // transposed taps, T <= 32
constexpr int kRfSlotBase = kRfHdrFloats + kRfTapFloats;
static_assert(sizeof(RowTileDev) == 96, "tile record is six 16-byte words");
static_assert(kRowStageFloats - kRfSlotBase >= kRowSlotFloats + 28, "slot area: nrows * ss plus the spreading offsets");

__device__ __forceinline__ void flag(unsigned* err, unsigned bit) {
    if (err) atomicOr(err, bit);
}

// Shared offset of row slot k (k < 32; ss a multiple of 32): congruent to
// 4 ((k >> 2) & 7) modulo 32, and increasing with k by at least ss, so slots
// never overlap (a tile's slots span nrows * ss + 28 floats).
__device__ __forceinline__ int slot_offset(int k, int ss) { return k * ss + 4 * (k >> 2); }

__device__ __forceinline__ RowTileDev load_tile(const RowTileDev* p) {
    RowTileDev r;
    const uint4* s = reinterpret_cast<const uint4*>(p);
    uint4* d = reinterpret_cast<uint4*>(&r);
#pragma unroll
    for (int i = 0; i < 6; ++i) d[i] = __ldg(s + i);
    return r;
}

template <int M>
__device__ __forceinline__ void load_taps(const float* hrow, float (&h)[M]) {
#pragma unroll
    for (int j = 0; j + 4 <= M; j += 4) {
        const float4 v = *reinterpret_cast<const float4*>(hrow + j);
        h[j] = v.x;
        h[j + 1] = v.y;
        h[j + 2] = v.z;
        h[j + 3] = v.w;
    }
    constexpr int j0 = M / 4 * 4;
    if (M - j0 >= 2) {
        const float2 v = *reinterpret_cast<const float2*>(hrow + j0);
        h[j0] = v.x;
        h[j0 + 1] = v.y;
    }
    if ((M - j0) & 1) h[M - 1] = hrow[M - 1];
}

struct UnitPos {
    bool valid;
    int k, j;   // row of the tile, repetition of the row
};

__device__ __forceinline__ UnitPos unit_pos(int u, int nb, int la, int kl, int jl, int nrows, int cnt) {
    UnitPos p;
    const int g = u / nb, blk = u - g * nb;
    p.k = (g << la) + kl;
    p.j = (blk << (5 - la)) + jl;
    p.valid = p.k < nrows && p.j < cnt;
    return p;
}

// Shared address (floats from the slot area) of window word 0 of repetition
// j of row k.
__device__ __forceinline__ int unit_base(const RowTileDev& h, int k, int j) {
    int ir = h.row0 + k;
    if (ir >= h.H) ir -= h.H;
    const uint64_t g = ((uint64_t)reinterpret_cast<uintptr_t>(h.x) >> 2) + (uint64_t)ir * (uint32_t)h.W + (uint32_t)h.c0;
    return slot_offset(k, h.ss) + (int)(g & 3u) + h.S * j;
}

template <int M>
__device__ __forceinline__ void store_unit(const RowTileDev& h, int k, int j, const float (&acc)[M]) {
    int orow = h.orow0 + k;
    if (orow >= h.Hout) orow -= h.Hout;
    float* yr = h.y + (int64_t)orow * h.Wout;
    int c = h.oc0 + M * j;
    if (!h.out_wrap) {
#pragma unroll
        for (int jj = 0; jj < M; ++jj) yr[c + jj] = acc[jj];
        return;
    }
    if (c >= h.Wout) c -= h.Wout;
#pragma unroll
    for (int jj = 0; jj < M; ++jj) {
        yr[c] = acc[jj];
        c = c + 1 == h.Wout ? 0 : c + 1;
    }
}

// Consumer warp `warp`: units warp, warp + kRfCWarps, ... of the tile, two at
// a time (they share every tap load).  A unit is a rows x 32/a repetitions;
// lanes past the tile's edge compute from slot 0 and store nothing.
template <int M>
__device__ __forceinline__ void tile_compute(const RowTileDev& h, const float* stage, int warp, int lane) {
    const float* ht = stage + kRfHdrFloats;
    const float* slots = stage + kRfSlotBase;
    const int la = __ffs(h.a) - 1;                // a = 2^la rows per unit
    const int kl = lane >> (5 - la), jl = lane & ((32 >> la) - 1);
    const int nb = (h.cnt + (32 >> la) - 1) >> (5 - la);
    const int U = ((h.nrows + h.a - 1) >> la) * nb;
    const int T = h.T;
    for (int u0 = warp; u0 < U; u0 += 2 * kRfCWarps) {
        const int u1 = u0 + kRfCWarps;
        const UnitPos p0 = unit_pos(u0, nb, la, kl, jl, h.nrows, h.cnt);
        const UnitPos p1 = u1 < U ? unit_pos(u1, nb, la, kl, jl, h.nrows, h.cnt) : UnitPos{false, 0, 0};
        const float* w0 = slots + (p0.valid ? unit_base(h, p0.k, p0.j) : 0);
        const float* w1 = slots + (p1.valid ? unit_base(h, p1.k, p1.j) : 0);
        float acc0[M], acc1[M];
#pragma unroll
        for (int j = 0; j < M; ++j) acc0[j] = acc1[j] = 0.f;
#pragma unroll 4
        for (int kk = 0; kk < T; ++kk) {
            const float v0 = w0[kk], v1 = w1[kk];
            float hh[M];
            load_taps<M>(ht + kk * 16, hh);
#pragma unroll
            for (int j = 0; j < M; ++j) {
                acc0[j] = fmaf(hh[j], v0, acc0[j]);
                acc1[j] = fmaf(hh[j], v1, acc1[j]);
            }
        }
        if (p0.valid) store_unit<M>(h, p0.k, p0.j, acc0);
        if (p1.valid) store_unit<M>(h, p1.k, p1.j, acc1);
    }
}

__device__ __forceinline__ void tile_dispatch(const RowTileDev& h, const float* stage, int warp, int lane) {
#define AROL_RF_CASE(M) \
    case M: tile_compute<M>(h, stage, warp, lane); break;
    switch (h.M) {
        AROL_RF_CASE(1) AROL_RF_CASE(2) AROL_RF_CASE(3) AROL_RF_CASE(4)
        AROL_RF_CASE(5) AROL_RF_CASE(6) AROL_RF_CASE(7) AROL_RF_CASE(8)
        AROL_RF_CASE(9) AROL_RF_CASE(10) AROL_RF_CASE(11) AROL_RF_CASE(12)
        AROL_RF_CASE(13) AROL_RF_CASE(14) AROL_RF_CASE(15) AROL_RF_CASE(16)
        default: break;
    }
#undef AROL_RF_CASE
}

// Producer: issues the copies of one tile into `stage` (shared address
// `stage_s`), completing on mbarrier `full`.  Lane k < nrows handles row k.
__device__ __forceinline__ void produce_tile(const RowTileDev& h, float* stage, uint32_t full, int lane) {
    const uintptr_t xs = reinterpret_cast<uintptr_t>(h.x);
    const uintptr_t xe = xs + (uintptr_t)h.H * (uintptr_t)h.W * 4u;
    uint32_t bulk_bytes = 0;
    uint32_t dst_s = 0;
    uintptr_t gA = 0;
    if (lane < h.nrows) {
        int ir = h.row0 + lane;
        if (ir >= h.H) ir -= h.H;
        const float* row = h.x + (int64_t)ir * h.W;
        const uintptr_t a0 = reinterpret_cast<uintptr_t>(row + h.c0);
        const int delta = (int)((a0 >> 2) & 3u);
        float* slot = stage + kRfSlotBase + slot_offset(lane, h.ss);   // word w of the window at slot[delta + w]
        const int L1 = min(h.lw, h.W - h.c0);                          // the run before the row's end
        const uintptr_t a1 = a0 + 4u * (uintptr_t)L1;
        gA = a0 & ~(uintptr_t)15;
        if (gA < xs) gA += 16;
        uintptr_t gB = (a1 + 15) & ~(uintptr_t)15;
        if (L1 < h.lw || gB > xe) gB = a1 & ~(uintptr_t)15;   // wrapped words follow, or the array ends
        if (gB <= gA) gA = gB = a0;                              // nothing to bulk-copy
        // 4-byte copies: the run's words outside [gA, gB), then the wrapped words
        for (uintptr_t g = a0; g < gA; g += 4) {
            const int w = (int)((g - a0) >> 2);
            ptx::cp_async4(slot + delta + w, row + h.c0 + w);
        }
        for (uintptr_t g = gB > a0 ? gB : a0; g < a1; g += 4) {
            const int w = (int)((g - a0) >> 2);
            ptx::cp_async4(slot + delta + w, row + h.c0 + w);
        }
        int col = h.c0 + L1 - h.W;   // 0 when the window wraps
        for (int w = L1; w < h.lw; ++w) {
            while (col >= h.W) col -= h.W;
            ptx::cp_async4(slot + delta + w, row + col);
            ++col;
        }
        bulk_bytes = (uint32_t)(gB - gA);
        dst_s = ptx::smem_addr(slot) + (uint32_t)(gA - (a0 & ~(uintptr_t)15));
    }
    // the mbarrier tracks this lane's 4-byte copies (net zero on its count)
    asm volatile("cp.async.mbarrier.arrive.shared::cta.b64 [%0];" ::"r"(full) : "memory");
    uint32_t total = bulk_bytes;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) total += __shfl_xor_sync(0xffffffffu, total, off);
    const uint32_t tap_bytes = (uint32_t)h.T * 16u * 4u;
    __syncwarp();
    if (lane == 0) {
        // the tile record for the consumers, then the stage's single arrival
        const uint4* src = reinterpret_cast<const uint4*>(&h);
        uint4* dst = reinterpret_cast<uint4*>(stage);
#pragma unroll
        for (int i = 0; i < 6; ++i) dst[i] = src[i];
        ptx::mbar_expect_tx(full, total + tap_bytes);
    }
    __syncwarp();
    if (bulk_bytes) ptx::bulk_g2s(dst_s, reinterpret_cast<const void*>(gA), bulk_bytes, full);
    if (lane == 0) ptx::bulk_g2s(ptx::smem_addr(stage + kRfHdrFloats), h.taps_t, tap_bytes, full);
}

// Persistent over the tile list: CTA b takes tiles b, b + gridDim.x, ...
__global__ void __launch_bounds__(kRfThreads, 2) rowfir_batch_kernel(const RowTileDev* __restrict__ tiles, int ntiles,
                                                                    unsigned* err) {
    extern __shared__ __align__(128) float rsm[];
    uint64_t* bars = reinterpret_cast<uint64_t*>(rsm + kRfStages * kRowStageFloats);
    const uint32_t full0 = ptx::smem_addr(bars), empty0 = ptx::smem_addr(bars + kRfStages);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int st = 0; st < kRfStages; ++st) {
            ptx::mbar_init(full0 + 8 * st, 1);
            ptx::mbar_init(empty0 + 8 * st, kRfCWarps);
        }
        ptx::fence_barrier_init();
    }
    __syncthreads();
    const int G = gridDim.x;
    if (warp == kRfCWarps) {
        int last[kRfStages];
#pragma unroll
        for (int st = 0; st < kRfStages; ++st) last[st] = -1;
        RowTileDev nxt;
        if ((int)blockIdx.x < ntiles) nxt = load_tile(tiles + blockIdx.x);
        int i = 0;
        for (int t = blockIdx.x; t < ntiles; t += G, ++i) {
            const int st = i % kRfStages;
            if (i >= kRfStages && !ptx::mbar_wait(empty0 + 8 * st, ((uint32_t)(i / kRfStages) & 1u) ^ 1u)) {
                if (lane == 0) flag(err, 1u);
                break;
            }
            const RowTileDev cur = nxt;
            if (t + G < ntiles) nxt = load_tile(tiles + t + G);
            produce_tile(cur, rsm + st * kRowStageFloats, full0 + 8 * st, lane);
            last[st] = i;
        }
        // every issued copy lands before the CTA's shared memory goes away
#pragma unroll
        for (int st = 0; st < kRfStages; ++st)
            if (last[st] >= 0 && !ptx::mbar_wait(full0 + 8 * st, ((uint32_t)last[st] / kRfStages) & 1u) && lane == 0)
                flag(err, 4u);
        ptx::cp_async_wait_all();
        return;
    }
    int i = 0;
    for (int t = blockIdx.x; t < ntiles; t += G, ++i) {
        const int st = i % kRfStages;
        if (!ptx::mbar_wait(full0 + 8 * st, (uint32_t)(i / kRfStages) & 1u)) {
            if (lane == 0) flag(err, 2u);
            break;
        }
        const float* stage = rsm + st * kRowStageFloats;
        const RowTileDev h = *reinterpret_cast<const RowTileDev*>(stage);
        tile_dispatch(h, stage, warp, lane);
        __syncwarp();
        if (lane == 0) ptx::mbar_arrive(empty0 + 8 * st);
    }
}

size_t rowfir_smem() { return (size_t)kRfStages * kRowStageFloats * sizeof(float) + 2 * kRfStages * sizeof(uint64_t); }

}  // namespace

int rowfir_ctas_per_sm() {
    static int occ = 0;
    if (!occ) {
        const size_t smem = rowfir_smem();
        cudaFuncSetAttribute(rowfir_batch_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        int n = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, rowfir_batch_kernel, kRfThreads, smem);
        occ = n > 0 ? n : 1;
    }
    return occ;
}

cudaError_t launch_rowfir_batch(const RowTileDev* tiles, int ntiles, int grid, unsigned* err, cudaStream_t s) {
    if (ntiles <= 0) return cudaSuccess;
    const int cap = device_sm_count() * rowfir_ctas_per_sm();
    if (grid <= 0 || grid > cap) grid = cap;
    if (grid > ntiles) grid = ntiles;
    rowfir_batch_kernel<<<grid, kRfThreads, rowfir_smem(), s>>>(tiles, ntiles, err);
    return cudaGetLastError();
}

}  // namespace arol
