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
// Two producer warps stream tiles into a ring of shared-memory stages: each
// row's contiguous part by one cp.async.bulk (16-byte aligned interior), the
// few words that wrap around the row's end or straddle a 16-byte boundary by
// 4-byte cp.async tracked on the same mbarrier, the task's transposed taps
// and the tile record by two more bulk copies.  Each consumer warp computes
// whole tiles from shared memory (per-tile set-up paid once per tile) and
// writes its outputs straight from registers; it gives the stage back on the
// stage's "empty" mbarrier.
//
// Bank spreading.  A bulk copy keeps an element's address modulo 16 bytes,
// so the low two bits of a word's shared index are its global ones.  Row
// slot k starts at a shared index congruent to 4 ((k >> 2) & 7) modulo 32,
// and a warp covers a rows x 32/a consecutive repetitions: lanes at stride S
// within a row fill one coset of gcd(S, 32), the rows the others (the host
// picks a).  In the tap loop every lane then reads word `kk` past its own
// base: immediate offsets, no per-tap address arithmetic.
#include <cuda_runtime.h>

#include "arol_internal.h"
#include "ptx.h"

namespace arol {
namespace {

#ifndef AROL_ROW_SHARE
#define AROL_ROW_SHARE 2
#endif
#ifndef AROL_ROW_UNROLL
#define AROL_ROW_UNROLL 4
#endif
constexpr int kRfShare = AROL_ROW_SHARE;            // consumer warps per tile
constexpr int kRfUnroll = AROL_ROW_UNROLL;          // tap-loop unroll
constexpr int kRfGroups = 4;                        // consumer groups (kRfShare warps each)
constexpr int kRfCWarps = kRfGroups * kRfShare;     // consumer warps
constexpr int kRfPWarps = 2;                        // producer warps
constexpr int kRfThreads = (kRfCWarps + kRfPWarps) * 32;
constexpr int kRfStages = 2 * kRfGroups;            // two per consumer group
constexpr int kRfRecs = 8;                         // tile records read ahead by the producers
static_assert(kRfRecs % kRfPWarps == 0 && kRfStages % kRfPWarps == 0, "each producer owns its stages and slots");
// Stage layout (floats): the tile record, the row table, the row slots, and
// at the stage's end the tile's taps (T x 32: transposed, each twice).
constexpr int kRfRecFloats = 32;                    // the tile record (96 bytes), padded
constexpr int kRfRowFloats = 32 * 4;                // the row table: one RowInfo per row
constexpr int kRfSlotBase = kRfRecFloats + kRfRowFloats;

// Row k of a tile, written by the producer: where its window starts in the
// slot area and where its output row starts.
struct RowInfo {
    int32_t base;   // shared offset (floats from the slot area) of window word 0
    int32_t pad_;
    float* out;     // output row (oo0 + r0 + k) mod Hout
};
static_assert(sizeof(RowInfo) == 16, "row table entries are 16 bytes");
static_assert(sizeof(RowTileDev) == 96, "tile record is six 16-byte words");
// (a tile of T taps has at most kRowSlotFloats - 32 (T - 1) slot floats)
static_assert(kRowStageFloats - kRfSlotBase - 32 >= kRowSlotFloats + 28,
              "slots of nrows * ss floats plus the spreading offsets, then the taps");
static_assert(kRfSlotBase % 4 == 0 && kRowStageFloats % 4 == 0, "16-byte aligned stage regions");

// Where a tile's taps start in its stage.
__device__ __forceinline__ float* stage_taps(float* stage, int T) { return stage + kRowStageFloats - 32 * T; }
__device__ __forceinline__ const float* stage_taps(const float* stage, int T) { return stage + kRowStageFloats - 32 * T; }

__device__ __forceinline__ void flag(unsigned* err, unsigned bit) {
    if (err) atomicOr(err, bit);
}

// Shared offset of row slot k (k < 32; ss a multiple of 32): congruent to
// 4 ((k >> 2) & 7) modulo 32, and increasing with k by at least ss, so slots
// never overlap (a tile's slots span nrows * ss + 28 floats).
__device__ __forceinline__ int slot_offset(int k, int ss) { return k * ss + 4 * (k >> 2); }

// Per-tile constants of a consumer warp.
struct TileGeom {
    int la;        // a = 2^la rows per unit
    int b;         // repetitions per unit row: 32 / a
    int kl, jl;    // this lane's row and repetition within a unit
    int nb;        // unit columns: ceil(cnt / b)
    int U;         // units: ceil(nrows / a) * nb
};

__device__ __forceinline__ TileGeom tile_geom(const RowTileDev& h, int lane) {
    TileGeom g;
    g.la = __ffs(h.a) - 1;
    g.b = 32 >> g.la;
    g.kl = lane >> (5 - g.la);
    g.jl = lane & (g.b - 1);
    g.nb = (h.cnt + g.b - 1) >> (5 - g.la);
    g.U = ((h.nrows + h.a - 1) >> g.la) * g.nb;
    return g;
}

// This lane's repetition of unit (grp, blk): its window in shared memory
// and its first output (with columns that wrap: the row and the column).
struct UnitPos {
    bool valid;
    int base;
    float* out;
    int col;
};

__device__ __forceinline__ UnitPos unit_pos(const RowTileDev& h, const TileGeom& g, const RowInfo* rows, int grp,
                                            int blk) {
    UnitPos p;
    const int k = (grp << g.la) + g.kl, j = blk * g.b + g.jl;
    p.valid = k < h.nrows && j < h.cnt;
    const RowInfo ri = rows[k & 31];
    p.base = p.valid ? ri.base + h.S * j : 0;
    const int c = h.oc0 + h.M * j;
    p.out = h.out_wrap ? ri.out : ri.out + c;
    p.col = c;
    return p;
}

// Outputs j0 .. j0 + G - 1 of one unit.
template <int G>
__device__ __forceinline__ void store_group(const RowTileDev& h, const UnitPos& p, int j0, const float* acc) {
    if (!h.out_wrap) {
#pragma unroll
        for (int jj = 0; jj < G; ++jj) p.out[j0 + jj] = acc[jj];
        return;
    }
    int c = p.col + j0;
    while (c >= h.Wout) c -= h.Wout;
#pragma unroll
    for (int jj = 0; jj < G; ++jj) {
        p.out[c] = acc[jj];
        c = c + 1 == h.Wout ? 0 : c + 1;
    }
}

// Outputs j0 .. j0 + G - 1 of R units (R even): the units go in pairs
// through paired FP32 FMAs (each lane of a pair rounds like fmaf), the
// window words of a pair's two units form one operand, and the taps are
// stored twice in a row (ht[kk * 32 + 2 j + e] = H[j, kk], e = 0, 1) so that
// one shared load gives a tap as a pair.  The R units share every tap load.
template <int G, int R>
__device__ __forceinline__ void unit_group(const RowTileDev& h, const UnitPos (&p)[R], const float* const (&w)[R],
                                           const float* ht, int j0) {
    static_assert(R % 2 == 0, "units go in pairs");
    constexpr int P = R / 2;
    float2 acc[P][G];
#pragma unroll
    for (int q = 0; q < P; ++q)
#pragma unroll
        for (int j = 0; j < G; ++j) acc[q][j] = make_float2(0.f, 0.f);
    const float* hp = ht + 2 * j0;
    const int T = h.T;
#pragma unroll kRfUnroll
    for (int kk = 0; kk < T; ++kk) {
        float2 v[P];
#pragma unroll
        for (int q = 0; q < P; ++q) v[q] = make_float2(w[2 * q][kk], w[2 * q + 1][kk]);
        float2 hh[G];
        const float* t = hp + kk * 32;
        if (G >= 2) {
#pragma unroll
            for (int j = 0; j + 2 <= G; j += 2) {
                const float4 d = *reinterpret_cast<const float4*>(t + 2 * j);
                hh[j] = make_float2(d.x, d.y);
                hh[j + 1 < G ? j + 1 : j] = make_float2(d.z, d.w);
            }
        } else {
            hh[0] = *reinterpret_cast<const float2*>(t);
        }
#pragma unroll
        for (int q = 0; q < P; ++q)
#pragma unroll
            for (int j = 0; j < G; ++j) acc[q][j] = __ffma2_rn(hh[j], v[q], acc[q][j]);
    }
#pragma unroll
    for (int q = 0; q < P; ++q) {
        float a0[G], a1[G];
#pragma unroll
        for (int j = 0; j < G; ++j) {
            a0[j] = acc[q][j].x;
            a1[j] = acc[q][j].y;
        }
        if (p[2 * q].valid) store_group<G>(h, p[2 * q], j0, a0);
        if (p[2 * q + 1].valid) store_group<G>(h, p[2 * q + 1], j0, a1);
    }
}

// R units starting at (grp, blk), all m outputs of each: four at a time,
// then two and one as needed (three small loop bodies serve every m, so
// warps on tasks of different m share the instruction cache).
template <int R>
__device__ __forceinline__ void units(const RowTileDev& h, const TileGeom& g, const RowInfo* rows, const float* slots,
                                      const float* ht, int& grp, int& blk) {
    UnitPos p[R];
    const float* w[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
        p[r] = unit_pos(h, g, rows, grp, blk);
        w[r] = slots + p[r].base;
        if (++blk == g.nb) {
            blk = 0;
            ++grp;
        }
    }
    const int M = h.M;
    int j0 = 0;
    for (; j0 + 4 <= M; j0 += 4) unit_group<4, R>(h, p, w, ht, j0);
    if (M - j0 >= 2) {
        unit_group<2, R>(h, p, w, ht, j0);
        j0 += 2;
    }
    if (j0 < M) unit_group<1, R>(h, p, w, ht, j0);
}

// One consumer warp computes a whole tile: units in (grp, blk) order, blk
// fastest, four at a time, the last U mod 4 two at a time.  A unit is a rows
// x 32/a repetitions; lanes past the tile's edge compute from slot 0 and
// store nothing.
__device__ __forceinline__ void tile_compute(const RowTileDev& h, const float* stage, int lane, int sub) {
    const RowInfo* rows = reinterpret_cast<const RowInfo*>(stage + kRfRecFloats);
    const float* ht = stage_taps(stage, h.T);
    const float* slots = stage + kRfSlotBase;
    const TileGeom g = tile_geom(h, lane);
    // the kRfShare warps of a group take alternate chunks of units
    int grp = 0, blk = 0, u = 0, c = 0;
    auto skip = [&](int n) {
        blk += n;
        while (blk >= g.nb) {
            blk -= g.nb;
            ++grp;
        }
    };
    for (; u + 4 <= g.U; u += 4, ++c) {
        if (c % kRfShare == sub) units<4>(h, g, rows, slots, ht, grp, blk);
        else skip(4);
    }
    for (; u < g.U; u += 2, ++c) {
        if (c % kRfShare == sub) units<2>(h, g, rows, slots, ht, grp, blk);
        else skip(2);
    }
}

// Producer: issues the copies of tile record `src` (its fields in h) into
// `stage`, completing on mbarrier `full`.  Lane k < nrows handles row k's
// bulk copy and the at most six 4-byte copies at its 16-byte edges; the
// words that wrap past the row's end (the same count nw in every row) are
// spread over all lanes as (row, word) pairs.
__device__ __forceinline__ void produce_tile(const RowTileDev& h, const RowTileDev* src, float* stage, uint32_t full,
                                             int lane) {
    const uintptr_t xs = reinterpret_cast<uintptr_t>(h.x);
    const uintptr_t xe = xs + (uintptr_t)h.H * (uintptr_t)h.W * 4u;
    float* slots = stage + kRfSlotBase;
    const int L1 = min(h.lw, h.W - h.c0);                          // each row's run before its end
    const int nw = h.lw - L1;                                      // words past the end, per row
    const uint32_t d0 = (uint32_t)((xs >> 2) + (uint64_t)h.row0 * (uint32_t)h.W + (uint32_t)h.c0) & 3u;
    uint32_t bulk_bytes = 0;
    uint32_t dst_s = 0;
    uintptr_t gA = 0;
    if (lane < h.nrows) {
        int ir = h.row0 + lane;
        if (ir >= h.H) ir -= h.H;
        const float* row = h.x + (int64_t)ir * h.W;
        const uintptr_t a0 = reinterpret_cast<uintptr_t>(row + h.c0);
        const int delta = (int)((a0 >> 2) & 3u);
        float* slot = slots + slot_offset(lane, h.ss);   // word w of the window at slot[delta + w]
        // this row's entry of the row table
        int orow = h.orow0 + lane;
        if (orow >= h.Hout) orow -= h.Hout;
        RowInfo* ri = reinterpret_cast<RowInfo*>(stage + kRfRecFloats) + lane;
        ri->base = slot_offset(lane, h.ss) + delta;
        ri->out = h.y + (int64_t)orow * h.Wout;
        const uintptr_t a1 = a0 + 4u * (uintptr_t)L1;
        gA = a0 & ~(uintptr_t)15;
        if (gA < xs) gA += 16;
        uintptr_t gB = (a1 + 15) & ~(uintptr_t)15;
        if (nw > 0 || gB > xe) gB = a1 & ~(uintptr_t)15;   // wrapped words follow, or the array ends
        if (gB <= gA) gA = gB = a0;                       // nothing to bulk-copy
        // 4-byte copies: the run's words outside [gA, gB)
        for (uintptr_t g = a0; g < gA; g += 4) {
            const int w = (int)((g - a0) >> 2);
            ptx::cp_async4(slot + delta + w, row + h.c0 + w);
        }
        for (uintptr_t g = gB > a0 ? gB : a0; g < a1; g += 4) {
            const int w = (int)((g - a0) >> 2);
            ptx::cp_async4(slot + delta + w, row + h.c0 + w);
        }
        bulk_bytes = (uint32_t)(gB - gA);
        dst_s = ptx::smem_addr(slot) + (uint32_t)(gA - (a0 & ~(uintptr_t)15));
    }
    if (nw > 0) {
        // word L1 + e of row k comes from column (c0 + L1 + e) mod W = (e + c0 + L1 - W) mod W
        const int n = h.nrows * nw;
        for (int idx = lane; idx < n; idx += 32) {
            const int k = idx / nw, e = idx - k * nw;
            int ir = h.row0 + k;
            uint32_t wrap = 0;
            if (ir >= h.H) {
                ir -= h.H;
                wrap = (uint32_t)h.H * (uint32_t)h.W;
            }
            const uint32_t dk = (d0 + (uint32_t)k * (uint32_t)h.W - wrap) & 3u;
            int col = h.c0 + L1 - h.W + e;
            while (col >= h.W) col -= h.W;
            ptx::cp_async4(slots + slot_offset(k, h.ss) + (int)dk + L1 + e, h.x + (int64_t)ir * h.W + col);
        }
    }
    // the mbarrier tracks this lane's 4-byte copies (net zero on its count)
    asm volatile("cp.async.mbarrier.arrive.shared::cta.b64 [%0];" ::"r"(full) : "memory");
    uint32_t total = bulk_bytes;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) total += __shfl_xor_sync(0xffffffffu, total, off);
    const uint32_t tap_bytes = (uint32_t)h.T * 32u * 4u;
    __syncwarp();
    // the stage's 32 arrivals, one per lane (each releases the lane's row
    // table entry); lane 0's also expects every bulk byte of the tile, its
    // taps and its record
    if (lane == 0) ptx::mbar_expect_tx(full, total + tap_bytes + (uint32_t)sizeof(RowTileDev));
    else ptx::mbar_arrive(full);
    __syncwarp();
    if (bulk_bytes) ptx::bulk_g2s(dst_s, reinterpret_cast<const void*>(gA), bulk_bytes, full);
    if (lane == 0) {
        ptx::bulk_g2s(ptx::smem_addr(stage_taps(stage, h.T)), h.taps_t, tap_bytes, full);
        ptx::bulk_g2s(ptx::smem_addr(stage), src, (uint32_t)sizeof(RowTileDev), full);
    }
}

// Persistent over the tile list: CTA b takes tiles b, b + gridDim.x, ...;
// its i-th tile goes to stage i % kRfStages and consumer group i % kRfGroups
// (two stages per group: one computed, one filling).  The producer
// reads each tile's record from a ring of kRfRecs records in shared memory
// that bulk copies fill kRfRecs tiles ahead, so no global load latency stands
// between two tiles.
#ifndef AROL_ROW_MIN_CTAS
#define AROL_ROW_MIN_CTAS 2
#endif
__global__ void __launch_bounds__(kRfThreads, AROL_ROW_MIN_CTAS) rowfir_batch_kernel(const RowTileDev* __restrict__ tiles, int ntiles,
                                                                    unsigned* err) {
    extern __shared__ __align__(128) float rsm[];
    RowTileDev* recs = reinterpret_cast<RowTileDev*>(rsm + kRfStages * kRowStageFloats);
    uint64_t* bars = reinterpret_cast<uint64_t*>(recs + kRfRecs);
    const uint32_t full0 = ptx::smem_addr(bars), empty0 = ptx::smem_addr(bars + kRfStages);
    const uint32_t rec0 = ptx::smem_addr(bars + 2 * kRfStages);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int st = 0; st < kRfStages; ++st) {
            ptx::mbar_init(full0 + 8 * st, 32);
            ptx::mbar_init(empty0 + 8 * st, kRfShare);
        }
        for (int q = 0; q < kRfRecs; ++q) ptx::mbar_init(rec0 + 8 * q, 1);
        ptx::fence_barrier_init();
    }
    __syncthreads();
    const int G = gridDim.x;
    if (warp >= kRfCWarps) {
        // producer p takes this CTA's tiles i = p, p + kRfPWarps, ...; the
        // record of tile i lives in slot i % kRfRecs (kRfRecs a multiple of
        // kRfPWarps, so each producer owns its slots)
        const int pw = warp - kRfCWarps;
        if (lane == 0) {
            for (int q = pw; q < kRfRecs && (int)blockIdx.x + q * G < ntiles; q += kRfPWarps) {
                ptx::mbar_expect_tx(rec0 + 8 * q, (uint32_t)sizeof(RowTileDev));
                ptx::bulk_g2s(ptx::smem_addr(recs + q), tiles + blockIdx.x + q * G, (uint32_t)sizeof(RowTileDev),
                              rec0 + 8 * q);
            }
        }
        int i = pw;
        for (int t = blockIdx.x + pw * G; t < ntiles; t += kRfPWarps * G, i += kRfPWarps) {
            const int st = i % kRfStages, q = i % kRfRecs;
            if (i >= kRfStages && !ptx::mbar_wait(empty0 + 8 * st, ((uint32_t)(i / kRfStages) & 1u) ^ 1u)) {
                if (lane == 0) flag(err, 1u);
                break;
            }
            if (!ptx::mbar_wait(rec0 + 8 * q, (uint32_t)(i / kRfRecs) & 1u)) {
                if (lane == 0) flag(err, 8u);
                break;
            }
            const RowTileDev cur = recs[q];
            produce_tile(cur, tiles + t, rsm + st * kRowStageFloats, full0 + 8 * st, lane);
            // every lane has used its copy of the record: refill the slot with
            // the record kRfRecs tiles ahead
            __syncwarp();
            const int tn = t + kRfRecs * G;
            if (lane == 0 && tn < ntiles) {
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                ptx::mbar_expect_tx(rec0 + 8 * q, (uint32_t)sizeof(RowTileDev));
                ptx::bulk_g2s(ptx::smem_addr(recs + q), tiles + tn, (uint32_t)sizeof(RowTileDev), rec0 + 8 * q);
            }
        }
        // every issued copy lands before the CTA's shared memory goes away.
        // This producer issued its tiles pw, pw + kRfPWarps, ... below i, and
        // the records of its tiles below min(n, i + kRfRecs): on stage st
        // (slot q) the last is the largest such index congruent to st (q).
        const int n = (ntiles - (int)blockIdx.x + G - 1) / G;   // this CTA's tiles
#pragma unroll
        for (int st = pw; st < kRfStages; st += kRfPWarps) {
            if (i <= st) continue;
            const int last = st + kRfStages * ((i - 1 - st) / kRfStages);
            if (!ptx::mbar_wait(full0 + 8 * st, ((uint32_t)last / kRfStages) & 1u) && lane == 0) flag(err, 4u);
        }
        const int nrec = min(n, i + kRfRecs);
#pragma unroll
        for (int q = pw; q < kRfRecs; q += kRfPWarps) {
            if (nrec <= q) continue;
            const int last = q + kRfRecs * ((nrec - 1 - q) / kRfRecs);
            if (!ptx::mbar_wait(rec0 + 8 * q, ((uint32_t)last / kRfRecs) & 1u) && lane == 0) flag(err, 4u);
        }
        ptx::cp_async_wait_all();
        return;
    }
    const int group = warp / kRfShare, sub = warp - group * kRfShare;
    for (int i = group, t = blockIdx.x + group * G; t < ntiles; i += kRfGroups, t += kRfGroups * G) {
        const int st = i % kRfStages;
        if (!ptx::mbar_wait(full0 + 8 * st, (uint32_t)(i / kRfStages) & 1u)) {
            if (lane == 0) flag(err, 2u);
            break;
        }
        const float* stage = rsm + st * kRowStageFloats;
        const RowTileDev h = *reinterpret_cast<const RowTileDev*>(stage);
        tile_compute(h, stage, lane, sub);
        __syncwarp();
        if (lane == 0) ptx::mbar_arrive(empty0 + 8 * st);
    }
}

size_t rowfir_smem() {
    return (size_t)kRfStages * kRowStageFloats * sizeof(float) + kRfRecs * sizeof(RowTileDev) +
           (2 * kRfStages + kRfRecs) * sizeof(uint64_t);
}

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
