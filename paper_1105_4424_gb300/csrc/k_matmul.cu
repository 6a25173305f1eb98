// Matmul elementary task on the 5th-generation tensor cores.
//
// The repetitive task has repetition space (M/128, N/128): repetition r reads
// the 128 x K row panel r0 of A and the K x 128 column panel r1 of B, and its
// output tiler writes the 128 x 128 tile (r0, r1) of C (a partition of C).
// A tile is BN/128 neighbouring repetitions (128 x BN outputs); one
// persistent CTA per SM walks the tiles:
//
//   * TMA (cp.async.bulk.tensor, 128-byte swizzle) streams 128 x 64 slices of
//     A (K-major) and 64 x BN slices of B (N-major, as B is stored row-major)
//     into a STAGES-deep shared-memory ring guarded by mbarriers;
//   * one elected thread issues tcgen05.mma (kind::f16, bf16 x bf16 -> f32,
//     M = 128, N = BN, K = 16) with the accumulator in tensor memory; each
//     stage is released by tcgen05.commit onto its "empty" barrier;
//   * after a tile's last k-block a commit hands its TMEM accumulator (one of
//     two) to four epilogue warps, which read their 32 lanes (rows) with
//     tcgen05.ld and store f32 C while the next tile accumulates in the other.
//
// When M and N are multiples of 256 a two-SM kernel (tcgen05 cta_group::2,
// below) takes the task instead: a CTA pair computes 256 x 256 tiles with
// half of B in each CTA, six stages deep, and stores C through 128-byte
// swizzled shared-memory blocks and bulk tensor stores.  AROL_MATMUL_PAIR=0
// keeps the one-SM kernel.
//
// Every mbarrier wait is bounded (iteration count and wall time).  A wait that
// gives up sets a bit in *err and the kernel drains what it issued, frees its
// tensor memory and returns; the host reports AROL_ERR_TIMEOUT.
#include <cstdlib>

#include <cuda.h>
#include <cudaTypedefs.h>

#include "arol_internal.h"
#include "ptx.h"

namespace arol {
namespace {

constexpr int BM = 128, BK = 64, STAGES = 4;
// mbarriers with bounded waits, shared with the other pipelined kernels
using ptx::mbar_arrive;
using ptx::mbar_expect_tx;
using ptx::mbar_init;
using ptx::mbar_wait;
using ptx::smem_addr;

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, int x, int y, uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(bar)
        : "memory");
}

// Shared-memory matrix descriptor (tcgen05): start, leading and stride byte
// offsets (16-byte units), descriptor version 1, 128-byte swizzle.
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= 1ull << 46;
    d |= 2ull << 61;
    return d;
}

// Instruction descriptor, kind::f16: f32 accumulator, bf16 A and B, A K-major,
// B N-major, N = bn, M = 128.
__host__ __device__ constexpr uint32_t instr_desc(int bn) {
    return (1u << 4) | (1u << 7) | (1u << 10) | (0u << 15) | (1u << 16) | ((uint32_t)(bn >> 3) << 17) |
           ((uint32_t)(BM >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
        : "memory");
}

__device__ __forceinline__ void mma_commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

template <int BN>
struct Cfg {
    static constexpr int kABytes = BM * BK * 2;
    static constexpr int kBBytes = BK * BN * 2;
    static constexpr int kStageBytes = kABytes + kBBytes;
    static constexpr int kSmem = STAGES * kStageBytes + 1024 + 256;
    static constexpr uint32_t kTmemCols = 2 * BN;   // two accumulators, a power of two <= 512
    static constexpr int kThreads = 192;            // TMA warp, MMA warp, 4 epilogue warps
};

// Persistent CTAs (one per SM) walk the output tiles t = blockIdx.x + i * gridDim.x
// (N-fastest order).  Tile i accumulates into TMEM buffer i & 1, so the four
// epilogue warps drain tile i while the MMA warp already fills tile i + 1.
template <int BN>
__global__ void __launch_bounds__(192, 1) matmul_tc_kernel(const __grid_constant__ CUtensorMap tmA,
                                                           const __grid_constant__ CUtensorMap tmB, float* __restrict__ C,
                                                           int M, int N, int K, unsigned* __restrict__ err) {
    using G = Cfg<BN>;
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint8_t* sA = smem;
    uint8_t* sB = smem + STAGES * G::kABytes;
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem + STAGES * G::kStageBytes);
    // bars: [0,S) full, [S,2S) empty, 2S + a: accumulator a ready, 2S + 2 + a: accumulator a free
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * STAGES + 4);
    int* progress = reinterpret_cast<int*>(tmem_slot + 1);   // [0] k-blocks issued by TMA, [1] consumed by MMA

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nkb = K / BK;
    const int tiles_n = N / BN;
    const int ntiles = (M / BM) * tiles_n;
    const uint32_t full0 = smem_addr(bars), empty0 = smem_addr(bars + STAGES);
    const uint32_t accf0 = smem_addr(bars + 2 * STAGES), acce0 = smem_addr(bars + 2 * STAGES + 2);

    if (threadIdx.x == 0) {
        for (int st = 0; st < STAGES; ++st) {
            mbar_init(full0 + 8 * st, 1);
            mbar_init(empty0 + 8 * st, 1);
        }
        for (int a = 0; a < 2; ++a) {
            mbar_init(accf0 + 8 * a, 1);
            mbar_init(acce0 + 8 * a, 4);
        }
        progress[0] = 0;
        progress[1] = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (warp == 2) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(tmem_slot)),
                     "r"(G::kTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tmem_slot;

    if (warp == 0) {
        // ---------------- TMA producer (one lane)
        if (lane == 0) {
            uint32_t g = 0;
            bool ok = true;
            for (int t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
                const int m0 = (t / tiles_n) * BM, n0 = (t % tiles_n) * BN;
                for (int kb = 0; kb < nkb; ++kb, ++g) {
                    const int st = (int)(g % STAGES);
                    if (g >= (uint32_t)STAGES && !mbar_wait(empty0 + 8 * st, ((g / STAGES) & 1u) ^ 1u)) {
                        atomicOr(err, 1u);
                        ok = false;
                        break;
                    }
                    const uint32_t fb = full0 + 8 * st;
                    mbar_expect_tx(fb, G::kStageBytes);
                    tma_load_2d(smem_addr(sA + st * G::kABytes), &tmA, kb * BK, m0, fb);
#pragma unroll
                    for (int c = 0; c < BN / 64; ++c)
                        tma_load_2d(smem_addr(sB + st * G::kBBytes + c * (BK * 128)), &tmB, n0 + 64 * c, kb * BK, fb);
                }
            }
            progress[0] = (int)g;
        }
    } else if (warp == 1) {
        // ---------------- MMA issuer (one lane)
        if (lane == 0) {
            constexpr uint32_t idesc = instr_desc(BN);
            uint32_t g = 0;
            int i = 0;
            bool ok = true;
            for (int t = blockIdx.x; t < ntiles && ok; t += gridDim.x, ++i) {
                const int acc = i & 1;
                if (i >= 2 && !mbar_wait(acce0 + 8 * acc, (((uint32_t)i >> 1) & 1u) ^ 1u)) {
                    atomicOr(err, 8u);
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint32_t d = tmem + (uint32_t)(acc * BN);
                for (int kb = 0; kb < nkb; ++kb, ++g) {
                    const int st = (int)(g % STAGES);
                    if (!mbar_wait(full0 + 8 * st, (g / STAGES) & 1u)) {
                        atomicOr(err, 2u);
                        ok = false;
                        break;
                    }
                    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                    const uint32_t a0 = smem_addr(sA + st * G::kABytes);
                    const uint32_t b0 = smem_addr(sB + st * G::kBBytes);
#pragma unroll
                    for (int kk = 0; kk < BK / 16; ++kk) {
                        // A: K-major rows of 128 B, 8-row groups 1024 B apart; +32 B per 16 k.
                        const uint64_t ad = smem_desc(a0 + kk * 32, 16, 1024);
                        // B: N-major, 64-column chunks 8 KB apart (LBO), 8-row k groups
                        // 1024 B apart (SBO); +16 rows of 128 B per 16 k.
                        const uint64_t bd = smem_desc(b0 + kk * 16 * 128, BK * 128, 1024);
                        mma_bf16(d, ad, bd, idesc, (kb > 0 || kk > 0) ? 1u : 0u);
                    }
                    mma_commit(empty0 + 8 * st);
                }
                mma_commit(accf0 + 8 * acc);   // accumulator ready once these MMAs complete
            }
            progress[1] = (int)g;
        }
    } else {
        // ---------------- epilogue: warp w reads TMEM lanes 32 * (w % 4) .. + 31
        const int quad = warp & 3;
        int i = 0;
        for (int t = blockIdx.x; t < ntiles; t += gridDim.x, ++i) {
            const int acc = i & 1;
            if (!mbar_wait(accf0 + 8 * acc, ((uint32_t)i >> 1) & 1u)) {
                if (lane == 0) atomicOr(err, 4u);
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const int m0 = (t / tiles_n) * BM, n0 = (t % tiles_n) * BN;
            const int row = m0 + quad * 32 + lane;
            float* crow = C + (int64_t)row * N + n0;
#pragma unroll 1
            for (int c = 0; c < BN; c += 32) {
                float v[32];
                tmem_ld32(tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)(acc * BN + c), v);
#pragma unroll
                for (int q = 0; q < 8; ++q)
                    *reinterpret_cast<float4*>(crow + c + 4 * q) =
                        make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
            }
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            __syncwarp();
            if (lane == 0) mbar_arrive(acce0 + 8 * acc);   // this warp is done with accumulator acc
        }
    }
    __syncwarp();
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    // On an error path, let every copy that was issued but not consumed land
    // before the CTA's shared memory goes away.
    if (threadIdx.x == 0) {
        for (int g = progress[1]; g < progress[0]; ++g) mbar_wait(full0 + 8 * (g % STAGES), (g / STAGES) & 1);
    }
    if (warp == 2) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(G::kTmemCols) : "memory");
    }
}

// ---------------------------------------------------------------------------
// Two-SM variant (tcgen05 cta_group::2).  A cluster of two CTAs on two SMs
// computes a 256 x 256 tile: CTA r holds rows 128 r .. 128 r + 127 of the A
// panel and columns 128 r .. 128 r + 127 of the B panel in its own shared
// memory, and one thread of the even CTA issues M = 256, N = 256 MMAs that
// read both CTAs' stages and leave 128 rows x 256 columns in each CTA's
// tensor memory.  Per CTA a k-block stage is 16 KB of A plus 16 KB of B (one
// CTA alone needs 16 + 32 KB for 128 x 256), so six stages fit and the
// L2 -> SM traffic per FLOP drops by a third.
//
// Barriers: the even CTA's full[s] collects both CTAs' copies (its producer
// posts the expected bytes of both halves); the MMA commit is multicast to
// empty[s] and to the accumulator-ready barriers of both CTAs; the eight
// epilogue warps of the pair arrive on the even CTA's accumulator-free
// barriers.  Every wait is bounded as in the one-SM kernel.
// ---------------------------------------------------------------------------
// k-depth of a stage of the pair kernel (64 or 128: one or two 64-deep A
// boxes per stage, one barrier round trip per stage) and the stages.
#ifndef AROL_MM_BK2
#define AROL_MM_BK2 128
#endif
constexpr int BK2 = AROL_MM_BK2;
constexpr int STAGES2 = 6 * 64 / BK2;
static_assert(BK2 == 64 || BK2 == 128, "one or two 64-deep boxes of A per stage");

__device__ __forceinline__ uint32_t cluster_rank() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}

// Address of the same shared variable in CTA `rank` of the cluster.
__device__ __forceinline__ uint32_t map_to(uint32_t saddr, uint32_t rank) {
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(saddr), "r"(rank));
    return r;
}

__device__ __forceinline__ void cluster_sync() {
    asm volatile("barrier.cluster.arrive.release.aligned;" ::: "memory");
    asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_cluster(uint32_t cluster_addr) {
    asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(cluster_addr) : "memory");
}

// TMA into this CTA's shared memory, completing on a barrier of either CTA of the pair.
__device__ __forceinline__ void tma_load_2d_pair(uint32_t dst, const CUtensorMap* map, int x, int y, uint32_t bar_cluster) {
    asm volatile(
        "cp.async.bulk.tensor.2d.cta_group::2.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(bar_cluster)
        : "memory");
}

__device__ __forceinline__ void mma_bf16_pair(uint32_t tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::2.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
        : "memory");
}

// Arrive (once the issuing thread's MMAs complete) on the barrier at this
// shared offset in both CTAs of the pair.
__device__ __forceinline__ void mma_commit_pair(uint32_t bar) {
    const uint16_t mask = 0x3;
    asm volatile("tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64 [%0], %1;" ::"r"(bar),
                 "h"(mask)
                 : "memory");
}

// kind::f16 instruction descriptor for the pair: M = 256, N = bn.
// Bulk tensor store of a shared-memory box to global memory (bulk-group completion).
__device__ __forceinline__ void tma_store_2d(const CUtensorMap* map, int x, int y, uint32_t src) {
    asm volatile("cp.async.bulk.tensor.2d.global.shared::cta.bulk_group [%0, {%1, %2}], [%3];" ::"l"(
                     reinterpret_cast<uint64_t>(map)),
                 "r"(x), "r"(y), "r"(src)
                 : "memory");
}

__host__ __device__ constexpr uint32_t instr_desc_pair(int bn) {
    return (1u << 4) | (1u << 7) | (1u << 10) | (0u << 15) | (1u << 16) | ((uint32_t)(bn >> 3) << 17) |
           ((uint32_t)(256 >> 4) << 24);
}

// Work item i of the pair kernel.  Items below `full` are whole 256 x 256
// tiles in N-fastest order; when the whole tiles do not fill the last round,
// the host makes every remaining tile two 256 x 128 items (`full` .. `total`)
// so that round takes half as long.
struct PairItem {
    int m0, n0;   // first row of the 256-row tile, first column of the item
    bool wide;    // 256 columns (else 128)
};

__device__ __forceinline__ PairItem pair_item(int i, int full, int tiles_n) {
    if (i < full) return PairItem{(i / tiles_n) * 256, (i % tiles_n) * 256, true};
    const int j = i - full, t = full + (j >> 1);
    return PairItem{(t / tiles_n) * 256, (t % tiles_n) * 256 + (j & 1) * 128, false};
}

struct Cfg2 {
    static constexpr int kABytes = BM * BK2 * 2;           // 128 x BK2 of A (BK2 / 64 boxes of 128 x 64)
    static constexpr int kBBytes = BK2 * 128 * 2;          // BK2 x 128 of B (this CTA's half)
    static constexpr int kStageBytes = kABytes + kBBytes;
    static constexpr int kOutBytes = 32 * 32 * 4;          // one 32 x 32 f32 block of C, 128-byte swizzled
    static constexpr int kSmem = STAGES2 * kStageBytes + 4 * 2 * kOutBytes + 1024 + 256;
    static constexpr uint32_t kTmemCols = 512;             // two 256-column accumulators
    static constexpr int kThreads = 192;
};

__global__ void __launch_bounds__(192, 1) matmul_tc2_kernel(const __grid_constant__ CUtensorMap tmA,
                                                            const __grid_constant__ CUtensorMap tmB,
                                                            const __grid_constant__ CUtensorMap tmC,
                                                            int M, int N, int K, int full, int total,
                                                            unsigned* __restrict__ err) {
    using G = Cfg2;
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint8_t* sA = smem;
    uint8_t* sB = smem + STAGES2 * G::kABytes;
    uint8_t* sOut = smem + STAGES2 * G::kStageBytes;                 // 2 blocks per epilogue warp
    uint64_t* bars = reinterpret_cast<uint64_t*>(sOut + 4 * 2 * G::kOutBytes);
    // bars: [0,S) full, [S,2S) empty, 2S + a: accumulator a ready, 2S + 2 + a:
    // accumulator a free, 2S + 4: drain
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * STAGES2 + 5);
    int* progress = reinterpret_cast<int*>(tmem_slot + 1);   // [0] k-blocks issued by TMA, [1] consumed by MMA

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t rank = cluster_rank();
    const bool leader = rank == 0;
    const int nkb = K / BK2;
    const int tiles_n = N / 256;
    const int ntiles = total;
    const int cluster = blockIdx.x >> 1, nclusters = gridDim.x >> 1;
    const uint32_t full0 = smem_addr(bars), empty0 = smem_addr(bars + STAGES2);
    const uint32_t accf0 = smem_addr(bars + 2 * STAGES2), acce0 = smem_addr(bars + 2 * STAGES2 + 2);
    const uint32_t drain = smem_addr(bars + 2 * STAGES2 + 4);

    if (threadIdx.x == 0) {
        for (int st = 0; st < STAGES2; ++st) {
            mbar_init(full0 + 8 * st, 1);
            mbar_init(empty0 + 8 * st, 1);
        }
        for (int a = 0; a < 2; ++a) {
            mbar_init(accf0 + 8 * a, 1);
            mbar_init(acce0 + 8 * a, 8);
        }
        mbar_init(drain, 1);
        progress[0] = 0;
        progress[1] = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (warp == 2) {   // one warp of each CTA of the pair allocates, together
        asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(tmem_slot)),
                     "r"(G::kTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    cluster_sync();   // both CTAs' barriers are initialised before any remote use
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tmem_slot;

    if (warp == 0) {
        // ---------------- TMA producer (one lane per CTA)
        if (lane == 0) {
            uint32_t g = 0;
            bool ok = true;
            for (int t = cluster; t < ntiles && ok; t += nclusters) {
                const PairItem it = pair_item(t, full, tiles_n);
                const int m0 = it.m0 + (int)rank * 128;
                const int chunks = it.wide ? 2 : 1;                  // 64-column B chunks of this CTA's half
                const int n0 = it.n0 + (int)rank * 64 * chunks;
                const uint32_t bytes = 2u * (uint32_t)(G::kABytes + chunks * BK2 * 128);
                for (int kb = 0; kb < nkb; ++kb, ++g) {
                    const int st = (int)(g % STAGES2);
                    if (g >= (uint32_t)STAGES2 && !mbar_wait(empty0 + 8 * st, ((g / STAGES2) & 1u) ^ 1u)) {
                        atomicOr(err, 1u);
                        ok = false;
                        break;
                    }
                    const uint32_t fb = full0 + 8 * st;
                    if (leader) mbar_expect_tx(fb, bytes);
                    const uint32_t fb_pair = map_to(fb, 0);
#pragma unroll
                    for (int hb = 0; hb < BK2 / 64; ++hb)
                        tma_load_2d_pair(smem_addr(sA + st * G::kABytes + hb * (BM * 64 * 2)), &tmA, kb * BK2 + 64 * hb,
                                         m0, fb_pair);
                    for (int c = 0; c < chunks; ++c)
                        tma_load_2d_pair(smem_addr(sB + st * G::kBBytes + c * (BK2 * 128)), &tmB, n0 + 64 * c,
                                         kb * BK2, fb_pair);
                }
            }
            progress[0] = (int)g;
        }
    } else if (warp == 1) {
        // ---------------- MMA issuer (one lane of the even CTA)
        if (leader && lane == 0) {
            uint32_t g = 0;
            int i = 0;
            bool ok = true;
            for (int t = cluster; t < ntiles && ok; t += nclusters, ++i) {
                const uint32_t idesc = pair_item(t, full, tiles_n).wide ? instr_desc_pair(256) : instr_desc_pair(128);
                const int acc = i & 1;
                if (i >= 2 && !mbar_wait(acce0 + 8 * acc, (((uint32_t)i >> 1) & 1u) ^ 1u)) {
                    atomicOr(err, 8u);
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint32_t d = tmem + (uint32_t)(acc * 256);
                for (int kb = 0; kb < nkb; ++kb, ++g) {
                    const int st = (int)(g % STAGES2);
                    // the stage's bytes were written by the copy engine and
                    // completed on this barrier: no tcgen05 fence is needed here
                    if (!mbar_wait(full0 + 8 * st, (g / STAGES2) & 1u)) {
                        atomicOr(err, 2u);
                        ok = false;
                        break;
                    }
                    const uint32_t a0 = smem_addr(sA + st * G::kABytes);
                    const uint32_t b0 = smem_addr(sB + st * G::kBBytes);
#pragma unroll
                    for (int kk = 0; kk < BK2 / 16; ++kk) {
                        // A: box kk / 4 of the stage, 32 bytes per 16-deep step in its swizzle atom
                        const uint64_t ad = smem_desc(a0 + (kk >> 2) * (BM * 64 * 2) + (kk & 3) * 32, 16, 1024);
                        const uint64_t bd = smem_desc(b0 + kk * 16 * 128, BK2 * 128, 1024);
                        mma_bf16_pair(d, ad, bd, idesc, (kb > 0 || kk > 0) ? 1u : 0u);
                    }
                    mma_commit_pair(empty0 + 8 * st);
                }
                if (!ok) break;
                mma_commit_pair(accf0 + 8 * acc);
            }
            progress[1] = (int)g;
            // every MMA this thread issued has completed before the pair tears down
            mma_commit_pair(drain);
            if (!mbar_wait(drain, 0)) atomicOr(err, 16u);
        }
    } else {
        // ---------------- epilogue: warp w reads TMEM lanes 32 * (w % 4) .. + 31
        // (rows of C), 32 columns at a time, writes each 32 x 32 block into
        // a 128-byte-swizzled shared buffer (lane r's 16-byte chunk j at chunk
        // j ^ (r & 7): conflict-free) and stores it with one bulk tensor copy;
        // two buffers per warp alternate.
        const int quad = warp & 3;
        const uint32_t acce_leader = map_to(acce0, 0);
        const uint32_t out0 = smem_addr(sOut + quad * 2 * G::kOutBytes);
        int i = 0, nb = 0;
        for (int t = cluster; t < ntiles; t += nclusters, ++i) {
            const int acc = i & 1;
            if (!mbar_wait(accf0 + 8 * acc, ((uint32_t)i >> 1) & 1u)) {
                if (lane == 0) atomicOr(err, 4u);
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const PairItem it = pair_item(t, full, tiles_n);
            const int row0 = it.m0 + (int)rank * 128 + quad * 32;
            const int width = it.wide ? 256 : 128;
#pragma unroll 1
            for (int c = 0; c < width; c += 32, ++nb) {
                float v[32];
                tmem_ld32(tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)(acc * 256 + c), v);
                const uint32_t buf = out0 + (uint32_t)(nb & 1) * G::kOutBytes;
                // the store issued from this buffer two blocks ago has read it
                if (lane == 0) asm volatile("cp.async.bulk.wait_group.read 1;" ::: "memory");
                __syncwarp();
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    const uint32_t dst = buf + (uint32_t)lane * 128u + (uint32_t)((q ^ (lane & 7)) * 16);
                    asm volatile("st.shared.v4.f32 [%0], {%1, %2, %3, %4};" ::"r"(dst), "f"(v[4 * q]), "f"(v[4 * q + 1]),
                                 "f"(v[4 * q + 2]), "f"(v[4 * q + 3])
                                 : "memory");
                }
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");   // visible to the bulk copy
                __syncwarp();
                if (lane == 0) {
                    tma_store_2d(&tmC, it.n0 + c, row0, buf);
                    asm volatile("cp.async.bulk.commit_group;" ::: "memory");
                }
            }
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            __syncwarp();
            if (lane == 0) mbar_arrive_cluster(acce_leader + 8 * acc);
        }
        if (lane == 0) asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");   // every store has completed
        __syncwarp();
    }
    __syncwarp();
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    cluster_sync();
    // On an error path, let every copy either CTA issued but the MMA did not
    // consume land before the pair's shared memory goes away.
    if (leader && threadIdx.x == 0) {
        int peer_issued;
        asm volatile("ld.shared::cluster.u32 %0, [%1];" : "=r"(peer_issued) : "r"(map_to(smem_addr(progress), 1)) : "memory");
        const int issued = progress[0] > peer_issued ? progress[0] : peer_issued;
        for (int g = progress[1]; g < issued; ++g) mbar_wait(full0 + 8 * (g % STAGES2), (g / STAGES2) & 1);
    }
    __syncthreads();
    cluster_sync();
    if (warp == 2) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(G::kTmemCols) : "memory");
    }
}

using EncodeTiled = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                 const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                 CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiled encoder() {
    static EncodeTiled fn = nullptr;
    if (!fn) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiled>(p);
    }
    return fn;
}

// 2-D bf16 row-major (rows x cols) tensor map with a (box_rows x 64) box and
// 128-byte swizzle.
bool make_map(CUtensorMap* map, const void* base, uint64_t rows, uint64_t cols, uint32_t box_rows) {
    EncodeTiled enc = encoder();
    if (!enc) return false;
    const cuuint64_t dims[2] = {cols, rows};
    const cuuint64_t strides[1] = {cols * 2};
    const cuuint32_t box[2] = {64, box_rows};
    const cuuint32_t estr[2] = {1, 1};
    return enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box, estr,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_NONE,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <int BN>
cudaError_t launch_bn(const CUtensorMap& ma, const CUtensorMap& mb, float* C, int M, int N, int K, unsigned* err,
                      cudaStream_t s) {
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(matmul_tc_kernel<BN>, cudaFuncAttributeMaxDynamicSharedMemorySize, Cfg<BN>::kSmem);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    const int ntiles = (M / BM) * (N / BN);
    const int grid = ntiles < device_sm_count() ? ntiles : device_sm_count();
    matmul_tc_kernel<BN><<<grid, Cfg<BN>::kThreads, Cfg<BN>::kSmem, s>>>(ma, mb, C, M, N, K, err);
    return cudaGetLastError();
}

// The two-SM kernel is the default for 256-divisible shapes; the variable
// AROL_MATMUL_PAIR=0 selects the one-SM kernel (for comparison).
bool pair_enabled() {
    static int v = -1;
    if (v < 0) {
        const char* e = std::getenv("AROL_MATMUL_PAIR");
        v = (e && e[0] == '0') ? 0 : 1;
    }
    return v == 1;
}

// 2-D f32 row-major (rows x cols) tensor map with a 32 x 32 box (128-byte
// rows), 128-byte swizzle: the pair kernel's output blocks.
bool make_map_f32(CUtensorMap* map, void* base, uint64_t rows, uint64_t cols) {
    EncodeTiled enc = encoder();
    if (!enc) return false;
    const cuuint64_t dims[2] = {cols, rows};
    const cuuint64_t strides[1] = {cols * 4};
    const cuuint32_t box[2] = {32, 32};
    const cuuint32_t estr[2] = {1, 1};
    return enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, base, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
               CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_NONE, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

cudaError_t launch_pair(const CUtensorMap& ma, const CUtensorMap& mb, float* C, int M, int N, int K, unsigned* err,
                        cudaStream_t s) {
    CUtensorMap mc;
    if (!make_map_f32(&mc, C, (uint64_t)M, (uint64_t)N)) return cudaErrorInvalidValue;
    static bool attr = false;
    static int max_clusters = 0;
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = 2;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.blockDim = dim3(Cfg2::kThreads);
    cfg.dynamicSmemBytes = Cfg2::kSmem;
    cfg.stream = s;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(matmul_tc2_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, Cfg2::kSmem);
        if (e != cudaSuccess) return e;
        cfg.gridDim = dim3(2 * device_sm_count());
        int n = 0;
        e = cudaOccupancyMaxActiveClusters(&n, matmul_tc2_kernel, &cfg);
        if (e != cudaSuccess) return e;
        max_clusters = n > 0 ? n : 1;
        attr = true;
    }
    const int ntiles = (M / 256) * (N / 256);
    int cap = max_clusters;
    if (const char* e = std::getenv("AROL_MATMUL_MAX_CLUSTERS")) {   // fewer clusters: exercises the schedule on small shapes
        const int v = std::atoi(e);
        if (v > 0 && v < cap) cap = v;
    }
    const int clusters = ntiles < cap ? ntiles : cap;
    // whole tiles fill `rounds` rounds; a partial last round of rem tiles is
    // run as 2 * rem half-width items when they fit one round
    const int rounds = ntiles / clusters, rem = ntiles - rounds * clusters;
    int full = ntiles, total = ntiles;
    if (rem > 0 && 2 * rem <= clusters && rounds > 0) {
        full = rounds * clusters;
        total = full + 2 * rem;
    }
    cfg.gridDim = dim3(2 * clusters);
    return cudaLaunchKernelEx(&cfg, matmul_tc2_kernel, ma, mb, mc, M, N, K, full, total, err);
}

}  // namespace

cudaError_t launch_matmul_tc(const void* A, const void* B, float* C, int M, int N, int K, unsigned* err_flag,
                             cudaStream_t s) {
    if ((reinterpret_cast<uintptr_t>(A) | reinterpret_cast<uintptr_t>(B)) & 15u) return cudaErrorMisalignedAddress;
    if ((reinterpret_cast<uintptr_t>(C) & 15u) != 0) return cudaErrorMisalignedAddress;
    if (M % BM || N % 128 || K % BK || K < BK) return cudaErrorInvalidValue;
    CUtensorMap ma, mb;
    if (!make_map(&ma, A, (uint64_t)M, (uint64_t)K, BM)) return cudaErrorInvalidValue;
    if (!make_map(&mb, B, (uint64_t)K, (uint64_t)N, BK)) return cudaErrorInvalidValue;
    cudaError_t e = cudaMemsetAsync(err_flag, 0, sizeof(unsigned), s);
    if (e != cudaSuccess) return e;
    if (M % 256 == 0 && N % 256 == 0 && K % BK2 == 0 && pair_enabled()) {
        CUtensorMap mb2;
        if (!make_map(&mb2, B, (uint64_t)K, (uint64_t)N, BK2)) return cudaErrorInvalidValue;
        return launch_pair(ma, mb2, C, M, N, K, err_flag, s);
    }
    if (N % 256 == 0) return launch_bn<256>(ma, mb, C, M, N, K, err_flag, s);
    return launch_bn<128>(ma, mb, C, M, N, K, err_flag, s);
}

}  // namespace arol
