// Streaming form of a fused two-pass separable chain: a row pass (taps
// Hh: m_h x T_h, step S_h, origin o_h along the columns) then a column pass
// (Hv: m_v x T_v, step S_v, origin o_v down the rows), on every frame
// (Sec. 5 associatedParts: the intermediate never reaches HBM).
//
// Work unit: one frame, one chunk of kSsChunk intermediate columns,
// one band of column-pass repetitions [rb0, rb0 + nrb).  The band needs the
// intermediate rows (o_v + S_v rb0 + i) mod H, i < S_v (nrb - 1) + T_v,
// which are the row pass of the same input rows.  Producer warps copy those
// input rows' windows (the row pass's input columns of the chunk, wrapped at
// the row end), kSsRows rows per stage, into a ring of `nst` shared-memory
// stages: one cp.async.bulk per row for its 16-byte interior and 4-byte
// cp.async for its ragged ends and wrapped words, all completing on the
// stage's mbarrier.
//
// One launch serves one chain or, in a batch, many: the units of chain c
// follow those of chain c - 1 (a unit prefix in device memory), and each
// consumer warp copies its unit's chain taps into its own shared area when
// the chain changes.
//
// Consumer lane l of warp w owns intermediate columns q and q + 1, q = q0 +
// 2 (32 w + l).  For every staged row it computes its two intermediate
// values (row pass, paired FMAs; the rows of a stage are independent, so
// their sums overlap), releases the stage, keeps the values in its warp's
// ring of the last kSsRing rows (a float2 per lane: no bank conflicts), and
// whenever the window of a column-pass repetition is complete (T_v rows,
// every S_v rows), computes that repetition's m_v outputs for its columns
// and stores them.
// Warps never wait on each other; each input row of a band is read from HBM
// once (the halo rows that neighbouring bands share, T_v - S_v of them, twice).
#include "arol_internal.h"
#include "ptx.h"
#include "sepchain.h"

#ifndef AROL_SS_STAGES
#define AROL_SS_STAGES 16
#endif
#ifndef AROL_SS_STAGE_KB
#define AROL_SS_STAGE_KB 40
#endif
#ifndef AROL_SS_SLEEP_NS
#define AROL_SS_SLEEP_NS 20000
#endif
#ifndef AROL_SS_MIN_CTAS
#define AROL_SS_MIN_CTAS 3
#endif
#ifndef AROL_SS_CWARPS
#define AROL_SS_CWARPS 4
#endif
#ifndef AROL_SS_ROWS
#define AROL_SS_ROWS 4
#endif

namespace arol {
namespace {

constexpr int kSsCWarps = AROL_SS_CWARPS;          // consumer warps
constexpr int kSsCols = 2;                         // intermediate columns per consumer lane
constexpr int kSsChunk = 32 * kSsCWarps * kSsCols; // intermediate columns per unit
constexpr int kSsPWarps = 2;                       // producer warps (alternate stages)
constexpr int kSsThreads = (kSsCWarps + kSsPWarps) * 32;
constexpr int kSsMaxStages = AROL_SS_STAGES;       // stages (an even number, 2 .. this, set by the window)
constexpr int kSsRows = AROL_SS_ROWS;              // input rows per stage
// intermediate rows kept per column: a window of T_v rows plus the
// kSsRows - 1 rows of its stage stored after its last one
constexpr int kSsRing = 32;
constexpr size_t kSsStageBudget = AROL_SS_STAGE_KB * 1024;   // bytes of stages aimed at
static_assert(kSsPWarps == 2 && kSsRing % kSsRows == 0, "producers alternate stages; stages fill whole ring runs");

__device__ __forceinline__ void flag(unsigned* err, unsigned bit) {
    if (err) atomicOr(err, bit);
}

// One band unit's geometry, the same in every thread.
struct SsUnit {
    uint32_t f;       // frame
    int q0, nq;       // intermediate columns q0 .. q0 + nq - 1
    int ra;           // first row-pass repetition of the chunk
    int c0, xw;       // input window: columns (c0 + w) mod W, w < xw
    int rb0, nrb;     // column-pass repetitions rb0 .. rb0 + nrb - 1
    int row0, nrows;  // intermediate (= input) rows (row0 + i) mod H, i < nrows
};

__host__ __device__ __forceinline__ SsUnit ss_unit(const SsChain& c, int u) {
    SsUnit s;
    const int per_frame = c.chunks * c.bands;
    s.f = (uint32_t)(u / per_frame);
    const int v = u - (int)s.f * per_frame, band = v / c.chunks, chunk = v - band * c.chunks;
    s.q0 = chunk * kSsChunk;
    s.nq = c.W1 - s.q0 < kSsChunk ? c.W1 - s.q0 : kSsChunk;
    s.ra = s.q0 / c.mh;
    const int rb = (s.q0 + s.nq - 1) / c.mh;
    s.xw = c.Sh * (rb - s.ra) + c.Th;
    s.c0 = (int)(((int64_t)c.oh + (int64_t)c.Sh * s.ra) % c.W);
    s.rb0 = band * c.BH;
    s.nrb = c.Rv - s.rb0 < c.BH ? c.Rv - s.rb0 : c.BH;
    s.nrows = c.Sv * (s.nrb - 1) + c.Tv;
    s.row0 = (int)(((int64_t)c.ov + (int64_t)c.Sv * s.rb0) % c.H);
    return s;
}

// Copies one input row's window, columns (c0 + w) mod W for w < xw, into
// `dst` (16-byte aligned) at dst[delta + w], delta the low two bits of the
// window's first word's address; lane-parallel.  The 4-byte copies are
// issued by every lane, the bulk copy by lane 0, which returns its bytes.
__device__ __forceinline__ uint32_t ss_copy_row(const float* row, const float* xs, const float* xe, int W, int c0, int xw,
                                                float* dst, uint32_t full, int lane) {
    const uintptr_t a0 = reinterpret_cast<uintptr_t>(row + c0);
    const int delta = (int)((a0 >> 2) & 3u);
    const int L1 = min(xw, W - c0);                       // the run before the row's end
    const uintptr_t a1 = a0 + 4u * (uintptr_t)L1;
    uintptr_t gA = a0 & ~(uintptr_t)15;
    if (gA < reinterpret_cast<uintptr_t>(xs)) gA += 16;
    uintptr_t gB = (a1 + 15) & ~(uintptr_t)15;
    if (L1 < xw || gB > reinterpret_cast<uintptr_t>(xe)) gB = a1 & ~(uintptr_t)15;
    if (gB <= gA) gA = gB = a0;
    // 4-byte copies: the run's words outside [gA, gB), then the wrapped words
    const int nhead = (int)((gA > a0 ? gA - a0 : 0) >> 2);
    const int tail0 = (int)(((gB > a0 ? gB : a0) - a0) >> 2);
    for (int w = lane; w < nhead; w += 32) ptx::cp_async4(dst + delta + w, row + c0 + w);
    for (int w = tail0 + lane; w < L1; w += 32) ptx::cp_async4(dst + delta + w, row + c0 + w);
    for (int w = L1 + lane; w < xw; w += 32) {
        int col = c0 + w - W;
        while (col >= W) col -= W;
        ptx::cp_async4(dst + delta + w, row + col);
    }
    const uint32_t bytes = (uint32_t)(gB - gA);
    if (lane == 0 && bytes)
        ptx::bulk_g2s(ptx::smem_addr(dst) + (uint32_t)(gA - (a0 & ~(uintptr_t)15)), reinterpret_cast<const void*>(gA),
                      bytes, full);
    return bytes;
}

// Row-pass sums of a lane's two intermediate values (paired FMAs, each an
// IEEE fma rounded to nearest).  h2[k] holds the two columns' taps k.  One
// window (`one`, both columns from the same repetition) or two (src0,
// src1).  TH > 0: T_h = TH, taps in registers; TH = 0: any T_h, taps read
// from shared memory (rows h0, h1).
template <int TH>
__device__ __forceinline__ float2 ss_dot2(const float2* h2, const float* h0, const float* h1, const float* src0,
                                          const float* src1, bool one, int T) {
    float2 acc = make_float2(0.f, 0.f);
    if (TH > 0) {
        if (one) {
#pragma unroll
            for (int k = 0; k < TH; ++k) {
                const float v = src0[k];
                acc = __ffma2_rn(h2[k], make_float2(v, v), acc);
            }
        } else {
#pragma unroll
            for (int k = 0; k < TH; ++k) acc = __ffma2_rn(h2[k], make_float2(src0[k], src1[k]), acc);
        }
    } else {
#pragma unroll 4
        for (int k = 0; k < T; ++k) acc = __ffma2_rn(make_float2(h0[k], h1[k]), make_float2(src0[k], src1[k]), acc);
    }
    return acc;
}

// The same sums (TH in 1 .. 8, one window) from 16-byte loads: `src` is
// 16-byte aligned and the staged row extends at least 8 words past it (the
// words past the window are loaded and not used).
template <int TH>
__device__ __forceinline__ float2 ss_dot2_v4(const float2* h2, const float* src) {
    float w[8];
    const float4 a = *reinterpret_cast<const float4*>(src);
    w[0] = a.x, w[1] = a.y, w[2] = a.z, w[3] = a.w;
    if (TH > 4) {
        const float4 b = *reinterpret_cast<const float4*>(src + 4);
        w[4] = b.x, w[5] = b.y, w[6] = b.z, w[7] = b.w;
    }
    float2 acc = make_float2(0.f, 0.f);
#pragma unroll
    for (int k = 0; k < (TH > 0 && TH <= 8 ? TH : 1); ++k) acc = __ffma2_rn(h2[k], make_float2(w[k], w[k]), acc);
    return acc;
}

// Column pass of one repetition: the m_v outputs of the lane's two columns
// from intermediate rows t .. t + T_v - 1 (ring slots mod kSsRing, a float2
// per lane and row), stored at yo[j * ys] and yo[j * ys + 1] by active
// lanes.  TV > 0: T_v = TV, the window loaded once into registers; TV = 0:
// any T_v, one ring sweep (in two runs that do not wrap) per output.
template <int TV>
__device__ __forceinline__ void ss_column_pass(const float2* hv, int m, int T, const float2* ring, int t, int lane,
                                               float* yo, int64_t ys, bool act0, bool act1) {
    const int s0 = t & (kSsRing - 1);
    if (TV > 0) {
        float2 rv[TV > 0 ? TV : 1];
        if (s0 + TV <= kSsRing) {
            const float2* a = ring + s0 * 32 + lane;
#pragma unroll
            for (int k = 0; k < TV; ++k) rv[k] = a[32 * k];
        } else {
#pragma unroll
            for (int k = 0; k < TV; ++k) rv[k] = ring[((s0 + k) & (kSsRing - 1)) * 32 + lane];
        }
        for (int j = 0; j < m; ++j) {
            const float2* h = hv + j * TV;
            float2 acc = make_float2(0.f, 0.f);
#pragma unroll
            for (int k = 0; k < TV; ++k) acc = __ffma2_rn(h[k], rv[k], acc);
            if (act0) yo[j * ys] = acc.x;
            if (act1) yo[j * ys + 1] = acc.y;
        }
    } else {
        const int n1 = min(T, kSsRing - s0);
        for (int j = 0; j < m; ++j) {
            const float2* h = hv + j * T;
            const float2* a = ring + s0 * 32 + lane;
            float2 acc = make_float2(0.f, 0.f);
#pragma unroll 4
            for (int k = 0; k < n1; ++k) acc = __ffma2_rn(h[k], a[32 * k], acc);
            const float2* b = ring + lane;
            const float2* hb = h + n1;
#pragma unroll 4
            for (int k = 0; k < T - n1; ++k) acc = __ffma2_rn(hb[k], b[32 * k], acc);
            if (act0) yo[j * ys] = acc.x;
            if (act1) yo[j * ys + 1] = acc.y;
        }
    }
}

// The chain of unit u: the last chain whose first unit is <= u, searched
// forward from the previous one (a CTA's units increase).
__device__ __forceinline__ int ss_find(const int* ustart, int nchains, int u, int c) {
    while (c + 1 < nchains && __ldg(ustart + c + 1) <= u) ++c;
    return c;
}

template <int TH, int TV, bool BATCH>
__global__ void __launch_bounds__(kSsThreads, AROL_SS_MIN_CTAS)
    sepstream_kernel(const SsChain one, const SsChain* chains, const int* ustart, int nchains, int units, int xw_max,
                     int nst, int tapw, unsigned* err) {
    extern __shared__ __align__(128) float ssm[];
    const int sr = (xw_max + 4 + 3) & ~3;                  // floats per staged row (window plus alignment slack)
    const int sf = kSsRows * sr;                           // floats per stage
    float* stages = ssm;
    float* rings = stages + nst * sf;                      // kSsCWarps x kSsRing x 32 x kSsCols
    float* wtaps = rings + kSsCWarps * kSsRing * 32 * kSsCols;   // per consumer warp: Hh, then Hv doubled
    uint64_t* bars = reinterpret_cast<uint64_t*>(wtaps + kSsCWarps * tapw);
    const uint32_t full0 = ptx::smem_addr(bars), empty0 = ptx::smem_addr(bars + nst);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int st = 0; st < nst; ++st) {
            ptx::mbar_init(full0 + 8 * st, 1);
            ptx::mbar_init(empty0 + 8 * st, kSsCWarps);
        }
        ptx::fence_barrier_init();
    }
    __syncthreads();

    if (warp >= kSsCWarps) {
        // producers: stages g = pw, pw + kSsPWarps, ... of this CTA's stage
        // sequence (nst is even, so each producer owns the stages of its parity)
        const int pw = warp - kSsCWarps;
        uint32_t g = 0;                                    // this CTA's stages so far (all units)
        int st = 0;
        uint32_t phase = 0;                                // parity of stage st's current use
        bool ok = true;
        int c = 0;
        for (int u = blockIdx.x; u < units && ok; u += gridDim.x) {
            if (BATCH) c = ss_find(ustart, nchains, u, c);
            const SsChain ch = BATCH ? chains[c] : one;
            const SsUnit s = ss_unit(ch, BATCH ? u - __ldg(ustart + c) : u);
            const int H = ch.H, W = ch.W;
            const int64_t frame_in = (int64_t)H * W;
            const float* xf = ch.x + (int64_t)s.f * frame_in;
            for (int base = 0; base < s.nrows; base += kSsRows) {
                const bool mine = (int)(g & 1u) == pw;
                if (mine) {
                    if (g >= (uint32_t)nst && !ptx::mbar_wait_sleep(empty0 + 8 * st, phase ^ 1u, AROL_SS_SLEEP_NS)) {
                        if (lane == 0) flag(err, 1u);
                        ok = false;
                        break;
                    }
                    const uint32_t full = full0 + 8 * st;
                    const int n = min(kSsRows, s.nrows - base);
                    int ir = (s.row0 + base) % H;
                    uint32_t bytes = 0;
                    for (int r = 0; r < n; ++r) {
                        bytes += ss_copy_row(xf + (int64_t)ir * W, xf, xf + frame_in, W, s.c0, s.xw,
                                             stages + st * sf + r * sr, full, lane);
                        if (++ir == H) ir = 0;
                    }
                    // each lane's 4-byte copies arrive on the barrier when they
                    // land (pending count raised now, lowered then); lane 0 then
                    // arrives with the bulk bytes it issued (the transaction
                    // count may dip below zero meanwhile: the phase cannot
                    // complete before this arrival)
                    asm volatile("cp.async.mbarrier.arrive.shared::cta.b64 [%0];" ::"r"(full) : "memory");
                    __syncwarp();
                    if (lane == 0) ptx::mbar_expect_tx(full, bytes);
                }
                ++g;
                if (++st == nst) st = 0, phase ^= 1u;
            }
        }
        // every issued copy lands before the CTA's shared memory goes away:
        // this producer's last use of stage t is the largest issued index
        // congruent to t
        for (int t = pw; t < nst; t += kSsPWarps) {
            if (g <= (uint32_t)t) continue;
            const uint32_t last = (uint32_t)t + (uint32_t)nst * ((g - 1 - (uint32_t)t) / (uint32_t)nst);
            if (!ptx::mbar_wait(full0 + 8 * t, (last / (uint32_t)nst) & 1u) && lane == 0) flag(err, 4u);
        }
        ptx::cp_async_wait_all();
        return;
    }

    // consumers: lane pair of columns q, q + 1
    const float2* ring = reinterpret_cast<const float2*>(rings) + warp * kSsRing * 32;
    float2* ringw = reinterpret_cast<float2*>(rings) + warp * kSsRing * 32;
    float* wt = wtaps + warp * tapw;                       // this warp's copy of its chain's taps
    int st = 0;
    uint32_t phase = 0;
    int c = 0, cur = -1;
    for (int u = blockIdx.x; u < units; u += gridDim.x) {
        if (BATCH) c = ss_find(ustart, nchains, u, c);
        const SsChain ch = BATCH ? chains[c] : one;
        const SsUnit s = ss_unit(ch, BATCH ? u - __ldg(ustart + c) : u);
        if (c != cur) {
            // the chain's taps: Hh (m_h x T_h), then Hv with each tap doubled
            __syncwarp();
            const int nh = ch.mh * ch.Th, hoff = (nh + 1) & ~1, nv = ch.mv * ch.Tv;
            for (int i = lane; i < nh; i += 32) wt[i] = __ldg(ch.hh + i);
            for (int i = lane; i < nv; i += 32) {
                const float h = __ldg(ch.hv + i);
                reinterpret_cast<float2*>(wt + hoff)[i] = make_float2(h, h);
            }
            __syncwarp();
            cur = c;
        }
        const float2* hv2 = reinterpret_cast<const float2*>(wt + ((ch.mh * ch.Th + 1) & ~1));
        const int H = ch.H, W = ch.W;
        const bool one2 = (ch.mh & 1) == 0;                // q even: q and q + 1 share a repetition
        const int cc = kSsCols * (32 * warp + lane);       // column of the pair within the chunk
        const int q = s.q0 + cc;
        const bool act0 = cc < s.nq, act1 = cc + 1 < s.nq;
        const int rh0 = act0 ? q / ch.mh : s.ra, jh0 = act0 ? q - rh0 * ch.mh : 0;
        const int rh1 = act1 ? (q + 1) / ch.mh : rh0, jh1 = act1 ? q + 1 - rh1 * ch.mh : jh0;
        const int xoff0 = ch.Sh * (rh0 - s.ra), xoff1 = ch.Sh * (rh1 - s.ra);
        const float* h0 = wt + jh0 * ch.Th;
        const float* h1 = wt + jh1 * ch.Th;
        float2 h2[TH > 0 ? TH : 1];
#pragma unroll
        for (int k = 0; k < (TH > 0 ? TH : 1); ++k) h2[k] = TH > 0 ? make_float2(h0[k], h1[k]) : make_float2(0.f, 0.f);
        // the window's first word sits at the low two bits of its global word index
        const int64_t frame_in = (int64_t)H * W;
        const uint32_t wbase = (uint32_t)(reinterpret_cast<uintptr_t>(ch.x) >> 2) +
                               (uint32_t)(s.f * (uint64_t)frame_in) + (uint32_t)s.c0;
        float* yf = ch.y + (int64_t)s.f * ch.H2 * ch.W1 + q;
        // every row's window starts on a 16-byte boundary and each lane's
        // repetition at a multiple of 4 words: 16-byte loads, no conflicts
        const bool v4 = TH > 0 && TH <= 8 && one2 && (ch.Sh & 3) == 0 && (wbase & 3u) == 0 && (W & 3) == 0;
        int ir = s.row0;
        int due = ch.Tv - 1;                               // next row that completes a column-pass window
        int64_t yrow = (int64_t)ch.mv * s.rb0 * ch.W1;     // offset of that repetition's first output row
        const int64_t ystep = (int64_t)ch.mv * ch.W1;
        for (int base = 0; base < s.nrows; base += kSsRows) {
            if (!ptx::mbar_wait_sleep(full0 + 8 * st, phase, AROL_SS_SLEEP_NS)) {
                if (lane == 0) flag(err, 2u);
                return;
            }
            // row pass of the stage's rows (rows past the unit's end read
            // stale words; their sums are dropped)
            const float* sp = stages + st * sf;
            float2 mid[kSsRows];
            int irk = ir;
            if (v4) {
#pragma unroll
                for (int k = 0; k < kSsRows; ++k) mid[k] = ss_dot2_v4<TH>(h2, sp + k * sr + xoff0);
                irk += kSsRows;
                while (irk >= H) irk -= H;
            } else {
#pragma unroll
                for (int k = 0; k < kSsRows; ++k) {
                    const float* row = sp + k * sr + (int)((wbase + (uint32_t)irk * (uint32_t)W) & 3u);
                    mid[k] = ss_dot2<TH>(h2, h0, h1, row + xoff0, row + xoff1, one2, ch.Th);
                    if (++irk == H) irk = 0;
                }
            }
            __syncwarp();
            if (lane == 0) ptx::mbar_arrive(empty0 + 8 * st);
            if (++st == nst) st = 0, phase ^= 1u;
            const int n = min(kSsRows, s.nrows - base);
            float2* rp = ringw + (base & (kSsRing - 1)) * 32 + lane;   // base is a multiple of kSsRows: no wrap
            if (n == kSsRows) {
#pragma unroll
                for (int k = 0; k < kSsRows; ++k) rp[32 * k] = mid[k];
                ir = irk;
            } else {
#pragma unroll
                for (int k = 0; k < kSsRows; ++k)
                    if (k < n) rp[32 * k] = mid[k];
                ir += n;
                while (ir >= H) ir -= H;
            }
            // column pass of every repetition whose window ends in this stage:
            // rows S_v r .. S_v r + T_v - 1 of the band
            for (; due < base + n; due += ch.Sv, yrow += ystep)
                ss_column_pass<TV>(hv2, ch.mv, ch.Tv, ring, due - (ch.Tv - 1), lane, yf + yrow, ch.W1, act0, act1);
        }
    }
}

}  // namespace

SsChain ss_chain_of(const SepChainDev& d) {
    SsChain c{};
    const SepPassDev &ph = d.p[0], &pv = d.p[1];
    c.F = d.F;
    c.H = d.H[0];
    c.W = d.W[0];
    c.W1 = d.W[1];
    c.H2 = d.H[2];
    c.Th = ph.T, c.mh = ph.m, c.Sh = ph.S, c.oh = ph.o;
    c.Tv = pv.T, c.mv = pv.m, c.Sv = pv.S, c.ov = pv.o;
    c.Rv = pv.R;
    c.BH = d.BH > 0 ? d.BH : pv.R;
    c.chunks = (c.W1 + kSsChunk - 1) / kSsChunk;
    c.bands = (c.Rv + c.BH - 1) / c.BH;
    return c;
}

int sepstream_window(const SsChain& c) {
    int xw = 0;
    for (int k = 0; k < c.chunks; ++k) {
        const int64_t q0 = (int64_t)k * kSsChunk, nq = std::min<int64_t>(kSsChunk, c.W1 - q0);
        const int64_t ra = q0 / c.mh, rb = (q0 + nq - 1) / c.mh;
        xw = (int)std::max<int64_t>(xw, c.Sh * (rb - ra) + c.Th);
    }
    return xw;
}

int sepstream_tap_floats(const SsChain& c) { return (((c.mh * c.Th + 1) & ~1) + 2 * c.mv * c.Tv + 3) & ~3; }

int sepstream_stages(int xw_max) {
    const size_t stage = (size_t)kSsRows * ((xw_max + 4 + 3) & ~3) * sizeof(float);
    size_t n = kSsStageBudget / stage;
    n = n < 2 ? 2 : n > (size_t)kSsMaxStages ? (size_t)kSsMaxStages : n;
    return (int)(n & ~(size_t)1);
}

size_t sepstream_smem(int xw_max, int nst, int tap_floats) {
    const int sr = (xw_max + 4 + 3) & ~3;
    return ((size_t)nst * kSsRows * sr + (size_t)kSsCWarps * kSsRing * 32 * kSsCols + (size_t)kSsCWarps * tap_floats) *
               sizeof(float) +
           2 * (size_t)nst * sizeof(uint64_t);
}

int sepstream_chunk_cols() { return kSsChunk; }
int sepstream_max_taps() { return kSsRing - kSsRows + 1; }

namespace {

// The kernel for the passes' tap counts: both exact when T_h = T_v <= 8,
// the row pass exact when T_h <= 8 (one chain), else the general forms.
using SsKernel = void (*)(const SsChain, const SsChain*, const int*, int, int, int, int, int, unsigned*);

template <int T>
SsKernel ss_pick(int Tv, bool batch) {
    if (batch) return Tv == T ? sepstream_kernel<T, T, true> : sepstream_kernel<0, 0, true>;
    return Tv == T ? sepstream_kernel<T, T, false> : sepstream_kernel<T, 0, false>;
}

SsKernel ss_kernel_for(int Th, int Tv, bool batch) {
    switch (Th) {
        case 1: return ss_pick<1>(Tv, batch);
        case 2: return ss_pick<2>(Tv, batch);
        case 3: return ss_pick<3>(Tv, batch);
        case 4: return ss_pick<4>(Tv, batch);
        case 5: return ss_pick<5>(Tv, batch);
        case 6: return ss_pick<6>(Tv, batch);
        case 7: return ss_pick<7>(Tv, batch);
        case 8: return ss_pick<8>(Tv, batch);
        default: return batch ? sepstream_kernel<0, 0, true> : sepstream_kernel<0, 0, false>;
    }
}

// cudaFuncSetAttribute once per kernel and size (the largest so far).
cudaError_t ss_set_smem(SsKernel k, size_t smem) {
    constexpr int kMax = 32;
    static SsKernel seen[kMax] = {};
    static size_t attr[kMax] = {};
    int i = 0;
    while (i < kMax && seen[i] && seen[i] != k) ++i;
    if (i == kMax) return cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    seen[i] = k;
    if (smem > attr[i]) {
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        attr[i] = smem;
    }
    return cudaSuccess;
}

}  // namespace

int sepstream_ctas_per_sm(int Th, int Tv, bool batch, size_t smem) {
    int occ = 0;
    const SsKernel k = ss_kernel_for(Th, Tv, batch);
    if (ss_set_smem(k, smem) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k, kSsThreads, smem) != cudaSuccess)
        return 1;
    return occ > 0 ? occ : 1;
}

cudaError_t launch_sepstream(const SsChain& one, const SsChain* chains, const int* ustart, int nchains, int units,
                             int Th, int Tv, int xw_max, int nst, int tap_floats, unsigned* err, cudaStream_t s) {
    if (units <= 0) return cudaSuccess;
    const bool batch = chains != nullptr;
    const size_t smem = sepstream_smem(xw_max, nst, tap_floats);
    const SsKernel k = ss_kernel_for(Th, Tv, batch);
    cudaError_t e = ss_set_smem(k, smem);
    if (e != cudaSuccess) return e;
    const int cap = device_sm_count() * sepstream_ctas_per_sm(Th, Tv, batch, smem);
    const int grid = units < cap ? units : cap;
    k<<<grid, kSsThreads, smem, s>>>(one, chains, ustart, nchains, units, xw_max, nst, tap_floats, err);
    return cudaGetLastError();
}

}  // namespace arol
