// Internal declarations shared by the host runtime (arol_host.cpp) and the
// CUDA kernels (k_*.cu).  Not part of the public ABI.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace arol {

// One array port bound to the repetition space, prepared on the host for the
// generic tiler kernel.  Every entry of origin/paving/fitting is already
// reduced into [0, shape_k) (Euclidean mod), so the device only ever adds
// non-negative values and subtracts shape_k once on overflow.  Unused array
// dimensions have shape 1 and zero coefficients; unused pattern dimensions
// have extent 1.
// n / d for every n < 2^31 as (n * m) >> s (multiply-shift division with a
// rounded-up reciprocal; m < 2^32).  Prepared on the host by make_fastdiv.
struct FastDiv {
    uint32_t d, m, s, pad_;
};

struct PortDev {
    int32_t shape[4];
    FastDiv shape_div[4];   // division by shape[k]
    int32_t fast;           // 1: the pattern walks one contiguous dimension with step 1
    int32_t fdim;           // that dimension
    int64_t stride[4];      // row-major element strides; 0 for unused dims
    int64_t lin[2];         // element offset of one step along pattern dim 0 / 1: sum_k fitting[k][c] stride[k]
    uint32_t ext[4];        // largest coordinate a pattern adds along each array dim (fittings reduced)
    int32_t linear;         // 1: ext < 2^31, so a pattern with base b and b + ext < shape never wraps
    int32_t pad_;
    uint32_t origin[4];
    uint32_t paving[4][4];  // [array dim][repetition dim]
    uint32_t fitting[4][2]; // [array dim][pattern dim]
    int32_t pattern[2];
};

enum ElemCode : int32_t { ELEM_COPY = 0, ELEM_FIR = 1 };

// Element storage of a FIR task's arrays: the arol_dtype codes.
enum StorageCode : int32_t { kStF32 = 0, kStBf16 = 1, kStF16 = 2 };

// A copy or fir task for the generic tiler kernel (and one entry of a batch).
struct TaskDev {
    int32_t rep[4];         // repetition space, last dimension fastest; unused = 1
    FastDiv rep_div[4];
    int64_t nreps;
    PortDev in, out;
    int32_t T, m;           // fir: pattern size and outputs; copy: both = pattern size
    int32_t elem;           // ElemCode
    int32_t esize;          // copy: element size in bytes (2 or 4)
    int32_t in_dt;          // fir: input storage, a StorageCode (16-bit values widen exactly to f32)
    int32_t out_dt;         // fir: output storage, a StorageCode (16-bit stores round to nearest even)
    int32_t wide;           // 1 when repetition indices or base sums reach 2^31 (64-bit path)
    int32_t rowfir;         // 1: rank-2 row FIR (paving [[1,0],[0,step]], fitting [[0],[1]], output
                            //    paving [[1,0],[0,m]]) with step, T <= 32 and m <= 16: row-tile path
    int32_t colfir;         // 1: rank-2 column FIR (paving [[step,0],[0,1]], fitting [[1],[0]], output
                            //    paving [[m,0],[0,1]], fitting [[1],[0]]) with T <= 32 and m <= 16
    int32_t fir2d;          // 1: rank-2 FIR on a 2-D pattern (paving [[s0,0],[0,s1]], fitting identity,
                            //    outputs m consecutive along the row): 2-D window tiles
    int32_t s0, s1, p0, p1; // fir2d: steps and pattern extents (rows, columns)
    int32_t bh, bw;         // fir2d: repetitions per CTA tile (rows, columns)
    int32_t step;           // input paving along the row (row FIR) or down the column (column FIR), reduced
    int32_t cf_frames;      // column FIR: frames (rep[1]); the ports describe one frame
    int64_t cf_in_frame, cf_out_frame;   // column FIR: input and output elements per frame
    const float* taps;      // m x T (fir)
    const float* taps_t;    // column-FIR tasks in a batch: taps transposed, T x 16, zero padded;
                            // row-FIR tasks: transposed and doubled, T x 32 (see RowTileDev)
    const void* x;
    void* y;
    int64_t in_elems, out_elems;   // array sizes, for the bounds checks of AROL_DEBUG builds
    unsigned* err;                 // AROL_DEBUG builds: bit 0x100 (input) / 0x200 (output) on an out-of-range index
};

// One unit of work of a batch: repetitions [start, start + count) of a task.
struct TileDev {
    int32_t task;
    int32_t count;
    int64_t start;
};

// One tile of a row-FIR task in a batch (see k_rowfir.cu): rows row0 ..
// row0 + nrows - 1 (mod H) of the input, repetitions a0 .. a0 + cnt - 1 of
// each row.  Built on the host; x, y and taps_t are filled in when the
// batch's buffers are known.
struct RowTileDev {
    const float* x;         // input array, rows of W floats
    float* y;               // output array, rows of Wout floats
    const float* taps_t;    // the task's taps transposed and doubled, T x 32: [k * 32 + 2 j + e] = H[j, k]
                            // (e = 0, 1; zero for j >= m), 16-byte aligned
    int32_t W, H;           // input row length and row count
    int32_t Wout, Hout;     // output row length and row count
    int32_t row0, orow0;    // input and output row of the tile's first row (reduced)
    int32_t nrows;          // rows in the tile, 1..32
    int32_t c0;             // window's first input column: (o1 + S a0) mod W
    int32_t oc0;            // first output column: (oo1 + M a0) mod Wout
    int32_t cnt;            // repetitions per row
    int32_t S, T, M;        // step (1..32), taps (<= 32), outputs per repetition (<= 16)
    int32_t lw;             // window words per row: S (cnt - 1) + T
    int32_t ss;             // row slot stride in floats: a multiple of 32, >= lw + 6
    int32_t a;              // rows per warp unit: 1, 2, 4, ..., 32 (the unit has 32 / a repetitions per row)
    int32_t out_wrap;       // 1 when the tile's output columns wrap at Wout
    int32_t task;           // the batch task this tile belongs to (host bookkeeping)
};
// Shared-memory stage of the row-FIR kernel (floats): the tile record, a
// table of its rows, the row slots, and the taps (32 T floats) at its end; a
// tile's slots take nrows * ss floats, at most kRowSlotFloats - 32 (T - 1)
// (kRowSlotFloats leaves room for T = 1).
#ifndef AROL_ROW_STAGE_FLOATS
#define AROL_ROW_STAGE_FLOATS 3456
#endif
constexpr int kRowStageFloats = AROL_ROW_STAGE_FLOATS;
constexpr int kRowSlotFloats = kRowStageFloats - 32 - 32 * 4 - 32 - 28;
cudaError_t launch_rowfir_batch(const RowTileDev* tiles, int ntiles, int grid, unsigned* err, cudaStream_t s);
int rowfir_ctas_per_sm();

// Parameters of the fused separable downscaler chain (8-tap -> 3-output on
// both axes, step 8, no wrap): x (frames, H, W) -> y (frames, 3H/8, 3W/8).
struct DownscaleDev {
    const float* x;
    float* y;
    const float* taps;      // 3x8 horizontal, then 3x8 vertical
    const float* gy;        // backward: dL/dy
    float* gx;              // backward: dL/dx
    float* partials;        // backward: per-CTA tap-gradient partials (48 floats each)
    unsigned* err;          // nullable: bit set when a bounded wait gives up
    int32_t in16;           // forward: x stored in 16 bits
    int32_t mid16;          // forward: the intermediate array is declared 16-bit (rounded)
    int32_t out16;          // forward: y stored in 16 bits
    int32_t half16;         // forward: the 16-bit arrays are IEEE half (else bfloat16)
    float* grad_taps;       // backward: 48 tap gradients, written by the last CTA (nullable)
    unsigned* ticket;       // backward: CTAs done (zero before the launch; the last CTA resets it)
    int64_t frames;
    int32_t H, W;
};

// One member of a batch of separable 8 -> 3 chains (k_downscale.cu): f32
// frames (frames x H x W, 16-byte aligned), taps 3x8 horizontal then 3x8
// vertical, column chunks of Wc (downscale_chunk), nch of them.
struct DsMember {
    const float* x;
    float* y;
    const float* taps;
    int64_t frames;
    int32_t H, W, Wc, nch;
};
int downscale_chunk(int W);
// One launch over the units of nmem members (unit prefix ustart[0 .. nmem],
// staged row stride Ws >= every member's Wc).
cudaError_t launch_downscale_batch(const DsMember* mem, const int* ustart, int nmem, int units, int Ws, unsigned* err,
                                   cudaStream_t s);

// Launchers (return cudaGetLastError() of the launch).
// Block tiling of the generic walk (tiler_tiled_kernel): a tile is R 2^lb
// consecutive repetitions along dim db (lane l takes l, l + 2^lb, ...)
// times ta along dim da (da = -1: none), so that the overlapping or
// neighbouring patterns of nearby repetitions share cache lines within one
// SM.
struct GenGeom {
    int32_t da, db;        // tiled repetition dims; every dim after da other than db has extent 1
    int32_t lb, ta;        // log2 of the threads along db; threads along da
    uint32_t na, nb;       // tiles along da and db
    uint32_t ntiles;       // (repetitions before the tiled dims) x na x nb, < 2^31
    int32_t tap_floats;    // taps staged in shared memory, transposed T x MAXM; 0: read from global memory
    FastDiv na_div, nb_div;
    uint32_t istep[4], ostep[4];   // base-coordinate step of 2^lb repetitions along db, reduced mod shape
    int64_t idelta, odelta;        // the element offsets of those steps when no coordinate wraps
};
cudaError_t launch_tiler_generic(const TaskDev& t, int max_m, cudaStream_t s);
cudaError_t launch_tiler_tiled(const TaskDev& t, const GenGeom& g, int max_m, cudaStream_t s);
int tiler_tiled_maxm(int max_m);
int tiler_tiled_reps(int max_m);   // repetitions per thread (R) of the tiled kernel for that bank size
// CTA b takes tiles b, b + grid, ... (a static schedule; `counter` is unused).
cudaError_t launch_fir2d(const TaskDev& t, cudaStream_t s);
// A 2-D window task that launch_fir2d runs on the register-blocked stencil
// kernel (steps 1, one output, a 3x3 or 5x5 pattern).
bool fir2d_uses_stencil(const TaskDev& t);
cudaError_t launch_wait_selftest(unsigned* err, cudaStream_t s);
cudaError_t launch_batch_persistent(const TaskDev* tasks, const TileDev* tiles, int ntiles,
                                    unsigned* counter, int grid, int threads, int max_m,
                                    cudaStream_t s);
constexpr int kBatchThreads = 128;                  // threads of the batch kernel (its launch bound)
cudaError_t launch_downscale_fwd(const DownscaleDev& p, cudaStream_t s);
cudaError_t launch_downscale_bwd(const DownscaleDev& p, float* grad_taps, int nparts, bool with_fwd,
                                 cudaStream_t s);
int downscale_bwd_partials(int sm_count, int W);   // per-CTA partial slots the backward uses for width W

// Fused chains of separable FIR passes (sepchain.h).
struct SepChainDev;
struct SepPassDev;
cudaError_t launch_sepchain(const SepChainDev& d, cudaStream_t s);
// dL/dIn of one pass of a separable chain (k_sepchain.cu): input F x Hin x
// Win, output F x Hout x Wout, taps the pass's m x T block.
cudaError_t launch_sep_adjoint(const SepPassDev& p, int64_t F, int Hin, int Win, int Hout, int Wout, const float* taps,
                               const float* gy, float* gx, cudaStream_t s);
// dL/dH of one pass (m <= 8, T <= 16; false otherwise, nothing launched):
// per-block partials (sep_dh_blocks() x m T floats) reduced into grad_taps.
int sep_dh_blocks();
bool sep_dh_supported(const SepPassDev& p);
cudaError_t launch_sep_dh(const SepPassDev& p, int64_t F, int Hin, int Win, int Hout, int Wout, const void* x, int x_dt,
                          const float* gy, float* partials, float* grad_taps, cudaStream_t s);   // x_dt: arol_dtype
// Backward of one separable pass in one sweep (k_sepbwd.cu): dX (gx, may be
// null) and the tap gradients (grad_taps, may be null; plan.blocks x m T
// partials), for repetitions that tile the axis and data that fit one of the
// kernels' forms (sep_bwd_plan false otherwise).
struct SepBwdPlan {
    int form;       // 0 column passes; 1 row passes, staged rows; 2 row passes in 16-word regions
    int bin;        // the kernel's (windows, outputs, taps) bank
    int ss;         // compile-time step (0: the pass's)
    int mm;         // outputs bank of form 2
    bool async;     // form 1: rows copied ahead
    size_t smem;    // dynamic shared memory per block
    int threads;
    int blocks;     // grid: one row of tap-gradient partials per block
};
bool sep_bwd_plan(const SepPassDev& p, int64_t F, int Hin, int Win, int x_dt, const void* x, const float* gy,
                  const float* gx, bool want_taps, SepBwdPlan* plan);
cudaError_t launch_sep_bwd(const SepBwdPlan& plan, const SepPassDev& p, int64_t F, int Hin, int Win, const float* taps,
                           const void* x, int x_dt, const float* gy, float* gx, float* partials, float* grad_taps,
                           cudaStream_t s);
// Row FIR in 16-word regions (k_rowregion.cu): repetitions that tile each row
// (S R = W), S in {2, 4, 8}, T <= 8, M <= 4 (2 for S = 2), W a multiple of
// 16, origin o a multiple of 16, output rows of M R words from column 0, one
// per input row; x and y 16-byte aligned.
bool rowfir_region_supported(int S, int T, int M, int64_t W, int64_t Wout, int64_t o, int64_t rows);
cudaError_t launch_rowfir_region(int S, int T, int M, int64_t rows, int W, int o, const float* taps, const float* x,
                                 float* y, unsigned* err, cudaStream_t s);
// Sum of nblocks rows of npairs partials, in a fixed order (k_tiler.cu).
cudaError_t launch_tap_reduce(const float* partials, int nblocks, int npairs, float* out, cudaStream_t s);
size_t sepchain_smem(const SepChainDev& d);
// One chain of the streaming row-then-column kernel (k_sepstream.cu): a row
// pass (taps hh, m_h x T_h, step S_h, origin o_h) then a column pass (hv,
// m_v x T_v, S_v, o_v) on F frames of H x W, intermediate and output W1
// columns, H2 = m_v R_v output rows; units of one frame, one chunk of
// sepstream_chunk_cols() intermediate columns and one band of BH column-pass
// repetitions.
struct SsChain {
    const float* x;
    float* y;
    const float* hh;
    const float* hv;
    int64_t F;
    int32_t H, W, W1, H2;
    int32_t Th, mh, Sh, oh;   // oh in [0, W)
    int32_t Tv, mv, Sv, ov;   // ov in [0, H)
    int32_t Rv, BH;
    int32_t chunks, bands;
};
SsChain ss_chain_of(const SepChainDev& d);           // BH, chunks and bands from d.BH; pointers left null
int sepstream_window(const SsChain& c);               // widest input window of a chunk, words
int sepstream_tap_floats(const SsChain& c);           // shared taps per consumer warp
size_t sepstream_smem(int xw_max, int nst, int tap_floats);
int sepstream_stages(int xw_max);
int sepstream_chunk_cols();
int sepstream_max_taps();
int sepstream_ctas_per_sm(int Th, int Tv, bool batch, size_t smem);
// One launch over the units of one chain (chains = nullptr: `one`) or of
// nchains chains in device memory (unit prefix ustart[0 .. nchains]).  Th,
// Tv pick the exact-tap variant when every chain has those tap counts
// (0: any).
cudaError_t launch_sepstream(const SsChain& one, const SsChain* chains, const int* ustart, int nchains, int units,
                             int Th, int Tv, int xw_max, int nst, int tap_floats, unsigned* err, cudaStream_t s);

// tcgen05 matmul: C (M x N, f32) = A (M x K, bf16 row-major) . B (K x N, bf16 row-major).
cudaError_t launch_matmul_tc(const void* A, const void* B, float* C, int M, int N, int K,
                             unsigned* err_flag, cudaStream_t s);

int device_sm_count();

}  // namespace arol
