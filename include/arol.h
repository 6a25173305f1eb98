/*
 * arol.h — C ABI of the GB300 Array-OL repetitive-task library.
 *
 * A repetitive task (MARTE Repetitive Structure Modeling, named in Sec. 3 of
 * Rodrigues, Guyomarc'h and Dekeyser 2011; "repetitive and thus potentially
 * parallel" tasks mapped onto GPU processors, Sec. 7) runs one elementary task
 * per point r of a repetition space R.  Its ports are arrays whose shape and
 * element type come from the flow ports (Sec. 5: dimAllocation and
 * typeAllocation; Sec. 6.3: direction — input ports are read-only).  A tiler
 * connects a port to the repetition space: for repetition r and pattern index i
 * it names the array element
 *
 *     e(r, i) = (origin + paving . r + fitting . i) mod shape
 *
 * componentwise with a Euclidean mod (result in [0, shape_k)).  Input tilers
 * gather patterns, the elementary task maps them, the output tiler scatters
 * the result and must write every element of its array exactly once.
 *
 * Conventions for every entry point
 *  - Arrays are dense and row-major (last dimension contiguous).  Array and
 *    pattern pointers passed to run calls are DEVICE pointers owned by the
 *    caller; the library never frees them.  The only host-pointer entry point
 *    is arol_task_run_host.
 *  - `stream` is a cudaStream_t passed as void* (NULL = the legacy default
 *    stream).  Work is enqueued asynchronously on it; the call returns after
 *    enqueueing (arol_task_run_host is the exception: it synchronizes).
 *  - Every call returns an arol_status and, on failure, records a message
 *    readable with arol_last_error (thread-local).  No C++ exception crosses
 *    the ABI.  A failed call enqueues nothing.
 *  - Handles (arol_task, arol_batch) own copies of their descriptors, taps and
 *    any scratch or staging memory they allocate; destroy them with
 *    arol_task_destroy / arol_batch_destroy after the streams they were used
 *    on have finished.
 *  - Calls on one handle must not run concurrently from several host threads.
 */
#ifndef AROL_H
#define AROL_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define AROL_VERSION 101            /* 1.0.1: arol_task_info_t.path */
#define AROL_MAX_RANK 4             /* array rank and repetition-space rank */
#define AROL_MAX_PATTERN_RANK 2     /* pattern rank */
#define AROL_MAX_FIR_M 32           /* outputs per pattern of a FIR bank */
#define AROL_MAX_FIR_TAPS 8192      /* m * T */

typedef enum {
    AROL_OK = 0,
    AROL_ERR_INVALID = 1,        /* malformed descriptor, null handle/pointer, bad size */
    AROL_ERR_NOT_PARTITION = 2,  /* an output tiler does not write each element exactly once */
    AROL_ERR_UNSUPPORTED = 3,    /* well formed, but outside what the kernels implement */
    AROL_ERR_CUDA = 4,           /* a CUDA runtime call or kernel launch failed */
    AROL_ERR_TIMEOUT = 5,        /* a bounded device-side wait gave up */
    AROL_ERR_OOB = 6             /* a device-side bounds check fired (checked builds only) */
} arol_status;

/* Element storage (Sec. 5 typeAllocation).  FIR arithmetic is f32 for every
 * storage type: 16-bit inputs are widened exactly, 16-bit outputs (and a
 * 16-bit chain intermediate) are rounded to nearest even.  Copy tasks move
 * raw bits of any type; matmul inputs are bfloat16 only; backward passes of
 * fir tasks read saved inputs of any storage (widened exactly) and take and
 * give gradients in float32; a chain's intermediates must be float32 there;
 * copy tasks differentiate on float32 only. */
typedef enum {
    AROL_F32 = 0,    /* IEEE binary32 */
    AROL_BF16 = 1,   /* bfloat16: the upper 16 bits of a binary32 */
    AROL_F16 = 2     /* IEEE binary16 (half) */
} arol_dtype;

typedef enum {
    AROL_ELEM_COPY = 0,    /* y[j] = p[j]: raw bits, NaN payloads kept */
    AROL_ELEM_FIR = 1,     /* y[j] = sum_k H[j,k] p[k], H is m x T (a bank of m tap rows) */
    AROL_ELEM_MATMUL = 2   /* y = p_A . p_B, patterns (a x K) and (K x b), bf16 in, f32 out */
} arol_elem_kind;

/* An array port (Sec. 5 MemoryMap/DataAllocate: dimAllocation = shape,
 * typeAllocation = dtype).  rank in [1, 4]; shape entries in [0, 2^31).  An
 * array with no elements is only allowed in a task whose repetition space is
 * empty (the output must then be empty too: the empty partition). */
typedef struct {
    int32_t rank;
    int32_t dtype;                 /* arol_dtype */
    int64_t shape[AROL_MAX_RANK];
} arol_array_desc;

/* A tiler: origin (rank entries), paving [array dim][repetition dim],
 * fitting [array dim][pattern dim], pattern shape (pattern_rank entries in
 * [1, 2], each >= 1).  Entries may be negative; they are taken mod shape. */
typedef struct {
    int64_t origin[AROL_MAX_RANK];
    int64_t paving[AROL_MAX_RANK][AROL_MAX_RANK];
    int64_t fitting[AROL_MAX_RANK][AROL_MAX_PATTERN_RANK];
    int32_t pattern_rank;
    int32_t reserved_;
    int64_t pattern[AROL_MAX_PATTERN_RANK];
} arol_tiler;

/* One repetitive task.  copy and fir take one input port, matmul two; every
 * task has one output port.  A repetition-space entry may be 0 (empty task).
 * fir_taps_host (m x T, row-major, float) is copied at create time; it may be
 * NULL, in which case arol_task_set_taps must be called before running. */
typedef struct {
    int32_t rep_rank;
    int32_t elem;                  /* arol_elem_kind */
    int64_t rep[AROL_MAX_RANK];
    int32_t n_in;
    int32_t n_out;
    arol_array_desc in[2];
    arol_array_desc out[1];
    arol_tiler in_tiler[2];
    arol_tiler out_tiler[1];
    int32_t fir_T;
    int32_t fir_m;
    const float* fir_taps_host;
} arol_task_desc;

typedef struct arol_task_s* arol_task;
typedef struct arol_batch_s* arol_batch;

/* What the library chose for a task (filled by arol_task_info). */
typedef struct {
    int32_t kind;              /* 0 single task, 1 chain */
    int32_t kernel;            /* 0 generic tiler, 1 fused separable downscaler (8 -> 3, step 8), 2 tcgen05 matmul,
                                  3 unfused chain, 4 fused separable chain (any row and column passes),
                                  5 fused row-then-column chain (streaming rows) */
    int64_t reps;              /* repetitions of the task (sum over a chain's tasks) */
    int64_t gathered_elems;    /* pattern elements gathered over all inputs (and tasks) */
    int64_t scattered_elems;   /* elements scattered (sum over a chain's tasks) */
    int64_t unique_bytes;      /* algorithmic bytes: every external input element read once,
                                  every final output element written once */
    double flops;              /* arithmetic of the elementary tasks (2 per multiply-add) */
    int32_t path;              /* a single task with kernel 0 and taps given on the host: 0 per-repetition
                                  walk, 1 row-FIR tiles, 2 column-FIR tiles, 3 2-D window tiles,
                                  4 register-blocked stencil (3x3 or 5x5, steps 1, one output),
                                  5 row FIR in 16-word regions (repetitions tiling each row, step 2, 4
                                  or 8, T <= 8, m <= 4, rows of a multiple of 16 words, origin a
                                  multiple of 16, output columns from 0; row-FIR tiles when a buffer
                                  is not 16-byte aligned); -1 otherwise */
    int32_t reserved_;
} arol_task_info_t;

/* ---- tasks --------------------------------------------------------------- */

/* Validate `desc` and build a task handle.  Host only: touches no GPU state.
 * Checks ranks, shapes, the elementary-task/pattern/dtype combination (copy:
 * same dtype and pattern size in and out; fir: f32, bf16 or f16 in and out,
 * pattern size T, output pattern size m; matmul: bf16 inputs with the panel
 * tilers of a tiled
 * product, f32 output) and that the output tiler partitions its array
 * (AROL_ERR_NOT_PARTITION otherwise).  On success *out owns a copy of the
 * descriptor and of the taps. */
arol_status arol_task_create(const arol_task_desc* desc, arol_task* out);

/* Chain n >= 2 single tasks through shared arrays (Sec. 5, associatedParts:
 * all elements of the model that use the same allocation): the output array
 * of tasks[k] is the input array of tasks[k+1] (same shape and dtype,
 * AROL_ERR_INVALID otherwise).  The chain copies what it needs from the tasks;
 * they may be destroyed afterwards.  Its run, backward and fwd_bwd take the
 * first task's inputs and the last task's output.  Fused chains never write
 * their intermediates to HBM:
 *  - the separable 8 -> 3 block downscaler (horizontal then vertical fir,
 *    step 8, no wrap) runs on its own kernel (kernel 1) when its storage is
 *    all f32, or 16-bit frames (bf16 or f16) with an intermediate and an
 *    output each f32 or of the frames' type;
 *  - any other f32 chain of 2 to 4 row passes (a fir along each row) and
 *    column passes (down each column), each identity on the other axis and
 *    the frames, with T <= 32, m <= 16, any step and input origin (wrap
 *    included), runs on a fused kernel: a row pass then a column pass on the
 *    streaming kernel (kernel 5: rows of the input streamed through shared
 *    memory, each intermediate column's last rows in a shared ring; T_v <= 29),
 *    other chains on the tile kernel (kernel 4: tiles of the
 *    last array, every pass in shared memory); the environment variable
 *    AROL_SEPSTREAM=off (or 0), read here, keeps a row-then-column chain on
 *    the tile kernel;
 * other chains run stage by stage through intermediates the chain owns. */
arol_status arol_chain_create(const arol_task* tasks, int n, arol_task* out);

/* Equal partition of a task over devices (Sec. 7: the generated host code
 * spreads the repetitive tasks equally over 1, 2 or 4 GPUs; every repetition
 * is independent, so the parts need no exchange).  Host only.  `desc` must
 * have a frame dimension: in every port, array dimension 0 is repetition
 * dimension 0 (extent rep[0], paving 1 on it and 0 elsewhere, fitting 0,
 * origin 0).  Part `part` (0 <= part < parts) gets frames [*first_frame,
 * *first_frame + count), count = rep[0] / parts, plus one for the first
 * rep[0] % parts parts; *out is `desc` on those frames alone (rep[0] and
 * every port's dimension 0 set to count), whose arrays are the frame slices
 * of the full ones: the part's device holds only its slices.  A chain is
 * sharded task by task with the same part.  Taps are not copied (the
 * fir_taps_host pointer is kept).  The tap gradients of a backward are
 * partial sums per part: their sum over the parts (an all-reduce) is the
 * full gradient; grad_in is the part's slice.  AROL_ERR_UNSUPPORTED without
 * a frame dimension, AROL_ERR_INVALID for a bad part. */
arol_status arol_task_shard_frames(const arol_task_desc* desc, int parts, int part, arol_task_desc* out,
                                   int64_t* first_frame);

/* Replace the fir taps.  on_device = 0: `taps` is host memory, copied now.
 * on_device = 1: `taps` is a device pointer the caller keeps alive and
 * unchanged while runs that use it are in flight (it is read, never written).
 * For a chain the taps are the concatenation of each task's m x T block in
 * task order. */
arol_status arol_task_set_taps(arol_task t, const float* taps, int on_device);

/* Run the task: in[k] is the device pointer of input port k, out[0] of the
 * output port.  Inputs are read-only (Sec. 6.3); they must not overlap the
 * output.  Row-FIR tasks that the 16-word-region kernel takes (info path 5)
 * run there when both buffers are 16-byte aligned.  Other row- and
 * column-FIR tasks and chains outside the fused kernel run on the batch
 * engine as a one-member batch the handle owns (built at the first run,
 * rebuilt after arol_task_set_taps); with taps on the device they take the
 * per-repetition kernel.  A handle may be used from several streams:
 * a change of buffers is ordered after its launches on any stream. */
arol_status arol_task_run(arol_task t, const void* const* in, void* const* out, void* stream);

/* Same computation from HOST buffers: copies each input from host memory to
 * device staging buffers owned by the task, runs, copies the output back to
 * host memory, and synchronizes `stream` before returning.  Host buffers
 * should be page-locked for full bandwidth. */
arol_status arol_task_run_host(arol_task t, const void* const* host_in, void* const* host_out, void* stream);

/* Reverse mode of a fir task or chain for a loss L with dL/d(out) = grad_out
 * (float32, output shape).  saved_in: the forward inputs (device, their own
 * storage: 16-bit inputs are widened exactly).  grad_in (nullable, device,
 * float32, input shape) is OVERWRITTEN with dL/d(in): the transposed-tiler
 * scatter-add, which
 * sums over every (r, i) whose gather visited an element (overlaps and modulo
 * wrap included).  grad_taps (nullable, device, m x T floats, a chain's blocks
 * concatenated) is OVERWRITTEN with dL/dH.  Deterministic: no atomics.
 * Row and column FIR passes (single tasks and the passes of a separable
 * chain) whose repetitions tile their axis take one sweep per pass for dX and
 * the tap gradients; a chain recomputes its intermediates from saved_in, and
 * a separable chain does so only when grad_taps is given. */
arol_status arol_task_backward(arol_task t, const void* grad_out, const void* const* saved_in,
                               void* grad_in, float* grad_taps, void* stream);

/* Forward and reverse mode in one pass when grad_out is known before the
 * forward runs (e.g. loss = sum(W * out)): writes out, grad_in and grad_taps
 * as arol_task_run followed by arol_task_backward would.  The f32 fused
 * separable downscaler (kernel 1, 16-byte aligned buffers) does both in one
 * kernel that reads the inputs once; every other fir task or chain runs the
 * forward, then the backward, on `stream`. */
arol_status arol_task_fwd_bwd(arol_task t, const void* const* in, const void* grad_out, void* out,
                              void* grad_in, float* grad_taps, void* stream);

/* Sizes and work of a task (host only). */
arol_status arol_task_info(arol_task t, arol_task_info_t* info);

void arol_task_destroy(arol_task t);

/* Host-side partition check (no task needed): *count_max and *count_min
 * receive the largest and smallest number of (r, j) pairs that the tiler maps
 * onto one element of the array; a partition has both equal to 1. */
arol_status arol_tiler_cover(const arol_array_desc* array, const arol_tiler* tiler,
                             int rep_rank, const int64_t* rep, int64_t* count_min, int64_t* count_max);

/* Self-test of failure detection (no counterpart in the paper).  Launches a
 * kernel whose thread waits on an mbarrier that nothing completes, through
 * the same bounded wait the pipelined kernels use: the wait gives up after
 * its limit (about 2 s), sets an error word and the kernel returns.  Returns
 * AROL_ERR_TIMEOUT when that happens (the expected result), AROL_OK if the
 * wait completed.  No trap or fault is involved; the context stays usable.
 * Synchronizes the stream. */
arol_status arol_selftest_wait_timeout(void* stream);

/* ---- batches of independent tasks ---------------------------------------- */

/* Build a batch of n independent members (uneven shapes allowed).  A member
 * is a single-input copy/fir task or a chain of them from arol_chain_create
 * (Sec. 5: tasks linked through shared arrays).  Chain members keep their
 * intermediates on chip when a fused form serves them all in one launch:
 * chains the fused 8 -> 3 downscaler takes (f32) run on its batched form
 * while their input is 16-byte aligned (checked every run; a change of that
 * set rebuilds the work lists and the graph), row-then-column chains (kernel
 * 5 of arol_task_info) on the batched streaming chain kernel.  Other chains
 * enter as their tasks, one per stage.  The batch copies the descriptors and
 * host taps (the handles may be destroyed afterwards), owns one device arena
 * for the staged chain intermediates, a device work list of tiles grouped by
 * stage, built on first run, and a CUDA graph that launches the fused chain
 * kernels, then the persistent kernels of each stage: stage k of every chain
 * runs after stage k - 1 of every chain.  Row-FIR tasks (one row per repetition row,
 * step <= 32 along it, T <= 32, m <= 16, f32) run as tiles of whole rows or
 * row pieces on the row-FIR kernel; the others as repetition ranges on the
 * general persistent kernel.  Matmul tasks and tasks whose
 * taps live on the device are rejected (AROL_ERR_UNSUPPORTED /
 * AROL_ERR_INVALID). */
arol_status arol_batch_create(const arol_task* tasks, int n, arol_batch* out);

/* Run every member of the batch in one graph launch: in[k] / out[k] are
 * member k's input and output device pointers (for a chain, the first task's
 * input and the last task's output).  When the pointers differ from the
 * previous call the device table is refreshed (one copy) before the launch. */
arol_status arol_batch_run(arol_batch b, const void* const* in, void* const* out, void* stream);

/* The same tasks with one kernel launch per task (each stage of a staged
 * chain is a task; a chain on a fused kernel is one launch), in order, on
 * `stream`:
 * the same kernel over each task's own tiles, without the graph or the shared
 * tile counter (for comparison with arol_batch_run). */
arol_status arol_batch_run_per_task(arol_batch b, const void* const* in, void* const* out, void* stream);

/* Autotune the batch's tile shapes and grid sizes by timing candidates on
 * the given buffers (outputs are overwritten): for row-FIR tasks the shared
 * memory a row tile may fill and the CTAs per SM of the row-FIR kernel, for
 * the other tasks the repetitions per tile and CTAs per SM of the persistent
 * kernel.  Results are
 * cached per process by batch signature and device, and persisted as JSON in
 * the file named by the AROL_TUNE_CACHE environment variable when it is set.
 * force = 1 re-times even when a cached choice exists.  Synchronizes.
 * The AROL_TUNE environment variable overrides: "off" returns AROL_OK at once
 * and keeps the current launch shape (no device work, buffers not read),
 * "force" re-times as force = 1 does. */
arol_status arol_batch_tune(arol_batch b, const void* const* in, void* const* out, void* stream, int force);

/* The tile size (repetitions per tile) and CTAs per SM in use. */
arol_status arol_batch_config(arol_batch b, int64_t* tile_reps, int32_t* ctas_per_sm, int32_t* threads);

/* Synchronizes `stream`, then reports AROL_ERR_TIMEOUT if a bounded wait
 * inside the batch's kernels gave up since the last query (the word is
 * cleared), else AROL_OK. */
arol_status arol_batch_sync_status(arol_batch b, void* stream);

void arol_batch_destroy(arol_batch b);

/* ---- errors and version --------------------------------------------------- */

/* Copy the calling thread's last error message into buf (NUL-terminated,
 * truncated to len).  Returns AROL_OK. */
arol_status arol_last_error(char* buf, size_t len);

int arol_version(void);

/* sizeof of the ABI structs as this library was compiled (0: arol_array_desc,
 * 1: arol_tiler, 2: arol_task_desc, 3: arol_task_info_t; -1 otherwise), so a
 * binding can check its own struct layout against the library's. */
int64_t arol_abi_struct_size(int which);

/* Synchronize `stream`, then report device-side failures recorded by kernels
 * of task t since the last report: AROL_ERR_TIMEOUT when a bounded wait inside
 * a pipelined kernel (the tensor-core matmul, the fused downscaler) gave up —
 * its outputs are then incomplete — AROL_OK otherwise.  Reporting clears the
 * record. */
arol_status arol_task_sync_status(arol_task t, void* stream);

/* ---- sparse rows and conjugate gradient (Sec. 7 case study) -------------- */

/* The case study of Sec. 7 solves a symmetric positive definite system stored
 * in Compressed Sparse Row format with conjugate gradient; its DGEMV(sparse)
 * step is a repetitive task over the rows, where row i gathers the columns of
 * its nonzeros, and a continue-condition ends the loop (Table 1: N = 132651,
 * NNZ = 3442951, tol = 1e-10, double precision).  All matrix and vector
 * pointers are DEVICE pointers owned by the caller: row_ptr (n_rows + 1
 * int64, row_ptr[0] = 0, non-decreasing, row_ptr[n_rows] = nnz), col_idx
 * (nnz int32 in [0, n_rows)), vals (nnz float64).  Column indices are not
 * checked on the device: out-of-range entries are the caller's error. */
typedef struct arol_cg_s* arol_cg;

/* y = A x (float64) with a fixed summation order: 1, 2, 4 or 8 lanes per row
 * chosen from the mean row length (or by the AROL_SPMV_LPR environment
 * variable).  x and y have n_rows entries and must not overlap. */
arol_status arol_csr_spmv(int64_t n_rows, int64_t nnz, const int64_t* row_ptr, const int32_t* col_idx,
                          const double* vals, const double* x, double* y, void* stream);

/* Check a CSR matrix on the device: row_ptr[0] == 0, row_ptr[n_rows] == nnz,
 * row_ptr non-decreasing, every col_idx in [0, n_rows).  Returns
 * AROL_ERR_INVALID (with the failed rule in arol_cg_last_error) for a
 * malformed matrix, AROL_ERR_UNSUPPORTED for n_rows >= 2^31.  Device
 * pointers; synchronizes the stream.  arol_cg_create runs it; arol_csr_spmv
 * does not (call it once per matrix). */
arol_status arol_csr_check(int64_t n_rows, int64_t nnz, const int64_t* row_ptr, const int32_t* col_idx, void* stream);

/* Prepare conjugate gradient on A: allocates five float64 work vectors, the
 * reduction scratch and the device-side state, and captures a CUDA graph of
 * eight iterations.  The matrix buffers must stay alive and unchanged while
 * the handle is used.  A must be symmetric positive definite (not checked). */
arol_status arol_cg_create(int64_t n_rows, int64_t nnz, const int64_t* row_ptr, const int32_t* col_idx,
                           const double* vals, arol_cg* out);

/* Solve A x = b: x holds the initial guess on entry and the solution on
 * return.  Iterates r = b - A x, p = r; alpha = r.r / p.Ap; x += alpha p;
 * r -= alpha Ap; beta = r.r(new) / r.r(old); p = r + beta p, until
 * ||r|| <= tol ||b|| or max_iter iterations.  The whole loop runs on the
 * device (reductions in a fixed order: the same bits every run); the call
 * synchronizes `stream` and reports the iteration count and ||r|| / ||b||. */
arol_status arol_cg_solve(arol_cg h, const double* b, double* x, double tol, int max_iter, int* iterations,
                          double* rel_residual, void* stream);

void arol_cg_destroy(arol_cg h);

/* The calling thread's last error message of the sparse/CG entry points. */
arol_status arol_cg_last_error(char* buf, size_t len);

/* ---- backward without device allocation ---------------------------------- */

/* The paper has no counterpart to this entry point; it serves callers that
 * cannot allocate device memory: code running while a stream is captured into
 * a CUDA graph (an allocation there breaks the capture), real-time or embedded
 * hosts whose device-memory budget is fixed at start-up, and programs whose
 * memory belongs to an allocator that must not be bypassed.
 *
 * Same result as arol_task_backward on the fused separable downscaler chain
 * (horizontal then vertical 8-tap -> 3-output fir, step 8): x (frames, height,
 * width) f32 and grad_out (frames, 3*height/8, 3*width/8) f32 are read;
 * grad_in (nullable, x's shape) and grad_taps (nullable, 48 floats: the 3x8
 * horizontal block, then the 3x8 vertical block) are OVERWRITTEN; taps (48
 * floats, same layout) is read.  All pointers are device pointers owned by the
 * caller; x, grad_out and grad_in must be 16-byte aligned; height and width
 * must be multiples of 8.
 *
 * Nothing is allocated: not by cudaMalloc, cudaFree or any allocating library
 * routine.  The only scratch (one 48-float partial per CTA, a ticket word and
 * an error word) is a static device array of 1024 partials (192 KiB) that
 * every GPU loading this library keeps until the process exits; the launch
 * uses at most 1024 CTAs (the kernels stride over the work, so a device that
 * could hold more still gets the whole result).  frames * height/8 * width/4
 * >= 2^31 work items gives AROL_ERR_UNSUPPORTED.  The first call on each
 * device looks up the array's device address (with that device current);
 * make that first call before any stream capture.  All calls share the array:
 * every CTA overwrites its partials before they are read and every launch
 * leaves the ticket at zero, so nothing needs clearing, but calls that
 * overlap on the GPU (two streams, or two host threads) race on it and must
 * be serialized by the caller.  Returns AROL_ERR_INVALID for null inputs,
 * unaligned buffers or sizes not multiples of 8; this entry point does not
 * record a message for arol_last_error.
 *
 * Device-side timeouts: every wait inside the kernel is bounded; a wait that
 * gives up sets the array's error word and leaves the gradients incomplete.
 * The call itself returns before the kernel runs, so it cannot see that;
 * arol_downscale_backward_noalloc_status reports it. */
arol_status arol_downscale_backward_noalloc(const float* x, const float* grad_out, const float* taps,
                                            int64_t frames, int32_t height, int32_t width,
                                            float* grad_in, float* grad_taps, void* stream);

/* Status of the no-allocation backward on the current device (the paper has
 * no counterpart either): synchronizes `stream`, then returns
 * AROL_ERR_TIMEOUT if a bounded wait of any arol_downscale_backward_noalloc
 * launch gave up since the last query (clearing the error word), else
 * AROL_OK; AROL_ERR_CUDA if the copy fails.  Allocates nothing; it is a
 * synchronizing call, so it does not belong inside a stream capture. */
arol_status arol_downscale_backward_noalloc_status(void* stream);

#ifdef __cplusplus
}
#endif

#endif /* AROL_H */
