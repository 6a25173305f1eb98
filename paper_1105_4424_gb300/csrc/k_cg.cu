// Sparse matrix-vector product over CSR rows and the conjugate-gradient loop
// (Sec. 7 of the paper: the DGEMV(sparse) step of CG is a repetitive task over
// the rows of a Compressed Sparse Row matrix, scalar steps run between the
// repetitive ones, and a continue-condition ends the loop; Table 1 solves
// N = 132651, NNZ = 3442951 to tol = 1e-10 in double precision).
//
// Row i gathers its nonzeros k in [row_ptr[i], row_ptr[i+1]): LPR lanes
// share a row (chosen from the mean row length), each summing every LPR-th
// product, then a fixed shuffle tree adds their partial sums.  Dot products are reduced per warp, per CTA
// (fixed order) and across CTAs by the last CTA to take a ticket (fixed
// order): results are identical run to run.  One CG iteration is three
// kernels (A p with p.Ap; x, r update with r.r; the new direction), all on the
// device; the scalars live in device memory, a "done" word turns later
// iterations into no-ops, and the host captures iterations into a CUDA graph
// and polls a page-locked copy of the state between graph launches.
#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <new>
#include <string>

#include "arol.h"
#include "arol_internal.h"

namespace arol {
namespace {

constexpr int kCgThreads = 256;
constexpr unsigned kFullMask = 0xffffffffu;

struct CgState {
    double rr, bb, alpha, beta, pap, tol2, rr_old;
    int32_t done, iters, max_iter, pad_;
    unsigned ticket, pad2_;
};

struct Csr {
    const int64_t* row_ptr;
    const int32_t* col;
    const double* val;
    int64_t n;
};

// (A v)_row with LPR lanes per row (a power of two <= 8); every lane of the
// group returns the sum.  Lane `sub` adds products k = a + sub, + LPR, ... in
// order, four per step with all loads issued first; then a fixed shuffle
// tree adds the LPR partial sums.  Fewer lanes per row means fewer
// predicated FMAs and adds on the float64 pipe, more means wider loads.
template <int LPR>
__device__ __forceinline__ double row_dot(const Csr& A, const double* __restrict__ v, int64_t row, int sub) {
    double s = 0.0;
    if (row < A.n) {
        const int64_t a = __ldg(A.row_ptr + row), z = __ldg(A.row_ptr + row + 1);
        int64_t k0 = a + sub;
        // whole steps of four products, all loads issued first ...
        for (; k0 + 3 * LPR < z; k0 += 4 * LPR) {
            double w[4], xv[4];
            int32_t c[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                w[u] = __ldg(A.val + k0 + u * LPR);
                c[u] = __ldg(A.col + k0 + u * LPR);
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) xv[u] = __ldg(v + c[u]);
#pragma unroll
            for (int u = 0; u < 4; ++u) s = fma(w[u], xv[u], s);
        }
        // ... then the remaining products one by one, in the same order
        for (; k0 < z; k0 += LPR) s = fma(__ldg(A.val + k0), __ldg(v + __ldg(A.col + k0)), s);
    }
#pragma unroll
    for (int off = LPR / 2; off > 0; off >>= 1) s += __shfl_xor_sync(kFullMask, s, off, LPR);
    return s;
}

// Block sum of one value per thread in a fixed order (warp tree, then warps in order).
__device__ __forceinline__ double block_sum(double v, double* s_warp) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(kFullMask, v, off);
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) s_warp[w] = v;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x == 0)
        for (int i = 0; i < kCgThreads / 32; ++i) t += s_warp[i];
    __syncthreads();
    return t;   // valid in thread 0
}

// Stores this CTA's partial(s); returns true in every thread of the last CTA
// to finish, after which partials of all CTAs are visible.
__device__ __forceinline__ bool last_cta(CgState* st) {
    __shared__ int s_last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) s_last = atomicAdd(&st->ticket, 1u) == gridDim.x - 1 ? 1 : 0;
    __syncthreads();
    if (s_last) __threadfence();
    return s_last != 0;
}

// Sum of n partials in a fixed order by the whole CTA (valid in thread 0).
__device__ __forceinline__ double sum_partials(const double* __restrict__ part, int n, double* s_warp) {
    double a = 0.0;
    for (int i = threadIdx.x; i < n; i += kCgThreads) a += __ldcg(part + i);
    return block_sum(a, s_warp);
}

template <int LPR>
__global__ void __launch_bounds__(kCgThreads) spmv_kernel(const Csr A, const double* __restrict__ x, double* __restrict__ y) {
    constexpr int kRowsPerBlock = kCgThreads / LPR;
    const int sub = threadIdx.x & (LPR - 1);
    const int64_t stride = (int64_t)gridDim.x * kRowsPerBlock;
    for (int64_t base = (int64_t)blockIdx.x * kRowsPerBlock; base < A.n; base += stride) {
        const int64_t row = base + threadIdx.x / LPR;
        const double s = row_dot<LPR>(A, x, row, sub);
        if (sub == 0 && row < A.n) y[row] = s;
    }
}

// r = b - A x, p = r; rr = r.r, bb = b.b; done if ||r|| <= tol ||b||.
template <int LPR>
__global__ void __launch_bounds__(kCgThreads) cg_init_kernel(const Csr A, const double* __restrict__ b,
                                                             const double* __restrict__ x, double* __restrict__ r,
                                                             double* __restrict__ p, double* __restrict__ part,
                                                             CgState* st) {
    __shared__ double s_warp[kCgThreads / 32];
    constexpr int kRowsPerBlock = kCgThreads / LPR;
    const int sub = threadIdx.x & (LPR - 1);
    double rr = 0.0, bb = 0.0;
    const int64_t stride = (int64_t)gridDim.x * kRowsPerBlock;
    for (int64_t base = (int64_t)blockIdx.x * kRowsPerBlock; base < A.n; base += stride) {
        const int64_t row = base + threadIdx.x / LPR;
        const double ax = row_dot<LPR>(A, x, row, sub);
        if (sub == 0 && row < A.n) {
            const double bi = b[row], ri = bi - ax;
            r[row] = ri;
            p[row] = ri;
            rr = fma(ri, ri, rr);
            bb = fma(bi, bi, bb);
        }
    }
    const double trr = block_sum(rr, s_warp), tbb = block_sum(bb, s_warp);
    if (threadIdx.x == 0) {
        part[blockIdx.x] = trr;
        part[gridDim.x + blockIdx.x] = tbb;
    }
    if (!last_cta(st)) return;
    const double srr = sum_partials(part, gridDim.x, s_warp), sbb = sum_partials(part + gridDim.x, gridDim.x, s_warp);
    if (threadIdx.x == 0) {
        st->rr = srr;
        st->bb = sbb;
        st->iters = 0;
        st->done = (srr <= st->tol2 * sbb || st->max_iter <= 0) ? 1 : 0;
        st->ticket = 0u;
    }
}

// One CG iteration is three kernels.  Each posts one partial sum per CTA;
// the next kernel sums all of them in every CTA, in the same fixed order,
// so every CTA sees the same scalar (no fence, ticket or last-CTA pass), and
// CTA 0 records it in the state.  part[0, grid_rows) holds the p.Ap
// partials, part[grid_rows, grid_rows + grid_vec) the r.r partials.

// Ap = A p; p.Ap partial per CTA.
template <int LPR>
__global__ void __launch_bounds__(kCgThreads) cg_ap_kernel(const Csr A, const double* __restrict__ p,
                                                           double* __restrict__ ap, double* __restrict__ part,
                                                           const CgState* st) {
    __shared__ double s_warp[kCgThreads / 32];
    if (st->done) return;
    constexpr int kRowsPerBlock = kCgThreads / LPR;
    const int sub = threadIdx.x & (LPR - 1);
    double pap = 0.0;
    const int64_t stride = (int64_t)gridDim.x * kRowsPerBlock;
    for (int64_t base = (int64_t)blockIdx.x * kRowsPerBlock; base < A.n; base += stride) {
        const int64_t row = base + threadIdx.x / LPR;
        const double s = row_dot<LPR>(A, p, row, sub);
        if (sub == 0 && row < A.n) {
            ap[row] = s;
            pap = fma(p[row], s, pap);
        }
    }
    const double t = block_sum(pap, s_warp);
    if (threadIdx.x == 0) part[blockIdx.x] = t;
}

// alpha = rr / p.Ap; x += alpha p, r -= alpha Ap; r.r partial per CTA.
__global__ void __launch_bounds__(kCgThreads) cg_update_kernel(int64_t n, double* __restrict__ x, double* __restrict__ r,
                                                               const double* __restrict__ p, const double* __restrict__ ap,
                                                               const double* __restrict__ pap_part, int n_pap,
                                                               double* __restrict__ rr_part, CgState* st) {
    __shared__ double s_warp[kCgThreads / 32];
    __shared__ double s_alpha;
    if (st->done) return;
    const double pap = sum_partials(pap_part, n_pap, s_warp);
    if (threadIdx.x == 0) {
        const double rr = st->rr;
        s_alpha = rr / pap;
        if (blockIdx.x == 0) {
            st->pap = pap;
            st->alpha = s_alpha;
            st->rr_old = rr;   // the direction kernel reads this while CTA 0 there overwrites rr
        }
    }
    __syncthreads();
    const double alpha = s_alpha;
    double rr = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * kCgThreads + threadIdx.x; i < n; i += (int64_t)gridDim.x * kCgThreads) {
        x[i] = fma(alpha, p[i], x[i]);
        const double ri = fma(-alpha, ap[i], r[i]);
        r[i] = ri;
        rr = fma(ri, ri, rr);
    }
    const double t = block_sum(rr, s_warp);
    if (threadIdx.x == 0) rr_part[blockIdx.x] = t;
}

// rr_new = r.r, beta = rr_new / rr_old; p = r + beta p; stop test.
__global__ void __launch_bounds__(kCgThreads) cg_direction_kernel(int64_t n, const double* __restrict__ r,
                                                                  double* __restrict__ p,
                                                                  const double* __restrict__ rr_part, int n_rr,
                                                                  CgState* st) {
    __shared__ double s_warp[kCgThreads / 32];
    __shared__ double s_beta;
    if (st->done) return;   // only CTA 0 below sets it, after this iteration's work
    const double rr_new = sum_partials(rr_part, n_rr, s_warp);
    if (threadIdx.x == 0) s_beta = rr_new / st->rr_old;
    __syncthreads();
    const double beta = s_beta;
    for (int64_t i = (int64_t)blockIdx.x * kCgThreads + threadIdx.x; i < n; i += (int64_t)gridDim.x * kCgThreads)
        p[i] = fma(beta, p[i], r[i]);
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        st->beta = beta;
        st->rr = rr_new;
        st->iters += 1;
        if (rr_new <= st->tol2 * st->bb || st->iters >= st->max_iter) st->done = 1;
    }
}

// CSR structure check: row_ptr[0] == 0, row_ptr[n] == nnz, row_ptr
// non-decreasing, every column index in [0, n).  Bits of *bad: 1 ends, 2
// order, 4 column range.
__global__ void __launch_bounds__(kCgThreads) csr_check_kernel(const Csr A, int64_t nnz, unsigned* bad) {
    const int64_t stride = (int64_t)gridDim.x * kCgThreads;
    const int64_t t0 = (int64_t)blockIdx.x * kCgThreads + threadIdx.x;
    if (t0 == 0 && (__ldg(A.row_ptr) != 0 || __ldg(A.row_ptr + A.n) != nnz)) atomicOr(bad, 1u);
    for (int64_t i = t0; i < A.n; i += stride)
        if (__ldg(A.row_ptr + i + 1) < __ldg(A.row_ptr + i)) atomicOr(bad, 2u);
    for (int64_t k = t0; k < nnz; k += stride) {
        const int32_t c = __ldg(A.col + k);
        if (c < 0 || (int64_t)c >= A.n) atomicOr(bad, 4u);
    }
}

// Lanes per row: AROL_SPMV_LPR (1, 2, 4 or 8) when set, else about 8 to 16
// products per lane from the mean row length (on the 27-point system, mean 26,
// two lanes per row beat one, four and eight).  Fixed per matrix, so results
// are reproducible.
int choose_lpr(int64_t n, int64_t nnz) {
    const char* e = std::getenv("AROL_SPMV_LPR");
    const int v = e ? std::atoi(e) : 0;
    if (v == 1 || v == 2 || v == 4 || v == 8) return v;
    const double mean = n > 0 ? (double)nnz / (double)n : 0.0;
    return mean < 16 ? 1 : mean < 32 ? 2 : mean < 64 ? 4 : 8;
}

int row_grid(int64_t n, int lpr) {
    const int rows_per_block = kCgThreads / lpr;
    const int64_t want = (n + rows_per_block - 1) / rows_per_block;
    const int64_t cap = (int64_t)device_sm_count() * 8;
    return (int)(want < cap ? (want > 0 ? want : 1) : cap);
}

int vec_grid(int64_t n) {
    const int64_t want = (n + kCgThreads - 1) / kCgThreads;
    const int64_t cap = (int64_t)device_sm_count() * 8;
    return (int)(want < cap ? (want > 0 ? want : 1) : cap);
}

thread_local std::string t_cg_err;

}  // namespace
}  // namespace arol

using namespace arol;

struct arol_cg_s {
    Csr A{};
    int device = -1;
    int lpr = 8;
    double *r = nullptr, *p = nullptr, *ap = nullptr, *xw = nullptr, *bw = nullptr, *part = nullptr;
    CgState* st = nullptr;
    CgState* host_st = nullptr;   // page-locked copy for polling
    int grid_rows = 1, grid_vec = 1, chunk = 8;
    cudaStream_t cap_stream = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaGraph_t graph = nullptr;
};

namespace {

arol_status cg_fail(arol_status st, const std::string& msg) {
    t_cg_err = msg;
    return st;
}

#define CG_CUDA(call, what)                                                                 \
    do {                                                                                    \
        cudaError_t e_ = (call);                                                            \
        if (e_ != cudaSuccess) return cg_fail(AROL_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e_)); \
    } while (0)

}  // namespace

extern "C" {

arol_status arol_cg_last_error(char* buf, size_t len) {
    if (buf && len) {
        std::strncpy(buf, t_cg_err.c_str(), len - 1);
        buf[len - 1] = 0;
    }
    return AROL_OK;
}

arol_status arol_csr_spmv(int64_t n_rows, int64_t nnz, const int64_t* row_ptr, const int32_t* col_idx,
                          const double* vals, const double* x, double* y, void* stream) {
    if (n_rows < 0 || nnz < 0) return cg_fail(AROL_ERR_INVALID, "negative size");
    if (n_rows == 0) return AROL_OK;
    if (!row_ptr || !x || !y || (nnz > 0 && (!col_idx || !vals))) return cg_fail(AROL_ERR_INVALID, "null pointer");
    Csr A{row_ptr, col_idx, vals, n_rows};
    const int lpr = choose_lpr(n_rows, nnz);
    const int grid = row_grid(n_rows, lpr);
    cudaStream_t s = (cudaStream_t)stream;
    switch (lpr) {
    case 1: spmv_kernel<1><<<grid, kCgThreads, 0, s>>>(A, x, y); break;
    case 2: spmv_kernel<2><<<grid, kCgThreads, 0, s>>>(A, x, y); break;
    case 4: spmv_kernel<4><<<grid, kCgThreads, 0, s>>>(A, x, y); break;
    default: spmv_kernel<8><<<grid, kCgThreads, 0, s>>>(A, x, y); break;
    }
    CG_CUDA(cudaGetLastError(), "spmv launch");
    return AROL_OK;
}

arol_status arol_csr_check(int64_t n_rows, int64_t nnz, const int64_t* row_ptr, const int32_t* col_idx, void* stream) {
    if (n_rows < 0 || nnz < 0) return cg_fail(AROL_ERR_INVALID, "negative size");
    if (!row_ptr || (nnz > 0 && !col_idx)) return cg_fail(AROL_ERR_INVALID, "null pointer");
    if (n_rows >= 2147483647LL) return cg_fail(AROL_ERR_UNSUPPORTED, "column indices are 32-bit: n_rows < 2^31");
    cudaStream_t s = (cudaStream_t)stream;
    unsigned* bad = nullptr;
    CG_CUDA(cudaMalloc(&bad, sizeof(unsigned)), "cudaMalloc(check word)");
    unsigned host = 0;
    cudaError_t e = cudaMemsetAsync(bad, 0, sizeof(unsigned), s);
    if (e == cudaSuccess) {
        const int64_t work = n_rows > nnz ? n_rows : nnz;
        int64_t grid = (work + kCgThreads - 1) / kCgThreads;
        const int64_t cap = (int64_t)device_sm_count() * 8;
        grid = grid < 1 ? 1 : (grid > cap ? cap : grid);
        csr_check_kernel<<<(int)grid, kCgThreads, 0, s>>>(Csr{row_ptr, col_idx, nullptr, n_rows}, nnz, bad);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(&host, bad, sizeof(unsigned), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFree(bad);
    if (e != cudaSuccess) return cg_fail(AROL_ERR_CUDA, std::string("csr check: ") + cudaGetErrorString(e));
    if (host & 1u) return cg_fail(AROL_ERR_INVALID, "csr: row_ptr[0] must be 0 and row_ptr[n] must equal nnz");
    if (host & 2u) return cg_fail(AROL_ERR_INVALID, "csr: row_ptr must not decrease");
    if (host & 4u) return cg_fail(AROL_ERR_INVALID, "csr: a column index is outside [0, n)");
    return AROL_OK;
}

arol_status arol_cg_create(int64_t n_rows, int64_t nnz, const int64_t* row_ptr, const int32_t* col_idx,
                           const double* vals, arol_cg* out) {
    if (!out) return cg_fail(AROL_ERR_INVALID, "null handle pointer");
    *out = nullptr;
    if (n_rows < 1 || nnz < 0 || !row_ptr || (nnz > 0 && (!col_idx || !vals)))
        return cg_fail(AROL_ERR_INVALID, "bad matrix");
    // the products index x by col_idx: a malformed matrix is refused here
    {
        const arol_status cs = arol_csr_check(n_rows, nnz, row_ptr, col_idx, nullptr);
        if (cs != AROL_OK) return cs;
    }
    arol_cg h = new (std::nothrow) arol_cg_s();
    if (!h) return cg_fail(AROL_ERR_INVALID, "out of host memory");
    h->A = Csr{row_ptr, col_idx, vals, n_rows};
    cudaGetDevice(&h->device);
    h->lpr = choose_lpr(n_rows, nnz);
    h->grid_rows = row_grid(n_rows, h->lpr);
    h->grid_vec = vec_grid(n_rows);
    const size_t vb = (size_t)n_rows * sizeof(double);
    const int nparts = 2 * (h->grid_rows > h->grid_vec ? h->grid_rows : h->grid_vec);
    cudaError_t e = cudaSuccess;
    double** vecs[] = {&h->r, &h->p, &h->ap, &h->xw, &h->bw};
    for (double** v : vecs)
        if (e == cudaSuccess) e = cudaMalloc(v, vb);
    if (e == cudaSuccess) e = cudaMalloc(&h->part, (size_t)nparts * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(&h->st, sizeof(CgState));
    if (e == cudaSuccess) e = cudaMemset(h->st, 0, sizeof(CgState));
    if (e == cudaSuccess) e = cudaMallocHost(&h->host_st, sizeof(CgState));
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) {
        // one graph of `chunk` iterations (three kernels each)
        e = cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal);
        for (int it = 0; it < h->chunk && e == cudaSuccess; ++it) {
            switch (h->lpr) {
            case 1: cg_ap_kernel<1><<<h->grid_rows, kCgThreads, 0, h->cap_stream>>>(h->A, h->p, h->ap, h->part, h->st); break;
            case 2: cg_ap_kernel<2><<<h->grid_rows, kCgThreads, 0, h->cap_stream>>>(h->A, h->p, h->ap, h->part, h->st); break;
            case 4: cg_ap_kernel<4><<<h->grid_rows, kCgThreads, 0, h->cap_stream>>>(h->A, h->p, h->ap, h->part, h->st); break;
            default: cg_ap_kernel<8><<<h->grid_rows, kCgThreads, 0, h->cap_stream>>>(h->A, h->p, h->ap, h->part, h->st); break;
            }
            double* rr_part = h->part + h->grid_rows;
            cg_update_kernel<<<h->grid_vec, kCgThreads, 0, h->cap_stream>>>(n_rows, h->xw, h->r, h->p, h->ap, h->part,
                                                                            h->grid_rows, rr_part, h->st);
            cg_direction_kernel<<<h->grid_vec, kCgThreads, 0, h->cap_stream>>>(n_rows, h->r, h->p, rr_part, h->grid_vec,
                                                                               h->st);
            e = cudaGetLastError();
        }
        cudaError_t e2 = cudaStreamEndCapture(h->cap_stream, &h->graph);
        if (e == cudaSuccess) e = e2;
        if (e == cudaSuccess) e = cudaGraphInstantiate(&h->exec, h->graph, 0);
    }
    if (e != cudaSuccess) {
        arol_cg_destroy(h);
        return cg_fail(AROL_ERR_CUDA, std::string("cg setup: ") + cudaGetErrorString(e));
    }
    *out = h;
    return AROL_OK;
}

arol_status arol_cg_solve(arol_cg h, const double* b, double* x, double tol, int max_iter, int* iterations,
                          double* rel_residual, void* stream) {
    if (!h || !b || !x) return cg_fail(AROL_ERR_INVALID, "null argument");
    if (!(tol >= 0.0) || max_iter < 0) return cg_fail(AROL_ERR_INVALID, "bad tolerance or iteration limit");
    cudaStream_t s = (cudaStream_t)stream;
    const size_t vb = (size_t)h->A.n * sizeof(double);
    CgState init{};
    init.tol2 = tol * tol;
    init.max_iter = max_iter;
    std::memcpy(h->host_st, &init, sizeof init);
    CG_CUDA(cudaMemcpyAsync(h->st, h->host_st, sizeof(CgState), cudaMemcpyHostToDevice, s), "upload state");
    CG_CUDA(cudaMemcpyAsync(h->bw, b, vb, cudaMemcpyDeviceToDevice, s), "copy b");
    CG_CUDA(cudaMemcpyAsync(h->xw, x, vb, cudaMemcpyDeviceToDevice, s), "copy x0");
    switch (h->lpr) {
    case 1: cg_init_kernel<1><<<h->grid_rows, kCgThreads, 0, s>>>(h->A, h->bw, h->xw, h->r, h->p, h->part, h->st); break;
    case 2: cg_init_kernel<2><<<h->grid_rows, kCgThreads, 0, s>>>(h->A, h->bw, h->xw, h->r, h->p, h->part, h->st); break;
    case 4: cg_init_kernel<4><<<h->grid_rows, kCgThreads, 0, s>>>(h->A, h->bw, h->xw, h->r, h->p, h->part, h->st); break;
    default: cg_init_kernel<8><<<h->grid_rows, kCgThreads, 0, s>>>(h->A, h->bw, h->xw, h->r, h->p, h->part, h->st); break;
    }
    CG_CUDA(cudaGetLastError(), "cg init launch");
    for (int launched = 0;; launched += h->chunk) {
        CG_CUDA(cudaMemcpyAsync(h->host_st, h->st, sizeof(CgState), cudaMemcpyDeviceToHost, s), "read state");
        CG_CUDA(cudaStreamSynchronize(s), "synchronize");
        if (h->host_st->done || launched >= max_iter) break;
        CG_CUDA(cudaGraphLaunch(h->exec, s), "graph launch");
    }
    CG_CUDA(cudaMemcpyAsync(x, h->xw, vb, cudaMemcpyDeviceToDevice, s), "copy solution");
    CG_CUDA(cudaStreamSynchronize(s), "synchronize");
    if (iterations) *iterations = h->host_st->iters;
    if (rel_residual) *rel_residual = h->host_st->bb > 0 ? __builtin_sqrt(h->host_st->rr / h->host_st->bb) : 0.0;
    return AROL_OK;
}

void arol_cg_destroy(arol_cg h) {
    if (!h) return;
    if (h->exec) cudaGraphExecDestroy(h->exec);
    if (h->graph) cudaGraphDestroy(h->graph);
    if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
    cudaFree(h->r);
    cudaFree(h->p);
    cudaFree(h->ap);
    cudaFree(h->xw);
    cudaFree(h->bw);
    cudaFree(h->part);
    cudaFree(h->st);
    if (h->host_st) cudaFreeHost(h->host_st);
    delete h;
}

}  // extern "C"
