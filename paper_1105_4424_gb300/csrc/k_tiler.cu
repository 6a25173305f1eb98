// Generic Array-OL tiler kernel (gather -> copy/FIR -> scatter) and the
// persistent batched kernel that runs many such tasks from one work list.
//
// Address generation (the tiler of the MARTE RSM package, Sec. 3; repetitive
// tasks, Sec. 7): for repetition r and pattern index i an array element is
// e(r, i) = (o + P r + F i) mod s.  The host reduces o, P and F into [0, s)
// so the device computes the base (o + P r) mod s once per repetition and then
// walks the pattern by adding fitting columns with one conditional subtract
// per dimension (strength-reduced modulo), all in 32-bit registers.
#include "arol_internal.h"

namespace arol {
namespace {

constexpr int kThreads = 256;

__device__ __forceinline__ void base_index(const PortDev& p, const uint32_t r[4], bool wide, uint32_t e[4]) {
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        if (wide) {
            uint64_t v = p.origin[k];
#pragma unroll
            for (int q = 0; q < 4; ++q) v += (uint64_t)p.paving[k][q] * r[q];
            e[k] = (uint32_t)(v % (uint64_t)(uint32_t)p.shape[k]);
        } else {
            uint32_t v = p.origin[k];
#pragma unroll
            for (int q = 0; q < 4; ++q) v += p.paving[k][q] * r[q];
            e[k] = v % (uint32_t)p.shape[k];
        }
    }
}

// c += fitting column `col`, modulo the shape (every term already in [0, s)).
__device__ __forceinline__ void advance(const PortDev& p, int col, uint32_t c[4]) {
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        uint32_t v = c[k] + p.fitting[k][col];
        c[k] = v >= (uint32_t)p.shape[k] ? v - (uint32_t)p.shape[k] : v;
    }
}

__device__ __forceinline__ int64_t offset_of(const PortDev& p, const uint32_t c[4]) {
    return (int64_t)c[0] * p.stride[0] + (int64_t)c[1] * p.stride[1] +
           (int64_t)c[2] * p.stride[2] + (int64_t)c[3] * p.stride[3];
}

// Walks a pattern in row-major order: pattern dim 1 is the fast one.
struct PatternWalk {
    uint32_t row[4], cur[4];
    int i1;
    __device__ __forceinline__ void start(const uint32_t b[4]) {
#pragma unroll
        for (int k = 0; k < 4; ++k) row[k] = cur[k] = b[k];
        i1 = 0;
    }
    __device__ __forceinline__ void next(const PortDev& p) {
        if (++i1 == p.pattern[1]) {
            i1 = 0;
            advance(p, 0, row);
#pragma unroll
            for (int k = 0; k < 4; ++k) cur[k] = row[k];
        } else {
            advance(p, 1, cur);
        }
    }
};

__device__ __forceinline__ void decode_rep(const TaskDev& t, int64_t lr, bool wide, uint32_t r[4]) {
    if (wide) {
#pragma unroll
        for (int q = 3; q >= 0; --q) {
            int64_t d = t.rep[q];
            int64_t qq = lr / d;
            r[q] = (uint32_t)(lr - qq * d);
            lr = qq;
        }
    } else {
        uint32_t l = (uint32_t)lr;
#pragma unroll
        for (int q = 3; q >= 0; --q) {
            uint32_t d = (uint32_t)t.rep[q];
            uint32_t qq = l / d;
            r[q] = l - qq * d;
            l = qq;
        }
    }
}

// One repetition of a copy or fir task: gather, elementary task, scatter.
template <int MAXM>
__device__ __forceinline__ void process_rep(const TaskDev& t, int64_t lr) {
    const bool wide = t.wide != 0;
    uint32_t r[4], b[4];
    decode_rep(t, lr, wide, r);
    PatternWalk wi, wo;
    base_index(t.in, r, wide, b);
    wi.start(b);
    base_index(t.out, r, wide, b);
    wo.start(b);
    const int n = t.T;
    if (t.elem == ELEM_COPY) {
        if (t.esize == 4) {
            const uint32_t* x = static_cast<const uint32_t*>(t.x);
            uint32_t* y = static_cast<uint32_t*>(t.y);
            for (int k = 0; k < n; ++k) {
                y[offset_of(t.out, wo.cur)] = __ldg(x + offset_of(t.in, wi.cur));
                wi.next(t.in);
                wo.next(t.out);
            }
        } else {
            const uint16_t* x = static_cast<const uint16_t*>(t.x);
            uint16_t* y = static_cast<uint16_t*>(t.y);
            for (int k = 0; k < n; ++k) {
                y[offset_of(t.out, wo.cur)] = __ldg(x + offset_of(t.in, wi.cur));
                wi.next(t.in);
                wo.next(t.out);
            }
        }
        return;
    }
    // FIR bank: y[j] = sum_k H[j,k] p[k], accumulated in k order with fma.
    const float* x = static_cast<const float*>(t.x);
    float* y = static_cast<float*>(t.y);
    const int m = t.m;
    float acc[MAXM];
#pragma unroll
    for (int j = 0; j < MAXM; ++j) acc[j] = 0.f;
    for (int k = 0; k < n; ++k) {
        const float p = __ldg(x + offset_of(t.in, wi.cur));
        wi.next(t.in);
        const float* h = t.taps + k;
#pragma unroll
        for (int j = 0; j < MAXM; ++j)
            if (j < m) acc[j] = fmaf(__ldg(h + (int64_t)j * n), p, acc[j]);
    }
#pragma unroll
    for (int j = 0; j < MAXM; ++j) {
        if (j < m) {
            y[offset_of(t.out, wo.cur)] = acc[j];
            wo.next(t.out);
        }
    }
}

template <int MAXM>
__global__ void __launch_bounds__(kThreads) tiler_generic_kernel(const TaskDev t) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t lr = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; lr < t.nreps; lr += stride)
        process_rep<MAXM>(t, lr);
}

// Persistent batched kernel: CTAs take tiles (task, repetition range) from a
// shared counter until the list is exhausted.  No CTA waits on another.
template <int MAXM>
__global__ void __launch_bounds__(512) batch_persistent_kernel(const TaskDev* __restrict__ tasks,
                                                               const TileDev* __restrict__ tiles,
                                                               int ntiles, unsigned* counter) {
    __shared__ int s_tile;
    for (;;) {
        if (threadIdx.x == 0) s_tile = (int)atomicAdd(counter, 1u);
        __syncthreads();
        const int ti = s_tile;
        __syncthreads();
        if (ti >= ntiles) break;
        const TileDev tile = tiles[ti];
        const TaskDev& t = tasks[tile.task];
        const int64_t end = tile.start + tile.count;
        for (int64_t lr = tile.start + threadIdx.x; lr < end; lr += blockDim.x) process_rep<MAXM>(t, lr);
    }
}

// Element of port p at flat pattern index j of the repetition whose base is b
// (pattern dim 1 fastest); direct form, used by the backward kernels.
__device__ __forceinline__ int64_t pattern_offset(const PortDev& p, const uint32_t b[4], int j) {
    const uint32_t i0 = (uint32_t)j / (uint32_t)p.pattern[1];
    const uint32_t i1 = (uint32_t)j - i0 * (uint32_t)p.pattern[1];
    int64_t off = 0;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const uint64_t v = (uint64_t)b[k] + (uint64_t)p.fitting[k][0] * i0 + (uint64_t)p.fitting[k][1] * i1;
        off += (int64_t)(v % (uint64_t)(uint32_t)p.shape[k]) * p.stride[k];
    }
    return off;
}

// dL/dX by owner computes: input element e sums, over the (r, k) pairs whose
// gather visited it (inverse map, increasing order), sum_j H[j,k] g[e_out(r,j)]
// (fir) or g[e_out(r,k)] (copy).  Each element is written once: no atomics.
__global__ void __launch_bounds__(kThreads) tiler_bwd_dx_kernel(const TaskDev t, const int64_t* __restrict__ start,
                                                                const int32_t* __restrict__ list, float* __restrict__ gx,
                                                                const float* __restrict__ gy, int64_t n) {
    const bool wide = t.wide != 0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += stride) {
        float acc = 0.f;
        const int64_t a = start[e], z = start[e + 1];
        for (int64_t idx = a; idx < z; ++idx) {
            const int64_t rk = list[idx];
            const int64_t lr = rk / t.T;
            const int k = (int)(rk - lr * t.T);
            uint32_t r[4], b[4];
            decode_rep(t, lr, wide, r);
            base_index(t.out, r, wide, b);
            if (t.elem == ELEM_FIR) {
                for (int j = 0; j < t.m; ++j)
                    acc = fmaf(__ldg(t.taps + (int64_t)j * t.T + k), __ldg(gy + pattern_offset(t.out, b, j)), acc);
            } else {
                acc += __ldg(gy + pattern_offset(t.out, b, k));
            }
        }
        gx[e] = acc;
    }
}

// Per-block partial tap gradients: block b covers repetitions
// [b*chunk, (b+1)*chunk); thread p owns the pair (j, k) = (p / T, p % T) and
// sums g[e_out(r,j)] * x[e_in(r,k)] over them in order.
__global__ void __launch_bounds__(kThreads) tiler_bwd_dh_kernel(const TaskDev t, const float* __restrict__ gy,
                                                                float* __restrict__ partials, int64_t chunk) {
    const bool wide = t.wide != 0;
    const float* x = static_cast<const float*>(t.x);
    const int64_t r0 = (int64_t)blockIdx.x * chunk;
    const int64_t r1 = r0 + chunk < t.nreps ? r0 + chunk : t.nreps;
    const int npairs = t.m * t.T;
    for (int p = threadIdx.x; p < npairs; p += blockDim.x) {
        const int j = p / t.T, k = p - (p / t.T) * t.T;
        float acc = 0.f;
        for (int64_t lr = r0; lr < r1; ++lr) {
            uint32_t r[4], bi[4], bo[4];
            decode_rep(t, lr, wide, r);
            base_index(t.in, r, wide, bi);
            base_index(t.out, r, wide, bo);
            acc = fmaf(__ldg(gy + pattern_offset(t.out, bo, j)), __ldg(x + pattern_offset(t.in, bi, k)), acc);
        }
        partials[(int64_t)blockIdx.x * npairs + p] = acc;
    }
}

__global__ void __launch_bounds__(kThreads) tiler_bwd_reduce_kernel(const float* __restrict__ partials, int nblocks,
                                                                    int npairs, float* __restrict__ out) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= npairs) return;
    float s = 0.f;
    for (int b = 0; b < nblocks; ++b) s += partials[(int64_t)b * npairs + p];
    out[p] = s;
}

int grid_for(int64_t work, int threads) {
    const int64_t blocks = (work + threads - 1) / threads;
    const int64_t cap = (int64_t)device_sm_count() * 16;
    return (int)(blocks < cap ? (blocks > 0 ? blocks : 1) : cap);
}

}  // namespace

int device_sm_count() {
    static int sms = 0;
    if (!sms) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (sms <= 0) sms = 1;
    }
    return sms;
}

cudaError_t launch_tiler_generic(const TaskDev& t, int max_m, cudaStream_t s) {
    if (t.nreps == 0) return cudaSuccess;
    const int grid = grid_for(t.nreps, kThreads);
    if (max_m <= 4) tiler_generic_kernel<4><<<grid, kThreads, 0, s>>>(t);
    else if (max_m <= 8) tiler_generic_kernel<8><<<grid, kThreads, 0, s>>>(t);
    else if (max_m <= 16) tiler_generic_kernel<16><<<grid, kThreads, 0, s>>>(t);
    else tiler_generic_kernel<32><<<grid, kThreads, 0, s>>>(t);
    return cudaGetLastError();
}

cudaError_t launch_batch_persistent(const TaskDev* tasks, const TileDev* tiles, int ntiles, unsigned* counter,
                                    int grid, int threads, int max_m, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(counter, 0, sizeof(unsigned), s);
    if (e != cudaSuccess) return e;
    if (ntiles == 0) return cudaSuccess;
    if (max_m <= 4) batch_persistent_kernel<4><<<grid, threads, 0, s>>>(tasks, tiles, ntiles, counter);
    else if (max_m <= 8) batch_persistent_kernel<8><<<grid, threads, 0, s>>>(tasks, tiles, ntiles, counter);
    else if (max_m <= 16) batch_persistent_kernel<16><<<grid, threads, 0, s>>>(tasks, tiles, ntiles, counter);
    else batch_persistent_kernel<32><<<grid, threads, 0, s>>>(tasks, tiles, ntiles, counter);
    return cudaGetLastError();
}

int tiler_bwd_blocks(int64_t nreps, int64_t* chunk) {
    int64_t nb = (nreps + 63) / 64;
    const int64_t cap = (int64_t)device_sm_count() * 8;
    if (nb > cap) nb = cap;
    if (nb < 1) nb = 1;
    *chunk = (nreps + nb - 1) / nb;
    if (*chunk < 1) *chunk = 1;
    return (int)nb;
}

cudaError_t launch_tiler_bwd(const TaskDev& t, const int64_t* inv_start, const int32_t* inv_list, float* gx,
                             const float* gy, float* grad_taps, float* partials, int nblocks, int64_t chunk,
                             cudaStream_t s) {
    if (gx) {
        int64_t n = 1;
        for (int k = 0; k < 4; ++k) n *= t.in.shape[k];
        tiler_bwd_dx_kernel<<<grid_for(n, kThreads), kThreads, 0, s>>>(t, inv_start, inv_list, gx, gy, n);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    if (grad_taps) {
        const int npairs = t.m * t.T;
        tiler_bwd_dh_kernel<<<nblocks, kThreads, 0, s>>>(t, gy, partials, chunk);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        tiler_bwd_reduce_kernel<<<(npairs + kThreads - 1) / kThreads, kThreads, 0, s>>>(partials, nblocks, npairs, grad_taps);
        return cudaGetLastError();
    }
    return cudaSuccess;
}

}  // namespace arol
