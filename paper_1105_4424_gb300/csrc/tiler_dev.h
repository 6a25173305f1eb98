// Device helpers of the tiler kernels (k_tiler.cu, k_tiled.cu): repetition
// decode, base coordinates and offsets by multiply-shift division, the
// pattern walks, 16-bit storage reads and writes, the per-repetition FIR
// bank, and the test that a pattern cannot wrap.  Not part of the ABI.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "arol_internal.h"

namespace arol {
namespace {

constexpr int kThreads = 256;


// n / d for n < 2^31 by multiply-shift (host-prepared reciprocal).
__device__ __forceinline__ uint32_t fast_div(uint32_t n, const FastDiv& f) {
    return (uint32_t)(((uint64_t)n * f.m) >> f.s);
}

__device__ __forceinline__ void base_index(const PortDev& p, const uint32_t r[4], bool wide, uint32_t e[4]) {
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        if (wide) {
            uint64_t v = p.origin[k];
#pragma unroll
            for (int q = 0; q < 4; ++q) v += (uint64_t)p.paving[k][q] * r[q];
            e[k] = (uint32_t)(v % (uint64_t)(uint32_t)p.shape[k]);
        } else {
            // the host guarantees v < 2^31 on this path
            uint32_t v = p.origin[k];
#pragma unroll
            for (int q = 0; q < 4; ++q) v += p.paving[k][q] * r[q];
            e[k] = v - fast_div(v, p.shape_div[k]) * (uint32_t)p.shape[k];
        }
    }
}

__device__ __forceinline__ uint32_t pick(const uint32_t c[4], int k) {
    return k == 0 ? c[0] : k == 1 ? c[1] : k == 2 ? c[2] : c[3];
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
        uint32_t l = (uint32_t)lr;   // < 2^31 on this path
#pragma unroll
        for (int q = 3; q >= 0; --q) {
            const uint32_t qq = fast_div(l, t.rep_div[q]);
            r[q] = l - qq * (uint32_t)t.rep[q];
            l = qq;
        }
    }
}

// One repetition of a copy or fir task: gather, elementary task, scatter.
// FIR storage: f32, bfloat16 or IEEE half; 16-bit values are widened
// exactly on load and rounded to nearest even on store; the arithmetic is f32
// either way.
__device__ __forceinline__ float load_value(const TaskDev& t, int64_t off) {
    if (t.in_dt == kStBf16) return __uint_as_float((uint32_t)__ldg(static_cast<const unsigned short*>(t.x) + off) << 16);
    if (t.in_dt == kStF16) return __half2float(__ushort_as_half(__ldg(static_cast<const unsigned short*>(t.x) + off)));
    return __ldg(static_cast<const float*>(t.x) + off);
}

__device__ __forceinline__ void store_value(const TaskDev& t, int64_t off, float v) {
    if (t.out_dt == kStBf16) static_cast<__nv_bfloat16*>(t.y)[off] = __float2bfloat16_rn(v);
    else if (t.out_dt == kStF16) static_cast<__half*>(t.y)[off] = __float2half_rn(v);
    else static_cast<float*>(t.y)[off] = v;
}

// Contiguous-row pattern walk: offset of the row start plus a coordinate
// along the last dimension that wraps to 0 at its extent.
struct RowWalk {
    int64_t base;
    uint32_t c, extent;
    __device__ __forceinline__ void start(const PortDev& p, const uint32_t b[4]) {
        c = pick(b, p.fdim);
        extent = (uint32_t)p.shape[p.fdim];
        base = offset_of(p, b) - (int64_t)c;
    }
    __device__ __forceinline__ int64_t off() const { return base + (int64_t)c; }
    __device__ __forceinline__ void next() { c = (c + 1u == extent) ? 0u : c + 1u; }
};

// AROL_DEBUG builds check every index the per-repetition walk computes
// against its array before the access; an index out of range is skipped and
// recorded in *t.err, bit 0x100 (input) or 0x200 (output), which
// arol_task_sync_status reports as AROL_ERR_OOB.
// Release builds compile the checks away.
#ifdef AROL_DEBUG
__device__ __forceinline__ bool in_ok(const TaskDev& t, int64_t off) {
    if ((uint64_t)off < (uint64_t)t.in_elems) return true;
    if (t.err) atomicOr(t.err, 0x100u);
    return false;
}
__device__ __forceinline__ bool out_ok(const TaskDev& t, int64_t off) {
    if ((uint64_t)off < (uint64_t)t.out_elems) return true;
    if (t.err) atomicOr(t.err, 0x200u);
    return false;
}
#else
__device__ __forceinline__ constexpr bool in_ok(const TaskDev&, int64_t) { return true; }
__device__ __forceinline__ constexpr bool out_ok(const TaskDev&, int64_t) { return true; }
#endif

template <int MAXM>
__device__ __forceinline__ void process_rep_rows(const TaskDev& t, const uint32_t bi[4], const uint32_t bo[4]) {
    RowWalk wi, wo;
    wi.start(t.in, bi);
    wo.start(t.out, bo);
    const int n = t.T;
    if (t.elem == ELEM_COPY) {
        if (t.esize == 4) {
            const uint32_t* x = static_cast<const uint32_t*>(t.x);
            uint32_t* y = static_cast<uint32_t*>(t.y);
            for (int k = 0; k < n; ++k) {
                if (in_ok(t, wi.off()) && out_ok(t, wo.off())) y[wo.off()] = __ldg(x + wi.off());
                wi.next();
                wo.next();
            }
        } else {
            const uint16_t* x = static_cast<const uint16_t*>(t.x);
            uint16_t* y = static_cast<uint16_t*>(t.y);
            for (int k = 0; k < n; ++k) {
                if (in_ok(t, wi.off()) && out_ok(t, wo.off())) y[wo.off()] = __ldg(x + wi.off());
                wi.next();
                wo.next();
            }
        }
        return;
    }
    const int m = t.m;
    float acc[MAXM];
#pragma unroll
    for (int j = 0; j < MAXM; ++j) acc[j] = 0.f;
    for (int k = 0; k < n; ++k) {
        const float p = in_ok(t, wi.off()) ? load_value(t, wi.off()) : 0.f;
        wi.next();
        const float* h = t.taps + k;
#pragma unroll
        for (int j = 0; j < MAXM; ++j)
            if (j < m) acc[j] = fmaf(__ldg(h + j * n), p, acc[j]);
    }
#pragma unroll
    for (int j = 0; j < MAXM; ++j) {
        if (j < m) {
            if (out_ok(t, wo.off())) store_value(t, wo.off(), acc[j]);
            wo.next();
        }
    }
}

// One repetition from its input and output base coordinates b, bo: the
// pattern walks with a wrap test per step (PatternWalk), or with one per
// row pattern (process_rep_rows).
template <int MAXM>
__device__ __forceinline__ void process_rep_at(const TaskDev& t, const uint32_t b[4], const uint32_t bo[4]) {
    if (t.in.fast && t.out.fast) {
        process_rep_rows<MAXM>(t, b, bo);
        return;
    }
    PatternWalk wi, wo;
    wi.start(b);
    wo.start(bo);
    const int n = t.T;
    if (t.elem == ELEM_COPY) {
        if (t.esize == 4) {
            const uint32_t* x = static_cast<const uint32_t*>(t.x);
            uint32_t* y = static_cast<uint32_t*>(t.y);
            for (int k = 0; k < n; ++k) {
                const int64_t oi = offset_of(t.in, wi.cur), oo = offset_of(t.out, wo.cur);
                if (in_ok(t, oi) && out_ok(t, oo)) y[oo] = __ldg(x + oi);
                wi.next(t.in);
                wo.next(t.out);
            }
        } else {
            const uint16_t* x = static_cast<const uint16_t*>(t.x);
            uint16_t* y = static_cast<uint16_t*>(t.y);
            for (int k = 0; k < n; ++k) {
                const int64_t oi = offset_of(t.in, wi.cur), oo = offset_of(t.out, wo.cur);
                if (in_ok(t, oi) && out_ok(t, oo)) y[oo] = __ldg(x + oi);
                wi.next(t.in);
                wo.next(t.out);
            }
        }
        return;
    }
    // FIR bank: y[j] = sum_k H[j,k] p[k], accumulated in k order with fma.
    const int m = t.m;
    float acc[MAXM];
#pragma unroll
    for (int j = 0; j < MAXM; ++j) acc[j] = 0.f;
    for (int k = 0; k < n; ++k) {
        const int64_t oi = offset_of(t.in, wi.cur);
        const float p = in_ok(t, oi) ? load_value(t, oi) : 0.f;
        wi.next(t.in);
        const float* h = t.taps + k;
#pragma unroll
        for (int j = 0; j < MAXM; ++j)
            if (j < m) acc[j] = fmaf(__ldg(h + (int64_t)j * n), p, acc[j]);
    }
#pragma unroll
    for (int j = 0; j < MAXM; ++j) {
        if (j < m) {
            const int64_t oo = offset_of(t.out, wo.cur);
            if (out_ok(t, oo)) store_value(t, oo, acc[j]);
            wo.next(t.out);
        }
    }
}

// Taps of one tap index k for M outputs, from the transposed block
// ht[k * 16 + j] = H[j, k], as float4 / float2 / float pieces.
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

// A pattern whose base coordinates b satisfy b + ext < shape on every array
// dimension never wraps (fittings are reduced into [0, shape)): its elements
// sit at offset(b) + i0 lin[0] + i1 lin[1].
__device__ __forceinline__ bool pattern_fits(const PortDev& p, const uint32_t b[4]) {
    bool ok = p.linear != 0;
#pragma unroll
    for (int k = 0; k < 4; ++k) ok = ok && b[k] + p.ext[k] < (uint32_t)p.shape[k];
    return ok;
}

}  // namespace
}  // namespace arol
