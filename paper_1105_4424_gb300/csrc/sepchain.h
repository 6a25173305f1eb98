// A chain of separable FIR passes fused through shared memory (Sec. 5,
// associatedParts: the arrays the tasks share stay on chip).  Shared by the
// host runtime (planning) and the kernel (k_sepchain.cu); not part of the ABI.
//
// Every task of the chain is a row pass (a FIR along the last dimension) or
// a column pass (along the rows), identity on the other dimension and on the
// frames.  Pass k reads stage k (extents H[k] x W[k]) and writes stage k + 1;
// along its axis, output position p = m r + j (r < R, j < m) is
//
//     sum_{i < T} H_k[j, i] in[(o + S r + i) mod n_in].
//
// A CTA computes one tile of the last stage.  Walking back through the passes
// gives, for every stage, the circular row and column ranges [start, start +
// len) (mod the extent) that hold every value the tile needs:
// along a pass's axis the covering repetitions need a circular range of its
// input (sep_back).  The other axis passes through unchanged.
#pragma once

#include <cstdint>

namespace arol {

constexpr int kSepMaxPasses = 4;

struct SepPassDev {
    int32_t axis;      // 0: column pass (along the rows), 1: row pass (along the columns)
    int32_t T, m, S;   // taps, outputs per repetition, step
    int32_t o;         // input origin along the axis, reduced into [0, n_in)
    int32_t n_in;      // input extent along the axis
    int32_t n_out;     // output extent along the axis: m R
    int32_t R;         // repetitions along the axis
    int32_t tap_off;   // offset of H_k (m x T, row-major) in the chain's taps
    int32_t pad_;
};

struct SepChainDev {
    const float* x;    // stage 0: (F, H[0], W[0])
    float* y;          // stage K: (F, H[K], W[K])
    const float* taps;
    int64_t F;
    int32_t K;         // passes, 2 .. kSepMaxPasses
    int32_t BH, BW;    // tile of the last stage
    int32_t tiles_y, tiles_x;
    int32_t buf;       // floats of shared buffer 0: the largest region of the even stages < K (row stride odd)
    int32_t buf1;      // floats of shared buffer 1: the largest region of the odd stages < K
    int32_t ntaps;     // floats of all passes' taps
    int32_t H[kSepMaxPasses + 1], W[kSepMaxPasses + 1];
    SepPassDev p[kSepMaxPasses];
    // sep_regions, tabulated by the host: the rows of stages 0 .. K for every
    // tile row (row_tab[ty * (K + 1) + k]) and the columns for every tile
    // column (col_tab[tx * (K + 1) + k]); each is a SepRange (start, len)
    const int32_t* row_tab;
    const int32_t* col_tab;
};

// Range of one axis of one stage: local index i of the region holds the
// stage's element at position (start + i) mod extent.  len may exceed the
// extent (by less than 32): the region then holds some positions twice, so
// that a window of T consecutive positions never runs past its end.
struct SepRange {
    int32_t start, len;
};

// Unwrapped repetition of unwrapped output position u, and back: position u
// = w n_out + m r + j (r < R, j < m) is repetition w R + r.
__host__ __device__ inline int32_t sep_urep(const SepPassDev& p, int32_t u) {
    const int32_t w = u / p.n_out;
    return w * p.R + (u - w * p.n_out) / p.m;
}
__host__ __device__ inline int32_t sep_upos(const SepPassDev& p, int32_t ur) {
    const int32_t w = ur / p.R;
    return w * p.n_out + p.m * (ur - w * p.R);
}

// The input range of a pass along its axis that covers output range `out`
// (out.start < n_out).  It starts at the window of the first repetition ra,
// o + S ra.  If the range stays below n_out its repetitions end at rb and
// span S (rb - ra) + T.  If it wraps once, repetitions ra .. R - 1 span
// S (R - 1 - ra) + T and repetitions 0 .. rb follow at (-S ra) mod n_in + S r
// from the start.  A span of n_in or more, or an output range of n_out or
// more, takes the whole axis from o, extended by T - 1 positions (every
// window then fits without a wrap).
__host__ __device__ inline SepRange sep_back(const SepPassDev& p, SepRange out) {
    SepRange in;
    in.start = p.o;
    in.len = p.n_in + p.T - 1;
    if (out.len >= p.n_out) return in;
    const int32_t ra = out.start / p.m;
    const int32_t ue = sep_urep(p, out.start + out.len - 1);
    int64_t span;
    if (ue < p.R) {
        span = (int64_t)p.S * (ue - ra) + p.T;
    } else {
        const int64_t d0 = (p.n_in - ((int64_t)p.S * ra) % p.n_in) % p.n_in;
        const int64_t pre = (int64_t)p.S * (p.R - 1 - ra) + p.T, post = d0 + (int64_t)p.S * (ue - p.R) + p.T;
        span = pre > post ? pre : post;
    }
    if (span >= p.n_in) return in;
    in.len = (int32_t)span;
    in.start = (int32_t)(((int64_t)p.o + (int64_t)p.S * ra) % p.n_in);
    return in;
}

// Rows and columns of every stage 0 .. K for tile (ty, tx) of the last stage.
__host__ __device__ inline void sep_regions(const SepChainDev& d, int32_t ty, int32_t tx, SepRange* rows,
                                            SepRange* cols) {
    const int K = d.K;
    rows[K].start = ty * d.BH;
    rows[K].len = d.H[K] - rows[K].start < d.BH ? d.H[K] - rows[K].start : d.BH;
    cols[K].start = tx * d.BW;
    cols[K].len = d.W[K] - cols[K].start < d.BW ? d.W[K] - cols[K].start : d.BW;
    for (int k = K - 1; k >= 0; --k) {
        rows[k] = rows[k + 1];
        cols[k] = cols[k + 1];
        if (d.p[k].axis == 0) rows[k] = sep_back(d.p[k], rows[k + 1]);
        else cols[k] = sep_back(d.p[k], cols[k + 1]);
    }
}

}  // namespace arol
