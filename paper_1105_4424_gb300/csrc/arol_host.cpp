// Host runtime of the Array-OL repetitive-task library: descriptor validation,
// the output-partition check, kernel selection, tap buffers, chains (shared
// arrays, Sec. 5 associatedParts), batches (device work list + CUDA graph +
// autotuner) and the C ABI declared in include/arol.h.
#include "arol.h"
#include "arol_internal.h"
#include "sepchain.h"

#include <algorithm>
#include <cinttypes>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <fstream>
#include <map>
#include <mutex>
#include <sstream>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

using namespace arol;

namespace arol {
cudaError_t launch_tiler_bwd(const TaskDev& t, const int64_t* inv_start, const int32_t* inv_list,
                             float* gx, const float* gy, float* grad_taps, float* partials, int nblocks,
                             int64_t chunk, cudaStream_t s);
int tiler_bwd_blocks(int64_t nreps, int m, int T, int64_t* chunk);
}  // namespace arol

namespace {

thread_local std::string g_err;

arol_status fail(arol_status st, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return st;
}

arol_status cuda_fail(cudaError_t e, const char* what) {
    return fail(AROL_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define AROL_CUDA(call, what)                        \
    do {                                             \
        cudaError_t e_ = (call);                     \
        if (e_ != cudaSuccess) return cuda_fail(e_, what); \
    } while (0)

// An NVTX range named after the ABI call, for the duration of the call
// (shown by Nsight tools; nearly free without one attached).
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};
#define AROL_TRACE() NvtxRange arol_nvtx_range_(__func__)

// AROL_LOG=1: one line on stderr for each kernel-path decision (task and
// chain creation, one-member batches, batch layout).
bool log_enabled() {
    static const bool on = [] {
        const char* v = std::getenv("AROL_LOG");
        return v && v[0] && v[0] != '0';
    }();
    return on;
}

void log_line(const char* fmt, ...) {
    if (!log_enabled()) return;
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    std::fprintf(stderr, "arol: %s\n", buf);
}

int64_t emod(int64_t a, int64_t s) {
    int64_t r = a % s;
    return r < 0 ? r + s : r;
}

int64_t elems_of(const arol_array_desc& a) {
    int64_t n = 1;
    for (int k = 0; k < a.rank; ++k) n *= a.shape[k];
    return n;
}

int esize_of(int dtype) { return dtype == AROL_BF16 || dtype == AROL_F16 ? 2 : 4; }

int64_t pattern_size(const arol_tiler& t) {
    int64_t n = 1;
    for (int p = 0; p < t.pattern_rank; ++p) n *= t.pattern[p];
    return n;
}

int64_t reps_of(const arol_task_desc& d) {
    int64_t n = 1;
    for (int q = 0; q < d.rep_rank; ++q) n *= d.rep[q];
    return n;
}

constexpr int64_t kMaxDim = (int64_t(1) << 31) - 1;

arol_status check_array(const arol_array_desc& a, const char* name) {
    if (a.rank < 1 || a.rank > AROL_MAX_RANK) return fail(AROL_ERR_INVALID, "%s: rank %d not in [1,4]", name, a.rank);
    if (a.dtype != AROL_F32 && a.dtype != AROL_BF16 && a.dtype != AROL_F16)
        return fail(AROL_ERR_INVALID, "%s: unknown dtype %d", name, a.dtype);
    double total = 1;
    for (int k = 0; k < a.rank; ++k) {
        if (a.shape[k] < 0 || a.shape[k] > kMaxDim)
            return fail(AROL_ERR_INVALID, "%s: shape[%d] = %" PRId64 " not in [0, 2^31)", name, k, a.shape[k]);
        total *= (double)a.shape[k];
    }
    if (total > 4.0e18) return fail(AROL_ERR_INVALID, "%s: too many elements", name);
    return AROL_OK;
}

arol_status check_tiler(const arol_tiler& t, const char* name) {
    if (t.pattern_rank < 1 || t.pattern_rank > AROL_MAX_PATTERN_RANK)
        return fail(AROL_ERR_INVALID, "%s: pattern rank %d not in [1,2]", name, t.pattern_rank);
    double n = 1;
    for (int p = 0; p < t.pattern_rank; ++p) {
        if (t.pattern[p] < 1 || t.pattern[p] > kMaxDim)
            return fail(AROL_ERR_INVALID, "%s: pattern[%d] = %" PRId64 " not in [1, 2^31)", name, p, t.pattern[p]);
        n *= (double)t.pattern[p];
    }
    if (n > (double)kMaxDim) return fail(AROL_ERR_INVALID, "%s: pattern has 2^31 or more elements", name);
    return AROL_OK;
}

// ---------------------------------------------------------------- partition

// Sufficient closed-form test: every array dimension is a mixed-radix
// combination of repetition/pattern dimensions (coefficients 1, n1, n1*n2, ...
// whose extents multiply to the dimension's size), each repetition/pattern
// dimension of extent > 1 drives exactly one array dimension.  Such a map is
// a bijection onto the array (a cyclic shift by the origin keeps it one).
bool partition_closed_form(const arol_array_desc& a, const arol_tiler& t, int rep_rank, const int64_t* rep) {
    struct Term { int64_t coef, extent; };
    const int nd = rep_rank + t.pattern_rank;
    std::vector<int> used(nd, 0);
    for (int k = 0; k < a.rank; ++k) {
        std::vector<Term> terms;
        for (int q = 0; q < nd; ++q) {
            const int64_t ext = q < rep_rank ? rep[q] : t.pattern[q - rep_rank];
            const int64_t c = emod(q < rep_rank ? t.paving[k][q] : t.fitting[k][q - rep_rank], a.shape[k]);
            if (ext <= 1 || c == 0) continue;
            terms.push_back({c, ext});
            ++used[q];
        }
        std::sort(terms.begin(), terms.end(), [](const Term& x, const Term& y) { return x.coef < y.coef; });
        int64_t expect = 1;
        for (const Term& tm : terms) {
            if (tm.coef != expect) return false;
            if (expect > kMaxDim * 4 / tm.extent) return false;
            expect *= tm.extent;
        }
        if (expect != a.shape[k]) return false;
    }
    for (int q = 0; q < nd; ++q) {
        const int64_t ext = q < rep_rank ? rep[q] : t.pattern[q - rep_rank];
        if (ext > 1 && used[q] != 1) return false;
    }
    return true;
}

// Exact count by enumeration: the largest and smallest number of (r, j) that
// land on one element.  Address walk with one conditional subtract per step.
arol_status partition_count(const arol_array_desc& a, const arol_tiler& t, int rep_rank, const int64_t* rep,
                            int64_t* cmin, int64_t* cmax) {
    const int64_t n = elems_of(a);
    int64_t nreps = 1;
    for (int q = 0; q < rep_rank; ++q) nreps *= rep[q];
    const int64_t ns = pattern_size(t);
    std::vector<uint8_t> cnt;
    try {
        cnt.assign((size_t)n, 0);
    } catch (...) {
        return fail(AROL_ERR_INVALID, "partition check: cannot allocate %" PRId64 " counters", n);
    }
    int64_t stride[4] = {0, 0, 0, 0};
    {
        int64_t s = 1;
        for (int k = a.rank - 1; k >= 0; --k) { stride[k] = s; s *= a.shape[k]; }
    }
    int64_t pav[4][4] = {}, fit[4][2] = {}, org[4] = {};
    for (int k = 0; k < a.rank; ++k) {
        org[k] = emod(t.origin[k], a.shape[k]);
        for (int q = 0; q < rep_rank; ++q) pav[k][q] = emod(t.paving[k][q], a.shape[k]);
        for (int p = 0; p < t.pattern_rank; ++p) fit[k][p] = emod(t.fitting[k][p], a.shape[k]);
    }
    const int64_t P1 = t.pattern_rank == 2 ? t.pattern[1] : t.pattern[0];
    const int64_t P0 = t.pattern_rank == 2 ? t.pattern[0] : 1;
    const int c1 = t.pattern_rank == 2 ? 1 : 0;   // fitting column of the fast pattern dim
    std::vector<int64_t> r(std::max(rep_rank, 1), 0);
    int64_t base[4], row[4], cur[4];
    for (int64_t lr = 0; lr < nreps; ++lr) {
        for (int k = 0; k < a.rank; ++k) {
            __int128 v = org[k];
            for (int q = 0; q < rep_rank; ++q) v += (__int128)pav[k][q] * r[q];
            base[k] = (int64_t)(v % a.shape[k]);
            row[k] = base[k];
        }
        for (int64_t i0 = 0; i0 < P0; ++i0) {
            for (int k = 0; k < a.rank; ++k) cur[k] = row[k];
            for (int64_t i1 = 0; i1 < P1; ++i1) {
                int64_t off = 0;
                for (int k = 0; k < a.rank; ++k) off += cur[k] * stride[k];
                if (cnt[off] < 255) ++cnt[off];
                for (int k = 0; k < a.rank; ++k) {
                    cur[k] += fit[k][c1];
                    if (cur[k] >= a.shape[k]) cur[k] -= a.shape[k];
                }
            }
            if (t.pattern_rank == 2)
                for (int k = 0; k < a.rank; ++k) {
                    row[k] += fit[k][0];
                    if (row[k] >= a.shape[k]) row[k] -= a.shape[k];
                }
        }
        for (int q = rep_rank - 1; q >= 0; --q) {
            if (++r[q] < rep[q]) break;
            r[q] = 0;
        }
    }
    (void)ns;
    uint8_t lo = 255, hi = 0;
    for (int64_t e = 0; e < n; ++e) {
        lo = std::min(lo, cnt[e]);
        hi = std::max(hi, cnt[e]);
    }
    *cmin = lo;
    *cmax = hi;
    return AROL_OK;
}

arol_status check_partition(const arol_array_desc& a, const arol_tiler& t, int rep_rank, const int64_t* rep) {
    int64_t nreps = 1;
    for (int q = 0; q < rep_rank; ++q) nreps *= rep[q];
    if (nreps * pattern_size(t) != elems_of(a))
        return fail(AROL_ERR_NOT_PARTITION, "output tiler writes %" PRId64 " elements into an array of %" PRId64,
                    nreps * pattern_size(t), elems_of(a));
    if (nreps == 0) return AROL_OK;   // an empty repetition space partitions an empty array
    if (partition_closed_form(a, t, rep_rank, rep)) return AROL_OK;
    int64_t lo = 0, hi = 0;
    arol_status st = partition_count(a, t, rep_rank, rep, &lo, &hi);
    if (st != AROL_OK) return st;
    if (lo != 1 || hi != 1)
        return fail(AROL_ERR_NOT_PARTITION, "output tiler writes some element %" PRId64 " times and some %" PRId64 " times",
                    hi, lo);
    return AROL_OK;
}

// ------------------------------------------------------------ device params

FastDiv make_fastdiv(uint32_t d) {
    FastDiv f{};
    f.d = d ? d : 1;
    uint32_t l = 0;
    while ((uint64_t(1) << l) < f.d) ++l;          // l = ceil(log2 d)
    f.s = 31 + l;
    const uint64_t two_s = uint64_t(1) << f.s;
    f.m = (uint32_t)((two_s + f.d - 1) / f.d);       // < 2^32 for every d >= 1
    return f;
}

void make_port(const arol_array_desc& a, const arol_tiler& t, int rep_rank, PortDev& p) {
    std::memset(&p, 0, sizeof p);
    int64_t s = 1;
    for (int k = 3; k >= 0; --k) {
        if (k < a.rank) {
            p.shape[k] = (int32_t)a.shape[k];
            p.stride[k] = s;
            s *= a.shape[k];
        } else {
            p.shape[k] = 1;
            p.stride[k] = 0;
        }
    }
    for (int k = 0; k < a.rank; ++k) {
        if (a.shape[k] == 0) continue;   // empty array: never addressed
        p.origin[k] = (uint32_t)emod(t.origin[k], a.shape[k]);
        for (int q = 0; q < rep_rank; ++q) p.paving[k][q] = (uint32_t)emod(t.paving[k][q], a.shape[k]);
        if (t.pattern_rank == 1) {
            p.fitting[k][0] = 0;
            p.fitting[k][1] = (uint32_t)emod(t.fitting[k][0], a.shape[k]);
        } else {
            p.fitting[k][0] = (uint32_t)emod(t.fitting[k][0], a.shape[k]);
            p.fitting[k][1] = (uint32_t)emod(t.fitting[k][1], a.shape[k]);
        }
    }
    if (t.pattern_rank == 1) {
        p.pattern[0] = 1;
        p.pattern[1] = (int32_t)t.pattern[0];
    } else {
        p.pattern[0] = (int32_t)t.pattern[0];
        p.pattern[1] = (int32_t)t.pattern[1];
    }
    for (int k = 0; k < 4; ++k) p.shape_div[k] = make_fastdiv((uint32_t)p.shape[k]);
    // Linear walk: with every fitting reduced into [0, shape), a pattern whose
    // base coordinate plus its largest step stays inside the array never
    // wraps, and its elements sit at base + i0 lin[0] + i1 lin[1].
    p.linear = 1;
    for (int c = 0; c < 2; ++c) {
        p.lin[c] = 0;
        for (int k = 0; k < 4; ++k) p.lin[c] += (int64_t)p.fitting[k][c] * p.stride[k];
    }
    for (int k = 0; k < 4; ++k) {
        const uint64_t e = (uint64_t)p.fitting[k][0] * (uint64_t)(p.pattern[0] - 1) +
                           (uint64_t)p.fitting[k][1] * (uint64_t)(p.pattern[1] - 1);
        if (e >= 0x80000000ull) p.linear = 0;
        p.ext[k] = (uint32_t)std::min<uint64_t>(e, 0xFFFFFFFFull);
    }
    // Contiguous-row pattern: the whole pattern advances along the last array
    // dimension (stride 1) by one element per step, so the walk is an
    // increment with one wrap test.
    p.fdim = a.rank - 1;
    bool fast = p.pattern[0] == 1;                 // one pattern row
    if (p.pattern[1] > 1) {
        for (int k = 0; k < 4; ++k) {
            // reduced fittings: 1 along the last dimension (0 if its extent is 1), 0 elsewhere
            const uint32_t want = (k == p.fdim && a.shape[k] > 1) ? 1u : 0u;
            if (p.fitting[k][1] != want) fast = false;
        }
    }
    p.fast = (fast && p.stride[p.fdim] == 1) ? 1 : 0;
}

bool port_needs_wide(const PortDev& p, const arol_task_desc& d) {
    for (int k = 0; k < 4; ++k) {
        double v = p.origin[k];
        for (int q = 0; q < d.rep_rank; ++q) v += (double)p.paving[k][q] * (double)(d.rep[q] - 1);
        if (v >= 2147483647.0) return true;
    }
    return false;
}

// A FIR task whose leading array dimensions are frames (origin 0, paving 1
// on their own repetition dimension, fitting 0, iterated completely, the
// same extents in and out) is the same task on (frames x rows, W): the rows
// of every frame follow each other in memory, so every linear offset is
// unchanged.  This lets such tasks (and frames = 1) take the row-FIR path.
bool flatten_frames(const arol_task_desc& d, arol_task_desc* o) {
    const int R = d.in[0].rank;
    if (d.elem != AROL_ELEM_FIR || R < 3 || d.out[0].rank != R || d.rep_rank != R) return false;
    const arol_tiler &ti = d.in_tiler[0], &to = d.out_tiler[0];
    if (ti.pattern_rank != 1 || to.pattern_rank != 1) return false;
    int64_t rows = 1;
    for (int k = 0; k < R - 1; ++k) {
        if (d.in[0].shape[k] != d.rep[k] || d.out[0].shape[k] != d.rep[k]) return false;
        if (ti.origin[k] != 0 || to.origin[k] != 0 || ti.fitting[k][0] != 0 || to.fitting[k][0] != 0) return false;
        for (int q = 0; q < R; ++q)
            if (ti.paving[k][q] != (q == k ? 1 : 0) || to.paving[k][q] != (q == k ? 1 : 0)) return false;
        rows *= d.rep[k];
    }
    for (int q = 0; q < R - 1; ++q)
        if (ti.paving[R - 1][q] != 0 || to.paving[R - 1][q] != 0) return false;
    if (rows >= 2147483647LL) return false;
    *o = d;
    o->rep_rank = 2;
    o->rep[0] = rows;
    o->rep[1] = d.rep[R - 1];
    arol_array_desc* arrs[2] = {&o->in[0], &o->out[0]};
    const arol_array_desc* src[2] = {&d.in[0], &d.out[0]};
    for (int a = 0; a < 2; ++a) {
        arrs[a]->rank = 2;
        arrs[a]->shape[0] = rows;
        arrs[a]->shape[1] = src[a]->shape[R - 1];
        arrs[a]->shape[2] = arrs[a]->shape[3] = 1;
    }
    arol_tiler* tls[2] = {&o->in_tiler[0], &o->out_tiler[0]};
    const arol_tiler* tsrc[2] = {&ti, &to};
    for (int a = 0; a < 2; ++a) {
        arol_tiler& t = *tls[a];
        const arol_tiler& u = *tsrc[a];
        std::memset(&t, 0, sizeof t);
        t.origin[1] = u.origin[R - 1];
        t.paving[0][0] = 1;
        t.paving[1][1] = u.paving[R - 1][R - 1];
        t.fitting[1][0] = u.fitting[R - 1][0];
        t.pattern_rank = 1;
        t.pattern[0] = u.pattern[0];
    }
    return true;
}

// The column form: leading frames as above, then rows (step S down the
// rows per repetition, the pattern running down them) and columns (one per
// repetition).  Frames merge into rows only when every frame's rows are
// covered exactly without wrap (origin 0, rows = S * repetitions, T <= S, and
// the output likewise), or when there is a single frame.
bool flatten_frames_col(const arol_task_desc& d, arol_task_desc* o) {
    const int R = d.in[0].rank;
    if (d.elem != AROL_ELEM_FIR || R < 3 || d.out[0].rank != R || d.rep_rank != R) return false;
    const arol_tiler &ti = d.in_tiler[0], &to = d.out_tiler[0];
    if (ti.pattern_rank != 1 || to.pattern_rank != 1) return false;
    int64_t frames = 1;
    for (int k = 0; k < R - 2; ++k) {
        if (d.in[0].shape[k] != d.rep[k] || d.out[0].shape[k] != d.rep[k]) return false;
        if (ti.origin[k] != 0 || to.origin[k] != 0 || ti.fitting[k][0] != 0 || to.fitting[k][0] != 0) return false;
        for (int q = 0; q < R; ++q)
            if (ti.paving[k][q] != (q == k ? 1 : 0) || to.paving[k][q] != (q == k ? 1 : 0)) return false;
        frames *= d.rep[k];
    }
    const int rr = R - 2, cc = R - 1;
    for (int q = 0; q < R; ++q) {
        if (q != rr && (ti.paving[rr][q] != 0 || to.paving[rr][q] != 0)) return false;
        if (ti.paving[cc][q] != (q == cc ? 1 : 0) || to.paving[cc][q] != (q == cc ? 1 : 0)) return false;
    }
    if (ti.fitting[rr][0] != 1 || to.fitting[rr][0] != 1 || ti.fitting[cc][0] != 0 || to.fitting[cc][0] != 0) return false;
    const int64_t S = ti.paving[rr][rr], m = to.paving[rr][rr], R0 = d.rep[rr];
    if (frames > 1) {
        if (ti.origin[rr] != 0 || to.origin[rr] != 0 || S < 1 || d.in[0].shape[rr] != S * R0 ||
            d.out[0].shape[rr] != m * R0 || ti.pattern[0] > S)
            return false;
    }
    if (frames * d.in[0].shape[rr] >= 2147483647LL || frames * d.out[0].shape[rr] >= 2147483647LL ||
        frames * R0 >= 2147483647LL)
        return false;
    *o = d;
    o->rep_rank = 2;
    o->rep[0] = frames * R0;
    o->rep[1] = d.rep[cc];
    arol_array_desc* arrs[2] = {&o->in[0], &o->out[0]};
    const arol_array_desc* src[2] = {&d.in[0], &d.out[0]};
    for (int a = 0; a < 2; ++a) {
        arrs[a]->rank = 2;
        arrs[a]->shape[0] = frames * src[a]->shape[rr];
        arrs[a]->shape[1] = src[a]->shape[cc];
        arrs[a]->shape[2] = arrs[a]->shape[3] = 1;
    }
    arol_tiler* tls[2] = {&o->in_tiler[0], &o->out_tiler[0]};
    const arol_tiler* tsrc[2] = {&ti, &to};
    for (int a = 0; a < 2; ++a) {
        arol_tiler& t = *tls[a];
        const arol_tiler& u = *tsrc[a];
        std::memset(&t, 0, sizeof t);
        t.origin[0] = u.origin[rr];
        t.origin[1] = u.origin[cc];
        t.paving[0][0] = u.paving[rr][rr];
        t.paving[1][1] = 1;
        t.fitting[0][0] = 1;
        t.pattern_rank = 1;
        t.pattern[0] = u.pattern[0];
    }
    return true;
}

TaskDev make_taskdev_exact(const arol_task_desc& d);

// One frame of a rank-3 fir task whose dimension 0 is frames (origin 0,
// paving 1 on its own repetition dimension, fitting 0, the same extent in
// and out): the rank-2 task on (rows, cols).
bool strip_frame(const arol_task_desc& d, arol_task_desc* o) {
    if (d.elem != AROL_ELEM_FIR || d.in[0].rank != 3 || d.out[0].rank != 3 || d.rep_rank != 3 || d.n_in != 1) return false;
    const arol_tiler &ti = d.in_tiler[0], &to = d.out_tiler[0];
    if (ti.pattern_rank != 1 || to.pattern_rank != 1) return false;
    if (d.in[0].shape[0] != d.rep[0] || d.out[0].shape[0] != d.rep[0] || ti.origin[0] || to.origin[0] ||
        ti.fitting[0][0] || to.fitting[0][0])
        return false;
    for (int q = 0; q < 3; ++q)
        if (ti.paving[0][q] != (q == 0) || to.paving[0][q] != (q == 0) || (q > 0 && (ti.paving[q][0] || to.paving[q][0])))
            return false;
    *o = d;
    o->rep_rank = 2;
    o->rep[0] = d.rep[1];
    o->rep[1] = d.rep[2];
    o->rep[2] = o->rep[3] = 0;
    arol_array_desc* arrs[2] = {&o->in[0], &o->out[0]};
    const arol_array_desc* src[2] = {&d.in[0], &d.out[0]};
    for (int a = 0; a < 2; ++a) {
        arrs[a]->rank = 2;
        arrs[a]->shape[0] = src[a]->shape[1];
        arrs[a]->shape[1] = src[a]->shape[2];
        arrs[a]->shape[2] = arrs[a]->shape[3] = 1;
    }
    arol_tiler* tls[2] = {&o->in_tiler[0], &o->out_tiler[0]};
    const arol_tiler* tsrc[2] = {&ti, &to};
    for (int a = 0; a < 2; ++a) {
        arol_tiler& t = *tls[a];
        const arol_tiler& u = *tsrc[a];
        std::memset(&t, 0, sizeof t);
        for (int k = 0; k < 2; ++k) {
            t.origin[k] = u.origin[k + 1];
            t.fitting[k][0] = u.fitting[k + 1][0];
            for (int q = 0; q < 2; ++q) t.paving[k][q] = u.paving[k + 1][q + 1];
        }
        t.pattern_rank = 1;
        t.pattern[0] = u.pattern[0];
    }
    return true;
}

// batch_form: the form the batch engine runs (a column FIR over frames that
// cannot merge keeps the column-FIR path with frames as an outer
// repetition; its ports then describe one frame, so only the batch kernels'
// column-FIR path may take it).  Otherwise the exact or frame-merged form
// that the per-repetition kernels take.
TaskDev make_taskdev(const arol_task_desc& d, bool batch_form = false) {
    arol_task_desc flat;
    if (flatten_frames(d, &flat)) {
        const TaskDev t = make_taskdev_exact(flat);
        if (t.rowfir) return t;
    }
    if (flatten_frames_col(d, &flat)) {
        const TaskDev t = make_taskdev_exact(flat);
        if (t.colfir) return t;
    }
    // A column FIR on each frame of a rank-3 array whose frames cannot merge
    // into rows (windows that overlap or wrap within a frame): the column-FIR
    // path over one frame's ports, with the frame as an outer repetition.
    if (batch_form && strip_frame(d, &flat)) {
        TaskDev t = make_taskdev_exact(flat);
        if (t.colfir && (int64_t)t.nreps * d.rep[0] < 2147483647LL) {
            t.cf_frames = (int32_t)d.rep[0];
            t.rep[1] = t.cf_frames;
            t.rep_div[1] = make_fastdiv((uint32_t)t.cf_frames);
            t.cf_in_frame = elems_of(flat.in[0]);
            t.cf_out_frame = elems_of(flat.out[0]);
            t.nreps *= d.rep[0];
            t.in_elems = elems_of(d.in[0]);
            t.out_elems = elems_of(d.out[0]);
            return t;
        }
    }
    return make_taskdev_exact(d);
}

TaskDev make_taskdev_exact(const arol_task_desc& d) {
    TaskDev t;
    std::memset(&t, 0, sizeof t);
    for (int q = 0; q < 4; ++q) t.rep[q] = 1;
    // real repetition dims are right-aligned so that the last one is fastest
    // in decode_rep; paving columns are re-indexed to match.
    const int shift = 4 - d.rep_rank;
    arol_task_desc dd = d;
    for (int k = 0; k < AROL_MAX_RANK; ++k)
        for (int q = 0; q < 4; ++q) dd.in_tiler[0].paving[k][q] = dd.out_tiler[0].paving[k][q] = 0;
    for (int q = 0; q < d.rep_rank; ++q) {
        t.rep[q + shift] = (int32_t)d.rep[q];
        for (int k = 0; k < AROL_MAX_RANK; ++k) {
            dd.in_tiler[0].paving[k][q + shift] = d.in_tiler[0].paving[k][q];
            dd.out_tiler[0].paving[k][q + shift] = d.out_tiler[0].paving[k][q];
        }
    }
    t.nreps = reps_of(d);
    t.in_elems = elems_of(d.in[0]);
    t.out_elems = elems_of(d.out[0]);
    for (int q = 0; q < 4; ++q) t.rep_div[q] = make_fastdiv((uint32_t)t.rep[q]);
    make_port(d.in[0], dd.in_tiler[0], 4, t.in);
    make_port(d.out[0], dd.out_tiler[0], 4, t.out);
    t.elem = d.elem == AROL_ELEM_FIR ? ELEM_FIR : ELEM_COPY;
    t.T = (int32_t)pattern_size(d.in_tiler[0]);
    t.m = (int32_t)pattern_size(d.out_tiler[0]);
    t.esize = esize_of(d.in[0].dtype);
    t.in_dt = d.elem == AROL_ELEM_FIR ? d.in[0].dtype : kStF32;
    t.out_dt = d.elem == AROL_ELEM_FIR ? d.out[0].dtype : kStF32;
    arol_task_desc full = dd;
    full.rep_rank = 4;
    for (int q = 0; q < 4; ++q) full.rep[q] = t.rep[q];
    t.wide = (t.nreps >= 2147483647LL || port_needs_wide(t.in, full) || port_needs_wide(t.out, full)) ? 1 : 0;
    // Row FIR: one row per r0, step along the row per r1, one contiguous
    // pattern of T taps, m contiguous outputs per repetition.
    const arol_tiler &ti = d.in_tiler[0], &to = d.out_tiler[0];
    if (d.elem == AROL_ELEM_FIR && !t.wide && t.in_dt == kStF32 && t.out_dt == kStF32 && d.rep_rank == 2 && d.in[0].rank == 2 &&
        d.out[0].rank == 2 &&
        ti.pattern_rank == 1 && to.pattern_rank == 1 && ti.paving[0][0] == 1 && ti.paving[0][1] == 0 &&
        ti.paving[1][0] == 0 && ti.fitting[0][0] == 0 && ti.fitting[1][0] == 1 && to.paving[0][0] == 1 &&
        to.paving[0][1] == 0 && to.paving[1][0] == 0 && to.paving[1][1] == d.fir_m && to.fitting[0][0] == 0 &&
        to.fitting[1][0] == 1 && ti.paving[1][1] >= 1 && ti.paving[1][1] <= 32 && d.fir_T <= 32 && d.fir_m <= 16 &&
        d.in[0].shape[1] > 1 && d.out[0].shape[1] > 1) {
        t.rowfir = 1;
        t.step = (int32_t)emod(ti.paving[1][1], d.in[0].shape[1]);
        if (t.step < 1) t.rowfir = 0;
    }
    // Column FIR: one column per r1, step down the rows per r0, the pattern
    // running down the rows, m consecutive output rows per repetition.
    if (!t.rowfir && d.elem == AROL_ELEM_FIR && !t.wide && t.in_dt == kStF32 && t.out_dt == kStF32 && d.rep_rank == 2 &&
        d.in[0].rank == 2 && d.out[0].rank == 2 && ti.pattern_rank == 1 && to.pattern_rank == 1 &&
        ti.paving[0][0] >= 1 && ti.paving[0][1] == 0 && ti.paving[1][0] == 0 && ti.paving[1][1] == 1 &&
        ti.fitting[0][0] == 1 && ti.fitting[1][0] == 0 && to.paving[0][0] == d.fir_m && to.paving[0][1] == 0 &&
        to.paving[1][0] == 0 && to.paving[1][1] == 1 && to.fitting[0][0] == 1 && to.fitting[1][0] == 0 &&
        d.fir_T <= 32 && d.fir_m <= 16 && d.in[0].shape[0] > 1 && d.out[0].shape[0] > 1) {
        t.step = (int32_t)emod(ti.paving[0][0], d.in[0].shape[0]);
        t.colfir = t.step >= 1 ? 1 : 0;
    }
    // FIR on a 2-D pattern: pattern dims map to the array dims in order
    // (fitting identity), diagonal paving, m outputs along the output row.
    if (d.elem == AROL_ELEM_FIR && !t.wide && t.in_dt == kStF32 && t.out_dt == kStF32 && d.rep_rank == 2 && d.in[0].rank == 2 &&
        d.out[0].rank == 2 && ti.pattern_rank == 2 && to.pattern_rank == 1 && ti.fitting[0][0] == 1 &&
        ti.fitting[0][1] == 0 && ti.fitting[1][0] == 0 && ti.fitting[1][1] == 1 && ti.paving[0][1] == 0 &&
        ti.paving[1][0] == 0 && to.paving[0][0] == 1 && to.paving[0][1] == 0 && to.paving[1][0] == 0 &&
        to.paving[1][1] == d.fir_m && (d.fir_m == 1 || (to.fitting[0][0] == 0 && to.fitting[1][0] == 1)) &&
        d.fir_T <= 64 && d.fir_m <= 16 && elems_of(d.in[0]) > 0 && elems_of(d.out[0]) > 0) {
        const int64_t s0 = emod(ti.paving[0][0], d.in[0].shape[0]), s1 = emod(ti.paving[1][1], d.in[0].shape[1]);
        const int64_t p0 = ti.pattern[0], p1 = ti.pattern[1];
        // tile of 16 x 64 repetitions, or 32 x 32, whose input window fits 8192 floats
        const int shapes[2][2] = {{16, 64}, {32, 32}};
        for (const auto& sh : shapes) {
            const int64_t wh = s0 * (sh[0] - 1) + p0, ww = s1 * (sh[1] - 1) + p1;
            const int64_t tiles = ((d.rep[0] + sh[0] - 1) / sh[0]) * ((d.rep[1] + sh[1] - 1) / sh[1]);
            if (wh * ww <= 8192 && tiles < 2147483647LL) {
                t.fir2d = 1;
                t.s0 = (int32_t)s0;
                t.s1 = (int32_t)s1;
                t.p0 = (int32_t)p0;
                t.p1 = (int32_t)p1;
                t.bh = sh[0];
                t.bw = sh[1];
                break;
            }
        }
    }
    return t;
}

// ------------------------------------------------------------------ matchers

bool tiler_is(const arol_tiler& t, int rank, std::initializer_list<int64_t> origin,
              std::initializer_list<std::initializer_list<int64_t>> paving,
              std::initializer_list<std::initializer_list<int64_t>> fitting, int rep_rank) {
    int k = 0;
    for (int64_t o : origin) if (t.origin[k++] != o) return false;
    k = 0;
    for (auto& row : paving) {
        int q = 0;
        for (int64_t v : row) if (t.paving[k][q++] != v) return false;
        if (q != rep_rank) return false;
        ++k;
    }
    if (k != rank) return false;
    k = 0;
    for (auto& row : fitting) {
        int p = 0;
        for (int64_t v : row) if (t.fitting[k][p++] != v) return false;
        if (p != t.pattern_rank) return false;
        ++k;
    }
    return k == rank;
}

// The panel form of a tiled product: A (M,K) row panels, B (K,N) column
// panels, C (M,N) tiles, all 128 x 128 tiles, origins 0, fittings identity.
bool is_matmul_panels(const arol_task_desc& d, int* M, int* N, int* K) {
    if (d.n_in != 2 || d.rep_rank != 2 || d.in[0].rank != 2 || d.in[1].rank != 2 || d.out[0].rank != 2) return false;
    const int64_t m = d.in[0].shape[0], k = d.in[0].shape[1], n = d.in[1].shape[1];
    if (d.in[1].shape[0] != k || d.out[0].shape[0] != m || d.out[0].shape[1] != n) return false;
    const arol_tiler &A = d.in_tiler[0], &B = d.in_tiler[1], &C = d.out_tiler[0];
    if (A.pattern_rank != 2 || B.pattern_rank != 2 || C.pattern_rank != 2) return false;
    const int64_t tm = A.pattern[0], tn = B.pattern[1];
    if (A.pattern[1] != k || B.pattern[0] != k || C.pattern[0] != tm || C.pattern[1] != tn) return false;
    if (d.rep[0] * tm != m || d.rep[1] * tn != n) return false;
    if (!tiler_is(A, 2, {0, 0}, {{tm, 0}, {0, 0}}, {{1, 0}, {0, 1}}, 2)) return false;
    if (!tiler_is(B, 2, {0, 0}, {{0, 0}, {0, tn}}, {{1, 0}, {0, 1}}, 2)) return false;
    if (!tiler_is(C, 2, {0, 0}, {{tm, 0}, {0, tn}}, {{1, 0}, {0, 1}}, 2)) return false;
    *M = (int)m;
    *N = (int)n;
    *K = (int)k;
    return tm == 128 && tn == 128;
}

// A rank-3 (frames, rows, cols) view of a single fir task of the row form
// (axis = 2: horizontal) or column form (axis = 1: vertical), rank-2 arrays
// being one frame.  Fills frames/rows/cols/step/T/m; origins must be 0.
struct Pass { int64_t F, H, W; int64_t S, T, m; };

bool match_pass(const arol_task_desc& d, int axis, Pass* ps) {
    if (d.elem != AROL_ELEM_FIR || d.n_in != 1) return false;
    const arol_array_desc &a = d.in[0], &o = d.out[0];
    const arol_tiler &ti = d.in_tiler[0], &to = d.out_tiler[0];
    if (a.rank != o.rank || a.rank != d.rep_rank || (a.rank != 2 && a.rank != 3)) return false;
    if (ti.pattern_rank != 1 || to.pattern_rank != 1) return false;
    const int off = a.rank == 3 ? 1 : 0;   // index of the rows dim
    const int ax = axis - (3 - a.rank);     // axis in this rank
    const int64_t S = ti.paving[ax][ax], T = ti.pattern[0], m = to.pattern[0];
    for (int k = 0; k < a.rank; ++k) {
        if (ti.origin[k] != 0 || to.origin[k] != 0) return false;
        for (int q = 0; q < a.rank; ++q) {
            const int64_t want_in = (k == q) ? (k == ax ? S : 1) : 0;
            const int64_t want_out = (k == q) ? (k == ax ? m : 1) : 0;
            if (ti.paving[k][q] != want_in || to.paving[k][q] != want_out) return false;
        }
        if (ti.fitting[k][0] != (k == ax ? 1 : 0) || to.fitting[k][0] != (k == ax ? 1 : 0)) return false;
    }
    for (int k = 0; k < a.rank; ++k) {
        const int64_t want_rep = k == ax ? a.shape[k] / S : a.shape[k];
        if (d.rep[k] != want_rep) return false;
        const int64_t want_out = k == ax ? want_rep * m : a.shape[k];
        if (o.shape[k] != want_out) return false;
    }
    if (a.shape[ax] % S != 0) return false;
    ps->F = a.rank == 3 ? a.shape[0] : 1;
    ps->H = a.shape[off];
    ps->W = a.shape[off + 1];
    ps->S = S;
    ps->T = T;
    ps->m = m;
    return true;
}

// One task of a separable chain: a f32 fir along the columns of each row
// (row pass, axis 1) or down the rows of each column (column pass, axis 0) of
// a rank-2 array or of every frame of a rank-3 one: along its axis input
// paving S, fitting 1, any origin, output paving m, fitting 1, origin 0; the
// other axis and the frames identity.  Fills the pass (taps offset left 0)
// and the frame count and input/output extents.
bool match_sep_pass(const arol_task_desc& d, SepPassDev* p, int64_t* F, int64_t in_hw[2], int64_t out_hw[2],
                    bool any_storage = false) {
    if (d.elem != AROL_ELEM_FIR || d.n_in != 1) return false;
    const arol_array_desc &a = d.in[0], &o = d.out[0];
    if (!any_storage && (a.dtype != AROL_F32 || o.dtype != AROL_F32)) return false;
    const int r = a.rank;
    if ((r != 2 && r != 3) || o.rank != r || d.rep_rank != r) return false;
    const arol_tiler &ti = d.in_tiler[0], &to = d.out_tiler[0];
    if (ti.pattern_rank != 1 || to.pattern_rank != 1 || ti.pattern[0] > 32 || to.pattern[0] > 16) return false;
    if (r == 3) {   // frames
        if (a.shape[0] != d.rep[0] || o.shape[0] != d.rep[0] || ti.origin[0] || to.origin[0] || ti.fitting[0][0] ||
            to.fitting[0][0])
            return false;
        for (int q = 0; q < 3; ++q)
            if (ti.paving[0][q] != (q == 0) || to.paving[0][q] != (q == 0) || (q > 0 && (ti.paving[q][0] || to.paving[q][0])))
                return false;
    }
    const int ar = r - 2, ac = r - 1;
    int axis = -1;
    if (ti.fitting[ac][0] == 1 && ti.fitting[ar][0] == 0) axis = 1;
    else if (ti.fitting[ar][0] == 1 && ti.fitting[ac][0] == 0) axis = 0;
    else return false;
    const int ax = axis == 1 ? ac : ar, ot = axis == 1 ? ar : ac;
    if (to.fitting[ax][0] != 1 || to.fitting[ot][0] != 0) return false;
    if (ti.paving[ax][ot] || ti.paving[ot][ax] || ti.paving[ot][ot] != 1 || to.paving[ax][ot] || to.paving[ot][ax] ||
        to.paving[ot][ot] != 1 || ti.origin[ot] || to.origin[ot] || to.origin[ax])
        return false;
    const int64_t n_in = a.shape[ax], R = d.rep[ax], m = to.pattern[0];
    if (to.paving[ax][ax] != m || o.shape[ax] != m * R || d.rep[ot] != a.shape[ot] || o.shape[ot] != a.shape[ot]) return false;
    if (n_in < 1 || R < 1 || n_in >= (1 << 30) || m * R >= (1 << 30) || a.shape[ot] >= (1 << 30)) return false;
    const int64_t S = emod(ti.paving[ax][ax], n_in);
    if (S < 1 || S * R >= (1 << 30) || S * 8 >= (1 << 30)) return false;   // the kernel's 32-bit window arithmetic
    std::memset(p, 0, sizeof *p);
    p->axis = axis;
    p->T = (int32_t)ti.pattern[0];
    p->m = (int32_t)m;
    p->S = (int32_t)S;
    p->o = (int32_t)emod(ti.origin[ax], n_in);
    p->n_in = (int32_t)n_in;
    p->n_out = (int32_t)(m * R);
    p->R = (int32_t)R;
    *F = r == 3 ? a.shape[0] : 1;
    in_hw[0] = a.shape[ar];
    in_hw[1] = a.shape[ac];
    out_hw[0] = o.shape[ar];
    out_hw[1] = o.shape[ac];
    return true;
}

// Plans the streaming form of a chain of a row pass then a column pass
// (host only): chunks of sepstream_chunk_cols() intermediate columns, the
// widest input window of a chunk, the stages and the shared taps per warp;
// refused when the column pass's window outgrows the ring of intermediate
// rows or the shared memory would not leave two CTAs per SM.  The bands
// are chosen at the first run (sepstream_bands).
constexpr size_t kSsSmemMax = 110 * 1024;

bool plan_sepstream(const SepChainDev& d, SsChain* out, int* xw_max, int* nst, int* tapw) {
    if (d.K != 2 || d.p[0].axis != 1 || d.p[1].axis != 0) return false;
    if (d.p[1].T > sepstream_max_taps()) return false;
    SepChainDev one = d;
    one.BH = d.p[1].R;
    const SsChain c = ss_chain_of(one);
    const int xw = sepstream_window(c), ns = sepstream_stages(xw), tw = sepstream_tap_floats(c);
    if (sepstream_smem(xw, ns, tw) > kSsSmemMax || c.F * c.chunks * c.Rv >= 2147483647LL) return false;
    *out = c;
    *xw_max = xw;
    *nst = ns;
    *tapw = tw;
    return true;
}

// Bands of column-pass repetitions for the streaming chain kernel on the
// current device: the band height that minimises the rows the busiest CTA
// walks (waves of resident CTAs times the rows of one band, halo included).
void sepstream_bands(SsChain& c, int xw_max, int nst, int tapw, int* units) {
    const int64_t per = c.F * c.chunks;
    const int64_t cap =
        (int64_t)device_sm_count() * sepstream_ctas_per_sm(c.Th, c.Tv, false, sepstream_smem(xw_max, nst, tapw));
    int64_t best = -1, best_bh = c.Rv;
    for (int64_t nb = 1; nb <= std::min<int64_t>(c.Rv, 4096); ++nb) {
        const int64_t bh = (c.Rv + nb - 1) / nb, u = per * ((c.Rv + bh - 1) / bh);
        const int64_t cost = ((u + cap - 1) / cap) * ((int64_t)c.Sv * (bh - 1) + c.Tv);
        if (best < 0 || cost < best) best = cost, best_bh = bh;
    }
    c.BH = (int32_t)best_bh;
    c.bands = (c.Rv + c.BH - 1) / c.BH;
    *units = (int)(per * c.bands);
}

// The tile kernel's plan: region sizes separate into a row part (depending
// on the tile row only) and a column part (tile column only), so the largest
// shared buffer and the total work of a tile shape take one pass over tile
// rows and one over tile columns.  Among the shapes whose shared memory
// (taps and two buffers) fits kSepSmemFloats, the one with the least work
// wins: staging the window, and T multiply-adds per output of every pass
// (halos included) divided by the pass's lane use, weighted up for narrow
// tiles whose row segments use DRAM sectors poorly; shapes with fewer tiles
// than kSepFillTiles pay for the idle SMs.
constexpr int kSepSmemFloats = 14 * 1024;   // 56 KB: four CTAs per SM
constexpr double kSepFillTiles = 4.0 * 152;  // four tiles per SM of a 152-SM GB300 (planning stays host-only)

// The passes and stage extents of a chain of 2 .. 4 row and column passes
// (false for any other chain).
bool describe_sepchain(const std::vector<arol_task_desc>& descs, SepChainDev* out, bool any_storage = false) {
    const int K = (int)descs.size();
    if (K < 2 || K > kSepMaxPasses) return false;
    SepChainDev d;
    std::memset(&d, 0, sizeof d);
    d.K = K;
    int64_t F0 = -1, ntaps = 0;
    for (int k = 0; k < K; ++k) {
        int64_t F, ihw[2], ohw[2];
        if (!match_sep_pass(descs[k], &d.p[k], &F, ihw, ohw, any_storage)) return false;
        if (k == 0) {
            F0 = F;
            d.H[0] = (int32_t)ihw[0];
            d.W[0] = (int32_t)ihw[1];
        } else if (F != F0 || ihw[0] != d.H[k] || ihw[1] != d.W[k]) {
            return false;
        }
        d.H[k + 1] = (int32_t)ohw[0];
        d.W[k + 1] = (int32_t)ohw[1];
        d.p[k].tap_off = (int32_t)ntaps;
        ntaps += (int64_t)d.p[k].m * d.p[k].T;
    }
    d.F = F0;
    d.ntaps = (int32_t)ntaps;
    *out = d;
    return true;
}

// Tiles of the last stage for the shared-memory tile kernel (false when no
// tile's regions fit shared memory).
bool plan_sepchain(const SepChainDev& d, SepChainDev* out) {
    const int K = d.K;
    int max_m = 1;
    for (int k = 0; k < K; ++k) max_m = std::max(max_m, (int)d.p[k].m);
    const int taps4 = kSepMaxPasses * 32 * (max_m <= 4 ? 4 : 16);   // every pass's taps, transposed
    // tile heights: powers of two, and those whose window, through the first
    // column pass, is just under a multiple of 32 rows (the row passes' lanes
    // walk rows 32 at a time)
    std::vector<int> bhs = {4, 8, 16, 32, 64, 128};
    for (int k = 0; k < K; ++k) {
        if (d.p[k].axis != 0) continue;
        for (int rows = 32; rows <= 128; rows += 32) {
            const int reps = (rows - d.p[k].T) / d.p[k].S + 1;
            if (reps >= 1) bhs.push_back(reps * d.p[k].m);
        }
        break;
    }
    static const int bws[] = {16, 32, 64, 128, 256, 512};
    double best = 1e300;
    bool found = false;
    for (int bh : bhs)
        for (int bw : bws) {
            SepChainDev c = d;
            c.BH = std::min<int32_t>(bh, std::max<int32_t>(d.H[K], 1));
            c.BW = std::min<int32_t>(bw, std::max<int32_t>(d.W[K], 1));
            c.tiles_y = (int32_t)((d.H[K] + c.BH - 1) / c.BH);
            c.tiles_x = (int32_t)((d.W[K] + c.BW - 1) / c.BW);
            if (c.tiles_y == 0 || c.tiles_x == 0) continue;
            int64_t rmax[kSepMaxPasses + 1] = {}, cmax[kSepMaxPasses + 1] = {};
            double rsum[kSepMaxPasses + 1] = {}, csum[kSepMaxPasses + 1] = {};
            SepRange rows[kSepMaxPasses + 1], cols[kSepMaxPasses + 1];
            for (int ty = 0; ty < c.tiles_y; ++ty) {
                sep_regions(c, ty, 0, rows, cols);
                for (int k = 0; k <= K; ++k) {
                    rmax[k] = std::max<int64_t>(rmax[k], rows[k].len);
                    rsum[k] += rows[k].len;
                }
            }
            for (int tx = 0; tx < c.tiles_x; ++tx) {
                sep_regions(c, 0, tx, rows, cols);
                for (int k = 0; k <= K; ++k) {
                    cmax[k] = std::max<int64_t>(cmax[k], cols[k].len);
                    csum[k] += cols[k].len;
                }
            }
            int64_t buf[2] = {0, 0};
            double work = 2.0 * rsum[0] * csum[0];   // staging the window
            for (int k = 0; k < K; ++k) {
                // rows of an odd stride (cols | 1), whole 16-byte units per buffer
                buf[k & 1] = std::max<int64_t>(buf[k & 1], (rmax[k] * (cmax[k] | 1) + 3) & ~int64_t(3));
                // a pass's lanes walk the region's rows (row pass) or columns
                // (column pass) 32 at a time: T multiply-adds per output,
                // lanes past the region's edge idle
                const int64_t lanes = d.p[k].axis == 1 ? rmax[k] : cmax[k];
                const double util = (double)lanes / (32.0 * (double)((lanes + 31) / 32));
                work += d.p[k].T * rsum[k + 1] * csum[k + 1] / util;
            }
            if (taps4 + buf[0] + buf[1] > kSepSmemFloats) continue;
            const double tiles = (double)d.F * c.tiles_y * c.tiles_x;
            if (tiles >= 2147483647.0) continue;   // the kernel counts tiles in 32 bits
            const double fill = kSepFillTiles;
            // narrow tiles read short row segments: a sector-efficiency factor
            const double cost = work * std::max(1.0, fill / tiles) * (1.0 + 8.0 / c.BW);
            if (cost < best) {
                best = cost;
                c.buf = (int32_t)buf[0];
                c.buf1 = (int32_t)buf[1];
                *out = c;
                found = true;
            }
        }
    return found;
}

}  // namespace

// ===================================================================== tasks

constexpr int kPipeChunks = 8;   // frame chunks of the host-buffer pipeline

struct arol_task_s {
    int kind = 0;                        // 0 single, 1 chain
    int kernel = 0;                      // arol_task_info_t.kernel
    std::vector<arol_task_desc> descs;   // one per task (fir_taps_host cleared)
    std::vector<int64_t> tap_off;        // offset of each task's taps in taps_host
    std::vector<float> taps_host;
    bool taps_ready = true;
    const float* taps_borrowed = nullptr;
    float* taps_dev = nullptr;
    bool taps_dirty = true;
    int device = -1;
    // unfused chain intermediates
    std::vector<void*> mids;
    // row/column-FIR tasks and unfused chains run as a one-member batch
    arol_batch ib = nullptr;
    bool ib_checked = false;
    // a row-FIR task in 16-word regions (rr_ok)
    bool rr_ok = false;
    int rr_S = 0, rr_T = 0, rr_M = 0, rr_W = 0, rr_o = 0;
    int64_t rr_rows = 0;
    // fused downscaler
    int64_t ds_frames = 0;
    int ds_H = 0, ds_W = 0;
    bool ds_in16 = false, ds_mid16 = false, ds_out16 = false, ds_half16 = false;
    // matmul
    int mm_M = 0, mm_N = 0, mm_K = 0;
    // fused separable chain (kernel 4): parameters and region tables (rows
    // per tile row, then columns per tile column), on the host and the device
    SepChainDev sc{};
    std::vector<int32_t> sc_tab;
    int32_t* sc_tab_dev = nullptr;
    // streaming row-then-column chain (kernel 5)
    SepChainDev sd{};     // the chain as separable passes (sd_ok), for the backward
    bool sd_ok = false;
    SsChain ss{};
    int ss_units = 0, ss_xw = 0, ss_nst = 2, ss_tapw = 0;
    unsigned* err_flag = nullptr;        // device word: bounded waits that gave up
    // backward scratch and inverse maps
    float* partials = nullptr;
    int64_t partials_cap = 0;
    std::vector<int64_t*> inv_start;
    std::vector<int32_t*> inv_list;
    std::vector<float*> grad_mids;
    // chain backward: per intermediate, a one-pass task over the same tiler
    // and taps that recomputes it on the batch engine (row- and column-FIR
    // passes); null where the per-repetition walk recomputes it
    std::vector<arol_task> rc;
    bool rc_checked = false;
    // host-buffer staging
    void* stage_in[2] = {nullptr, nullptr};
    void* stage_out = nullptr;
    bool pipe_ready = false;             // chunked host-buffer pipeline (fused downscaler)
    cudaStream_t pipe_stream[2] = {nullptr, nullptr};
    cudaEvent_t pipe_in[8] = {}, pipe_done[8] = {};
    cudaEvent_t pipe_last = nullptr;
    arol_task_info_t info{};
};

namespace {

arol_status remember_device(arol_task t) {
    int dev = 0;
    AROL_CUDA(cudaGetDevice(&dev), "cudaGetDevice");
    if (t->device < 0) t->device = dev;
    else if (t->device != dev)
        return fail(AROL_ERR_INVALID, "task used on device %d but its buffers live on device %d", dev, t->device);
    return AROL_OK;
}

// Device allocations go through here.  AROL_FAIL_ALLOC=1 makes every one
// fail as if the device were out of memory (failure injection for tests;
// nothing is allocated), so callers' error paths can be exercised on the host.
cudaError_t arol_malloc(void** p, size_t bytes) {
    const char* v = std::getenv("AROL_FAIL_ALLOC");
    if (v && v[0] == '1') {
        *p = nullptr;
        return cudaErrorMemoryAllocation;
    }
    return cudaMalloc(p, bytes);
}

arol_status dev_alloc(arol_task t, void** p, size_t bytes, const char* what) {
    arol_status st = remember_device(t);
    if (st != AROL_OK) return st;
    if (*p) return AROL_OK;
    cudaError_t e = arol_malloc(p, bytes ? bytes : 16);
    if (e != cudaSuccess) {
        *p = nullptr;
        return cuda_fail(e, what);
    }
    return AROL_OK;
}

// The task's device error word (bounded device-side waits that gave up),
// cleared when allocated and after arol_task_sync_status reports it.
arol_status ensure_err(arol_task t, cudaStream_t s) {
    if (t->err_flag) return AROL_OK;
    arol_status st = dev_alloc(t, (void**)&t->err_flag, sizeof(unsigned), "cudaMalloc(error flag)");
    if (st != AROL_OK) return st;
    AROL_CUDA(cudaMemsetAsync(t->err_flag, 0, sizeof(unsigned), s), "clear error flag");
    return AROL_OK;
}

arol_status ensure_taps(arol_task t, cudaStream_t s, const float** out) {
    *out = nullptr;
    if (t->taps_host.empty() && !t->taps_borrowed) return AROL_OK;
    if (t->taps_borrowed) {
        *out = t->taps_borrowed;
        return AROL_OK;
    }
    if (!t->taps_ready) return fail(AROL_ERR_INVALID, "fir taps were never set");
    arol_status st = dev_alloc(t, (void**)&t->taps_dev, t->taps_host.size() * sizeof(float), "cudaMalloc(taps)");
    if (st != AROL_OK) return st;
    if (t->taps_dirty) {
        AROL_CUDA(cudaMemcpyAsync(t->taps_dev, t->taps_host.data(), t->taps_host.size() * sizeof(float),
                                  cudaMemcpyHostToDevice, s),
                  "upload taps");
        t->taps_dirty = false;
    }
    *out = t->taps_dev;
    return AROL_OK;
}

arol_status validate_desc(const arol_task_desc& d) {
    if (d.rep_rank < 1 || d.rep_rank > AROL_MAX_RANK) return fail(AROL_ERR_INVALID, "rep_rank %d not in [1,4]", d.rep_rank);
    for (int q = 0; q < d.rep_rank; ++q)
        if (d.rep[q] < 0 || d.rep[q] > kMaxDim) return fail(AROL_ERR_INVALID, "rep[%d] = %" PRId64 " out of range", q, d.rep[q]);
    if (d.n_out != 1) return fail(AROL_ERR_INVALID, "n_out must be 1 (got %d)", d.n_out);
    const int want_in = d.elem == AROL_ELEM_MATMUL ? 2 : 1;
    if (d.elem < AROL_ELEM_COPY || d.elem > AROL_ELEM_MATMUL) return fail(AROL_ERR_INVALID, "unknown elementary task %d", d.elem);
    if (d.n_in != want_in) return fail(AROL_ERR_INVALID, "elementary task %d takes %d inputs (got %d)", d.elem, want_in, d.n_in);
    arol_status st;
    for (int i = 0; i < d.n_in; ++i) {
        if ((st = check_array(d.in[i], "input")) != AROL_OK) return st;
        if ((st = check_tiler(d.in_tiler[i], "input tiler")) != AROL_OK) return st;
    }
    if ((st = check_array(d.out[0], "output")) != AROL_OK) return st;
    if ((st = check_tiler(d.out_tiler[0], "output tiler")) != AROL_OK) return st;
    if (reps_of(d) > 0) {
        for (int i = 0; i < d.n_in; ++i)
            if (elems_of(d.in[i]) == 0) return fail(AROL_ERR_INVALID, "input %d is empty but the repetition space is not", i);
        if (elems_of(d.out[0]) == 0) return fail(AROL_ERR_INVALID, "output is empty but the repetition space is not");
    }
    const int64_t ns_in = pattern_size(d.in_tiler[0]), ns_out = pattern_size(d.out_tiler[0]);
    switch (d.elem) {
    case AROL_ELEM_COPY:
        if (d.in[0].dtype != d.out[0].dtype) return fail(AROL_ERR_INVALID, "copy: input and output dtypes differ");
        if (ns_in != ns_out) return fail(AROL_ERR_INVALID, "copy: input pattern has %" PRId64 " elements, output %" PRId64, ns_in, ns_out);
        break;
    case AROL_ELEM_FIR:
        // f32 or bf16 storage on either side (Sec. 5 typeAllocation); arithmetic in f32
        if (d.fir_T != ns_in || d.fir_m != ns_out)
            return fail(AROL_ERR_INVALID, "fir: T=%d m=%d but patterns have %" PRId64 " and %" PRId64 " elements",
                        d.fir_T, d.fir_m, ns_in, ns_out);
        if (d.fir_m < 1 || d.fir_m > AROL_MAX_FIR_M) return fail(AROL_ERR_UNSUPPORTED, "fir: m=%d not in [1,32]", d.fir_m);
        if ((int64_t)d.fir_m * d.fir_T > AROL_MAX_FIR_TAPS) return fail(AROL_ERR_UNSUPPORTED, "fir: m*T above 8192");
        break;
    case AROL_ELEM_MATMUL: {
        if (d.in[0].dtype != AROL_BF16 || d.in[1].dtype != AROL_BF16 || d.out[0].dtype != AROL_F32)
            return fail(AROL_ERR_UNSUPPORTED, "matmul: bf16 inputs and float32 output only");
        int M, N, K;
        if (!is_matmul_panels(d, &M, &N, &K))
            return fail(AROL_ERR_UNSUPPORTED, "matmul: only the 128 x 128 panel/tile tilers of a tiled product are supported");
        if (K % 64 != 0 || K < 64) return fail(AROL_ERR_UNSUPPORTED, "matmul: K must be a positive multiple of 64");
        break;
    }
    }
    return check_partition(d.out[0], d.out_tiler[0], d.rep_rank, d.rep);
}

// A single row-FIR task that the region kernel takes (host only): one output
// row per input row, repetitions tiling the rows, output columns from 0.
void plan_row_region(arol_task t) {
    t->rr_ok = false;
    const arol_task_desc& d = t->descs[0];
    if (d.elem != AROL_ELEM_FIR || d.n_in != 1) return;
    const TaskDev td = make_taskdev(d, true);
    if (!td.rowfir || td.in_dt != kStF32 || td.out_dt != kStF32) return;
    const int64_t H = td.in.shape[0], W = td.in.shape[1], Ho = td.out.shape[0], Wo = td.out.shape[1];
    const int64_t R0 = td.rep[2], R1 = td.rep[3];
    if (R0 != H || Ho != H || td.in.origin[0] != 0 || td.out.origin[0] != 0 || td.out.origin[1] != 0) return;
    if ((int64_t)td.step * R1 != W) return;
    const int64_t o = td.in.origin[1];
    if (!rowfir_region_supported(td.step, td.T, td.m, W, Wo, o, R0)) return;
    t->rr_ok = true;
    t->rr_S = td.step;
    t->rr_T = td.T;
    t->rr_M = td.m;
    t->rr_W = (int)W;
    t->rr_o = (int)o;
    t->rr_rows = R0;
}

void fill_info_single(arol_task t) {
    const arol_task_desc& d = t->descs[0];
    arol_task_info_t& in = t->info;
    in.kind = 0;
    in.kernel = t->kernel;
    in.reps = reps_of(d);
    in.gathered_elems = 0;
    in.unique_bytes = 0;
    for (int i = 0; i < d.n_in; ++i) {
        in.gathered_elems += in.reps * pattern_size(d.in_tiler[i]);
        in.unique_bytes += elems_of(d.in[i]) * esize_of(d.in[i].dtype);
    }
    in.scattered_elems = in.reps * pattern_size(d.out_tiler[0]);
    in.unique_bytes += elems_of(d.out[0]) * esize_of(d.out[0].dtype);
    if (d.elem == AROL_ELEM_FIR) in.flops = 2.0 * d.fir_m * d.fir_T * (double)in.reps;
    else if (d.elem == AROL_ELEM_MATMUL)
        in.flops = 2.0 * (double)d.in_tiler[0].pattern[0] * d.in_tiler[0].pattern[1] * d.in_tiler[1].pattern[1] * (double)in.reps;
    else in.flops = 0;
    in.path = -1;
    if (t->kernel == 0 && d.elem != AROL_ELEM_MATMUL) {
        const TaskDev td = make_taskdev(d, true);
        in.path = t->rr_ok ? 5 : td.rowfir ? 1 : td.colfir ? 2 : td.fir2d ? (fir2d_uses_stencil(td) ? 4 : 3) : 0;
    }
    in.reserved_ = 0;
}

void free_dev(void* p) {
    if (p) cudaFree(p);
}

}  // namespace

extern "C" {

int arol_version(void) { return AROL_VERSION; }

int64_t arol_abi_struct_size(int which) {
    switch (which) {
    case 0: return (int64_t)sizeof(arol_array_desc);
    case 1: return (int64_t)sizeof(arol_tiler);
    case 2: return (int64_t)sizeof(arol_task_desc);
    case 3: return (int64_t)sizeof(arol_task_info_t);
    default: return -1;
    }
}

arol_status arol_last_error(char* buf, size_t len) {
    if (buf && len) {
        std::strncpy(buf, g_err.c_str(), len - 1);
        buf[len - 1] = 0;
    }
    return AROL_OK;
}

arol_status arol_selftest_wait_timeout(void* stream) {
    AROL_TRACE();
    cudaStream_t s = (cudaStream_t)stream;
    unsigned* err = nullptr;
    AROL_CUDA(arol_malloc((void**)&err, sizeof(unsigned)), "cudaMalloc(error word)");
    unsigned host = 0;
    cudaError_t e = cudaMemsetAsync(err, 0, sizeof(unsigned), s);
    if (e == cudaSuccess) e = launch_wait_selftest(err, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&host, err, sizeof(unsigned), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFree(err);
    if (e != cudaSuccess) return cuda_fail(e, "wait self-test");
    if (host) return fail(AROL_ERR_TIMEOUT, "wait self-test: the bounded wait gave up as designed");
    return AROL_OK;
}

arol_status arol_tiler_cover(const arol_array_desc* array, const arol_tiler* tiler, int rep_rank, const int64_t* rep,
                             int64_t* count_min, int64_t* count_max) {
    AROL_TRACE();
    if (!array || !tiler || !rep || !count_min || !count_max) return fail(AROL_ERR_INVALID, "null argument");
    if (rep_rank < 1 || rep_rank > AROL_MAX_RANK) return fail(AROL_ERR_INVALID, "rep_rank %d not in [1,4]", rep_rank);
    for (int q = 0; q < rep_rank; ++q)
        if (rep[q] < 0 || rep[q] > kMaxDim) return fail(AROL_ERR_INVALID, "rep[%d] out of range", q);
    arol_status st = check_array(*array, "array");
    if (st != AROL_OK) return st;
    if ((st = check_tiler(*tiler, "tiler")) != AROL_OK) return st;
    int64_t nreps = 1;
    for (int q = 0; q < rep_rank; ++q) nreps *= rep[q];
    if (elems_of(*array) == 0) {
        if (nreps > 0) return fail(AROL_ERR_INVALID, "tiler addresses an empty array");
        *count_min = *count_max = 0;
        return AROL_OK;
    }
    return partition_count(*array, *tiler, rep_rank, rep, count_min, count_max);
}

arol_status arol_task_create(const arol_task_desc* desc, arol_task* out) {
    AROL_TRACE();
    if (!desc || !out) return fail(AROL_ERR_INVALID, "null argument");
    *out = nullptr;
    arol_status st = validate_desc(*desc);
    if (st != AROL_OK) return st;
    arol_task t = new (std::nothrow) arol_task_s();
    if (!t) return fail(AROL_ERR_INVALID, "out of host memory");
    t->descs.push_back(*desc);
    t->descs[0].fir_taps_host = nullptr;
    t->tap_off.push_back(0);
    if (desc->elem == AROL_ELEM_FIR) {
        t->taps_host.assign((size_t)desc->fir_m * desc->fir_T, 0.f);
        if (desc->fir_taps_host) std::memcpy(t->taps_host.data(), desc->fir_taps_host, t->taps_host.size() * sizeof(float));
        else t->taps_ready = false;
    }
    int M, N, K;
    if (desc->elem == AROL_ELEM_MATMUL && is_matmul_panels(*desc, &M, &N, &K)) {
        t->kernel = 2;
        t->mm_M = M;
        t->mm_N = N;
        t->mm_K = K;
    }
    if (t->kernel == 0) plan_row_region(t);
    fill_info_single(t);
    if (log_enabled()) {
        const TaskDev td = make_taskdev(t->descs[0], true);
        const char* path = t->kernel == 2 ? (M % 256 == 0 && N % 256 == 0 ? "tcgen05 matmul, CTA pairs" : "tcgen05 matmul")
                           : t->rr_ok ? "row FIR (16-word regions)"
                           : td.rowfir ? "row FIR (staged row tiles)"
                           : td.colfir ? "column FIR (column tiles)"
                           : td.fir2d ? (fir2d_uses_stencil(td) ? "register-blocked stencil" : "2-D window FIR")
                                      : "per-repetition walk";
        log_line("task %p: rank %d, %lld repetitions, %s", (void*)t, desc->in[0].rank, (long long)reps_of(*desc), path);
    }
    *out = t;
    return AROL_OK;
}

arol_status arol_chain_create(const arol_task* tasks, int n, arol_task* out) {
    AROL_TRACE();
    if (!tasks || !out || n < 2) return fail(AROL_ERR_INVALID, "a chain needs at least 2 tasks");
    *out = nullptr;
    for (int i = 0; i < n; ++i) {
        if (!tasks[i]) return fail(AROL_ERR_INVALID, "null task %d", i);
        if (tasks[i]->kind != 0) return fail(AROL_ERR_INVALID, "task %d is itself a chain", i);
        const arol_task_desc& d = tasks[i]->descs[0];
        if (d.elem == AROL_ELEM_MATMUL) return fail(AROL_ERR_UNSUPPORTED, "matmul tasks cannot be chained");
        if (i > 0) {
            const arol_array_desc &a = tasks[i - 1]->descs[0].out[0], &b = d.in[0];
            bool same = a.rank == b.rank && a.dtype == b.dtype;
            for (int k = 0; same && k < a.rank; ++k) same = a.shape[k] == b.shape[k];
            if (!same) return fail(AROL_ERR_INVALID, "output of task %d is not the input array of task %d", i - 1, i);
        }
    }
    arol_task t = new (std::nothrow) arol_task_s();
    if (!t) return fail(AROL_ERR_INVALID, "out of host memory");
    t->kind = 1;
    for (int i = 0; i < n; ++i) {
        t->descs.push_back(tasks[i]->descs[0]);
        t->tap_off.push_back((int64_t)t->taps_host.size());
        t->taps_host.insert(t->taps_host.end(), tasks[i]->taps_host.begin(), tasks[i]->taps_host.end());
        t->taps_ready = t->taps_ready && tasks[i]->taps_ready && !tasks[i]->taps_borrowed;
    }
    // Fused separable downscaler: horizontal 8->3 then vertical 8->3, step 8.
    Pass h, v;
    t->kernel = 3;
    if (n == 2 && match_pass(t->descs[0], 2, &h) && match_pass(t->descs[1], 1, &v) && h.S == 8 && h.T == 8 &&
        h.m == 3 && v.S == 8 && v.T == 8 && v.m == 3 && v.F == h.F && v.H == h.H && v.W == h.W / 8 * 3 &&
        h.W % 8 == 0 && h.H % 8 == 0 && (double)h.F * (h.H / 8) * (h.W / 4) < 2147483647.0) {
        // fused storage combinations: all f32, or 16-bit frames (bfloat16 or
        // IEEE half) with an intermediate and an output each f32 or of the
        // frames' type; others run task by task
        const int di = t->descs[0].in[0].dtype, dm = t->descs[0].out[0].dtype, dy = t->descs[1].out[0].dtype;
        const bool fused = di == AROL_F32 ? dm == AROL_F32 && dy == AROL_F32
                                          : (dm == AROL_F32 || dm == di) && (dy == AROL_F32 || dy == di);
        if (fused) {
            t->kernel = 1;
            t->ds_frames = h.F;
            t->ds_H = (int)h.H;
            t->ds_W = (int)h.W;
            t->ds_in16 = di != AROL_F32;
            t->ds_mid16 = dm != AROL_F32;
            t->ds_out16 = dy != AROL_F32;
            t->ds_half16 = di == AROL_F16;
        }
    }
    // Any other chain of 2 .. 4 row and column passes (f32): the general
    // fused separable chain kernel, when a tile shape fits shared memory.
    // A row pass then a column pass runs on the streaming kernel when its
    // ring fits, unless AROL_SEPSTREAM is off.
    SepChainDev sd;
    t->sd_ok = describe_sepchain(t->descs, &t->sd, true);   // the backward reads any storage
    const char* e = std::getenv("AROL_SEPSTREAM");
    const bool stream = !(e && (!std::strcmp(e, "off") || !std::strcmp(e, "0")));
    if (t->kernel == 3 && describe_sepchain(t->descs, &sd)) {
        if (stream && plan_sepstream(sd, &t->ss, &t->ss_xw, &t->ss_nst, &t->ss_tapw)) t->kernel = 5;
        else if (plan_sepchain(sd, &t->sc)) t->kernel = 4;
    }
    if (t->kernel == 4) {
        const SepChainDev& c = t->sc;
        const int K1 = c.K + 1;
        t->sc_tab.assign((size_t)2 * K1 * (c.tiles_y + c.tiles_x), 0);
        SepRange rows[kSepMaxPasses + 1], cols[kSepMaxPasses + 1];
        for (int ty = 0; ty < c.tiles_y; ++ty) {
            sep_regions(c, ty, 0, rows, cols);
            for (int k = 0; k < K1; ++k) {
                t->sc_tab[(size_t)2 * (ty * K1 + k)] = rows[k].start;
                t->sc_tab[(size_t)2 * (ty * K1 + k) + 1] = rows[k].len;
            }
        }
        const size_t coff = (size_t)2 * K1 * c.tiles_y;
        for (int tx = 0; tx < c.tiles_x; ++tx) {
            sep_regions(c, 0, tx, rows, cols);
            for (int k = 0; k < K1; ++k) {
                t->sc_tab[coff + (size_t)2 * (tx * K1 + k)] = cols[k].start;
                t->sc_tab[coff + (size_t)2 * (tx * K1 + k) + 1] = cols[k].len;
            }
        }
    }
    arol_task_info_t& in = t->info;
    in.kind = 1;
    in.kernel = t->kernel;
    in.path = -1;
    in.reserved_ = 0;
    for (int i = 0; i < n; ++i) {
        const arol_task_info_t& s = tasks[i]->info;
        in.reps += s.reps;
        in.gathered_elems += s.gathered_elems;
        in.scattered_elems += s.scattered_elems;
        in.flops += s.flops;
    }
    const arol_task_desc &first = t->descs.front(), &last = t->descs.back();
    in.unique_bytes = elems_of(first.in[0]) * esize_of(first.in[0].dtype) + elems_of(last.out[0]) * esize_of(last.out[0].dtype);
    t->mids.assign(n - 1, nullptr);
    log_line("chain %p: %d tasks, %s", (void*)t, n,
             t->kernel == 1 ? "fused separable downscaler"
             : t->kernel == 4 ? "fused separable chain (shared-memory tiles)"
             : t->kernel == 5 ? "fused row-then-column chain (streaming rows)"
                              : "stage by stage through a one-member batch");
    if (t->kernel == 5)
        log_line("chain %p: input windows of %d words, %d stages, %zu B of shared memory", (void*)t, t->ss_xw,
                 t->ss_nst, sepstream_smem(t->ss_xw, t->ss_nst, t->ss_tapw));
    if (t->kernel == 4)
        log_line("chain %p: tiles of %d x %d, %lld tiles per frame, %zu B of shared memory", (void*)t, t->sc.BH,
                 t->sc.BW, (long long)t->sc.tiles_y * t->sc.tiles_x, sepchain_smem(t->sc));
    *out = t;
    return AROL_OK;
}

arol_status arol_task_shard_frames(const arol_task_desc* desc, int parts, int part, arol_task_desc* out,
                                   int64_t* first_frame) {
    if (!desc || !out || !first_frame) return fail(AROL_ERR_INVALID, "null argument");
    if (parts < 1 || part < 0 || part >= parts) return fail(AROL_ERR_INVALID, "part %d of %d", part, parts);
    const arol_task_desc& d = *desc;
    if (d.rep_rank < 1 || d.n_in < 1 || d.n_in > 2 || d.n_out != 1) return fail(AROL_ERR_INVALID, "malformed descriptor");
    const int64_t F = d.rep[0];
    // every port: array dimension 0 is repetition dimension 0 (the frames)
    auto frame_port = [&](const arol_array_desc& a, const arol_tiler& t) {
        if (a.rank < 2 || a.shape[0] != F || t.origin[0] != 0) return false;
        for (int q = 0; q < d.rep_rank; ++q)
            if (t.paving[0][q] != (q == 0 ? 1 : 0)) return false;
        for (int k = 1; k < a.rank; ++k)
            if (t.paving[k][0] != 0) return false;
        for (int i = 0; i < t.pattern_rank; ++i)
            if (t.fitting[0][i] != 0) return false;
        return true;
    };
    for (int i = 0; i < d.n_in; ++i)
        if (!frame_port(d.in[i], d.in_tiler[i]))
            return fail(AROL_ERR_UNSUPPORTED, "shard: input %d has no frame dimension (array dim 0 = repetition dim 0)", i);
    if (!frame_port(d.out[0], d.out_tiler[0]))
        return fail(AROL_ERR_UNSUPPORTED, "shard: the output has no frame dimension (array dim 0 = repetition dim 0)");
    const int64_t base = F / parts, extra = F % parts;
    const int64_t count = base + (part < extra ? 1 : 0);
    *first_frame = part * base + std::min<int64_t>(part, extra);
    *out = d;
    out->rep[0] = count;
    for (int i = 0; i < d.n_in; ++i) out->in[i].shape[0] = count;
    out->out[0].shape[0] = count;
    return AROL_OK;
}

arol_status arol_task_set_taps(arol_task t, const float* taps, int on_device) {
    if (!t || !taps) return fail(AROL_ERR_INVALID, "null argument");
    if (t->taps_host.empty()) return fail(AROL_ERR_INVALID, "task has no fir taps");
    if (t->ib) {   // rebuilt with the new taps at the next run
        arol_batch_destroy(t->ib);
        t->ib = nullptr;
    }
    t->ib_checked = false;
    for (arol_task& r : t->rc) {
        arol_task_destroy(r);
        r = nullptr;
    }
    t->rc_checked = false;
    if (on_device) {
        t->taps_borrowed = taps;
    } else {
        std::memcpy(t->taps_host.data(), taps, t->taps_host.size() * sizeof(float));
        t->taps_borrowed = nullptr;
        t->taps_ready = true;
        t->taps_dirty = true;
    }
    return AROL_OK;
}

arol_status arol_task_info(arol_task t, arol_task_info_t* info) {
    if (!t || !info) return fail(AROL_ERR_INVALID, "null argument");
    *info = t->info;
    return AROL_OK;
}

}  // extern "C"

namespace {

uint32_t pow2_at_least(uint32_t v) {
    uint32_t p = 1;
    while (p < v && p < (1u << 30)) p <<= 1;
    return p;
}

// Block tiling of the generic walk over the last two repetition dims of
// extent > 1 (db the last, da the one before): 256 threads, at most 8 rows
// of repetitions along da, the rest along db, each thread R repetitions
// 2^lb apart along db.
bool gen_geom(const TaskDev& t, GenGeom* out) {
    GenGeom g{};
    g.db = 3;
    while (g.db > 0 && t.rep[g.db] <= 1) --g.db;
    g.da = g.db - 1;
    while (g.da >= 0 && t.rep[g.da] <= 1) --g.da;
    const uint32_t RB = (uint32_t)std::max(t.rep[g.db], 1), RA = g.da >= 0 ? (uint32_t)t.rep[g.da] : 1u;
    const uint32_t rows = std::min<uint32_t>(8, pow2_at_least(RA));
    const uint32_t tb = std::min<uint32_t>(pow2_at_least(RB), 256 / rows);
    const uint32_t ta = std::min<uint32_t>(256 / tb, pow2_at_least(RA));
    g.lb = 0;
    while ((1u << g.lb) < tb) ++g.lb;
    g.ta = (int32_t)ta;
    const uint32_t R = (uint32_t)tiler_tiled_reps(t.elem == ELEM_FIR ? t.m : 1);
    g.na = (RA + ta - 1) / ta;
    g.nb = (RB + R * tb - 1) / (R * tb);
    g.idelta = g.odelta = 0;
    for (int k = 0; k < 4; ++k) {
        g.istep[k] = t.in.shape[k] ? (uint32_t)(((uint64_t)tb * t.in.paving[k][g.db]) % (uint32_t)t.in.shape[k]) : 0u;
        g.ostep[k] = t.out.shape[k] ? (uint32_t)(((uint64_t)tb * t.out.paving[k][g.db]) % (uint32_t)t.out.shape[k]) : 0u;
        g.idelta += (int64_t)g.istep[k] * t.in.stride[k];
        g.odelta += (int64_t)g.ostep[k] * t.out.stride[k];
    }
    uint64_t outer = 1;
    for (int q = 0; q < (g.da >= 0 ? g.da : g.db); ++q) outer *= (uint64_t)std::max(t.rep[q], 1);
    const uint64_t nt = outer * g.na * g.nb;
    if (nt >= 0x80000000ull) return false;
    g.ntiles = (uint32_t)nt;
    g.na_div = make_fastdiv(g.na);
    g.nb_div = make_fastdiv(g.nb);
    const int mx = (tiler_tiled_maxm(t.elem == ELEM_FIR ? t.m : 1) + 3) & ~3;   // taps staged in 16-byte rows
    g.tap_floats = t.elem == ELEM_FIR && (int64_t)t.T * mx <= 12288 ? t.T * mx : 0;
    *out = g;
    return true;
}

arol_status run_generic(const arol_task_desc& d, const float* taps, const void* x, void* y, cudaStream_t s,
                        unsigned* err = nullptr) {
    TaskDev td = make_taskdev(d);
    td.taps = taps;
    td.x = x;
    td.y = y;
    td.err = err;
    if (td.fir2d) {
        AROL_CUDA(launch_fir2d(td, s), "2-D FIR kernel launch");
        return AROL_OK;
    }
    GenGeom g;
    if (!td.wide && gen_geom(td, &g)) {
        AROL_CUDA(launch_tiler_tiled(td, g, td.elem == ELEM_FIR ? td.m : 1, s), "tiler kernel launch");
        return AROL_OK;
    }
    AROL_CUDA(launch_tiler_generic(td, td.elem == ELEM_FIR ? td.m : 1, s), "tiler kernel launch");
    return AROL_OK;
}

DownscaleDev ds_params(arol_task t, const float* taps) {
    DownscaleDev p;
    std::memset(&p, 0, sizeof p);
    p.err = t->err_flag;
    p.in16 = t->ds_in16;
    p.mid16 = t->ds_mid16;
    p.out16 = t->ds_out16;
    p.half16 = t->ds_half16;
    p.taps = taps;
    p.frames = t->ds_frames;
    p.H = t->ds_H;
    p.W = t->ds_W;
    return p;
}

size_t array_bytes(const arol_array_desc& a) { return (size_t)elems_of(a) * esize_of(a.dtype); }

// The fused downscaler moves X and dX with 128-bit accesses: both must be
// 16-byte aligned (a null pointer counts as aligned).
bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

}  // namespace

extern "C" {

}  // extern "C"

namespace {

// Row- and column-FIR tasks and unfused chains run on the batch engine, as a
// one-member batch owned by the task (staged row tiles, column tiles, one
// launch per chain stage, in one graph).  *used stays false when the task
// does not qualify (other elementary tasks, taps on the device), and the
// caller takes the per-repetition path.
arol_status run_internal_batch(arol_task t, const void* const* in, void* const* out, cudaStream_t s, bool* used) {
    *used = false;
    if (t->taps_borrowed || !t->taps_ready) return AROL_OK;
    if (!t->ib_checked) {
        t->ib_checked = true;
        bool want = true;
        for (const arol_task_desc& d : t->descs)
            if (d.elem != AROL_ELEM_FIR) want = false;
        if (want && t->kind == 0) {
            const TaskDev td = make_taskdev(t->descs[0], true);
            want = td.rowfir || td.colfir;
        }
        if (want) {
            arol_task self = t;
            if (arol_batch_create(&self, 1, &t->ib) != AROL_OK) t->ib = nullptr;
        }
        log_line("task %p: %s", (void*)t, t->ib ? "runs as a one-member batch" : "runs its per-task kernel");
    }
    if (!t->ib) return AROL_OK;
    *used = true;
    return arol_batch_run(t->ib, in, out, s);
}

}  // namespace

extern "C" {

arol_status arol_task_run(arol_task t, const void* const* in, void* const* out, void* stream) {
    AROL_TRACE();
    if (!t || !in || !out) return fail(AROL_ERR_INVALID, "null argument");
    cudaStream_t s = (cudaStream_t)stream;
    const arol_task_desc& d0 = t->descs[0];
    for (int i = 0; i < d0.n_in; ++i)
        if (!in[i] && elems_of(d0.in[i]) > 0) return fail(AROL_ERR_INVALID, "null input pointer %d", i);
    if (!out[0] && elems_of(t->descs.back().out[0]) > 0) return fail(AROL_ERR_INVALID, "null output pointer");
    if (t->kind == 0 && reps_of(d0) == 0) return AROL_OK;
    arol_status st = remember_device(t);
    if (st != AROL_OK) return st;
    const float* taps = nullptr;
    if ((st = ensure_taps(t, s, &taps)) != AROL_OK) return st;
    if (t->kind == 0) {
        if (reps_of(d0) == 0) return AROL_OK;
        if (t->kernel == 2) {
            if ((st = ensure_err(t, s)) != AROL_OK) return st;
            AROL_CUDA(launch_matmul_tc(in[0], in[1], (float*)out[0], t->mm_M, t->mm_N, t->mm_K, t->err_flag, s),
                      "matmul kernel launch");
            return AROL_OK;
        }
        if (t->rr_ok && aligned16(in[0]) && aligned16(out[0])) {
            if ((st = ensure_err(t, s)) != AROL_OK) return st;
            AROL_CUDA(launch_rowfir_region(t->rr_S, t->rr_T, t->rr_M, t->rr_rows, t->rr_W, t->rr_o, taps,
                                           (const float*)in[0], (float*)out[0], t->err_flag, s),
                      "row-FIR region kernel launch");
            return AROL_OK;
        }
        bool used = false;
        st = run_internal_batch(t, in, out, s, &used);
        if (used) return st;
        if ((st = ensure_err(t, s)) != AROL_OK) return st;
        return run_generic(d0, taps, in[0], out[0], s, t->err_flag);
    }
    if (t->kernel == 1 && aligned16(in[0])) {
        if ((st = ensure_err(t, s)) != AROL_OK) return st;
        DownscaleDev p = ds_params(t, taps);
        p.x = (const float*)in[0];
        p.y = (float*)out[0];
        AROL_CUDA(launch_downscale_fwd(p, s), "downscale kernel launch");
        return AROL_OK;
    }
    if (t->kernel == 5) {
        if ((st = ensure_err(t, s)) != AROL_OK) return st;
        if (!t->ss_units) {
            sepstream_bands(t->ss, t->ss_xw, t->ss_nst, t->ss_tapw, &t->ss_units);
            log_line("chain %p: %d units, bands of %d repetitions", (void*)t, t->ss_units, t->ss.BH);
        }
        SsChain c = t->ss;
        c.x = (const float*)in[0];
        c.y = (float*)out[0];
        c.hh = taps;
        c.hv = taps + (size_t)c.mh * c.Th;
        AROL_CUDA(launch_sepstream(c, nullptr, nullptr, 1, t->ss_units, c.Th, c.Tv, t->ss_xw, t->ss_nst, t->ss_tapw,
                                   t->err_flag, s),
                  "fused chain kernel launch");
        return AROL_OK;
    }
    if (t->kernel == 4) {
        if (!t->sc_tab_dev) {
            if ((st = dev_alloc(t, (void**)&t->sc_tab_dev, t->sc_tab.size() * sizeof(int32_t), "cudaMalloc(chain tiles)")) !=
                AROL_OK)
                return st;
            AROL_CUDA(cudaMemcpyAsync(t->sc_tab_dev, t->sc_tab.data(), t->sc_tab.size() * sizeof(int32_t),
                                      cudaMemcpyHostToDevice, s),
                      "upload chain tiles");
        }
        SepChainDev d = t->sc;
        d.x = (const float*)in[0];
        d.y = (float*)out[0];
        d.taps = taps;
        d.row_tab = t->sc_tab_dev;
        d.col_tab = t->sc_tab_dev + (size_t)2 * (d.K + 1) * d.tiles_y;
        AROL_CUDA(launch_sepchain(d, s), "fused chain kernel launch");
        return AROL_OK;
    }
    bool used = false;
    st = run_internal_batch(t, in, out, s, &used);
    if (used) return st;
    // Unfused chain through intermediates owned by the chain.
    const size_t n = t->descs.size();
    const void* cur = in[0];
    for (size_t i = 0; i < n; ++i) {
        void* dst = out[0];
        if (i + 1 < n) {
            if ((st = dev_alloc(t, &t->mids[i], array_bytes(t->descs[i].out[0]), "cudaMalloc(chain intermediate)")) != AROL_OK)
                return st;
            dst = t->mids[i];
        }
        if (reps_of(t->descs[i]) > 0) {
            const float* tp = taps ? taps + t->tap_off[i] : nullptr;
            if ((st = ensure_err(t, s)) != AROL_OK) return st;
            if ((st = run_generic(t->descs[i], tp, cur, dst, s, t->err_flag)) != AROL_OK) return st;
        }
        cur = dst;
    }
    return AROL_OK;
}

}  // extern "C"

namespace {

// Host buffers through the fused downscaler, pipelined over frame chunks on
// three streams: the copy of chunk c+1 to the device overlaps the kernel on
// chunk c and the copy of chunk c-1 back to the host.  `s` (the caller's
// stream) carries the input copies; the caller's prior work on it is ordered
// before everything, and the call returns after the last output copy.
arol_status run_host_pipelined(arol_task t, const void* hin, void* hout, cudaStream_t s) {
    if (!t->pipe_ready) {
        AROL_CUDA(cudaStreamCreateWithFlags(&t->pipe_stream[0], cudaStreamNonBlocking), "cudaStreamCreate");
        AROL_CUDA(cudaStreamCreateWithFlags(&t->pipe_stream[1], cudaStreamNonBlocking), "cudaStreamCreate");
        for (int c = 0; c < kPipeChunks; ++c) {
            AROL_CUDA(cudaEventCreateWithFlags(&t->pipe_in[c], cudaEventDisableTiming), "cudaEventCreate");
            AROL_CUDA(cudaEventCreateWithFlags(&t->pipe_done[c], cudaEventDisableTiming), "cudaEventCreate");
        }
        AROL_CUDA(cudaEventCreateWithFlags(&t->pipe_last, cudaEventDisableTiming), "cudaEventCreate");
        t->pipe_ready = true;
    }
    const float* taps = nullptr;
    arol_status st = ensure_taps(t, s, &taps);
    if (st != AROL_OK) return st;
    if ((st = ensure_err(t, s)) != AROL_OK) return st;
    const int64_t F = t->ds_frames;
    const int nch = (int)std::min<int64_t>(kPipeChunks, F);
    const int64_t in_frame = (int64_t)t->ds_H * t->ds_W, out_frame = (int64_t)(t->ds_H / 8 * 3) * (t->ds_W / 8 * 3);
    cudaStream_t ks = t->pipe_stream[0], os = t->pipe_stream[1];
    // the compute and output streams start after everything already queued on s
    AROL_CUDA(cudaEventRecord(t->pipe_last, s), "cudaEventRecord");
    AROL_CUDA(cudaStreamWaitEvent(ks, t->pipe_last, 0), "cudaStreamWaitEvent");
    AROL_CUDA(cudaStreamWaitEvent(os, t->pipe_last, 0), "cudaStreamWaitEvent");
    for (int c = 0; c < nch; ++c) {
        const int64_t f0 = F * c / nch, f1 = F * (c + 1) / nch;
        const float* hx = static_cast<const float*>(hin) + f0 * in_frame;
        float* dx = static_cast<float*>(t->stage_in[0]) + f0 * in_frame;
        float* dy = static_cast<float*>(t->stage_out) + f0 * out_frame;
        AROL_CUDA(cudaMemcpyAsync(dx, hx, (size_t)((f1 - f0) * in_frame) * 4, cudaMemcpyHostToDevice, s),
                  "copy input chunk to device");
        AROL_CUDA(cudaEventRecord(t->pipe_in[c], s), "cudaEventRecord");
        AROL_CUDA(cudaStreamWaitEvent(ks, t->pipe_in[c], 0), "cudaStreamWaitEvent");
        DownscaleDev p = ds_params(t, taps);
        p.x = dx;
        p.y = dy;
        p.frames = f1 - f0;
        AROL_CUDA(launch_downscale_fwd(p, ks), "downscale kernel launch");
        AROL_CUDA(cudaEventRecord(t->pipe_done[c], ks), "cudaEventRecord");
        AROL_CUDA(cudaStreamWaitEvent(os, t->pipe_done[c], 0), "cudaStreamWaitEvent");
        AROL_CUDA(cudaMemcpyAsync(static_cast<float*>(hout) + f0 * out_frame, dy, (size_t)((f1 - f0) * out_frame) * 4,
                                  cudaMemcpyDeviceToHost, os),
                  "copy output chunk to host");
    }
    AROL_CUDA(cudaStreamSynchronize(os), "synchronize");
    AROL_CUDA(cudaStreamSynchronize(s), "synchronize");
    return AROL_OK;
}

}  // namespace

extern "C" {

arol_status arol_task_run_host(arol_task t, const void* const* host_in, void* const* host_out, void* stream) {
    AROL_TRACE();
    if (!t || !host_in || !host_out) return fail(AROL_ERR_INVALID, "null argument");
    cudaStream_t s = (cudaStream_t)stream;
    const arol_task_desc& d0 = t->descs[0];
    const arol_array_desc& od = t->descs.back().out[0];
    arol_status st;
    const bool pipelined = t->kind == 1 && t->kernel == 1 && t->ds_frames >= 2 && !t->ds_in16 && !t->ds_out16;
    void* dins[2] = {nullptr, nullptr};
    for (int i = 0; i < d0.n_in; ++i) {
        if (!host_in[i]) return fail(AROL_ERR_INVALID, "null input pointer %d", i);
        if ((st = dev_alloc(t, &t->stage_in[i], array_bytes(d0.in[i]), "cudaMalloc(staging)")) != AROL_OK) return st;
        if (!pipelined)
            AROL_CUDA(cudaMemcpyAsync(t->stage_in[i], host_in[i], array_bytes(d0.in[i]), cudaMemcpyHostToDevice, s),
                      "copy input to device");
        dins[i] = t->stage_in[i];
    }
    if (!host_out[0]) return fail(AROL_ERR_INVALID, "null output pointer");
    if ((st = dev_alloc(t, &t->stage_out, array_bytes(od), "cudaMalloc(staging)")) != AROL_OK) return st;
    void* douts[1] = {t->stage_out};
    if (pipelined) return run_host_pipelined(t, host_in[0], host_out[0], s);
    if ((st = arol_task_run(t, dins, douts, stream)) != AROL_OK) return st;
    AROL_CUDA(cudaMemcpyAsync(host_out[0], t->stage_out, array_bytes(od), cudaMemcpyDeviceToHost, s),
              "copy output to host");
    AROL_CUDA(cudaStreamSynchronize(s), "synchronize");
    return AROL_OK;
}

}  // extern "C"

namespace {

// Per-CTA tap-gradient partials (n floats) followed by one word, the ticket
// of the last-CTA reduction; zeroed once here, left at zero by every launch.
arol_status ensure_partials(arol_task t, int64_t n, cudaStream_t s) {
    if (t->partials && t->partials_cap >= n) return AROL_OK;
    if (t->partials) AROL_CUDA(cudaStreamSynchronize(s), "synchronize");   // earlier launches may still use it
    free_dev(t->partials);
    t->partials = nullptr;
    arol_status st = dev_alloc(t, (void**)&t->partials, (size_t)(n + 4) * sizeof(float), "cudaMalloc(tap-gradient partials)");
    if (st != AROL_OK) return st;
    AROL_CUDA(cudaMemsetAsync(t->partials, 0, (size_t)(n + 4) * sizeof(float), s), "clear tap-gradient partials");
    t->partials_cap = n;
    return AROL_OK;
}

unsigned* partials_ticket(arol_task t) { return reinterpret_cast<unsigned*>(t->partials + t->partials_cap); }

// Owner-computes inverse of an input tiler: for every input element e, the
// list of flat (r * T + k) indices whose gather visits e, in increasing order.
arol_status ensure_inverse(arol_task t, size_t i) {
    if (t->inv_start.size() <= i) {
        t->inv_start.resize(t->descs.size(), nullptr);
        t->inv_list.resize(t->descs.size(), nullptr);
    }
    if (t->inv_start[i]) return AROL_OK;
    const arol_task_desc& d = t->descs[i];
    const TaskDev td = make_taskdev(d);
    const int64_t n = elems_of(d.in[0]);
    const int64_t total = td.nreps * td.T;
    if (total >= 2147483647LL) return fail(AROL_ERR_UNSUPPORTED, "backward: more than 2^31 gathered elements");
    std::vector<int64_t> offs((size_t)total);
    // host walk of the input tiler (same definition as the device walk)
    {
        const PortDev& p = td.in;
        uint32_t r[4] = {0, 0, 0, 0};
        for (int64_t lr = 0; lr < td.nreps; ++lr) {
            int64_t l = lr;
            for (int q = 3; q >= 0; --q) { r[q] = (uint32_t)(l % td.rep[q]); l /= td.rep[q]; }
            int64_t row[4], cur[4];
            for (int k = 0; k < 4; ++k) {
                __int128 v = p.origin[k];
                for (int q = 0; q < 4; ++q) v += (__int128)p.paving[k][q] * r[q];
                row[k] = (int64_t)(v % p.shape[k]);
            }
            int64_t kk = 0;
            for (int i0 = 0; i0 < p.pattern[0]; ++i0) {
                for (int k = 0; k < 4; ++k) cur[k] = row[k];
                for (int i1 = 0; i1 < p.pattern[1]; ++i1) {
                    offs[(size_t)(lr * td.T + kk++)] = cur[0] * p.stride[0] + cur[1] * p.stride[1] + cur[2] * p.stride[2] + cur[3] * p.stride[3];
                    for (int k = 0; k < 4; ++k) { cur[k] += p.fitting[k][1]; if (cur[k] >= p.shape[k]) cur[k] -= p.shape[k]; }
                }
                for (int k = 0; k < 4; ++k) { row[k] += p.fitting[k][0]; if (row[k] >= p.shape[k]) row[k] -= p.shape[k]; }
            }
        }
    }
    std::vector<int64_t> start((size_t)n + 1, 0);
    for (int64_t o : offs) ++start[(size_t)o + 1];
    for (int64_t e = 0; e < n; ++e) start[(size_t)e + 1] += start[(size_t)e];
    std::vector<int32_t> list((size_t)std::max<int64_t>(total, 1));
    std::vector<int64_t> fillp(start.begin(), start.end() - 1);
    for (int64_t idx = 0; idx < total; ++idx) list[(size_t)fillp[(size_t)offs[(size_t)idx]]++] = (int32_t)idx;
    arol_status st;
    if ((st = dev_alloc(t, (void**)&t->inv_start[i], start.size() * sizeof(int64_t), "cudaMalloc(inverse map)")) != AROL_OK) return st;
    if ((st = dev_alloc(t, (void**)&t->inv_list[i], list.size() * sizeof(int32_t), "cudaMalloc(inverse map)")) != AROL_OK) return st;
    AROL_CUDA(cudaMemcpy(t->inv_start[i], start.data(), start.size() * sizeof(int64_t), cudaMemcpyHostToDevice), "upload inverse map");
    AROL_CUDA(cudaMemcpy(t->inv_list[i], list.data(), list.size() * sizeof(int32_t), cudaMemcpyHostToDevice), "upload inverse map");
    return AROL_OK;
}

arol_status backward_generic_task(arol_task t, size_t i, const float* taps, const void* x, const float* gy, float* gx,
                                  float* gtaps, cudaStream_t s) {
    const arol_task_desc& d = t->descs[i];
    if (d.elem == AROL_ELEM_COPY && d.in[0].dtype != AROL_F32)
        return fail(AROL_ERR_UNSUPPORTED, "backward: copy tasks on float32 only");
    arol_status st;
    if (gx && (st = ensure_inverse(t, i)) != AROL_OK) return st;
    TaskDev td = make_taskdev(d);
    td.taps = taps;
    td.x = x;
    int64_t chunk = 0;
    const int nb = tiler_bwd_blocks(td.nreps, td.m, td.T, &chunk);
    if (gtaps && d.elem == AROL_ELEM_FIR && (st = ensure_partials(t, (int64_t)nb * td.m * td.T, s)) != AROL_OK) return st;
    AROL_CUDA(launch_tiler_bwd(td, gx ? t->inv_start[i] : nullptr, gx ? t->inv_list[i] : nullptr, gx, gy,
                               d.elem == AROL_ELEM_FIR ? gtaps : nullptr, t->partials, nb, chunk, s),
              "tiler backward launch");
    return AROL_OK;
}

// Backward of one separable pass (task ii of t): the one-sweep kernel when
// the repetitions tile the axis and the data fit its forms, else the adjoint
// gather and the tap-gradient walk (no inverse map); tap gradients of larger
// banks by the owner-computes walk.  gx and gt may be null.
arol_status sep_pass_backward(arol_task t, size_t ii, const SepPassDev& p, int64_t F, const int64_t ihw[2],
                              const int64_t ohw[2], const float* tp, const void* x, const float* g, float* gx, float* gt,
                              cudaStream_t s) {
    const int x_dt = t->descs[ii].in[0].dtype;
    const int Hin = (int)ihw[0], Win = (int)ihw[1], Hout = (int)ohw[0], Wout = (int)ohw[1];
    arol_status st = AROL_OK;
    if (!gx && !gt) return AROL_OK;
    SepBwdPlan plan;
    if (sep_bwd_plan(p, F, Hin, Win, x_dt, x, g, gx, gt != nullptr, &plan)) {
        if (gt && (st = ensure_partials(t, (int64_t)plan.blocks * p.m * p.T, s)) != AROL_OK) return st;
        AROL_CUDA(launch_sep_bwd(plan, p, F, Hin, Win, tp, x, x_dt, g, gx, t->partials, gt, s), "backward launch");
        return AROL_OK;
    }
    if (gx) AROL_CUDA(launch_sep_adjoint(p, F, Hin, Win, Hout, Wout, tp, g, gx, s), "backward launch");
    if (gt && sep_dh_supported(p)) {
        if ((st = ensure_partials(t, (int64_t)sep_dh_blocks() * p.m * p.T, s)) != AROL_OK) return st;
        AROL_CUDA(launch_sep_dh(p, F, Hin, Win, Hout, Wout, x, x_dt, g, t->partials, gt, s), "backward launch");
    } else if (gt) {
        return backward_generic_task(t, ii, tp, x, g, nullptr, gt, s);
    }
    return AROL_OK;
}

// The chain backward's recompute tasks: one single-pass task per
// intermediate whose pass is a row or column FIR with host taps (it runs as a
// one-member batch: staged row tiles or column tiles); the others stay null.
void build_recompute_tasks(arol_task t) {
    t->rc_checked = true;
    t->rc.assign(t->descs.size(), nullptr);
    if (t->taps_borrowed || !t->taps_ready) return;
    for (size_t i = 0; i + 1 < t->descs.size(); ++i) {
        const arol_task_desc& d = t->descs[i];
        if (d.elem != AROL_ELEM_FIR || d.n_in != 1) continue;
        const TaskDev td = make_taskdev(d, true);
        if (!td.rowfir && !td.colfir) continue;
        arol_task_desc di = d;
        di.fir_taps_host = t->taps_host.data() + t->tap_off[i];
        arol_task sub = nullptr;
        if (arol_task_create(&di, &sub) == AROL_OK) t->rc[i] = sub;
    }
}

}  // namespace

extern "C" {

arol_status arol_task_backward(arol_task t, const void* grad_out, const void* const* saved_in, void* grad_in,
                               float* grad_taps, void* stream) {
    AROL_TRACE();
    if (!t || !grad_out || !saved_in || !saved_in[0]) return fail(AROL_ERR_INVALID, "null argument");
    cudaStream_t s = (cudaStream_t)stream;
    for (size_t i = 0; i < t->descs.size(); ++i) {
        const arol_task_desc& d = t->descs[i];
        if (d.elem == AROL_ELEM_MATMUL) return fail(AROL_ERR_UNSUPPORTED, "backward of matmul tasks is not implemented");
        if (d.elem == AROL_ELEM_COPY && (d.in[0].dtype != AROL_F32 || d.out[0].dtype != AROL_F32))
            return fail(AROL_ERR_UNSUPPORTED, "backward: copy tasks on float32 only");
        if (i + 1 < t->descs.size() && d.out[0].dtype != AROL_F32)
            return fail(AROL_ERR_UNSUPPORTED, "backward: chain intermediates must be float32");
    }
    arol_status st = remember_device(t);
    if (st != AROL_OK) return st;
    const float* taps = nullptr;
    if ((st = ensure_taps(t, s, &taps)) != AROL_OK) return st;
    if (t->kind == 1 && t->kernel == 1 && !t->ds_in16 && !t->ds_mid16 && !t->ds_out16 && aligned16(saved_in[0]) &&
        aligned16(grad_in) && aligned16(grad_out)) {
        const int nparts = downscale_bwd_partials(device_sm_count(), t->ds_W);
        if ((st = ensure_partials(t, (int64_t)nparts * 48, s)) != AROL_OK) return st;
        if ((st = ensure_err(t, s)) != AROL_OK) return st;
        DownscaleDev p = ds_params(t, taps);
        p.x = (const float*)saved_in[0];
        p.gy = (const float*)grad_out;
        p.gx = (float*)grad_in;
        p.partials = t->partials;
        p.ticket = partials_ticket(t);
        AROL_CUDA(launch_downscale_bwd(p, grad_taps, nparts, false, s), "downscale backward launch");
        return AROL_OK;
    }
    if (t->kind == 0) {
        // a row or column FIR pass: the separable adjoint and tap-gradient
        // kernels (no inverse map); any other tiler: owner computes
        SepPassDev pass;
        int64_t F = 0, ihw[2], ohw[2];
        if (match_sep_pass(t->descs[0], &pass, &F, ihw, ohw, true)) {
            pass.tap_off = 0;
            return sep_pass_backward(t, 0, pass, F, ihw, ohw, taps, saved_in[0], (const float*)grad_out,
                                     (float*)grad_in, grad_taps, s);
        }
        return backward_generic_task(t, 0, taps, saved_in[0], (const float*)grad_out, (float*)grad_in, grad_taps, s);
    }
    // Unfused chain: recompute the intermediates, then reverse task by task.
    // Separable passes read a pass's input only for its tap gradients, so
    // without tap gradients nothing is recomputed.
    const size_t n = t->descs.size();
    if (!t->rc_checked) build_recompute_tasks(t);
    if (t->grad_mids.size() < n) t->grad_mids.resize(n, nullptr);
    const bool need_mids = !(t->sd_ok && !grad_taps);
    const void* cur = saved_in[0];
    for (size_t i = 0; need_mids && i + 1 < n; ++i) {
        if ((st = dev_alloc(t, &t->mids[i], array_bytes(t->descs[i].out[0]), "cudaMalloc(chain intermediate)")) != AROL_OK)
            return st;
        if (reps_of(t->descs[i]) > 0) {
            if (t->rc[i]) {
                const void* rin[1] = {cur};
                void* rout[1] = {t->mids[i]};
                if ((st = arol_task_run(t->rc[i], rin, rout, stream)) != AROL_OK) return st;
            } else if ((st = run_generic(t->descs[i], taps ? taps + t->tap_off[i] : nullptr, cur, t->mids[i], s)) !=
                       AROL_OK) {
                return st;
            }
        }
        cur = t->mids[i];
    }
    const float* g = (const float*)grad_out;
    for (size_t ii = n; ii-- > 0;) {
        const void* xin = ii == 0 ? saved_in[0] : need_mids ? t->mids[ii - 1] : nullptr;
        float* gx = nullptr;
        if (ii == 0) gx = (float*)grad_in;
        else {
            if ((st = dev_alloc(t, (void**)&t->grad_mids[ii], array_bytes(t->descs[ii].in[0]), "cudaMalloc(chain gradient)")) != AROL_OK)
                return st;
            gx = t->grad_mids[ii];
        }
        const float* tp = taps ? taps + t->tap_off[ii] : nullptr;
        float* gt = grad_taps ? grad_taps + t->tap_off[ii] : nullptr;
        if (reps_of(t->descs[ii]) == 0) {
            if (gx) AROL_CUDA(cudaMemsetAsync(gx, 0, (size_t)elems_of(t->descs[ii].in[0]) * sizeof(float), s), "zero gradient");
            if (gt) AROL_CUDA(cudaMemsetAsync(gt, 0, sizeof(float) * t->descs[ii].fir_m * t->descs[ii].fir_T, s), "zero gradient");
        } else if (t->sd_ok) {
            // separable passes: dX by the pass's transposed tiler as a
            // gather (no inverse map), the tap gradients as for any task
            const SepChainDev& c = t->sd;
            const int64_t ihw[2] = {c.H[ii], c.W[ii]}, ohw[2] = {c.H[ii + 1], c.W[ii + 1]};
            if ((st = sep_pass_backward(t, ii, c.p[ii], c.F, ihw, ohw, tp, xin, g, gx, gt, s)) != AROL_OK) return st;
        } else if ((st = backward_generic_task(t, ii, tp, xin, g, gx, gt, s)) != AROL_OK) {
            return st;
        }
        g = gx;
    }
    return AROL_OK;
}

arol_status arol_task_fwd_bwd(arol_task t, const void* const* in, const void* grad_out, void* out, void* grad_in,
                              float* grad_taps, void* stream) {
    AROL_TRACE();
    if (!t || !in || !in[0] || !grad_out || !out) return fail(AROL_ERR_INVALID, "null argument");
    cudaStream_t s = (cudaStream_t)stream;
    if (!(t->kind == 1 && t->kernel == 1) || t->ds_in16 || t->ds_mid16 || t->ds_out16 || !aligned16(in[0]) ||
        !aligned16(grad_in) || !aligned16(grad_out)) {
        // every other task: the forward, then the backward (same results)
        void* outs[1] = {out};
        arol_status st = arol_task_run(t, in, outs, stream);
        if (st != AROL_OK) return st;
        return arol_task_backward(t, grad_out, in, grad_in, grad_taps, stream);
    }
    const float* taps = nullptr;
    arol_status st = remember_device(t);
    if (st != AROL_OK) return st;
    if ((st = ensure_taps(t, s, &taps)) != AROL_OK) return st;
    const int nparts = downscale_bwd_partials(device_sm_count(), t->ds_W);
    if ((st = ensure_partials(t, (int64_t)nparts * 48, s)) != AROL_OK) return st;
    if ((st = ensure_err(t, s)) != AROL_OK) return st;
    DownscaleDev p = ds_params(t, taps);
    p.x = (const float*)in[0];
    p.y = (float*)out;
    p.gy = (const float*)grad_out;
    p.gx = (float*)grad_in;
    p.partials = t->partials;
    p.ticket = partials_ticket(t);
    AROL_CUDA(launch_downscale_bwd(p, grad_taps, nparts, true, s), "downscale fwd_bwd launch");
    return AROL_OK;
}

arol_status arol_task_sync_status(arol_task t, void* stream) {
    if (!t) return fail(AROL_ERR_INVALID, "null task");
    AROL_CUDA(cudaStreamSynchronize((cudaStream_t)stream), "synchronize");
    if (t->ib) {
        const arol_status bs = arol_batch_sync_status(t->ib, stream);
        if (bs != AROL_OK) return bs;
    }
    for (arol_task r : t->rc)
        if (r) {
            const arol_status rs = arol_task_sync_status(r, stream);
            if (rs != AROL_OK) return rs;
        }
    if (t->err_flag) {
        unsigned flag = 0;
        AROL_CUDA(cudaMemcpy(&flag, t->err_flag, sizeof flag, cudaMemcpyDeviceToHost), "read error flag");
        if (flag) {
            cudaMemset(t->err_flag, 0, sizeof(unsigned));
            if (flag & 0x300u)
                return fail(AROL_ERR_OOB, "a device-side index was out of range (%s; flags 0x%x)",
                            (flag & 0x100u) ? "input" : "output", flag);
            return fail(AROL_ERR_TIMEOUT, "a bounded device-side wait gave up (flags 0x%x)", flag);
        }
    }
    return AROL_OK;
}

void arol_task_destroy(arol_task t) {
    if (!t) return;
    if (t->ib) arol_batch_destroy(t->ib);
    for (arol_task r : t->rc) arol_task_destroy(r);
    if (t->device >= 0) {
        int cur = 0;
        cudaGetDevice(&cur);
        if (cur != t->device) cudaSetDevice(t->device);
        free_dev(t->taps_dev);
        free_dev(t->sc_tab_dev);
        for (void* p : t->mids) free_dev(p);
        free_dev(t->err_flag);
        free_dev(t->partials);
        for (auto* p : t->inv_start) free_dev(p);
        for (auto* p : t->inv_list) free_dev(p);
        for (auto* p : t->grad_mids) free_dev(p);
        free_dev(t->stage_in[0]);
        free_dev(t->stage_in[1]);
        free_dev(t->stage_out);
        if (t->pipe_ready) {
            cudaStreamDestroy(t->pipe_stream[0]);
            cudaStreamDestroy(t->pipe_stream[1]);
            for (int c = 0; c < 8; ++c) {
                cudaEventDestroy(t->pipe_in[c]);
                cudaEventDestroy(t->pipe_done[c]);
            }
            cudaEventDestroy(t->pipe_last);
        }
        if (cur != t->device) cudaSetDevice(cur);
    }
    delete t;
}

}  // extern "C"

// ==================================================================== batches

struct arol_batch_s {
    // Internal tasks, member-major: member i (a task or a chain of len_of[i]
    // tasks) owns internal tasks first_of[i] .. first_of[i] + len_of[i] - 1.
    std::vector<arol_task_desc> descs;
    std::vector<std::vector<float>> taps;
    std::vector<TaskDev> host_tasks;
    std::vector<int> member_of, stage_of;
    std::vector<int> first_of, len_of;
    int nstages = 1;
    std::vector<int> stage_off, stage_cnt;   // tile range of each stage in dev_tiles
    std::vector<size_t> mid_off;             // arena offset of a non-final task's output
    unsigned char* arena = nullptr;          // chain intermediates, owned
    std::vector<const void*> last_in;        // per member
    std::vector<void*> last_out;
    int device = -1;
    int max_m = 1;
    // device state
    TaskDev* dev_tasks = nullptr;
    TaskDev* pinned_tasks = nullptr;
    cudaEvent_t table_copied = nullptr;
    cudaEvent_t launched = nullptr;   // after the latest launch: a new table waits for it, on any stream
    TileDev* dev_tiles = nullptr;
    int64_t tiles_cap = 0;
    int ntiles = 0;
    TileDev* dev_tiles_pt = nullptr;      // the same tiles grouped by task, for one launch per task
    std::vector<int> pt_off, pt_cnt;
    // row-FIR tiles (k_rowfir.cu): by stage, and the same grouped by task
    std::vector<RowTileDev> rtiles, rtiles_pt;
    std::vector<int> rstage_off, rstage_cnt, rpt_off, rpt_cnt;
    RowTileDev* dev_rtiles = nullptr;
    RowTileDev* dev_rtiles_pt = nullptr;
    RowTileDev* pinned_rtiles = nullptr;  // both lists back to back, for the upload
    int64_t rtiles_cap = 0;
    int row_budget = kRowSlotFloats;      // slot floats a row tile may fill (autotuned)
    int row_ctas = 0;                     // row-FIR CTAs per SM (0: as many as fit; autotuned)
    unsigned* err = nullptr;              // bounded device waits that gave up (bits)
    unsigned* counter = nullptr;
    float* taps_dev = nullptr;
    bool tables_built = false;
    // launch configuration
    int64_t tile_reps = 2048;
    int threads = kBatchThreads;
    int ctas_per_sm = 4;
    // members that are a row pass then a column pass run on the streaming
    // chain kernel, all in one launch: their plans (pointers set per run),
    // the unit prefix over them, and the common launch shape
    std::vector<char> streamed;           // per internal task: its member is streamed
    std::vector<int> ss_members;
    std::vector<SsChain> ss_chains;
    std::vector<int> ss_ustart;
    int ss_xw = 0, ss_nst = 2, ss_tapw = 0, ss_th = 0, ss_tv = 0, ss_units = 0;
    SsChain* dev_ss = nullptr;
    SsChain* pinned_ss = nullptr;
    int* dev_ss_ustart = nullptr;
    // chain members the fused 8 -> 3 kernel would run alone (f32): one
    // launch of its batched form over those whose input is 16-byte aligned
    // (checked every run; a change of the set rebuilds tiles and graph)
    std::vector<char> ds_ok;              // per member: eligible
    std::vector<char> ds_on;              // per member: on the batched kernel in the current tables
    std::vector<int> ds_members;
    std::vector<DsMember> ds_geom;        // per member: frames, H, W and chunks (eligible members)
    std::vector<DsMember> ds_mem;
    float* ds_taps = nullptr;             // per eligible member: its 48 taps back to back
    std::vector<int> ds_ustart;
    int ds_units = 0, ds_ws = 0;
    DsMember* dev_ds = nullptr;
    DsMember* pinned_ds = nullptr;
    int* dev_ds_ustart = nullptr;
    std::vector<char> skip;               // per internal task: no tiles (its member runs on a chain kernel)
    // graph
    cudaStream_t cap_stream = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
};

namespace {

std::mutex g_tune_mu;
std::map<std::string, std::vector<int64_t>> g_tune_cache;   // signature -> {tile, threads, ctas}
bool g_tune_loaded = false;

uint64_t fnv1a(const void* data, size_t n, uint64_t h) {
    const unsigned char* p = (const unsigned char*)data;
    for (size_t i = 0; i < n; ++i) { h ^= p[i]; h *= 1099511628211ULL; }
    return h;
}

std::string batch_signature(arol_batch b) {
    uint64_t h = 1469598103934665603ULL;
    for (size_t j = 0; j < b->host_tasks.size(); ++j) {
        TaskDev c = b->host_tasks[j];
        c.x = nullptr; c.y = nullptr; c.taps = nullptr; c.taps_t = nullptr;
        h = fnv1a(&c, sizeof c, h);
        h = fnv1a(&b->stage_of[j], sizeof(int), h);
    }
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, dev) == cudaSuccess) {
        h = fnv1a(prop.name, std::strlen(prop.name), h);
        h = fnv1a(&prop.multiProcessorCount, sizeof prop.multiProcessorCount, h);
    }
    char buf[32];
    std::snprintf(buf, sizeof buf, "%016" PRIx64, h);
    return buf;
}

// The cache file is a flat JSON object:
// {"<signature>": [tile, threads, ctas, row_budget, row_ctas], ...}
void tune_cache_load() {
    if (g_tune_loaded) return;
    g_tune_loaded = true;
    const char* path = std::getenv("AROL_TUNE_CACHE");
    if (!path) return;
    std::ifstream f(path);
    if (!f) return;
    std::stringstream ss;
    ss << f.rdbuf();
    std::string s = ss.str();
    size_t pos = 0;
    while ((pos = s.find('"', pos)) != std::string::npos) {
        size_t end = s.find('"', pos + 1);
        if (end == std::string::npos) break;
        std::string key = s.substr(pos + 1, end - pos - 1);
        long long v[5] = {0, 0, 0, 0, 0};
        size_t lb = s.find('[', end);
        if (lb == std::string::npos) break;
        if (std::sscanf(s.c_str() + lb, "[%lld , %lld , %lld , %lld , %lld]", &v[0], &v[1], &v[2], &v[3], &v[4]) == 5)
            g_tune_cache[key] = {v[0], v[1], v[2], v[3], v[4]};
        pos = s.find(']', lb);
        if (pos == std::string::npos) break;
    }
}

void tune_cache_save() {
    const char* path = std::getenv("AROL_TUNE_CACHE");
    if (!path) return;
    std::string tmp = std::string(path) + ".tmp";
    std::ofstream f(tmp);
    if (!f) return;
    f << "{";
    bool first = true;
    for (auto& kv : g_tune_cache) {
        f << (first ? "\n" : ",\n") << "  \"" << kv.first << "\": [";
        for (size_t q = 0; q < kv.second.size(); ++q) f << (q ? ", " : "") << kv.second[q];
        f << "]";
        first = false;
    }
    f << "\n}\n";
    f.close();
    std::rename(tmp.c_str(), path);
}

void invalidate_graph(arol_batch b) {
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    b->exec = nullptr;
    b->graph = nullptr;
}

// Shared-memory bank conflict degree of one warp of the row-FIR kernel that
// covers a rows x 32/a consecutive repetitions: lane (k, j) reads word
// 4 ((k >> 2) & 7) + (k W mod 4) + S j (mod 32) of its tile at every tap
// (row slot placement and 16-byte-preserving bulk copies; the tile's first
// row and column shift every lane alike).
int rowfir_conflicts(int a, int64_t W, int S) {
    int count[32] = {0}, worst = 0;
    for (int k = 0; k < a; ++k)
        for (int j = 0; j < 32 / a; ++j) {
            const int bank = (int)((4 * ((k >> 2) & 7) + (int)((k * W) & 3) + S * j) & 31);
            worst = std::max(worst, ++count[bank]);
        }
    return worst;
}

// Row tiles of a row-FIR task: rows per warp unit (a), repetitions per row
// piece (cnt) and rows per tile (<= 32), within `budget` slot floats per
// tile, chosen by a cost model in warp instructions: a fixed cost per tile
// (record, waits, set-up), a cost per unit (addresses, stores) and per unit
// and tap the shared-memory wavefronts of the window load (its bank
// conflict degree) plus m FMAs, lanes past a tile's edge included.
void build_row_tiles(const TaskDev& t, int task, int budget, std::vector<RowTileDev>& out) {
    const int S = t.step, T = t.T, M = t.m;
    const int64_t W = t.in.shape[1], H = t.in.shape[0], Wo = t.out.shape[1], Ho = t.out.shape[0];
    const int64_t R0 = t.rep[2], R1 = t.rep[3];
    if (R0 <= 0 || R1 <= 0) return;
    auto ss_of = [&](int64_t cnt) { return (int)((S * (cnt - 1) + T + 6 + 31) & ~int64_t(31)); };
    budget = std::min(budget, kRowSlotFloats - 32 * (T - 1));   // the taps sit at the stage's end
    constexpr double kTile = 400, kUnit = 40;
    double best = 1e300;
    int ba = 1;
    int64_t bcnt = 1, brows = 1;
    for (int a = 1; a <= 32; a *= 2) {
        if (a > 1 && a > R0) break;
        const int b = 32 / a;
        const int64_t cmax = ((budget / a) - T - 37) / S + 1;   // ss_of(cmax) * a <= budget
        if (cmax < 1) break;
        int64_t cnt = std::min<int64_t>(R1, cmax);
        const int64_t pieces = (R1 + cnt - 1) / cnt;
        cnt = (R1 + pieces - 1) / pieces;
        int64_t rows = std::min<int64_t>({32, R0, (int64_t)(budget / ss_of(cnt))});
        rows = rows / a * a;
        if (rows < a) continue;
        const double tiles = (double)((R0 + rows - 1) / rows) * (double)pieces;
        const double units = tiles * (double)(rows / a) * (double)((cnt + b - 1) / b);
        const double cost = tiles * kTile + units * (kUnit + T * (double)(rowfir_conflicts(a, W, S) + M));
        if (cost < best) {
            best = cost;
            ba = a;
            bcnt = cnt;
            brows = rows;
        }
    }
    for (int64_t r0 = 0; r0 < R0; r0 += brows)
        for (int64_t a0 = 0; a0 < R1; a0 += bcnt) {
            RowTileDev rt;
            std::memset(&rt, 0, sizeof rt);
            const int64_t cnt = std::min<int64_t>(bcnt, R1 - a0);
            rt.W = (int32_t)W;
            rt.H = (int32_t)H;
            rt.Wout = (int32_t)Wo;
            rt.Hout = (int32_t)Ho;
            rt.row0 = (int32_t)(((int64_t)t.in.origin[0] + r0) % H);
            rt.orow0 = (int32_t)(((int64_t)t.out.origin[0] + r0) % Ho);
            rt.nrows = (int32_t)std::min<int64_t>(brows, R0 - r0);
            rt.c0 = (int32_t)(((int64_t)t.in.origin[1] + (int64_t)S * a0) % W);
            rt.oc0 = (int32_t)(((int64_t)t.out.origin[1] + (int64_t)M * a0) % Wo);
            rt.cnt = (int32_t)cnt;
            rt.S = S;
            rt.T = T;
            rt.M = M;
            rt.lw = (int32_t)(S * (cnt - 1) + T);
            rt.ss = ss_of(cnt);
            rt.a = ba;
            rt.out_wrap = rt.oc0 + M * cnt > Wo ? 1 : 0;
            rt.task = task;
            out.push_back(rt);
        }
}

// Row tiles carry their task's current buffers and transposed taps.
void fill_row_tile_ptrs(arol_batch b) {
    for (std::vector<RowTileDev>* v : {&b->rtiles, &b->rtiles_pt})
        for (RowTileDev& rt : *v) {
            const TaskDev& t = b->host_tasks[rt.task];
            rt.x = static_cast<const float*>(t.x);
            rt.y = static_cast<float*>(t.y);
            rt.taps_t = t.taps_t;
        }
}

// Tiles of at most tile_reps repetitions, grouped by chain stage (stage k of
// every chain runs in the k-th launch, after stage k-1 has finished), most
// expensive tasks first within a stage (a longest-processing-time order for
// the static round-robin schedule).
arol_status build_tiles(arol_batch b) {
    auto cost = [&](int i) {
        const TaskDev& t = b->host_tasks[i];
        return (double)t.nreps * (t.T + t.m);
    };
    std::vector<TileDev> tiles;
    std::vector<RowTileDev> rtiles;
    b->stage_off.assign(b->nstages, 0);
    b->stage_cnt.assign(b->nstages, 0);
    b->rstage_off.assign(b->nstages, 0);
    b->rstage_cnt.assign(b->nstages, 0);
    for (int stage = 0; stage < b->nstages; ++stage) {
        b->stage_off[stage] = (int)std::min<size_t>(tiles.size(), 2147483647);
        std::vector<int> order;
        for (size_t i = 0; i < b->host_tasks.size(); ++i)
            if (b->stage_of[i] == stage) order.push_back((int)i);
        std::stable_sort(order.begin(), order.end(), [&](int a, int c) { return cost(a) > cost(c); });
        b->rstage_off[stage] = (int)std::min<size_t>(rtiles.size(), 2147483647);
        for (int i : order) {
            if (b->skip[i]) continue;
            const TaskDev& t = b->host_tasks[i];
            if (t.rowfir) {
                build_row_tiles(t, i, b->row_budget, rtiles);
                continue;
            }
            for (int64_t s = 0; s < t.nreps; s += b->tile_reps) {
                TileDev td;
                td.task = i;
                td.start = s;
                td.count = (int32_t)std::min<int64_t>(b->tile_reps, t.nreps - s);
                tiles.push_back(td);
            }
        }
        b->stage_cnt[stage] = (int)std::min<size_t>(tiles.size() - b->stage_off[stage], 2147483647);
        b->rstage_cnt[stage] = (int)std::min<size_t>(rtiles.size() - b->rstage_off[stage], 2147483647);
    }
    if ((int64_t)tiles.size() >= 2147483647LL || (int64_t)rtiles.size() >= 2147483647LL)
        return fail(AROL_ERR_UNSUPPORTED, "batch: too many tiles");
    // row tiles: the same list grouped by task, for one launch per task
    b->rtiles = rtiles;
    b->rtiles_pt = rtiles;
    std::stable_sort(b->rtiles_pt.begin(), b->rtiles_pt.end(),
                     [](const RowTileDev& x, const RowTileDev& y) { return x.task < y.task; });
    b->rpt_off.assign(b->host_tasks.size(), 0);
    b->rpt_cnt.assign(b->host_tasks.size(), 0);
    for (size_t k = 0; k < b->rtiles_pt.size(); ++k)
        if (b->rpt_cnt[b->rtiles_pt[k].task]++ == 0) b->rpt_off[b->rtiles_pt[k].task] = (int)k;
    if ((int64_t)rtiles.size() > b->rtiles_cap) {
        free_dev(b->dev_rtiles);
        free_dev(b->dev_rtiles_pt);
        if (b->pinned_rtiles) cudaFreeHost(b->pinned_rtiles);
        b->dev_rtiles = b->dev_rtiles_pt = b->pinned_rtiles = nullptr;
        b->rtiles_cap = 0;
        const size_t bytes = std::max<size_t>(rtiles.size(), 1) * sizeof(RowTileDev);
        AROL_CUDA(arol_malloc((void**)&b->dev_rtiles, bytes), "cudaMalloc(row tiles)");
        AROL_CUDA(arol_malloc((void**)&b->dev_rtiles_pt, bytes), "cudaMalloc(row tiles)");
        AROL_CUDA(cudaMallocHost((void**)&b->pinned_rtiles, 2 * bytes), "cudaMallocHost(row tiles)");
        b->rtiles_cap = (int64_t)rtiles.size();
    }
    fill_row_tile_ptrs(b);
    if (!b->rtiles.empty()) {
        AROL_CUDA(cudaMemcpy(b->dev_rtiles, b->rtiles.data(), b->rtiles.size() * sizeof(RowTileDev),
                             cudaMemcpyHostToDevice),
                  "upload row tiles");
        AROL_CUDA(cudaMemcpy(b->dev_rtiles_pt, b->rtiles_pt.data(), b->rtiles_pt.size() * sizeof(RowTileDev),
                             cudaMemcpyHostToDevice),
                  "upload row tiles");
    }
    b->ntiles = (int)tiles.size();
    std::vector<TileDev> by_task(tiles);
    std::stable_sort(by_task.begin(), by_task.end(), [](const TileDev& x, const TileDev& y) { return x.task < y.task; });
    b->pt_off.assign(b->host_tasks.size(), 0);
    b->pt_cnt.assign(b->host_tasks.size(), 0);
    for (size_t k = 0; k < by_task.size(); ++k) {
        if (b->pt_cnt[by_task[k].task]++ == 0) b->pt_off[by_task[k].task] = (int)k;
    }
    if ((int64_t)tiles.size() > b->tiles_cap) {
        free_dev(b->dev_tiles);
        free_dev(b->dev_tiles_pt);
        b->dev_tiles = b->dev_tiles_pt = nullptr;
        AROL_CUDA(arol_malloc((void**)&b->dev_tiles, std::max<size_t>(tiles.size(), 1) * sizeof(TileDev)), "cudaMalloc(tiles)");
        AROL_CUDA(arol_malloc((void**)&b->dev_tiles_pt, std::max<size_t>(tiles.size(), 1) * sizeof(TileDev)), "cudaMalloc(tiles)");
        b->tiles_cap = (int64_t)tiles.size();
    }
    if (!tiles.empty()) {
        AROL_CUDA(cudaMemcpy(b->dev_tiles, tiles.data(), tiles.size() * sizeof(TileDev), cudaMemcpyHostToDevice),
                  "upload tiles");
        AROL_CUDA(cudaMemcpy(b->dev_tiles_pt, by_task.data(), by_task.size() * sizeof(TileDev), cudaMemcpyHostToDevice),
                  "upload tiles");
    }
    invalidate_graph(b);
    return AROL_OK;
}

// Bands of the streamed chain members, sized for about four units per
// resident CTA over the whole batch (16 to 1024 rows per unit), the unit
// prefix, and the device chain table.
arol_status batch_stream_plan(arol_batch b) {
    const size_t ns = b->ss_members.size();
    if (!ns || b->dev_ss) return AROL_OK;
    const size_t smem = sepstream_smem(b->ss_xw, b->ss_nst, b->ss_tapw);
    const double cap = (double)device_sm_count() * sepstream_ctas_per_sm(b->ss_th, b->ss_tv, true, smem);
    double rows = 0;
    for (const SsChain& c : b->ss_chains) rows += (double)c.F * c.chunks * c.H;
    const double target = std::min(1024.0, std::max(16.0, rows / (4.0 * cap)));
    b->ss_ustart.assign(ns + 1, 0);
    int64_t units = 0;
    for (size_t k = 0; k < ns; ++k) {
        SsChain& c = b->ss_chains[k];
        const int64_t bh = std::max<int64_t>(1, std::min<int64_t>(c.Rv, (int64_t)((target - c.Tv) / c.Sv) + 1));
        c.BH = (int32_t)bh;
        c.bands = (int32_t)((c.Rv + bh - 1) / bh);
        b->ss_ustart[k] = (int)units;
        units += c.F * c.chunks * c.bands;
        if (units >= 2147483647LL) return fail(AROL_ERR_UNSUPPORTED, "batch: too many streamed chain units");
    }
    b->ss_ustart[ns] = (int)units;
    b->ss_units = (int)units;
    AROL_CUDA(arol_malloc((void**)&b->dev_ss, ns * sizeof(SsChain)), "cudaMalloc(chain table)");
    AROL_CUDA(arol_malloc((void**)&b->dev_ss_ustart, (ns + 1) * sizeof(int)), "cudaMalloc(chain units)");
    AROL_CUDA(cudaMallocHost((void**)&b->pinned_ss, ns * sizeof(SsChain)), "cudaMallocHost(chain table)");
    AROL_CUDA(cudaMemcpy(b->dev_ss_ustart, b->ss_ustart.data(), (ns + 1) * sizeof(int), cudaMemcpyHostToDevice),
              "upload chain units");
    log_line("batch %p: %lld streamed chain units (%.0f rows per unit aimed at)", (void*)b, (long long)units, target);
    return AROL_OK;
}

// The members on the batched 8 -> 3 kernel (ds_on), their column chunks,
// the unit prefix, and device tables sized for every eligible member.
arol_status batch_ds_plan(arol_batch b) {
    b->ds_members.clear();
    b->ds_mem.clear();
    b->ds_ustart.assign(1, 0);
    b->ds_ws = 32;
    int64_t units = 0;
    size_t cap = 0;
    for (char e : b->ds_ok) cap += e ? 1 : 0;
    if (cap && !b->dev_ds) {
        AROL_CUDA(arol_malloc((void**)&b->dev_ds, cap * sizeof(DsMember)), "cudaMalloc(chain table)");
        AROL_CUDA(arol_malloc((void**)&b->dev_ds_ustart, (cap + 1) * sizeof(int)), "cudaMalloc(chain units)");
        AROL_CUDA(cudaMallocHost((void**)&b->pinned_ds, cap * sizeof(DsMember)), "cudaMallocHost(chain table)");
        AROL_CUDA(arol_malloc((void**)&b->ds_taps, cap * 48 * sizeof(float)), "cudaMalloc(chain taps)");
        std::vector<float> h;
        for (size_t i = 0; i < b->ds_ok.size(); ++i) {
            if (!b->ds_ok[i]) continue;
            const int f = b->first_of[i];
            h.insert(h.end(), b->taps[f].begin(), b->taps[f].end());
            h.insert(h.end(), b->taps[f + 1].begin(), b->taps[f + 1].end());
        }
        if (h.size() != cap * 48) return fail(AROL_ERR_INVALID, "batch: 8 -> 3 chain taps");
        AROL_CUDA(cudaMemcpy(b->ds_taps, h.data(), h.size() * sizeof(float), cudaMemcpyHostToDevice), "upload chain taps");
    }
    int e = 0;   // eligible members so far: their taps' slot
    for (size_t i = 0; i < b->ds_on.size(); ++i) {
        if (!b->ds_ok[i]) continue;
        const int slot = e++;
        if (!b->ds_on[i]) continue;
        DsMember d = b->ds_geom[i];
        d.taps = b->ds_taps + (size_t)48 * slot;
        b->ds_members.push_back((int)i);
        b->ds_mem.push_back(d);
        b->ds_ws = std::max(b->ds_ws, d.Wc);
        units += d.frames * (d.H / 8) * d.nch;
        if (units >= 2147483647LL) return fail(AROL_ERR_UNSUPPORTED, "batch: too many chain units");
        b->ds_ustart.push_back((int)units);
    }
    b->ds_units = (int)units;
    if (!b->ds_members.empty()) {
        AROL_CUDA(cudaMemcpy(b->dev_ds_ustart, b->ds_ustart.data(), b->ds_ustart.size() * sizeof(int),
                             cudaMemcpyHostToDevice),
                  "upload chain units");
        log_line("batch %p: %zu 8 -> 3 chain members on the batched downscaler, %d units", (void*)b,
                 b->ds_members.size(), b->ds_units);
    }
    return AROL_OK;
}

arol_status batch_prepare(arol_batch b, const void* const* in, void* const* out, cudaStream_t s) {
    const size_t n = b->descs.size(), nm = b->first_of.size();
    int dev = 0;
    AROL_CUDA(cudaGetDevice(&dev), "cudaGetDevice");
    if (b->device < 0) b->device = dev;
    else if (b->device != dev) return fail(AROL_ERR_INVALID, "batch used on another device than its buffers");
    for (size_t i = 0; i < nm; ++i) {
        const int f = b->first_of[i], l = f + b->len_of[i] - 1;
        if (!in[i] && b->host_tasks[f].nreps > 0) return fail(AROL_ERR_INVALID, "null input pointer for task %zu", i);
        if (!out[i] && b->host_tasks[l].nreps > 0) return fail(AROL_ERR_INVALID, "null output pointer for task %zu", i);
    }
    // the batched 8 -> 3 kernel takes the eligible members whose input is
    // 16-byte aligned now; another set than the tables were built for
    // rebuilds them
    {
        bool same = true;
        std::vector<char> on(nm, 0);
        for (size_t i = 0; i < nm; ++i) {
            on[i] = b->ds_ok[i] && aligned16(in[i]);
            same = same && on[i] == b->ds_on[i];
        }
        if (!same) {
            b->ds_on = on;
            b->tables_built = false;
        }
    }
    if (!b->tables_built) {
        b->skip = b->streamed;
        for (size_t i = 0; i < nm; ++i)
            if (b->ds_on[i])
                for (int k = 0; k < b->len_of[i]; ++k) b->skip[b->first_of[i] + k] = 1;
        // each task's taps, then (row-FIR tasks) the same taps transposed and
        // zero padded to T x 16 for the row-tile path
        size_t ntaps = 0;
        for (size_t i = 0; i < n; ++i) {
            ntaps += b->taps[i].size();
            if (b->host_tasks[i].rowfir) ntaps += 3 + (size_t)b->host_tasks[i].T * 32;
            else if (b->host_tasks[i].colfir) ntaps += 3 + (size_t)b->host_tasks[i].T * 16;
        }
        // each resource is made once: a call that failed part-way (say, out of
        // memory) is retried without leaking what it had already made
        if (!b->dev_tasks)
            AROL_CUDA(arol_malloc((void**)&b->dev_tasks, std::max<size_t>(n, 1) * sizeof(TaskDev)), "cudaMalloc(task table)");
        if (!b->pinned_tasks)
            AROL_CUDA(cudaMallocHost(&b->pinned_tasks, std::max<size_t>(n, 1) * sizeof(TaskDev)), "cudaMallocHost(task table)");
        if (!b->table_copied)
            AROL_CUDA(cudaEventCreateWithFlags(&b->table_copied, cudaEventDisableTiming), "cudaEventCreate");
        if (!b->launched) AROL_CUDA(cudaEventCreateWithFlags(&b->launched, cudaEventDisableTiming), "cudaEventCreate");
        if (!b->counter) AROL_CUDA(arol_malloc((void**)&b->counter, sizeof(unsigned)), "cudaMalloc(counter)");
        if (!b->err) {
            AROL_CUDA(arol_malloc((void**)&b->err, sizeof(unsigned)), "cudaMalloc(error word)");
            AROL_CUDA(cudaMemset(b->err, 0, sizeof(unsigned)), "clear error word");
        }
        if (!b->taps_dev)
            AROL_CUDA(arol_malloc((void**)&b->taps_dev, std::max<size_t>(ntaps, 1) * sizeof(float)), "cudaMalloc(taps)");
        size_t off = 0;
        for (size_t i = 0; i < n; ++i) {
            if (!b->taps[i].empty()) {
                AROL_CUDA(cudaMemcpy(b->taps_dev + off, b->taps[i].data(), b->taps[i].size() * sizeof(float),
                                     cudaMemcpyHostToDevice),
                          "upload taps");
                b->host_tasks[i].taps = b->taps_dev + off;
                off += b->taps[i].size();
            }
            TaskDev& td = b->host_tasks[i];
            if (td.rowfir || td.colfir) {
                off = (off + 3) & ~size_t(3);   // 16-byte aligned: the row-FIR kernel bulk-copies these
                // column FIR: ht[k * 16 + j] = H[j, k]; row FIR: each tap twice,
                // ht[k * 32 + 2 j + e] = H[j, k] (pairs for paired FMAs)
                const int dup = td.rowfir ? 2 : 1;
                std::vector<float> ht((size_t)td.T * 16 * dup, 0.f);
                for (int k = 0; k < td.T; ++k)
                    for (int j = 0; j < td.m; ++j)
                        for (int e = 0; e < dup; ++e)
                            ht[((size_t)k * 16 + j) * dup + e] = b->taps[i][(size_t)j * td.T + k];
                AROL_CUDA(cudaMemcpy(b->taps_dev + off, ht.data(), ht.size() * sizeof(float), cudaMemcpyHostToDevice),
                          "upload taps");
                td.taps_t = b->taps_dev + off;
                off += ht.size();
            }
        }
        // one arena for every chain intermediate, 256-byte aligned slices
        size_t arena = 0;
        b->mid_off.assign(n, 0);
        for (size_t j = 0; j < n; ++j) {
            const int m = b->member_of[j];
            if (b->stage_of[j] == b->len_of[m] - 1 || b->streamed[j]) continue;
            b->mid_off[j] = arena;
            const arol_array_desc& o = b->descs[j].out[0];
            arena += ((size_t)elems_of(o) * esize_of(o.dtype) + 255) / 256 * 256;
        }
        if (arena && !b->arena) AROL_CUDA(arol_malloc((void**)&b->arena, arena), "cudaMalloc(chain intermediates)");
        if (!b->cap_stream) AROL_CUDA(cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking), "cudaStreamCreate");
        arol_status st = build_tiles(b);
        if (st != AROL_OK) return st;
        if ((st = batch_stream_plan(b)) != AROL_OK) return st;
        if ((st = batch_ds_plan(b)) != AROL_OK) return st;
        b->tables_built = true;
        b->last_in.assign(nm, (const void*)1);   // force the first table upload
        b->last_out.assign(nm, (void*)1);
    }
    bool changed = false;
    for (size_t i = 0; i < nm; ++i) changed = changed || in[i] != b->last_in[i] || out[i] != b->last_out[i];
    if (changed) {
        AROL_CUDA(cudaEventSynchronize(b->table_copied), "wait for previous table upload");
        for (size_t j = 0; j < n; ++j) {
            const int m = b->member_of[j], k = b->stage_of[j];
            b->host_tasks[j].x = k == 0 ? in[m] : (const void*)(b->arena + b->mid_off[j - 1]);
            b->host_tasks[j].y = k == b->len_of[m] - 1 ? out[m] : (void*)(b->arena + b->mid_off[j]);
        }
        for (size_t i = 0; i < nm; ++i) {
            b->last_in[i] = in[i];
            b->last_out[i] = out[i];
        }
        std::memcpy(b->pinned_tasks, b->host_tasks.data(), n * sizeof(TaskDev));
        fill_row_tile_ptrs(b);
        const size_t nr = b->rtiles.size();
        if (nr) {
            std::memcpy(b->pinned_rtiles, b->rtiles.data(), nr * sizeof(RowTileDev));
            std::memcpy(b->pinned_rtiles + nr, b->rtiles_pt.data(), nr * sizeof(RowTileDev));
        }
        // launches on other streams may still read the old table
        AROL_CUDA(cudaStreamWaitEvent(s, b->launched, 0), "wait for previous launches");
        AROL_CUDA(cudaMemcpyAsync(b->dev_tasks, b->pinned_tasks, n * sizeof(TaskDev), cudaMemcpyHostToDevice, s),
                  "upload task table");
        const size_t ns = b->ss_members.size();
        if (ns) {
            for (size_t k = 0; k < ns; ++k) {
                const int m = b->ss_members[k], f = b->first_of[m];
                SsChain c = b->ss_chains[k];
                c.x = (const float*)in[m];
                c.y = (float*)out[m];
                c.hh = b->host_tasks[f].taps;
                c.hv = b->host_tasks[f + 1].taps;
                b->pinned_ss[k] = c;
            }
            AROL_CUDA(cudaMemcpyAsync(b->dev_ss, b->pinned_ss, ns * sizeof(SsChain), cudaMemcpyHostToDevice, s),
                      "upload chain table");
        }
        const size_t nd = b->ds_members.size();
        if (nd) {
            for (size_t k = 0; k < nd; ++k) {
                const int m = b->ds_members[k];
                DsMember d = b->ds_mem[k];
                d.x = (const float*)in[m];
                d.y = (float*)out[m];
                b->pinned_ds[k] = d;
            }
            AROL_CUDA(cudaMemcpyAsync(b->dev_ds, b->pinned_ds, nd * sizeof(DsMember), cudaMemcpyHostToDevice, s),
                      "upload chain table");
        }
        if (nr) {
            AROL_CUDA(cudaMemcpyAsync(b->dev_rtiles, b->pinned_rtiles, nr * sizeof(RowTileDev), cudaMemcpyHostToDevice, s),
                      "upload row tiles");
            AROL_CUDA(cudaMemcpyAsync(b->dev_rtiles_pt, b->pinned_rtiles + nr, nr * sizeof(RowTileDev),
                                      cudaMemcpyHostToDevice, s),
                      "upload row tiles");
        }
        AROL_CUDA(cudaEventRecord(b->table_copied, s), "cudaEventRecord");
    }
    return AROL_OK;
}

arol_status batch_capture(arol_batch b) {
    if (b->exec) return AROL_OK;
    const int grid = device_sm_count() * b->ctas_per_sm;
    AROL_CUDA(cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeThreadLocal), "begin capture");
    // one launch per chain stage; stage k reads what stage k - 1 wrote
    cudaError_t le = cudaSuccess;
    const int rgrid = b->row_ctas > 0 ? device_sm_count() * b->row_ctas : 0;
    if (b->ss_units > 0)
        le = launch_sepstream(SsChain{}, b->dev_ss, b->dev_ss_ustart, (int)b->ss_members.size(), b->ss_units, b->ss_th,
                              b->ss_tv, b->ss_xw, b->ss_nst, b->ss_tapw, b->err, b->cap_stream);
    if (b->ds_units > 0 && le == cudaSuccess)
        le = launch_downscale_batch(b->dev_ds, b->dev_ds_ustart, (int)b->ds_members.size(), b->ds_units, b->ds_ws,
                                    b->err, b->cap_stream);
    for (int k = 0; k < b->nstages && le == cudaSuccess; ++k) {
        if (b->rstage_cnt[k] > 0)
            le = launch_rowfir_batch(b->dev_rtiles + b->rstage_off[k], b->rstage_cnt[k], rgrid, b->err, b->cap_stream);
        const int cnt = b->stage_cnt[k];
        if (cnt == 0 || le != cudaSuccess) continue;
        le = launch_batch_persistent(b->dev_tasks, b->dev_tiles + b->stage_off[k], cnt, b->counter,
                                     std::min(grid, cnt), b->threads, b->max_m, b->cap_stream);
    }
    cudaGraph_t g = nullptr;
    cudaError_t ee = cudaStreamEndCapture(b->cap_stream, &g);
    if (le != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return cuda_fail(le, "batch kernel capture");
    }
    AROL_CUDA(ee, "end capture");
    b->graph = g;
    AROL_CUDA(cudaGraphInstantiate(&b->exec, b->graph, 0), "graph instantiate");
    return AROL_OK;
}

}  // namespace

extern "C" {

arol_status arol_batch_create(const arol_task* tasks, int n, arol_batch* out) {
    AROL_TRACE();
    if (!tasks || !out || n < 1) return fail(AROL_ERR_INVALID, "a batch needs at least one task");
    *out = nullptr;
    for (int i = 0; i < n; ++i) {
        if (!tasks[i]) return fail(AROL_ERR_INVALID, "null task %d", i);
        for (const arol_task_desc& d : tasks[i]->descs)
            if (d.elem == AROL_ELEM_MATMUL) return fail(AROL_ERR_UNSUPPORTED, "batch: task %d is a matmul", i);
        if (tasks[i]->taps_borrowed || !tasks[i]->taps_ready) return fail(AROL_ERR_INVALID, "batch: task %d has no host taps", i);
    }
    arol_batch b = new (std::nothrow) arol_batch_s();
    if (!b) return fail(AROL_ERR_INVALID, "out of host memory");
    // a chain enters as its tasks, one per stage, in chain order
    for (int i = 0; i < n; ++i) {
        const arol_task t = tasks[i];
        const int len = (int)t->descs.size();
        b->first_of.push_back((int)b->descs.size());
        b->len_of.push_back(len);
        b->nstages = std::max(b->nstages, len);
        for (int k = 0; k < len; ++k) {
            const arol_task_desc& d = t->descs[k];
            // a chain's taps are its tasks' m x T blocks back to back
            const size_t a = t->kind == 0 ? 0 : (size_t)t->tap_off[k];
            const size_t z = t->kind == 0 || k + 1 == len ? t->taps_host.size() : (size_t)t->tap_off[k + 1];
            b->descs.push_back(d);
            b->taps.emplace_back(t->taps_host.begin() + a, t->taps_host.begin() + z);
            b->host_tasks.push_back(make_taskdev(d, true));
            b->member_of.push_back(i);
            b->stage_of.push_back(k);
            if (d.elem == AROL_ELEM_FIR) b->max_m = std::max(b->max_m, d.fir_m);
        }
    }
    // Members that are a row pass then a column pass run together on the
    // streaming chain kernel when its common launch shape (widest window,
    // most taps) fits shared memory; their tasks get no tiles and no
    // intermediates.
    b->streamed.assign(b->descs.size(), 0);
    {
        std::vector<int> mem;
        int xw = 0, tapw = 0, th = -1, tv = -1;
        for (int i = 0; i < n; ++i) {
            const arol_task t = tasks[i];
            if (t->kind != 1 || t->kernel != 5) continue;
            mem.push_back(i);
            xw = std::max(xw, t->ss_xw);
            tapw = std::max(tapw, t->ss_tapw);
            th = th == -1 || th == t->ss.Th ? t->ss.Th : 0;
            tv = tv == -1 || tv == t->ss.Tv ? t->ss.Tv : 0;
        }
        const int nst = sepstream_stages(std::max(xw, 1));
        if (!mem.empty() && sepstream_smem(xw, nst, tapw) <= kSsSmemMax) {
            b->ss_members = mem;
            b->ss_xw = xw;
            b->ss_nst = nst;
            b->ss_tapw = tapw;
            b->ss_th = th;
            b->ss_tv = tv;
            for (int i : mem) {
                b->ss_chains.push_back(tasks[i]->ss);
                for (int k = 0; k < b->len_of[i]; ++k) b->streamed[b->first_of[i] + k] = 1;
            }
        }
    }
    b->ds_ok.assign(n, 0);
    b->ds_on.assign(n, 0);
    for (int i = 0; i < n; ++i) {
        const arol_task t = tasks[i];
        b->ds_ok[i] = t->kind == 1 && t->kernel == 1 && !t->ds_in16 && !t->ds_mid16 && !t->ds_out16;
        DsMember d{};
        if (b->ds_ok[i]) {
            d.frames = t->ds_frames;
            d.H = t->ds_H;
            d.W = t->ds_W;
            d.Wc = downscale_chunk(d.W);
            d.nch = (d.W + d.Wc - 1) / d.Wc;
        }
        b->ds_geom.push_back(d);
    }
    // The persistent kernel's column-FIR path serves output counts up to 16;
    // a batch with a larger m runs other tiles on the per-repetition walk,
    // which needs every task's full ports: frame-stripped column FIRs go back
    // to their exact form there.
    if (b->max_m > 16)
        for (size_t j = 0; j < b->host_tasks.size(); ++j)
            if (b->host_tasks[j].cf_frames > 0) b->host_tasks[j] = make_taskdev_exact(b->descs[j]);
    if (log_enabled()) {
        int rows = 0, cols = 0;
        for (const TaskDev& td : b->host_tasks) {
            rows += td.rowfir;
            cols += td.colfir;
        }
        log_line("batch %p: %d members, %zu tasks in %d stage(s): %d row FIR, %d column FIR, %zu per-repetition",
                 (void*)b, n, b->host_tasks.size(), b->nstages, rows, cols, b->host_tasks.size() - rows - cols);
        if (!b->ss_members.empty())
            log_line("batch %p: %zu chain members on the streaming chain kernel (windows of %d words, %d stages)",
                     (void*)b, b->ss_members.size(), b->ss_xw, b->ss_nst);
    }
    *out = b;
    return AROL_OK;
}

arol_status arol_batch_run(arol_batch b, const void* const* in, void* const* out, void* stream) {
    AROL_TRACE();
    if (!b || !in || !out) return fail(AROL_ERR_INVALID, "null argument");
    cudaStream_t s = (cudaStream_t)stream;
    arol_status st = batch_prepare(b, in, out, s);
    if (st != AROL_OK) return st;
    if ((st = batch_capture(b)) != AROL_OK) return st;
    AROL_CUDA(cudaGraphLaunch(b->exec, s), "graph launch");
    AROL_CUDA(cudaEventRecord(b->launched, s), "cudaEventRecord");
    return AROL_OK;
}

arol_status arol_batch_run_per_task(arol_batch b, const void* const* in, void* const* out, void* stream) {
    AROL_TRACE();
    if (!b || !in || !out) return fail(AROL_ERR_INVALID, "null argument");
    cudaStream_t s = (cudaStream_t)stream;
    arol_status st = batch_prepare(b, in, out, s);
    if (st != AROL_OK) return st;
    // one launch of the batch kernel per task, over that task's tiles only
    const int cap = device_sm_count() * b->ctas_per_sm;
    const int rgrid = b->row_ctas > 0 ? device_sm_count() * b->row_ctas : 0;
    // 8 -> 3 chain members: one launch of the fused downscaler each
    for (size_t k = 0; k < b->ds_members.size(); ++k) {
        const DsMember& d = b->pinned_ds[k];
        DownscaleDev p{};
        p.x = d.x;
        p.y = d.y;
        p.taps = d.taps;
        p.err = b->err;
        p.frames = d.frames;
        p.H = d.H;
        p.W = d.W;
        AROL_CUDA(launch_downscale_fwd(p, s), "downscale kernel launch");
    }
    // streamed chain members: one launch of the streaming kernel each
    for (size_t k = 0; k < b->ss_members.size(); ++k) {
        const SsChain& c = b->pinned_ss[k];
        AROL_CUDA(launch_sepstream(c, nullptr, nullptr, 1, b->ss_ustart[k + 1] - b->ss_ustart[k], c.Th, c.Tv, b->ss_xw,
                                   b->ss_nst, b->ss_tapw, b->err, s),
                  "fused chain kernel launch");
    }
    for (size_t i = 0; i < b->host_tasks.size(); ++i) {
        if (b->rpt_cnt[i] > 0)
            AROL_CUDA(launch_rowfir_batch(b->dev_rtiles_pt + b->rpt_off[i], b->rpt_cnt[i], rgrid, b->err, s),
                      "row-FIR kernel launch");
        const int cnt = b->pt_cnt[i];
        if (cnt == 0) continue;
        AROL_CUDA(launch_batch_persistent(b->dev_tasks, b->dev_tiles_pt + b->pt_off[i], cnt, nullptr,
                                          std::min(cnt, cap), b->threads, b->max_m, s),
                  "tiler kernel launch");
    }
    AROL_CUDA(cudaEventRecord(b->launched, s), "cudaEventRecord");
    return AROL_OK;
}

arol_status arol_batch_config(arol_batch b, int64_t* tile_reps, int32_t* ctas_per_sm, int32_t* threads) {
    if (!b) return fail(AROL_ERR_INVALID, "null batch");
    if (tile_reps) *tile_reps = b->tile_reps;
    if (ctas_per_sm) *ctas_per_sm = b->ctas_per_sm;
    if (threads) *threads = b->threads;
    return AROL_OK;
}

arol_status arol_batch_tune(arol_batch b, const void* const* in, void* const* out, void* stream, int force) {
    AROL_TRACE();
    if (!b || !in || !out) return fail(AROL_ERR_INVALID, "null argument");
    // AROL_TUNE: "off" keeps the current launch shape (nothing is timed or
    // read), "force" re-times as force = 1 does, anything else is the default
    if (const char* mode = std::getenv("AROL_TUNE")) {
        if (std::strcmp(mode, "off") == 0) {
            log_line("batch tune: AROL_TUNE=off, keeping tile_reps %lld, %d CTAs per SM", (long long)b->tile_reps,
                     b->ctas_per_sm);
            return AROL_OK;
        }
        if (std::strcmp(mode, "force") == 0) force = 1;
    }
    cudaStream_t s = (cudaStream_t)stream;
    arol_status st = batch_prepare(b, in, out, s);
    if (st != AROL_OK) return st;
    const std::string sig = batch_signature(b);
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        tune_cache_load();
        auto it = g_tune_cache.find(sig);
        if (!force && it != g_tune_cache.end() && it->second.size() == 5) {
            b->tile_reps = it->second[0];
            b->threads = (int)it->second[1];
            b->ctas_per_sm = (int)it->second[2];
            b->row_budget = (int)it->second[3];
            b->row_ctas = (int)it->second[4];
            return build_tiles(b);
        }
    }
    bool has_rows = false, has_other = false;
    for (const TaskDev& t : b->host_tasks) {
        if (t.nreps == 0) continue;
        if (t.rowfir) has_rows = true;
        else has_other = true;
    }
    cudaEvent_t e0, e1;
    AROL_CUDA(cudaEventCreate(&e0), "cudaEventCreate");
    AROL_CUDA(cudaEventCreate(&e1), "cudaEventCreate");
    // one candidate: tiles rebuilt (when their shape changed), graph
    // captured, one warm-up launch, three timed
    auto time_it = [&](bool rebuild, float* ms) -> arol_status {
        arol_status r = AROL_OK;
        if (rebuild && (r = build_tiles(b)) != AROL_OK) return r;
        invalidate_graph(b);
        if ((r = batch_capture(b)) != AROL_OK) return r;
        cudaGraphLaunch(b->exec, s);
        cudaEventRecord(e0, s);
        for (int rep = 0; rep < 3; ++rep) cudaGraphLaunch(b->exec, s);
        cudaEventRecord(e1, s);
        cudaError_t ce = cudaEventSynchronize(e1);
        if (ce != cudaSuccess) return cuda_fail(ce, "autotune run");
        cudaEventElapsedTime(ms, e0, e1);
        return AROL_OK;
    };
    st = AROL_OK;
    // row-FIR tiles: slot floats per tile and CTAs per SM
    if (has_rows) {
        float best = 1e30f;
        int best_budget = b->row_budget, best_rc = b->row_ctas;
        const int budgets[] = {kRowSlotFloats / 2, kRowSlotFloats * 3 / 4, kRowSlotFloats};
        const int rcs[] = {1, 2};
        for (int bud : budgets) {
            b->row_budget = bud;
            bool rebuilt = false;
            for (int rc : rcs) {
                b->row_ctas = rc;
                float ms = 0;
                if ((st = time_it(!rebuilt, &ms)) != AROL_OK) break;
                rebuilt = true;
                if (ms < best) { best = ms; best_budget = bud; best_rc = rc; }
            }
            if (st != AROL_OK) break;
        }
        b->row_budget = best_budget;
        b->row_ctas = best_rc;
    }
    // other tiles: repetitions per tile and CTAs per SM of the persistent kernel
    if (st == AROL_OK && has_other) {
        float best = 1e30f;
        int64_t best_tile = b->tile_reps;
        int best_ctas = b->ctas_per_sm;
        const int64_t tiles[] = {512, 1024, 2048, 4096, 8192, 16384};
        const int ctas[] = {2, 4, 6, 8};
        for (int64_t tile : tiles) {
            b->tile_reps = tile;
            bool rebuilt = false;
            for (int c : ctas) {
                if ((int64_t)b->threads * c > 2048) continue;
                b->ctas_per_sm = c;
                float ms = 0;
                if ((st = time_it(!rebuilt, &ms)) != AROL_OK) break;
                rebuilt = true;
                if (ms < best) { best = ms; best_tile = tile; best_ctas = c; }
            }
            if (st != AROL_OK) break;
        }
        b->tile_reps = best_tile;
        b->ctas_per_sm = best_ctas;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != AROL_OK) return st;
    if ((st = build_tiles(b)) != AROL_OK) return st;
    log_line("batch tune: tile_reps %lld, %d CTAs per SM; row tiles of %d slot floats, %d CTAs per SM",
             (long long)b->tile_reps, b->ctas_per_sm, b->row_budget, b->row_ctas);
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune_cache[sig] = {b->tile_reps, (int64_t)b->threads, (int64_t)b->ctas_per_sm, (int64_t)b->row_budget,
                         (int64_t)b->row_ctas};
    tune_cache_save();
    return AROL_OK;
}

arol_status arol_batch_sync_status(arol_batch b, void* stream) {
    if (!b) return fail(AROL_ERR_INVALID, "null batch");
    AROL_CUDA(cudaStreamSynchronize((cudaStream_t)stream), "synchronize");
    if (!b->err) return AROL_OK;
    unsigned flag = 0;
    AROL_CUDA(cudaMemcpy(&flag, b->err, sizeof flag, cudaMemcpyDeviceToHost), "read error word");
    if (!flag) return AROL_OK;
    cudaMemset(b->err, 0, sizeof(unsigned));
    return fail(AROL_ERR_TIMEOUT, "a bounded device-side wait of the batch kernels gave up (flags 0x%x)", flag);
}

void arol_batch_destroy(arol_batch b) {
    if (!b) return;
    if (b->device >= 0) {
        int cur = 0;
        cudaGetDevice(&cur);
        if (cur != b->device) cudaSetDevice(b->device);
        invalidate_graph(b);
        if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
        if (b->table_copied) cudaEventDestroy(b->table_copied);
        if (b->launched) cudaEventDestroy(b->launched);
        if (b->pinned_tasks) cudaFreeHost(b->pinned_tasks);
        free_dev(b->dev_tasks);
        free_dev(b->dev_tiles);
        free_dev(b->dev_tiles_pt);
        free_dev(b->dev_rtiles);
        free_dev(b->dev_rtiles_pt);
        if (b->pinned_rtiles) cudaFreeHost(b->pinned_rtiles);
        free_dev(b->err);
        free_dev(b->counter);
        free_dev(b->taps_dev);
        free_dev(b->arena);
        free_dev(b->dev_ss);
        free_dev(b->dev_ss_ustart);
        if (b->pinned_ss) cudaFreeHost(b->pinned_ss);
        free_dev(b->dev_ds);
        free_dev(b->dev_ds_ustart);
        free_dev(b->ds_taps);
        if (b->pinned_ds) cudaFreeHost(b->pinned_ds);
        if (cur != b->device) cudaSetDevice(cur);
    }
    delete b;
}

}  // extern "C"
