/*
 * Array-OL repetitive task, written out as its definition in plain C.
 * TEST INFRASTRUCTURE ONLY: loaded by tests/, __graft_entry__.smoke() and
 * bench.py (CPU baseline and reference arm).  The product library never links
 * or calls it, and it shares no code with the CUDA path.
 *
 * Definition (MARTE Repetitive Structure Modeling, Sec. 3; repetitive tasks,
 * Sec. 7): a tiler with origin o, paving P (d x q), fitting F (d x p) names,
 * for repetition index r and pattern index i, the array element
 *     e(r, i) = (o + P r + F i) mod s     componentwise, Euclidean mod.
 * Input tilers gather patterns, the elementary task maps them, the output
 * tiler scatters the result.  Accumulation is in double.  The repetition loop
 * is split across OpenMP threads: distinct r write distinct output elements
 * once the output tiler is checked to be a partition (oref_cover_check).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct {
    int32_t rank;
    int32_t dtype;            /* 0: float32, 1: bfloat16 bits (uint16), 2: float64 */
    int64_t shape[4];
    int64_t origin[4];
    int64_t paving[4][4];     /* [array dim][repetition dim] */
    int64_t fitting[4][2];    /* [array dim][pattern dim] */
    int32_t pattern_rank;
    int32_t pad_;
    int64_t pattern[2];
} oref_port;

enum { OREF_COPY = 0, OREF_FIR = 1, OREF_MATMUL = 2 };

static int64_t emod(int64_t a, int64_t s) {
    int64_t r = a % s;
    return r < 0 ? r + s : r;
}

/* Row-major linear offset of e(r, i) in the port's array. */
static int64_t element_offset(const oref_port* t, int rep_rank, const int64_t* r, const int64_t* i) {
    int64_t off = 0;
    for (int k = 0; k < t->rank; ++k) {
        int64_t v = t->origin[k];
        for (int q = 0; q < rep_rank; ++q) v += t->paving[k][q] * r[q];
        for (int p = 0; p < t->pattern_rank; ++p) v += t->fitting[k][p] * i[p];
        off = off * t->shape[k] + emod(v, t->shape[k]);
    }
    return off;
}

static int64_t pattern_size(const oref_port* t) {
    int64_t n = 1;
    for (int p = 0; p < t->pattern_rank; ++p) n *= t->pattern[p];
    return n;
}

static int64_t array_size(const oref_port* t) {
    int64_t n = 1;
    for (int k = 0; k < t->rank; ++k) n *= t->shape[k];
    return n;
}

static void unflatten(int64_t lin, int n, const int64_t* dims, int64_t* idx) {
    for (int k = n - 1; k >= 0; --k) {
        idx[k] = lin % dims[k];
        lin /= dims[k];
    }
}

static double read_value(const oref_port* t, const void* data, int64_t off) {
    switch (t->dtype) {
    case 0: return (double)((const float*)data)[off];
    case 1: {
        uint32_t bits = (uint32_t)((const uint16_t*)data)[off] << 16;
        float f;
        memcpy(&f, &bits, 4);
        return (double)f;
    }
    default: return ((const double*)data)[off];
    }
}

static int itemsize(int dtype) { return dtype == 1 ? 2 : (dtype == 0 ? 4 : 8); }

int oref_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void oref_set_threads(int n) {
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

/* Returns 0 when the output tiler writes every element of its array exactly
 * once over the repetition space, 1 otherwise. */
int oref_cover_check(int rep_rank, const int64_t* rep, const oref_port* out) {
    int64_t n = array_size(out), nr = 1, ns = pattern_size(out);
    for (int q = 0; q < rep_rank; ++q) nr *= rep[q];
    if (nr * ns != n) return 1;
    uint8_t* seen = (uint8_t*)calloc((size_t)(n > 0 ? n : 1), 1);
    if (!seen) return 2;
    int bad = 0;
    int64_t r[4], j[2];
    for (int64_t lr = 0; lr < nr && !bad; ++lr) {
        unflatten(lr, rep_rank, rep, r);
        for (int64_t lj = 0; lj < ns; ++lj) {
            unflatten(lj, out->pattern_rank, out->pattern, j);
            int64_t e = element_offset(out, rep_rank, r, j);
            if (seen[e]) { bad = 1; break; }
            seen[e] = 1;
        }
    }
    free(seen);
    return bad;
}

/* One task.  out_data is float64 for fir/matmul; for copy it has the input's
 * element size and receives the raw bits.  taps: m x T row-major (fir only).
 * Returns 0 on success, 1 for a non-partitioning output tiler, 3 for an
 * unsupported combination, 2 for an allocation failure. */
int oref_run_task(int rep_rank, const int64_t* rep, int elem, int n_in,
                  const oref_port* in, const void* const* in_data,
                  const oref_port* out, void* out_data,
                  const double* taps, int m, int T) {
    int rc = oref_cover_check(rep_rank, rep, out);
    if (rc) return rc;
    int64_t nr = 1;
    for (int q = 0; q < rep_rank; ++q) nr *= rep[q];
    int64_t ns_out = pattern_size(out);
    if (elem == OREF_COPY && (n_in != 1 || pattern_size(&in[0]) != ns_out)) return 3;
    if (elem == OREF_FIR && (n_in != 1 || pattern_size(&in[0]) != T || ns_out != m)) return 3;
    if (elem == OREF_MATMUL && (n_in != 2 || in[0].pattern_rank != 2 || in[1].pattern_rank != 2 ||
                                in[0].pattern[1] != in[1].pattern[0] ||
                                ns_out != in[0].pattern[0] * in[1].pattern[1]))
        return 3;
    int64_t ns_in0 = pattern_size(&in[0]);
    int64_t ns_in1 = n_in > 1 ? pattern_size(&in[1]) : 0;
    int failed = 0;
#pragma omp parallel
    {
        double* pa = (double*)malloc(sizeof(double) * (size_t)(ns_in0 + ns_in1 + ns_out + 1));
        int64_t r[4], i[2];
        if (!pa) {
#pragma omp atomic write
            failed = 1;
        }
#pragma omp for schedule(static)
        for (int64_t lr = 0; lr < nr; ++lr) {
            if (!pa) continue;
            double* pb = pa + ns_in0;
            double* y = pb + ns_in1;
            unflatten(lr, rep_rank, rep, r);
            if (elem == OREF_COPY) {
                int sz = itemsize(in[0].dtype);
                for (int64_t li = 0; li < ns_out; ++li) {
                    unflatten(li, in[0].pattern_rank, in[0].pattern, i);
                    int64_t src = element_offset(&in[0], rep_rank, r, i);
                    unflatten(li, out->pattern_rank, out->pattern, i);
                    int64_t dst = element_offset(out, rep_rank, r, i);
                    memcpy((char*)out_data + dst * sz, (const char*)in_data[0] + src * sz, (size_t)sz);
                }
                continue;
            }
            for (int64_t li = 0; li < ns_in0; ++li) {
                unflatten(li, in[0].pattern_rank, in[0].pattern, i);
                pa[li] = read_value(&in[0], in_data[0], element_offset(&in[0], rep_rank, r, i));
            }
            for (int64_t li = 0; li < ns_in1; ++li) {
                unflatten(li, in[1].pattern_rank, in[1].pattern, i);
                pb[li] = read_value(&in[1], in_data[1], element_offset(&in[1], rep_rank, r, i));
            }
            if (elem == OREF_FIR) {
                for (int j = 0; j < m; ++j) {
                    double acc = 0.0;
                    for (int k = 0; k < T; ++k) acc += taps[(int64_t)j * T + k] * pa[k];
                    y[j] = acc;
                }
            } else {
                int64_t a = in[0].pattern[0], K = in[0].pattern[1], b = in[1].pattern[1];
                for (int64_t u = 0; u < a; ++u)
                    for (int64_t v = 0; v < b; ++v) {
                        double acc = 0.0;
                        for (int64_t k = 0; k < K; ++k) acc += pa[u * K + k] * pb[k * b + v];
                        y[u * b + v] = acc;
                    }
            }
            for (int64_t lj = 0; lj < ns_out; ++lj) {
                unflatten(lj, out->pattern_rank, out->pattern, i);
                ((double*)out_data)[element_offset(out, rep_rank, r, i)] = y[lj];
            }
        }
        free(pa);
    }
    return failed ? 2 : 0;
}

/* Sampled matmul-task outputs: for each of n (row, col) pairs of C, the dot
 * product of row `row` of A's pattern and column `col` of B's pattern for the
 * repetition that owns C[row, col].  The C tiler must be the plain tile
 * partition (paving diag(a, b), fitting identity, origin 0) so the owner of
 * (row, col) is r = (row / a, col / b), j = (row % a, col % b). */
int oref_matmul_sample(const oref_port* A, const void* a_data, const oref_port* B, const void* b_data,
                       const oref_port* C, int64_t n, const int64_t* rows, const int64_t* cols,
                       double* vals, double* absvals) {
    int64_t a = C->pattern[0], b = C->pattern[1], K = A->pattern[1];
#pragma omp parallel for schedule(static)
    for (int64_t t = 0; t < n; ++t) {
        int64_t r[2] = {rows[t] / a, cols[t] / b};
        int64_t iu[2], iv[2];
        double acc = 0.0, aacc = 0.0;
        for (int64_t k = 0; k < K; ++k) {
            iu[0] = rows[t] % a; iu[1] = k;
            iv[0] = k; iv[1] = cols[t] % b;
            double x = read_value(A, a_data, element_offset(A, 2, r, iu));
            double y = read_value(B, b_data, element_offset(B, 2, r, iv));
            acc += x * y;
            aacc += (x < 0 ? -x : x) * (y < 0 ? -y : y);
        }
        vals[t] = acc;
        absvals[t] = aacc;
    }
    return 0;
}

/* Reverse mode of one fir task for the loss sum(G * Y):
 *   dX[e_in(r,k)] += sum_j H[j,k] G[e_out(r,j)]   (scatter-add, serial)
 *   dH[j,k]       += G[e_out(r,j)] X[e_in(r,k)]
 * dX (float64, input shape) and dH (m x T) are overwritten. */
int oref_fir_vjp(int rep_rank, const int64_t* rep, const oref_port* in, const void* x,
                 const oref_port* out, const double* g, const double* taps, int m, int T,
                 double* dx, double* dh) {
    int64_t nr = 1;
    for (int q = 0; q < rep_rank; ++q) nr *= rep[q];
    memset(dx, 0, sizeof(double) * (size_t)array_size(in));
    memset(dh, 0, sizeof(double) * (size_t)m * (size_t)T);
    int64_t r[4], i[2];
    int64_t* ein = (int64_t*)malloc(sizeof(int64_t) * (size_t)T);
    double* gj = (double*)malloc(sizeof(double) * (size_t)m);
    if (!ein || !gj) { free(ein); free(gj); return 2; }
    for (int64_t lr = 0; lr < nr; ++lr) {
        unflatten(lr, rep_rank, rep, r);
        for (int k = 0; k < T; ++k) {
            unflatten(k, in->pattern_rank, in->pattern, i);
            ein[k] = element_offset(in, rep_rank, r, i);
        }
        for (int j = 0; j < m; ++j) {
            unflatten(j, out->pattern_rank, out->pattern, i);
            gj[j] = g[element_offset(out, rep_rank, r, i)];
        }
        for (int k = 0; k < T; ++k) {
            double xv = read_value(in, x, ein[k]);
            double s = 0.0;
            for (int j = 0; j < m; ++j) {
                s += taps[(int64_t)j * T + k] * gj[j];
                dh[(int64_t)j * T + k] += gj[j] * xv;
            }
            dx[ein[k]] += s;
        }
    }
    free(ein);
    free(gj);
    return 0;
}
