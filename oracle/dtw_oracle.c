/*
 * FP64 CPU oracle for exact DTW, the alignment that ParDTW computes.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path links, loads or
 * calls this file: only the tests, the smoke check and the bench's CPU
 * baseline do.  It shares no code, header, table or helper with the CUDA
 * library.
 *
 * What it computes (all in double precision):
 *
 *   r_x       = 1 / ||x||_2   (0 for a zero frame, so its cosine cost is 1)
 *   C[i][j]   = 1 - (a_i . b_j) * r_a[i] * r_b[j]       cosine distance, Sec. IV
 *   D[0][0]   = C[0][0]
 *   D[i][j]   = min( D[i-1][j-1] + 2 C[i][j],           step (1,1), weight 2
 *                    D[i-1][j-2] + 3 C[i][j],           step (1,2), weight 3
 *                    D[i-2][j-1] + 3 C[i][j] )          step (2,1), weight 3
 *   (out-of-range predecessors count as +inf)
 *
 * Steps and weights are those of the DTW baseline in Sec. V; ParDTW gives
 * exactly DTW's alignment (Sec. II-D, Sec. V).  Steps are (advance in A,
 * advance in B).  The cost of the optimal path is D[La-1][Lb-1]; the path
 * is recovered by backtracing a matrix of 2-bit step codes (Sec. II-D,
 * Sec. VI-D) from (La-1, Lb-1) to (0, 0).
 *
 * Readings where the paper is silent:
 *   - start cell: D[0][0] = C[0][0], unweighted.
 *   - tie-break: candidates are formed as one fma(w, C, D_pred) each and
 *     taken in the order (1,1), (1,2), (2,1); a later one replaces the
 *     current best only when strictly smaller.
 *   - a zero frame has r = 0, hence cost 1 against everything.
 *   - (La-1, Lb-1) unreachable (Lb-1 > 2(La-1) or La-1 > 2(Lb-1)) is an
 *     error, not a path.
 *
 * Step codes: 0 = (1,1), 1 = (1,2), 2 = (2,1), 3 = start / unreachable.
 * The DP runs row by row (the textbook order), keeping three rows of D and
 * a 2-bit code per cell, four cells per byte.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_OK 0
#define OR_ERR_INVALID 1
#define OR_ERR_UNREACHABLE 2
#define OR_ERR_NOMEM 3
#define OR_ERR_CAPACITY 4

int oracle_reachable(int La, int Lb) {
    if (La < 1 || Lb < 1) return 0;
    long long i = La - 1, j = Lb - 1;
    return j <= 2 * i && i <= 2 * j;
}

/* r[k] = 1/||X[k]|| in double, 0 for a zero frame. */
int oracle_inv_norms(const float* X, int L, int D, double* r) {
    if (!X || !r || L < 0 || D < 1) return OR_ERR_INVALID;
    for (int k = 0; k < L; ++k) {
        double s = 0.0;
        for (int d = 0; d < D; ++d) {
            double v = (double)X[(size_t)k * D + d];
            s += v * v;
        }
        r[k] = s > 0.0 ? 1.0 / sqrt(s) : 0.0;
    }
    return OR_OK;
}

static double cosine_cost(const float* a, const float* b, int D, double ra, double rb) {
    double dot = 0.0;
    for (int d = 0; d < D; ++d) dot += (double)a[d] * (double)b[d];
    return 1.0 - dot * ra * rb;
}

/* Full La x Lb cosine cost matrix, row-major. */
int oracle_cost_matrix(const float* A, int La, const float* B, int Lb, int D, double* C) {
    if (!A || !B || !C || La < 1 || Lb < 1 || D < 1) return OR_ERR_INVALID;
    double* ra = (double*)malloc(sizeof(double) * (size_t)La);
    double* rb = (double*)malloc(sizeof(double) * (size_t)Lb);
    if (!ra || !rb) { free(ra); free(rb); return OR_ERR_NOMEM; }
    oracle_inv_norms(A, La, D, ra);
    oracle_inv_norms(B, Lb, D, rb);
    for (int i = 0; i < La; ++i)
        for (int j = 0; j < Lb; ++j)
            C[(size_t)i * Lb + j] = cosine_cost(A + (size_t)i * D, B + (size_t)j * D, D, ra[i], rb[j]);
    free(ra);
    free(rb);
    return OR_OK;
}

/* Where the cost of row i comes from: a given matrix, or features. */
typedef struct {
    const double* C;          /* La x Lb, or NULL */
    const float* A;
    const float* B;
    const double* ra;
    const double* rb;
    int D;
} cost_src;

static void cost_row(const cost_src* s, int i, int Lb, double* out) {
    if (s->C) {
        memcpy(out, s->C + (size_t)i * Lb, sizeof(double) * (size_t)Lb);
        return;
    }
    const float* a = s->A + (size_t)i * s->D;
    for (int j = 0; j < Lb; ++j)   /* no norms given: the frames count as unit vectors */
        out[j] = cosine_cost(a, s->B + (size_t)j * s->D, s->D, s->ra ? s->ra[i] : 1.0,
                             s->rb ? s->rb[j] : 1.0);
}

static inline int get_code(const uint8_t* bp, size_t stride, int i, int j) {
    return (bp[(size_t)i * stride + (size_t)(j >> 2)] >> (2 * (j & 3))) & 3;
}

/*
 * The recurrence and the backtrace.  Optional outputs:
 *   Dfull  La x Lb cumulative costs (small inputs only)
 *   codes  La x Lb step codes, one byte per cell (small inputs only)
 * path receives len (i, j) pairs, ascending from (0, 0); cap = pairs it holds.
 */
static int run_dtw(const cost_src* s, int La, int Lb, double* Dfull, uint8_t* codes,
                   int32_t* path, int cap, int* len, double* total) {
    if (!oracle_reachable(La, Lb)) return OR_ERR_UNREACHABLE;
    const double inf = INFINITY;
    size_t stride = (size_t)(Lb + 3) / 4;
    uint8_t* bp = (uint8_t*)calloc((size_t)La * stride, 1);
    double* rows = (double*)malloc(sizeof(double) * 3 * (size_t)Lb);
    double* crow = (double*)malloc(sizeof(double) * (size_t)Lb);
    if (!bp || !rows || !crow) { free(bp); free(rows); free(crow); return OR_ERR_NOMEM; }
    double* prev2 = rows;               /* row i-2 */
    double* prev1 = rows + Lb;          /* row i-1 */
    double* cur = rows + 2 * (size_t)Lb;
    for (int j = 0; j < Lb; ++j) prev2[j] = prev1[j] = inf;

    for (int i = 0; i < La; ++i) {
        cost_row(s, i, Lb, crow);
        uint8_t* brow = bp + (size_t)i * stride;
        for (int j = 0; j < Lb; ++j) {
            double c = crow[j];
            double best;
            int code;
            if (i == 0 && j == 0) {
                best = c;
                code = 3;
            } else {
                double d11 = (j >= 1) ? prev1[j - 1] : inf;
                double d12 = (j >= 2) ? prev1[j - 2] : inf;
                double d21 = (j >= 1) ? prev2[j - 1] : inf;
                double c0 = fma(2.0, c, d11);
                double c1 = fma(3.0, c, d12);
                double c2 = fma(3.0, c, d21);
                best = c0;
                code = 0;
                if (c1 < best) { best = c1; code = 1; }
                if (c2 < best) { best = c2; code = 2; }
                if (isinf(best)) code = 3;
            }
            cur[j] = best;
            brow[j >> 2] |= (uint8_t)(code << (2 * (j & 3)));
            if (Dfull) Dfull[(size_t)i * Lb + j] = best;
            if (codes) codes[(size_t)i * Lb + j] = (uint8_t)code;
        }
        double* t = prev2;
        prev2 = prev1;
        prev1 = cur;
        cur = t;
    }
    double result = prev1[Lb - 1];   /* row La-1 */
    free(rows);
    free(crow);

    int rc = OR_OK;
    if (path || len) {
        /* walk back, writing pairs from the end of a scratch buffer */
        int maxlen = (La < Lb ? La : Lb);
        int32_t* tmp = (int32_t*)malloc(sizeof(int32_t) * 2 * (size_t)maxlen);
        if (!tmp) { free(bp); return OR_ERR_NOMEM; }
        int i = La - 1, j = Lb - 1, n = 0;
        for (;;) {
            if (n >= maxlen) { rc = OR_ERR_INVALID; break; }  /* cannot happen */
            tmp[2 * n] = i;
            tmp[2 * n + 1] = j;
            ++n;
            if (i == 0 && j == 0) break;
            int code = get_code(bp, stride, i, j);
            if (code == 0) { i -= 1; j -= 1; }
            else if (code == 1) { i -= 1; j -= 2; }
            else if (code == 2) { i -= 2; j -= 1; }
            else { rc = OR_ERR_INVALID; break; }
        }
        if (rc == OR_OK) {
            if (len) *len = n;
            if (path) {
                if (n > cap) rc = OR_ERR_CAPACITY;
                else
                    for (int k = 0; k < n; ++k) {
                        path[2 * k] = tmp[2 * (n - 1 - k)];
                        path[2 * k + 1] = tmp[2 * (n - 1 - k) + 1];
                    }
            }
        }
        free(tmp);
    }
    free(bp);
    if (total) *total = result;
    return rc;
}

/* Exact DTW over a given La x Lb cost matrix. */
int oracle_dtw_matrix(const double* C, int La, int Lb, double* Dfull, uint8_t* codes,
                      int32_t* path, int cap, int* len, double* total) {
    if (!C || La < 1 || Lb < 1) return OR_ERR_INVALID;
    cost_src s = {C, NULL, NULL, NULL, NULL, 0};
    return run_dtw(&s, La, Lb, Dfull, codes, path, cap, len, total);
}

/* Exact DTW of two feature sequences under the cosine cost (cost on the fly). */
int oracle_dtw(const float* A, int La, const float* B, int Lb, int D,
               int32_t* path, int cap, int* len, double* total) {
    if (!A || !B || La < 1 || Lb < 1 || D < 1) return OR_ERR_INVALID;
    double* ra = (double*)malloc(sizeof(double) * (size_t)La);
    double* rb = (double*)malloc(sizeof(double) * (size_t)Lb);
    if (!ra || !rb) { free(ra); free(rb); return OR_ERR_NOMEM; }
    oracle_inv_norms(A, La, D, ra);
    oracle_inv_norms(B, Lb, D, rb);
    cost_src s = {NULL, A, B, ra, rb, D};
    int rc = run_dtw(&s, La, Lb, NULL, NULL, path, cap, len, total);
    free(ra);
    free(rb);
    return rc;
}

/* Exact DTW of frames taken as given, C[i][j] = 1 - a_i . b_j (the cosine
 * cost of Sec. IV for frames that are already unit vectors; nothing is
 * renormalised).  Used for features that were normalised and then rounded
 * to a narrower type, whose norms are no longer exactly 1. */
int oracle_dtw_unit(const float* A, int La, const float* B, int Lb, int D,
                    int32_t* path, int cap, int* len, double* total) {
    if (!A || !B || La < 1 || Lb < 1 || D < 1) return OR_ERR_INVALID;
    cost_src s = {NULL, A, B, NULL, NULL, D};
    return run_dtw(&s, La, Lb, NULL, NULL, path, cap, len, total);
}

/* C[0,0] + sum over steps of w_step * C[destination], in double. */
int oracle_path_cost(const float* A, int La, const float* B, int Lb, int D,
                     const int32_t* path, int len, double* total) {
    if (!A || !B || !path || !total || len < 1 || D < 1) return OR_ERR_INVALID;
    double t = 0.0;
    for (int k = 0; k < len; ++k) {
        int i = path[2 * k], j = path[2 * k + 1];
        if (i < 0 || i >= La || j < 0 || j >= Lb) return OR_ERR_INVALID;
        double ra, rb;
        oracle_inv_norms(A + (size_t)i * D, 1, D, &ra);
        oracle_inv_norms(B + (size_t)j * D, 1, D, &rb);
        double c = cosine_cost(A + (size_t)i * D, B + (size_t)j * D, D, ra, rb);
        double w;
        if (k == 0) {
            w = 1.0;
        } else {
            int di = i - path[2 * (k - 1)], dj = j - path[2 * (k - 1) + 1];
            if (di == 1 && dj == 1) w = 2.0;
            else if ((di == 1 && dj == 2) || (di == 2 && dj == 1)) w = 3.0;
            else return OR_ERR_INVALID;
        }
        t += w * c;
    }
    *total = t;
    return OR_OK;
}
