/*
 * oracle.c -- plain, slow reference scorer for Beagle population fitness.
 *
 * TEST INFRASTRUCTURE ONLY. Only the tests, the package's smoke check and the benchmark's
 * CPU-baseline leg load this file's library. It shares no code, header, table or constant
 * with the CUDA path; the token numbering below is the wire format, written out again here.
 *
 * What it computes (Beagle tutorial, arXiv 2607.06731):
 *   - Genomes are GCL programs in reverse Polish notation run on a value stack
 *     (Section 3.2, Table 3). Unary ops replace the top; binary ops pop the top b and the
 *     element below it a, and push a (op) b: SUB is a - b, DIV is a / b (Table 3).
 *   - The stack holds at most 32 values (StackSize, Section 3.2).
 *   - Each program runs on every fitness case and one aggregated fitness per program is
 *     returned (Section 2.4).
 *   - Fitness: mean squared error, and 1 - r^2 with r the Pearson correlation of Eq. 1
 *     (Section 2.10: the paper squares r).
 * Readings where the paper is silent (protected operators, the validity rule, the
 * degenerate-r rule) are stated where they are used below.
 *
 * Two arithmetic modes:
 *   ORACLE_FP64   every operation in double; inputs are fp32 values widened exactly.
 *   ORACLE_FP32   every operation computed in double on fp32 operands and rounded to fp32
 *                 (for + - * / sqrt this equals IEEE fp32; for sin, cos, exp, log it is the
 *                 double result rounded once). Thresholds are read in fp32 too.
 * Aggregation (MSE, 1 - r^2) is in double in both modes, with Neumaier-compensated sums.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <float.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* Wire format: one byte per token. */
enum {
    T_CONST = 0, T_ADD = 1, T_SUB = 2, T_MUL = 3, T_PDIV = 4,
    T_SIN = 5, T_COS = 6, T_EXP = 7, T_PLOG = 8, T_PSQRT = 9, T_SQUARE = 10,
    T_DUP = 11, T_SWAP = 12, T_DEL = 13,
    T_LOAD0 = 32, T_LOAD_END = 48
};

enum { ORACLE_FP64 = 0, ORACLE_FP32 = 1 };

/* Result flags (same meaning as the library's, defined independently). */
#define OF_INVALID    1u    /* some value was non-finite or had |v| > 1e30 */
#define OF_DEGENERATE 2u    /* the program's output is the same on every case: r undefined */
#define OF_MALFORMED  4u    /* the token list is not a valid program */
#define OF_NEAR     256u    /* diagnostic: a value came within 1e-5 (relative) of a threshold */
#define OF_AMBIG    512u    /* error bound: a threshold or validity decision lies inside it */

#define ORACLE_STACK 32     /* StackSize (Section 3.2) */

/* Error codes of the check function. */
#define OE_OK 0
#define OE_UNDERFLOW 1
#define OE_OVERFLOW 2
#define OE_FINAL_DEPTH 3
#define OE_OPCODE 4
#define OE_VAR 5
#define OE_EMPTY 6

static double round_to(double v, int mode) {
    return mode == ORACLE_FP32 ? (double)(float)v : v;
}

/* Thresholds, read in the arithmetic's own precision. */
static double big_limit(int mode) { return mode == ORACLE_FP32 ? (double)1e30f : 1e30; }
static double tiny_limit(int mode) { return mode == ORACLE_FP32 ? (double)1e-3f : 1e-3; }

static int near_to(double v, double t) {
    double a = fabs(v);
    return isfinite(a) && fabs(a - t) <= 1e-5 * t;
}

/*
 * Structural check of one program (Section 3.2): every token finds enough operands, the
 * stack never exceeds max_depth, variables exist (inputs are zero-based, Table 3 LOAD),
 * and exactly one value remains at the end (the program's output).
 */
int oracle_check_program(const uint8_t *ops, int32_t L, int32_t d, int32_t max_depth) {
    if (L <= 0) return OE_EMPTY;
    int depth = 0;
    for (int32_t j = 0; j < L; ++j) {
        int op = ops[j], need, delta;
        if (op == T_CONST) { need = 0; delta = 1; }
        else if (op >= T_LOAD0 && op < T_LOAD_END) {
            if (op - T_LOAD0 >= d) return OE_VAR;
            need = 0; delta = 1;
        }
        else if (op >= T_ADD && op <= T_PDIV) { need = 2; delta = -1; }
        else if (op >= T_SIN && op <= T_SQUARE) { need = 1; delta = 0; }
        else if (op == T_DUP) { need = 1; delta = 1; }
        else if (op == T_SWAP) { need = 2; delta = 0; }
        else if (op == T_DEL) { need = 1; delta = -1; }
        else return OE_OPCODE;
        if (depth < need) return OE_UNDERFLOW;
        depth += delta;
        if (depth > max_depth) return OE_OVERFLOW;
    }
    return depth == 1 ? OE_OK : OE_FINAL_DEPTH;
}

/*
 * Run one program on one fitness case. x points at case i of variable 0; variable k is
 * x[k * ldx]. Returns the output; *bad is set when some pushed value fails the validity
 * rule and *near when some value lies within 1e-5 of a threshold.
 *
 * Validity rule (reading): every value pushed by an operator must be finite with
 * |v| <= 1e30; NaN fails. Leaves (CONST, LOAD) are checked the same way.
 * Protected operators (reading; the paper's own DIV, LN, SQRT are unprotected, Table 3):
 *   pdiv(a, b) = a / b    if |b| > 1e-3, else 1
 *   plog(a)    = ln |a|   if |a| > 1e-3, else 0
 *   psqrt(a)   = sqrt |a|
 */
static double run_case(const uint8_t *ops, const float *cs, int32_t L,
                       const float *x, int64_t ldx, int mode, int *bad, int *near) {
    double st[ORACLE_STACK + 1];
    int sp = 0;
    const double big = big_limit(mode), tiny = tiny_limit(mode);
    for (int32_t j = 0; j < L; ++j) {
        int op = ops[j];
        double v;
        if (op == T_CONST) {
            v = (double)cs[j];
            st[sp++] = v;
        } else if (op >= T_LOAD0) {
            v = (double)x[(int64_t)(op - T_LOAD0) * ldx];
            st[sp++] = v;
        } else if (op == T_DUP) {
            v = st[sp - 1];
            st[sp++] = v;
            continue;
        } else if (op == T_SWAP) {
            double t = st[sp - 1]; st[sp - 1] = st[sp - 2]; st[sp - 2] = t;
            continue;
        } else if (op == T_DEL) {
            --sp;
            continue;
        } else if (op <= T_PDIV) {
            double b = st[--sp];
            double a = st[--sp];
            switch (op) {
            case T_ADD: v = a + b; break;
            case T_SUB: v = a - b; break;
            case T_MUL: v = a * b; break;
            default:
                if (near_to(b, tiny)) *near = 1;
                v = fabs(b) > tiny ? a / b : 1.0;
                break;
            }
            v = round_to(v, mode);
            st[sp++] = v;
        } else {
            double a = st[--sp];
            switch (op) {
            case T_SIN: v = sin(a); break;
            case T_COS: v = cos(a); break;
            case T_EXP: v = exp(a); break;
            case T_PLOG:
                if (near_to(a, tiny)) *near = 1;
                v = fabs(a) > tiny ? log(fabs(a)) : 0.0;
                break;
            case T_PSQRT: v = sqrt(fabs(a)); break;
            default: v = a * a; break;   /* SQUARE */
            }
            v = round_to(v, mode);
            st[sp++] = v;
        }
        if (!(fabs(v) <= big)) *bad = 1;      /* also true for NaN */
        if (near_to(v, big)) *near = 1;
    }
    return st[0];
}

/* Neumaier's improvement of Kahan summation. */
typedef struct { double s, c; } nsum;
static void nadd(nsum *a, double x) {
    double t = a->s + x;
    if (fabs(a->s) >= fabs(x)) a->c += (a->s - t) + x;
    else a->c += (x - t) + a->s;
    a->s = t;
}
static double nval(const nsum *a) { return a->s + a->c; }

/*
 * Evaluate one program on all N cases. X is column-major [d][N] (row k holds variable
 * x_k for every case). f receives the N outputs. Returns the flags (OF_*).
 */
uint32_t oracle_eval(const uint8_t *ops, const float *cs, int32_t L, const float *X,
                     int64_t N, int32_t d, int32_t mode, double *f) {
    if (oracle_check_program(ops, L, d, ORACLE_STACK) != OE_OK) return OF_MALFORMED;
    uint32_t flags = 0;
    for (int64_t i = 0; i < N; ++i) {
        int bad = 0, near = 0;
        f[i] = run_case(ops, cs, L, X + i, N, mode, &bad, &near);
        if (bad) flags |= OF_INVALID;
        if (near) flags |= OF_NEAR;
    }
    return flags;
}

/*
 * Aggregate outputs f against targets y (Section 2.10).
 *   mse          = (1/N) sum (f_i - y_i)^2
 *   one_minus_r2 = 1 - r^2, r from Eq. 1 with means over all N cases.
 * Reading: when every f_i is the same value, r is undefined; 1 - r^2 := 1 and
 * OF_DEGENERATE is set. An invalid program gets +inf for both.
 */
void oracle_aggregate(const double *f, const float *y, int64_t N, uint32_t flags,
                      double *mse, double *omr2, uint32_t *flags_out) {
    if (flags & (OF_INVALID | OF_MALFORMED)) {
        *mse = INFINITY; *omr2 = INFINITY; *flags_out = flags; return;
    }
    nsum se = {0, 0}, sf = {0, 0}, sy = {0, 0};
    int constant = 1;
    for (int64_t i = 0; i < N; ++i) {
        double e = f[i] - (double)y[i];
        nadd(&se, e * e);
        nadd(&sf, f[i]);
        nadd(&sy, (double)y[i]);
        if (f[i] != f[0]) constant = 0;
    }
    *mse = nval(&se) / (double)N;
    if (constant) {
        *omr2 = 1.0; *flags_out = flags | OF_DEGENERATE; return;
    }
    double fbar = nval(&sf) / (double)N, ybar = nval(&sy) / (double)N;
    nsum sff = {0, 0}, syy = {0, 0}, sfy = {0, 0};
    for (int64_t i = 0; i < N; ++i) {
        double a = f[i] - fbar, b = (double)y[i] - ybar;
        nadd(&sff, a * a);
        nadd(&syy, b * b);
        nadd(&sfy, a * b);
    }
    double r = nval(&sfy) / sqrt(nval(&sff) * nval(&syy));
    *omr2 = 1.0 - r * r;
    *flags_out = flags;
}

/*
 * Score a population: programs concatenated, program p occupies tokens
 * [offsets[p], offsets[p] + lengths[p]); consts is token-aligned. One parallel loop over
 * programs (nthreads <= 0: the OpenMP default).
 */
int oracle_score(const uint8_t *programs, const int64_t *offsets, const int32_t *lengths,
                 const float *consts, int64_t P, const float *X, const float *y, int64_t N,
                 int32_t d, int32_t mode, int32_t nthreads,
                 double *mse, double *omr2, uint32_t *flags) {
    if (N <= 0 || P < 0) return -1;
#ifdef _OPENMP
    if (nthreads <= 0) nthreads = omp_get_max_threads();
#pragma omp parallel num_threads(nthreads)
#endif
    {
        double *f = (double *)malloc(sizeof(double) * (size_t)N);
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 4)
#endif
        for (int64_t p = 0; p < P; ++p) {
            const uint8_t *ops = programs + offsets[p];
            const float *cs = consts + offsets[p];
            uint32_t fl = oracle_eval(ops, cs, lengths[p], X, N, d, mode, f);
            oracle_aggregate(f, y, N, fl, &mse[p], &omr2[p], &flags[p]);
        }
        free(f);
    }
    return 0;
}

int oracle_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}


/* ------------------------------------------------------------------------------------
 * Running error analysis (first order, after Wilkinson): alongside each value v of the
 * oracle's evaluation in the given mode, carry a bound D on |v_dev - v|, where v_dev is the
 * value a device computes with the same operation order and precision but with sin, cos,
 * exp and log accurate only to dev_ulps[op] units in the last place (a library's documented
 * maximum error). + - * / sqrt are correctly rounded on both sides, so they add error only
 * when their inputs already differ. The oracle's own transcendental results are within
 * own_ulps (0.5 in FP32 mode: double results rounded to fp32; 1 in FP64 mode).
 * A decision (protection threshold, validity limit) whose operand lies within D of the
 * threshold is ambiguous and sets OF_AMBIG.
 * ---------------------------------------------------------------------------------- */
static double ulp_at(double r, int mode) {
    double a = fabs(r);
    if (!isfinite(a)) return INFINITY;
    if (mode == ORACLE_FP32) {
        float f = (float)a;
        return (double)nextafterf(f, INFINITY) - (double)f;
    }
    return nextafter(a, INFINITY) - a;
}

static double run_case_bound(const uint8_t *ops, const float *cs, int32_t L, const float *x,
                             int64_t ldx, int mode, const double *dev_ulps, double *delta,
                             int *bad, int *ambig) {
    double st[ORACLE_STACK + 1], dt[ORACLE_STACK + 1];
    int sp = 0;
    const double big = big_limit(mode), tiny = tiny_limit(mode);
    const double own = mode == ORACLE_FP32 ? 0.5 : 1.0;
    for (int32_t j = 0; j < L; ++j) {
        int op = ops[j];
        double v, d;
        if (op == T_CONST || op >= T_LOAD0) {
            v = op == T_CONST ? (double)cs[j] : (double)x[(int64_t)(op - T_LOAD0) * ldx];
            st[sp] = v; dt[sp] = 0.0; ++sp;
            if (!(fabs(v) <= big)) *bad = 1;
            continue;
        } else if (op == T_DUP) {
            st[sp] = st[sp - 1]; dt[sp] = dt[sp - 1]; ++sp;
            continue;
        } else if (op == T_SWAP) {
            double t = st[sp - 1]; st[sp - 1] = st[sp - 2]; st[sp - 2] = t;
            t = dt[sp - 1]; dt[sp - 1] = dt[sp - 2]; dt[sp - 2] = t;
            continue;
        } else if (op == T_DEL) {
            --sp;
            continue;
        } else if (op <= T_PDIV) {
            double b = st[--sp], db = dt[sp];
            double a = st[--sp], da = dt[sp];
            switch (op) {
            case T_ADD: v = a + b; d = da + db; break;
            case T_SUB: v = a - b; d = da + db; break;
            case T_MUL: v = a * b; d = fabs(b) * da + fabs(a) * db + da * db; break;
            default:
                if (fabs(fabs(b) - tiny) <= db) *ambig = 1;
                if (fabs(b) > tiny) {
                    v = a / b;
                    d = db > 0.0 ? (fabs(b) > db ? (da + fabs(v) * db) / (fabs(b) - db)
                                                 : INFINITY)
                                 : da / fabs(b);
                } else {
                    v = 1.0; d = 0.0;
                }
                break;
            }
            v = round_to(v, mode);
            if (d > 0.0) d += ulp_at(v, mode);
        } else {
            double a = st[--sp], da = dt[sp];
            double u = dev_ulps[op] + own;
            switch (op) {
            case T_SIN: v = sin(a); d = da + u * ulp_at(round_to(v, mode), mode); break;
            case T_COS: v = cos(a); d = da + u * ulp_at(round_to(v, mode), mode); break;
            case T_EXP:
                v = exp(a);
                d = fabs(v) * expm1(da) + u * ulp_at(round_to(v, mode), mode);
                break;
            case T_PLOG:
                if (fabs(fabs(a) - tiny) <= da) *ambig = 1;
                if (fabs(a) > tiny) {
                    v = log(fabs(a));
                    d = (fabs(a) > da ? da / (fabs(a) - da) : INFINITY) +
                        u * ulp_at(round_to(v, mode), mode);
                } else {
                    v = 0.0; d = 0.0;
                }
                break;
            case T_PSQRT:
                v = sqrt(fabs(a));
                d = da > 0.0 ? sqrt(fabs(a) + da) - sqrt(fmax(fabs(a) - da, 0.0)) : 0.0;
                if (d > 0.0) d += ulp_at(round_to(v, mode), mode);
                break;
            default:   /* SQUARE */
                v = a * a;
                d = 2.0 * fabs(a) * da + da * da;
                if (d > 0.0) d += ulp_at(round_to(v, mode), mode);
                break;
            }
            v = round_to(v, mode);
        }
        if (!isfinite(d)) *ambig = 1;
        if (fabs(v) <= big && fabs(v) + d > big) *ambig = 1;
        if (!(fabs(v) <= big)) {
            if (isfinite(fabs(v)) && fabs(v) - d <= big) *ambig = 1;
            *bad = 1;
        }
        st[sp] = v; dt[sp] = d; ++sp;
    }
    *delta = dt[0];
    return st[0];
}

/* Per-case values, error bounds and flags of one program (see run_case_bound). */
uint32_t oracle_eval_bound(const uint8_t *ops, const float *cs, int32_t L, const float *X,
                           int64_t N, int32_t d, int32_t mode, const double *dev_ulps,
                           double *f, double *delta) {
    if (oracle_check_program(ops, L, d, ORACLE_STACK) != OE_OK) return OF_MALFORMED;
    uint32_t flags = 0;
    for (int64_t i = 0; i < N; ++i) {
        int bad = 0, ambig = 0;
        f[i] = run_case_bound(ops, cs, L, X + i, N, mode, dev_ulps, &delta[i], &bad, &ambig);
        if (bad) flags |= OF_INVALID;
        if (ambig) flags |= OF_AMBIG;
    }
    return flags;
}

/*
 * Bounds on the fitness a device may report, from the per-case bounds D_i:
 *   |SSE_dev - SSE| <= sum (2 |e_i| D_i + D_i^2)
 *   S_fy moves by at most A = sum D_i |y_i - ybar|, S_ff by at most
 *   B = sum (2 |f_i - fbar| D_i + D_i^2); r^2 = S_fy^2 / (S_ff S_yy) then stays within the
 *   interval given by the extreme corners.
 * A program whose output is constant keeps it constant on the device (every case runs the
 * same operations on the same values); its 1 - r^2 bound is 0. The fp64 rounding of the
 * aggregation (both sides aggregate in fp64) is added to the S_fy and S_ff bounds.
 */
void oracle_fitness_bound(const double *f, const double *delta, const float *y, int64_t N,
                          uint32_t flags, double *bmse, double *bomr2) {
    if (flags & (OF_INVALID | OF_MALFORMED)) { *bmse = 0.0; *bomr2 = 0.0; return; }
    nsum sy = {0, 0}, sf = {0, 0};
    int constant = 1;
    for (int64_t i = 0; i < N; ++i) {
        nadd(&sy, (double)y[i]);
        nadd(&sf, f[i]);
        if (f[i] != f[0]) constant = 0;
    }
    const double ybar = nval(&sy) / (double)N, fbar = nval(&sf) / (double)N;
    nsum be = {0, 0}, ba = {0, 0}, bb = {0, 0}, sff = {0, 0}, syy = {0, 0}, sfy = {0, 0};
    for (int64_t i = 0; i < N; ++i) {
        const double e = f[i] - (double)y[i], yc = (double)y[i] - ybar, fc = f[i] - fbar;
        const double D = delta[i];
        nadd(&be, 2.0 * fabs(e) * D + D * D);
        nadd(&ba, D * fabs(yc));
        nadd(&bb, 2.0 * fabs(fc) * D + D * D);
        nadd(&sff, fc * fc);
        nadd(&syy, yc * yc);
        nadd(&sfy, fc * yc);
    }
    *bmse = nval(&be) / (double)N;
    if (constant) { *bomr2 = 0.0; return; }
    /* Rounding of the aggregation itself, in fp64 on either side: the mean carries an error
     * of a few units of 2^-53 |f|, which moves S_ff by about N (u max|f|)^2 -- dominant
     * when the outputs vary only in their last bits -- and each sum by a few u of its
     * absolute terms. */
    const double u = ldexp(1.0, -53);
    double fmaxabs = 0.0, sfyabs = 0.0;
    for (int64_t i = 0; i < N; ++i) {
        fmaxabs = fmax(fmaxabs, fabs(f[i]));
        sfyabs += fabs(f[i] - fbar) * fabs((double)y[i] - ybar);
    }
    const double Sff0 = nval(&sff);
    const double A = nval(&ba) + 8.0 * u * sfyabs + 8.0 * u * fmaxabs * fabs(nval(&sy) - N * ybar);
    const double B = nval(&bb) + 8.0 * (double)N * (u * fmaxabs) * (u * fmaxabs) + 8.0 * u * Sff0;
    const double Sff = Sff0, Syy = nval(&syy);
    const double Sfy = fabs(nval(&sfy));
    if (!(Sff - B > 0.0)) { *bomr2 = INFINITY; return; }
    const double r2 = Sfy * Sfy / (Sff * Syy);
    const double hi = (Sfy + A) * (Sfy + A) / ((Sff - B) * Syy);
    const double lo_n = Sfy > A ? (Sfy - A) : 0.0;
    const double lo = lo_n * lo_n / ((Sff + B) * Syy);
    *bomr2 = fmax(hi - r2, r2 - lo);
}

/* Population version: values, flags and fitness bounds (one parallel loop over programs). */
int oracle_score_bound(const uint8_t *programs, const int64_t *offsets, const int32_t *lengths,
                       const float *consts, int64_t P, const float *X, const float *y,
                       int64_t N, int32_t d, int32_t mode, const double *dev_ulps,
                       int32_t nthreads, double *mse, double *omr2, uint32_t *flags,
                       double *bmse, double *bomr2) {
    if (N <= 0 || P < 0) return -1;
#ifdef _OPENMP
    if (nthreads <= 0) nthreads = omp_get_max_threads();
#pragma omp parallel num_threads(nthreads)
#endif
    {
        double *f = (double *)malloc(sizeof(double) * (size_t)N);
        double *dl = (double *)malloc(sizeof(double) * (size_t)N);
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 4)
#endif
        for (int64_t p = 0; p < P; ++p) {
            uint32_t fl = oracle_eval_bound(programs + offsets[p], consts + offsets[p],
                                            lengths[p], X, N, d, mode, dev_ulps, f, dl);
            oracle_aggregate(f, y, N, fl, &mse[p], &omr2[p], &flags[p]);
            oracle_fitness_bound(f, dl, y, N, fl, &bmse[p], &bomr2[p]);
        }
        free(f);
        free(dl);
    }
    return 0;
}
