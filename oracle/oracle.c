/*
 * oracle.c -- plain, slow reference scorer for Beagle population fitness.
 *
 * TEST INFRASTRUCTURE ONLY. Only the tests, the package's smoke check and the benchmark's
 * CPU-baseline leg load this file's library. It shares no code, header, table or constant
 * with the CUDA path; the token numbering below is the wire format, written out again here.
 *
 * What it computes (Beagle tutorial, arXiv 2607.06731):
 *   - Genomes are GCL programs in reverse Polish notation run on a value stack
 *     (the GCL section, Table 3). Unary ops replace the top; binary ops pop the top b and the
 *     element below it a, and push a (op) b: SUB is a - b, DIV is a / b (Table 3).
 *   - The stack holds at most 32 values (StackSize, the GCL section).
 *   - Each program runs on every fitness case and one aggregated fitness per program is
 *     returned ("Dividing Tasks Between CPU and GPU").
 *   - Fitness: mean squared error, and 1 - r^2 with r the Pearson correlation of Eq. 1
 *     ("Fitness Functions": the paper squares r).
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
    T_POW = 14, T_SIGN = 15, T_CUBE = 16, T_CBRT = 17, T_TAN = 18, T_ASIN = 19,
    T_ACOS = 20, T_ATAN = 21, T_TANH = 22,
    T_LOAD0 = 32, T_LOAD_END = 48,
    T_COPY0 = 64, T_COPY_END = 72, T_PASTE0 = 80, T_PASTE_END = 88
};
#define ORACLE_REGS 8       /* COPY/PASTE variables @0..@7 */

static int is_binary(int op) { return (op >= T_ADD && op <= T_PDIV) || op == T_POW; }
static int is_unary(int op) {
    return (op >= T_SIN && op <= T_SQUARE) || (op >= T_SIGN && op <= T_TANH);
}

enum { ORACLE_FP64 = 0, ORACLE_FP32 = 1 };

/* Result flags (same meaning as the library's, defined independently). */
#define OF_INVALID    1u    /* some value was non-finite or had |v| > 1e30 */
#define OF_DEGENERATE 2u    /* the program's output is the same on every case: r undefined */
#define OF_MALFORMED  4u    /* the token list is not a valid program */
#define OF_NEAR     256u    /* diagnostic: a value came within 1e-5 (relative) of a threshold */
#define OF_AMBIG    512u    /* error bound: a threshold or validity decision lies inside it */

#define ORACLE_STACK 32     /* StackSize (the GCL section) */

/* Error codes of the check function. */
#define OE_OK 0
#define OE_UNDERFLOW 1
#define OE_OVERFLOW 2
#define OE_FINAL_DEPTH 3
#define OE_OPCODE 4
#define OE_VAR 5
#define OE_EMPTY 6
#define OE_REGISTER 7

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
 * Structural check of one program (the GCL section): every token finds enough operands, the
 * stack never exceeds max_depth, variables exist (inputs are zero-based, Table 3 LOAD),
 * COPY and PASTE come in pairs -- COPY @k fills variable k, which must be empty, PASTE @k
 * empties it, which must be full, and every variable is empty at the end (Table 3: each COPY
 * corresponds to exactly one PASTE) -- and exactly one value remains (the program's output).
 */
int oracle_check_program(const uint8_t *ops, int32_t L, int32_t d, int32_t max_depth) {
    if (L <= 0) return OE_EMPTY;
    int depth = 0;
    int full[ORACLE_REGS] = {0};
    for (int32_t j = 0; j < L; ++j) {
        int op = ops[j], need, delta;
        if (op == T_CONST) { need = 0; delta = 1; }
        else if (op >= T_LOAD0 && op < T_LOAD_END) {
            if (op - T_LOAD0 >= d) return OE_VAR;
            need = 0; delta = 1;
        }
        else if (is_binary(op)) { need = 2; delta = -1; }
        else if (is_unary(op)) { need = 1; delta = 0; }
        else if (op == T_DUP) { need = 1; delta = 1; }
        else if (op == T_SWAP) { need = 2; delta = 0; }
        else if (op == T_DEL) { need = 1; delta = -1; }
        else if (op >= T_COPY0 && op < T_COPY_END) {
            if (full[op - T_COPY0]) return OE_REGISTER;
            full[op - T_COPY0] = 1;
            need = 1; delta = 0;
        }
        else if (op >= T_PASTE0 && op < T_PASTE_END) {
            if (!full[op - T_PASTE0]) return OE_REGISTER;
            full[op - T_PASTE0] = 0;
            need = 0; delta = 1;
        }
        else return OE_OPCODE;
        if (depth < need) return OE_UNDERFLOW;
        depth += delta;
        if (depth > max_depth) return OE_OVERFLOW;
    }
    for (int k = 0; k < ORACLE_REGS; ++k)
        if (full[k]) return OE_REGISTER;
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
    double st[ORACLE_STACK + 1], reg[ORACLE_REGS];
    int sp = 0;
    const double big = big_limit(mode), tiny = tiny_limit(mode);
    for (int32_t j = 0; j < L; ++j) {
        int op = ops[j];
        double v;
        if (op == T_CONST) {
            v = (double)cs[j];
            st[sp++] = v;
        } else if (op >= T_COPY0 && op < T_COPY_END) {   /* the stack is unchanged */
            reg[op - T_COPY0] = st[sp - 1];
            continue;
        } else if (op >= T_PASTE0 && op < T_PASTE_END) {  /* a value checked when made */
            st[sp++] = reg[op - T_PASTE0];
            continue;
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
        } else if (is_binary(op)) {
            double b = st[--sp];
            double a = st[--sp];
            switch (op) {
            case T_ADD: v = a + b; break;
            case T_SUB: v = a - b; break;
            case T_MUL: v = a * b; break;
            case T_POW: v = pow(a, b); break;   /* second ^ top; unprotected (reading) */
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
            case T_SIGN: v = -a; break;   /* "changes the sign" */
            case T_CUBE: v = round_to(a * a, mode) * a; break;   /* (a a) a, each rounded */
            case T_CBRT: v = cbrt(a); break;
            case T_TAN: v = tan(a); break;
            case T_ASIN:   /* unprotected: NaN (invalid) outside [-1, 1] */
                if (near_to(a, 1.0)) *near = 1;
                v = asin(a);
                break;
            case T_ACOS:
                if (near_to(a, 1.0)) *near = 1;
                v = acos(a);
                break;
            case T_ATAN: v = atan(a); break;
            case T_TANH: v = tanh(a); break;
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
 * Aggregate outputs f against targets y ("Fitness Functions").
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

/* Largest change of a monotone function g over [a - da, a + da] (g increasing or
 * decreasing there): |g(a + da) - g(a - da)|. */
static double mono_spread(double (*g)(double), double a, double da) {
    return fabs(g(a + da) - g(a - da));
}

static double run_case_bound(const uint8_t *ops, const float *cs, int32_t L, const float *x,
                             int64_t ldx, int mode, const double *dev_ulps, double *delta,
                             int *bad, int *ambig) {
    double st[ORACLE_STACK + 1], dt[ORACLE_STACK + 1], reg[ORACLE_REGS], rdt[ORACLE_REGS];
    int sp = 0;
    const double big = big_limit(mode), tiny = tiny_limit(mode);
    const double own = mode == ORACLE_FP32 ? 0.5 : 1.0;
    for (int32_t j = 0; j < L; ++j) {
        int op = ops[j];
        double v, d;
        if (op >= T_COPY0 && op < T_COPY_END) {
            reg[op - T_COPY0] = st[sp - 1]; rdt[op - T_COPY0] = dt[sp - 1];
            continue;
        } else if (op >= T_PASTE0 && op < T_PASTE_END) {
            st[sp] = reg[op - T_PASTE0]; dt[sp] = rdt[op - T_PASTE0]; ++sp;
            continue;
        } else if (op == T_CONST || (op >= T_LOAD0 && op < T_LOAD_END)) {
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
        } else if (is_binary(op)) {
            double b = st[--sp], db = dt[sp];
            double a = st[--sp], da = dt[sp];
            switch (op) {
            case T_ADD: v = a + b; d = da + db; break;
            case T_SUB: v = a - b; d = da + db; break;
            case T_MUL: v = a * b; d = fabs(b) * da + fabs(a) * db + da * db; break;
            case T_POW: {
                /* first order in both operands: |b a^(b-1)| da + |a^b ln a| db; a perturbed
                 * base at or below zero, or a perturbed exponent of a negative base, can
                 * leave the domain: ambiguous */
                v = pow(a, b);
                if ((da > 0.0 && fabs(a) <= da) || (db > 0.0 && a < 0.0)) *ambig = 1;
                d = (da > 0.0 ? fabs(b * pow(a, b - 1.0)) * da : 0.0) +
                    (db > 0.0 ? fabs(v * log(fabs(a))) * db : 0.0);
                d += (dev_ulps[op] + own) * ulp_at(round_to(v, mode), mode);
                break;
            }
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
            if (d > 0.0 && op != T_POW) d += ulp_at(v, mode);
        } else {
            double a = st[--sp], da = dt[sp];
            double u = dev_ulps[op] + own;
            switch (op) {
            case T_SIGN: v = -a; d = da; break;
            case T_CUBE: {
                const double a2 = round_to(a * a, mode);
                v = a2 * a;
                d = da > 0.0 ? 3.0 * a * a * da + 3.0 * fabs(a) * da * da + da * da * da +
                               fabs(a) * ulp_at(a2, mode) : 0.0;
                if (d > 0.0) d += ulp_at(round_to(v, mode), mode);
                break;
            }
            case T_CBRT: v = cbrt(a); d = mono_spread(cbrt, a, da) + u * ulp_at(round_to(v, mode), mode); break;
            case T_TAN: {
                v = tan(a);
                /* a pole of tan inside [a - da, a + da] makes the value unbounded */
                const double pi = acos(-1.0);
                const double k0 = floor((a - da) / pi - 0.5), k1 = floor((a + da) / pi - 0.5);
                if (da > 0.0 && k0 != k1) { d = INFINITY; break; }
                d = mono_spread(tan, a, da) + u * ulp_at(round_to(v, mode), mode);
                break;
            }
            case T_ASIN:
            case T_ACOS:
                v = op == T_ASIN ? asin(a) : acos(a);
                if (fabs(a) <= 1.0 && fabs(a) + da > 1.0) *ambig = 1;   /* domain edge */
                d = fabs(a) + da <= 1.0 ? mono_spread(op == T_ASIN ? asin : acos, a, da) : 0.0;
                d += u * ulp_at(round_to(v, mode), mode);
                break;
            case T_ATAN: v = atan(a); d = da + u * ulp_at(round_to(v, mode), mode); break;
            case T_TANH: v = tanh(a); d = da + u * ulp_at(round_to(v, mode), mode); break;
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


/* ------------------------------------------------------------------------------------
 * The paper's own fitness functions ("Fitness Functions" in the overview and in the
 * configuration section, Eqs. 1-5; "Creating Custom Fit Functions"). Unlike the MSE / 1 - r^2
 * pair above, these judge every fitness case on its own: a case whose evaluation produced an
 * invalid value (non-finite or |v| > 1e30, the rule above, applied per case) is an invalid
 * model output, and a target that is non-finite or above 1e30 is an invalid target.
 *
 * Kinds:
 *   OFIT_CORRELATION  Eq. 1 over the valid pairs (both output and target valid), then Eq. 2:
 *                     score = M r^4 (N - (c1 + c2)) - M (c1 - c2), c1 = pairs with exactly one
 *                     invalid member, c2 = pairs with both invalid. Reading: r := 0 when it is
 *                     undefined (fewer than one valid pair, constant outputs or constant
 *                     targets over the valid pairs; flag DEGENERATE).
 *   OFIT_STD*         Eq. 5 per case, summed: q = min(|f|,|y|) / max(|f|,|y|); M when both are
 *                     0; round(M q^k - M/11) when f and y have opposite signs (f y < 0);
 *                     round(M q^k) otherwise. k = 1, 2, 3,
 *                     8 for StdFitFunc, StdSquareFitFunc, StdCubeFitFunc, StdHyperFitFunc
 *                     (reading: the power applies to the ratio, so the best case still earns
 *                     M). Invalid pairs (FitFunctionIfInvalid, reading): +M when both are
 *                     invalid, -M when exactly one is, as Eq. 2 treats c2 and c1. round() is
 *                     to nearest, ties to even, in the path's own precision.
 *   OFIT_VALIDATE     the interactive V command's test: a case passes when output and target
 *                     are valid and |f - y| <= 0.001 |y| (computed in double); score = number
 *                     of passing cases; flag PERFECT when every case passes.
 * asr = score / (M N) (the average score ratio of the sample run output; for VALIDATE
 * score / N). The length tax (ScriptLengthTaxRateInternal): taxed = score - tax * L.
 * ---------------------------------------------------------------------------------- */
enum { OFIT_MSE_R2 = 0, OFIT_CORRELATION = 1, OFIT_STD = 2, OFIT_STD_SQUARE = 3,
       OFIT_STD_CUBE = 4, OFIT_STD_HYPER = 5, OFIT_VALIDATE = 6 };
#define OF_PERFECT 16u

/* Per-case outputs and per-case validity of one program (bad[i] = 1: case i invalid). */
uint32_t oracle_eval_cases(const uint8_t *ops, const float *cs, int32_t L, const float *X,
                           int64_t N, int32_t d, int32_t mode, double *f, uint8_t *bad) {
    if (oracle_check_program(ops, L, d, ORACLE_STACK) != OE_OK) return OF_MALFORMED;
    uint32_t flags = 0;
    for (int64_t i = 0; i < N; ++i) {
        int b = 0, near = 0;
        f[i] = run_case(ops, cs, L, X + i, N, mode, &b, &near);
        bad[i] = (uint8_t)b;
        if (near) flags |= OF_NEAR;
    }
    return flags;
}

static int target_valid(float y) { return fabs((double)y) <= 1e30; }   /* NaN fails */

/* Eq. 5's "f y < 0", read as: the two are nonzero with opposite signs (the product itself
 * could underflow to zero in fp32). */
static int opposite_signs(double a, double b) { return (a < 0.0 && b > 0.0) || (a > 0.0 && b < 0.0); }

/* Eq. 5 reward of one valid pair, in the path's precision (mode). */
static int64_t std_reward(double fo, float yo, int32_t k, int32_t M, int mode) {
    if (mode == ORACLE_FP32) {
        float a = fabsf((float)fo), b = fabsf(yo);
        float mx = a > b ? a : b, mn = a > b ? b : a;
        if (mx == 0.0f) return M;
        float q = mn / mx, qk = q;
        if (k == 2) qk = q * q;
        else if (k == 3) { qk = q * q; qk = qk * q; }
        else if (k == 8) { qk = q * q; qk = qk * qk; qk = qk * qk; }
        float v = (float)M * qk;
        if (opposite_signs(fo, (double)yo)) v = v - (float)M / 11.0f;
        return (int64_t)rintf(v);
    } else {
        double a = fabs(fo), b = fabs((double)yo);
        double mx = a > b ? a : b, mn = a > b ? b : a;
        if (mx == 0.0) return M;
        double q = mn / mx, qk = q;
        if (k == 2) qk = q * q;
        else if (k == 3) { qk = q * q; qk = qk * q; }
        else if (k == 8) { qk = q * q; qk = qk * qk; qk = qk * qk; }
        double v = (double)M * qk;
        if (opposite_signs(fo, (double)yo)) v = v - (double)M / 11.0;
        return (int64_t)rint(v);
    }
}

/* Fitness of one program from its per-case outputs and validity. out[0] score, out[1] asr,
 * out[2] r^2, out[3] taxed score; cnt[0] c1, cnt[1] c2. */
void oracle_fit_aggregate(const double *f, const uint8_t *bad, const float *y, int64_t N,
                          uint32_t flags, int32_t kind, int32_t M, int32_t mode, double tax,
                          int32_t L, double *out, int64_t *cnt, uint32_t *flags_out) {
    out[0] = out[1] = out[2] = out[3] = 0.0;
    cnt[0] = cnt[1] = 0;
    if (flags & OF_MALFORMED) {
        out[0] = out[1] = out[3] = -INFINITY;
        *flags_out = flags;
        return;
    }
    int64_t c1 = 0, c2 = 0, n = 0;
    for (int64_t i = 0; i < N; ++i) {
        const int fv = !bad[i], tv = target_valid(y[i]);
        if (fv != tv) ++c1;
        else if (!fv) ++c2;
        else ++n;
    }
    cnt[0] = c1;
    cnt[1] = c2;
    double score = 0.0;
    if (kind == OFIT_CORRELATION) {
        /* Eq. 1 over the valid pairs: means, then centred sums (Neumaier). */
        double r = 0.0;
        if (n > 0) {
            nsum sf = {0, 0}, sy = {0, 0};
            int64_t first = -1;
            int fconst = 1, yconst = 1;   /* every valid pair has the same output / target */
            for (int64_t i = 0; i < N; ++i)
                if (!bad[i] && target_valid(y[i])) {
                    nadd(&sf, f[i]);
                    nadd(&sy, (double)y[i]);
                    if (first < 0) first = i;
                    if (f[i] != f[first]) fconst = 0;
                    if (y[i] != y[first]) yconst = 0;
                }
            const double fbar = nval(&sf) / (double)n, ybar = nval(&sy) / (double)n;
            nsum sff = {0, 0}, syy = {0, 0}, sfy = {0, 0};
            for (int64_t i = 0; i < N; ++i) {
                if (bad[i] || !target_valid(y[i])) continue;
                const double a = f[i] - fbar, b = (double)y[i] - ybar;
                nadd(&sff, a * a);
                nadd(&syy, b * b);
                nadd(&sfy, a * b);
            }
            if (!fconst && !yconst && nval(&sff) > 0.0 && nval(&syy) > 0.0)
                r = nval(&sfy) / sqrt(nval(&sff) * nval(&syy));
            else
                flags |= OF_DEGENERATE;
        } else {
            flags |= OF_DEGENERATE;
        }
        const double r2 = r * r;
        score = (double)M * r2 * r2 * (double)(N - (c1 + c2)) - (double)M * (double)(c1 - c2);
        out[2] = r2;
        out[1] = score / ((double)M * (double)N);
    } else if (kind >= OFIT_STD && kind <= OFIT_STD_HYPER) {
        const int32_t k = kind == OFIT_STD ? 1 : kind == OFIT_STD_SQUARE ? 2 :
                          kind == OFIT_STD_CUBE ? 3 : 8;
        int64_t total = 0;
        for (int64_t i = 0; i < N; ++i) {
            const int fv = !bad[i], tv = target_valid(y[i]);
            if (fv && tv) total += std_reward(f[i], y[i], k, M, mode);
            else total += (fv || tv) ? -(int64_t)M : (int64_t)M;
        }
        score = (double)total;
        out[1] = score / ((double)M * (double)N);
    } else if (kind == OFIT_VALIDATE) {
        int64_t pass = 0;
        for (int64_t i = 0; i < N; ++i) {
            if (bad[i] || !target_valid(y[i])) continue;
            if (fabs(f[i] - (double)y[i]) <= 0.001 * fabs((double)y[i])) ++pass;
        }
        score = (double)pass;
        out[1] = score / (double)N;
        if (pass == N) flags |= OF_PERFECT;
    }
    out[0] = score;
    out[3] = score - tax * (double)L;
    *flags_out = flags;
}

/* Population version of the paper's fitness functions (one parallel loop over programs).
 * out: [P][4] (score, asr, r^2, taxed); cnt: [P][2] (c1, c2). tax < 0: M N / 85. */
int oracle_fit_score(const uint8_t *programs, const int64_t *offsets, const int32_t *lengths,
                     const float *consts, int64_t P, const float *X, const float *y, int64_t N,
                     int32_t d, int32_t mode, int32_t kind, int32_t M, double tax,
                     int32_t nthreads, double *out, int64_t *cnt, uint32_t *flags) {
    if (N <= 0 || P < 0 || M <= 0 || kind < OFIT_CORRELATION || kind > OFIT_VALIDATE) return -1;
    if (tax < 0.0) tax = (double)M * (double)N / 85.0;
#ifdef _OPENMP
    if (nthreads <= 0) nthreads = omp_get_max_threads();
#pragma omp parallel num_threads(nthreads)
#endif
    {
        double *f = (double *)malloc(sizeof(double) * (size_t)N);
        uint8_t *bad = (uint8_t *)malloc((size_t)N);
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 4)
#endif
        for (int64_t p = 0; p < P; ++p) {
            uint32_t fl = oracle_eval_cases(programs + offsets[p], consts + offsets[p],
                                            lengths[p], X, N, d, mode, f, bad);
            oracle_fit_aggregate(f, bad, y, N, fl, kind, M, mode, tax, lengths[p],
                                 out + 4 * p, cnt + 2 * p, &flags[p]);
        }
        free(f);
        free(bad);
    }
    return 0;
}


/* ------------------------------------------------------------------------------------
 * Monte-Carlo ranking (the overview's section of that name, Table 2): instead of sorting the
 * population, a random sample of 100 individuals estimates its percentiles, and one pass
 * assigns every individual its percentile group and breeding rights whose expected number of
 * children per group is Table 2's.
 * Readings: key[p] ranks individual p, higher is better; a NaN key ranks below every other.
 * The sample's keys, sorted ascending, give the thresholds t_q = sorted[q] for q = 10, 20,
 * ..., 90 (the q-th order statistic of the 100, the q-th percentile's estimate); individual
 * p's group g = the number of thresholds with key[p] >= t_q (g = 9: the >= 90th percentile
 * row). Children of p: floor(E_g) plus one when u[p] < E_g - floor(E_g), u[p] a uniform number
 * in [0, 1) the caller draws (the method's randomness is an input).
 * ---------------------------------------------------------------------------------- */
static const double kTable2Children[10] = {0.01, 0.03, 0.06, 0.15, 0.25, 0.5, 1.0, 1.5, 2.5, 4.0};

static int cmp_key(const void *a, const void *b) {
    double x = *(const double *)a, y = *(const double *)b;
    int nx = isnan(x), ny = isnan(y);
    if (nx || ny) return nx - ny > 0 ? -1 : (nx == ny ? 0 : 1);   /* NaN first (lowest) */
    return x < y ? -1 : (x > y ? 1 : 0);
}

int oracle_rank(const double *key, int64_t P, const int64_t *sample, int32_t n_sample,
                const float *u, uint8_t *group, int32_t *children) {
    if (P < 0 || n_sample != 100) return -1;
    double s[100];
    for (int i = 0; i < 100; ++i) {
        if (sample[i] < 0 || sample[i] >= P) return -1;
        s[i] = key[sample[i]];
    }
    qsort(s, 100, sizeof(double), cmp_key);
    for (int64_t p = 0; p < P; ++p) {
        int g = 0;
        if (!isnan(key[p]))
            for (int q = 10; q <= 90; q += 10)
                if (!isnan(s[q]) && key[p] >= s[q]) ++g;
        group[p] = (uint8_t)g;
        const double e = kTable2Children[g], fl = floor(e);
        children[p] = (int32_t)fl + ((double)u[p] < e - fl ? 1 : 0);
    }
    return 0;
}
