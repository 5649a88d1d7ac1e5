// Interpreter loop for the FP32 path with 8 cases per lane (256 cases per pass): the threaded
// inline-PTX interpreter of interp_ptx.cuh on twice the cases per dispatch, with the value
// arithmetic in Blackwell's paired FP32 instructions (add/sub/mul/fma .rn.f32x2: two IEEE
// single-precision operations in one instruction, each rounded to nearest like its scalar
// form, so the results are bit-identical to the 4-case loop's).
//
// Lane l holds cases 4l..4l+3 (half 0) and 128+4l..128+4l+3 (half 1) of the pass: the pairs
// %0 = (4l, 4l+1), %1 = (4l+2, 4l+3), %2 and %3 the same in half 1. Input row k of the staged
// box is kBox floats (1 KB) further; half 1 is 128 floats into the row, so each half is one
// 16-byte load per lane, 512 contiguous bytes across the warp.
//
// The stack rows below the top live in tensor memory (TMEM): row r of the warp is the 8
// columns base + 8 r of its 32-lane quarter, register j of the top in column j. 15 rows take
// 120 of the warp's 128 columns, so 16 warps fill the SM's 512 columns x 4 quarters. A row
// load waits for the warp's earlier row stores and for itself before its values are used.
//
// Semantics are those of run_program in score.cuh, handler for handler: the same fp32
// operations in the same order, the same protected division and square root (Markstein's
// quotient rounded to nearest), the same validity decisions (results of psqrt, sin, cos and
// the protected log of valid operands are bounded, so they are not tracked). sin, cos, exp,
// the protected log, POW and the rest of Table 3's transcendentals leave the loop with their
// handler id; the caller applies them to the eight top values and re-enters.
#pragma once

#include "interp_ptx.cuh"
#include "score.cuh"

namespace beagle {

// The 8 top values as scalars t0..t7 (the pairs' halves: no data movement) and back.
#define BG8_UNPACK                                                                         \
    "mov.b64 {t0, t1}, %0;\n\tmov.b64 {t2, t3}, %1;\n\t"                                   \
    "mov.b64 {t4, t5}, %2;\n\tmov.b64 {t6, t7}, %3;\n\t"
#define BG8_PACK                                                                           \
    "mov.b64 %0, {t0, t1};\n\tmov.b64 %1, {t2, t3};\n\t"                                   \
    "mov.b64 %2, {t4, t5};\n\tmov.b64 %3, {t6, t7};\n\t"
// Validity tracker of one case: m = max.NaN(m, |t|).
#define BG8_TRK(T, M) "abs.f32 z, " T ";\n\tmax.NaN.f32 " M ", " M ", z;\n\t"
#define BG8_TRACK8                                                                         \
    BG8_UNPACK BG8_TRK("t0", "%4") BG8_TRK("t1", "%5") BG8_TRK("t2", "%6")                 \
    BG8_TRK("t3", "%7") BG8_TRK("t4", "%8") BG8_TRK("t5", "%9") BG8_TRK("t6", "%10")       \
    BG8_TRK("t7", "%11")
// Apply a paired operation to the four pairs: OP4(OP, "a", "b") gives OP %k, a(k), b(k).
#define BG8_PAIRS_TT(OP) OP " %0, %0, %0;\n\t" OP " %1, %1, %1;\n\t" OP " %2, %2, %2;\n\t" OP " %3, %3, %3;\n\t"
#define BG8_PAIRS_TA(OP) OP " %0, %0, A01;\n\t" OP " %1, %1, A23;\n\t" OP " %2, %2, A45;\n\t" OP " %3, %3, A67;\n\t"
#define BG8_PAIRS_AT(OP) OP " %0, A01, %0;\n\t" OP " %1, A23, %1;\n\t" OP " %2, A45, %2;\n\t" OP " %3, A67, %3;\n\t"
// Protected division of one pair, DST = |DEN| > 1e-3 ? NUM / DEN : 1 per half: y = rcp.approx
// refined by one Newton step to the correctly rounded 1/den, w = num y, then w + (num - den w) y
// with the remainder exact by FMA (the steps of Arith<float>::pdiv), the FMA steps paired.
#define BG8_PDIV2(DST, NUM, DEN)                                                           \
    "mov.b64 {d0, d1}, " DEN ";\n\t"                                                       \
    "abs.f32 z, d0;\n\tsetp.gt.f32 q0, z, 0f3A83126F;\n\t"                                 \
    "abs.f32 z, d1;\n\tsetp.gt.f32 q1, z, 0f3A83126F;\n\t"                                 \
    "rcp.approx.ftz.f32 d0, d0;\n\trcp.approx.ftz.f32 d1, d1;\n\tmov.b64 Y, {d0, d1};\n\t"  \
    "mul.rn.f32x2 ND, " DEN ", M1;\n\t"                                                     \
    "fma.rn.f32x2 E, ND, Y, ONE;\n\tfma.rn.f32x2 Y, E, Y, Y;\n\t"                           \
    "mul.rn.f32x2 Z, " NUM ", Y;\n\tfma.rn.f32x2 E, ND, Z, " NUM ";\n\t"                     \
    "fma.rn.f32x2 Z, E, Y, Z;\n\t"                                                          \
    "mov.b64 {d0, d1}, Z;\n\tselp.f32 d0, d0, 0f3F800000, q0;\n\t"                          \
    "selp.f32 d1, d1, 0f3F800000, q1;\n\tmov.b64 " DST ", {d0, d1};\n\t"
// Operands: %0-%3 top of stack (4 pairs), %4-%11 validity trackers, %12/%13 current token
// words, %14 shared address of the next token, %15 exit code (0 = program done, else the
// handler id of the operator the caller applies), %16 shared address of this lane's first
// case of input row 0, %17 tensor-memory address of the warp's stack row 0.
// Threaded dispatch as in the 4-case loop: the next token's handler id is in bits 24-28 of
// the current token, so the indexed branch does not wait for the load it covers.
#define BG8_DISPATCH                                                                       \
    "shr.b32 h, %12, 24;\n\t"                                                              \
    "ld.shared.v2.u32 {%12, %13}, [%14];\n\t"                                              \
    "add.u32 %14, %14, 8;\n\t"                                                             \
    "brx.idx.uni h, TBL_%=;\n"
#define BG8_ROW "bfe.u32 v, %12, 12, 8;\n\tmad.lo.u32 rp, v, 8, %17;\n\t"
#define BG8_XA "bfe.u32 v, %12, 8, 4;\n\tmad.lo.u32 xa, v, 1024, %16;\n\t"
#define BG8_C2 "mov.b64 C2, {%13, %13};\n\t"
#define BG8_STROW                                                                          \
    BG8_UNPACK "tcgen05.st.sync.aligned.32x32b.x8.b32 [rp], {t0, t1, t2, t3, t4, t5, t6, t7};\n\t"
#define BG8_LDROW(R)                                                                       \
    "tcgen05.wait::st.sync.aligned;\n\t"                                                   \
    "tcgen05.ld.sync.aligned.32x32b.x8.b32 {" R "0, " R "1, " R "2, " R "3, " R "4, " R "5, " \
    R "6, " R "7}, [rp];\n\t"                                                              \
    "tcgen05.wait::ld.sync.aligned;\n\t"
#define BG8_LDROW_A                                                                        \
    BG8_LDROW("a")                                                                         \
    "mov.b64 A01, {a0, a1};\n\tmov.b64 A23, {a2, a3};\n\t"                                 \
    "mov.b64 A45, {a4, a5};\n\tmov.b64 A67, {a6, a7};\n\t"
#define BG8_LDROW_T BG8_LDROW("t") BG8_PACK
#define BG8_LDX_A "ld.shared.v2.b64 {A01, A23}, [xa];\n\tld.shared.v2.b64 {A45, A67}, [xa+512];\n\t"
#define BG8_LDX_T "ld.shared.v2.b64 {%0, %1}, [xa];\n\tld.shared.v2.b64 {%2, %3}, [xa+512];\n\t"
#define BG8_EXIT(L, CODE) L "_%=:\n\tmov.u32 %15, " #CODE ";\n\tbra.uni OUT_%=;\n"

#define BG_PTX_INTERP8                                                                     \
    "{\n\t"                                                                                \
    ".reg .pred q0, q1;\n\t"                                                               \
    ".reg .b32 h, v, rp, xa;\n\t"                                                          \
    ".reg .b64 A01, A23, A45, A67, C2, S2, Y, ND, E, Z, ONE, M1;\n\t"                       \
    ".reg .f32 t0, t1, t2, t3, t4, t5, t6, t7, a0, a1, a2, a3, a4, a5, a6, a7, z, d0, d1;\n\t" \
    "TBL_%=: .branchtargets PUSHX_%=, PUSHC_%=, DUP_%=, SWAP_%=, DEL_%=, ADDSUB_%=, "      \
    "MUL_%=, PDIV_%=, SIN_%=, COS_%=, EXP_%=, PLOG_%=, PSQRT_%=, SQUARE_%=, ADDSUBX_%=, "   \
    "MULX_%=, PDIVX_%=, ADDC_%=, MULC_%=, PDIVC_%=, END_%=, POW_%=, SIGN_%=, CUBE_%=, "     \
    "CBRT_%=, TAN_%=, ASIN_%=, ACOS_%=, ATAN_%=, TANH_%=, PASTE_%=, END_%=;\n\t"           \
    "mov.b64 ONE, 0x3F8000003F800000;\n\tmov.b64 M1, 0xBF800000BF800000;\n\t"              \
    BG8_DISPATCH                                                                           \
    "PUSHX_%=:\n\t" BG8_ROW BG8_XA BG8_STROW BG8_LDX_T BG8_DISPATCH                        \
    "PUSHC_%=:\n\t" BG8_ROW BG8_STROW                                                      \
    "mov.b64 %0, {%13, %13};\n\tmov.b64 %1, %0;\n\tmov.b64 %2, %0;\n\tmov.b64 %3, %0;\n\t" \
    BG8_DISPATCH                                                                           \
    "DUP_%=:\n\t" BG8_ROW BG8_STROW BG8_DISPATCH                                           \
    "SWAP_%=:\n\t" BG8_ROW BG8_LDROW_A BG8_STROW                                           \
    "mov.b64 %0, A01;\n\tmov.b64 %1, A23;\n\tmov.b64 %2, A45;\n\tmov.b64 %3, A67;\n\t"     \
    BG8_DISPATCH                                                                           \
    "DEL_%=:\n\t" BG8_ROW BG8_LDROW_T BG8_DISPATCH                                         \
    /* top = s top + a: a +- top with s = +-1, rounded once like an add or a subtraction */ \
    "ADDSUB_%=:\n\t" BG8_ROW "mov.b64 S2, {%13, %13};\n\t" BG8_LDROW_A                      \
    "fma.rn.f32x2 %0, S2, %0, A01;\n\tfma.rn.f32x2 %1, S2, %1, A23;\n\t"                   \
    "fma.rn.f32x2 %2, S2, %2, A45;\n\tfma.rn.f32x2 %3, S2, %3, A67;\n\t"                   \
    BG8_TRACK8 BG8_DISPATCH                                                                \
    "MUL_%=:\n\t" BG8_ROW BG8_LDROW_A BG8_PAIRS_AT("mul.rn.f32x2") BG8_TRACK8 BG8_DISPATCH \
    "PDIV_%=:\n\t" BG8_ROW BG8_LDROW_A                                                     \
    BG8_PDIV2("%0", "A01", "%0") BG8_PDIV2("%1", "A23", "%1")                              \
    BG8_PDIV2("%2", "A45", "%2") BG8_PDIV2("%3", "A67", "%3")                              \
    BG8_TRACK8 BG8_DISPATCH                                                                \
    BG8_EXIT("SIN", 8) BG8_EXIT("COS", 9) BG8_EXIT("EXP", 10) BG8_EXIT("PLOG", 11)         \
    "PSQRT_%=:\n\t" BG8_UNPACK                                                             \
    "abs.f32 t0, t0;\n\tsqrt.rn.f32 t0, t0;\n\tabs.f32 t1, t1;\n\tsqrt.rn.f32 t1, t1;\n\t" \
    "abs.f32 t2, t2;\n\tsqrt.rn.f32 t2, t2;\n\tabs.f32 t3, t3;\n\tsqrt.rn.f32 t3, t3;\n\t" \
    "abs.f32 t4, t4;\n\tsqrt.rn.f32 t4, t4;\n\tabs.f32 t5, t5;\n\tsqrt.rn.f32 t5, t5;\n\t" \
    "abs.f32 t6, t6;\n\tsqrt.rn.f32 t6, t6;\n\tabs.f32 t7, t7;\n\tsqrt.rn.f32 t7, t7;\n\t" \
    BG8_PACK BG8_DISPATCH                                                                  \
    "SQUARE_%=:\n\t" BG8_PAIRS_TT("mul.rn.f32x2") BG8_TRACK8 BG8_DISPATCH                   \
    /* fused leaf + binary operator: top = s x + top; top + c (c negated for a subtraction) */ \
    "ADDSUBX_%=:\n\t" BG8_XA "mov.b64 S2, {%13, %13};\n\t" BG8_LDX_A                        \
    "fma.rn.f32x2 %0, S2, A01, %0;\n\tfma.rn.f32x2 %1, S2, A23, %1;\n\t"                   \
    "fma.rn.f32x2 %2, S2, A45, %2;\n\tfma.rn.f32x2 %3, S2, A67, %3;\n\t"                   \
    BG8_TRACK8 BG8_DISPATCH                                                                \
    "ADDC_%=:\n\t" BG8_C2                                                                  \
    "add.rn.f32x2 %0, %0, C2;\n\tadd.rn.f32x2 %1, %1, C2;\n\t"                             \
    "add.rn.f32x2 %2, %2, C2;\n\tadd.rn.f32x2 %3, %3, C2;\n\t"                             \
    BG8_TRACK8 BG8_DISPATCH                                                                \
    "MULX_%=:\n\t" BG8_XA BG8_LDX_A BG8_PAIRS_TA("mul.rn.f32x2") BG8_TRACK8 BG8_DISPATCH    \
    "MULC_%=:\n\t" BG8_C2                                                                  \
    "mul.rn.f32x2 %0, %0, C2;\n\tmul.rn.f32x2 %1, %1, C2;\n\t"                             \
    "mul.rn.f32x2 %2, %2, C2;\n\tmul.rn.f32x2 %3, %3, C2;\n\t"                             \
    BG8_TRACK8 BG8_DISPATCH                                                                \
    /* fused division by an input or a constant: one shared copy of the divisions */       \
    "PDIVX_%=:\n\t" BG8_XA BG8_LDX_A "bra.uni DIVTA_%=;\n"                                  \
    "PDIVC_%=:\n\t" "mov.b64 A01, {%13, %13};\n\tmov.b64 A23, A01;\n\t"                      \
    "mov.b64 A45, A01;\n\tmov.b64 A67, A01;\n"                                             \
    "DIVTA_%=:\n\t"                                                                         \
    BG8_PDIV2("%0", "%0", "A01") BG8_PDIV2("%1", "%1", "A23")                              \
    BG8_PDIV2("%2", "%2", "A45") BG8_PDIV2("%3", "%3", "A67")                              \
    BG8_TRACK8 BG8_DISPATCH                                                                \
    /* the rest of Table 3: SIGN (|v| unchanged, nothing to track), CUBE ((a a) a), PASTE */ \
    /* (push the top, load the register's row, its index in the constant word) */          \
    BG8_EXIT("POW", 21)                                                                    \
    "SIGN_%=:\n\t" "mul.rn.f32x2 %0, %0, M1;\n\tmul.rn.f32x2 %1, %1, M1;\n\t"               \
    "mul.rn.f32x2 %2, %2, M1;\n\tmul.rn.f32x2 %3, %3, M1;\n\t" BG8_DISPATCH                \
    "CUBE_%=:\n\t"                                                                         \
    "mul.rn.f32x2 A01, %0, %0;\n\tmul.rn.f32x2 A23, %1, %1;\n\t"                           \
    "mul.rn.f32x2 A45, %2, %2;\n\tmul.rn.f32x2 A67, %3, %3;\n\t"                           \
    BG8_PAIRS_AT("mul.rn.f32x2") BG8_TRACK8 BG8_DISPATCH                                   \
    BG8_EXIT("CBRT", 24) BG8_EXIT("TAN", 25) BG8_EXIT("ASIN", 26) BG8_EXIT("ACOS", 27)     \
    BG8_EXIT("ATAN", 28) BG8_EXIT("TANH", 29)                                              \
    "PASTE_%=:\n\t" BG8_ROW BG8_STROW "mad.lo.u32 rp, %13, 8, %17;\n\t" BG8_LDROW_T          \
    BG8_DISPATCH                                                                           \
    "END_%=:\n\tmov.u32 %15, 0;\n"                                                         \
    "OUT_%=:\n\t"                                                                          \
    "}"

static_assert(H_PUSHX == 0 && H_PUSHC == 1 && H_DUP == 2 && H_SWAP == 3 && H_DEL == 4 &&
                  H_ADDSUB == 5 && H_MUL == 6 && H_PDIV == 7 && H_SIN == 8 && H_COS == 9 &&
                  H_EXP == 10 && H_PLOG == 11 && H_PSQRT == 12 && H_SQUARE == 13 &&
                  H_ADDSUBX == 14 && H_MULX == 15 && H_PDIVX == 16 && H_ADDC == 17 &&
                  H_MULC == 18 && H_PDIVC == 19 && H_END == 20 && H_POW == 21 &&
                  H_SIGN == 22 && H_CUBE == 23 && H_CBRT == 24 && H_TAN == 25 &&
                  H_ASIN == 26 && H_ACOS == 27 && H_ATAN == 28 && H_TANH == 29 &&
                  H_PASTE == 30 && kNumHandlers == 31,
              "the PTX jump table lists the handlers in this order");
static_assert(kBoxShift == 10, "the 8-case loop hard-codes 1 KB input rows");

// prog: shared address of the packed program (bits 24-28 of each token: the next token's
// handler id); xrow: shared address of this lane's first case of input row 0 (half 0); tstk:
// tensor-memory address of the warp's stack row 0 (8 columns a row). top[0..3] are cases
// 4l..4l+3 and top[4..7] cases 128+4l..128+4l+3 of the pass.
__device__ __forceinline__ void run_program_ptx8(uint32_t prog, uint32_t xrow, uint32_t tstk,
                                                 float (&top)[8], bool (&bad)[8]) {
    using A = Arith<float>;
    unsigned long long p0 = 0ull, p1 = 0ull, p2 = 0ull, p3 = 0ull;
    float m0 = 0.f, m1 = 0.f, m2 = 0.f, m3 = 0.f, m4 = 0.f, m5 = 0.f, m6 = 0.f, m7 = 0.f;
    uint32_t cx = (lds_token(prog).x & 31u) << 24, cy = 0u, pa = prog;
    for (;;) {
        uint32_t code;
        asm volatile(BG_PTX_INTERP8
                     : "+l"(p0), "+l"(p1), "+l"(p2), "+l"(p3), "+f"(m0), "+f"(m1), "+f"(m2),
                       "+f"(m3), "+f"(m4), "+f"(m5), "+f"(m6), "+f"(m7), "+r"(cx), "+r"(cy),
                       "+r"(pa), "=r"(code)
                     : "r"(xrow), "r"(tstk)
                     : "memory");
        if (code == 0) break;
        // The eight values in two rounds of four through one copy of each function (the
        // loop is kept rolled so that the code stays small: each round works on the first
        // half, then swaps the halves); POW's base operands of half hh are columns 4 hh.. of
        // the token's stack row.
        const uint32_t base = tstk + 8u * ((cx >> 12) & 0xffu);
#pragma unroll 1
        for (uint32_t hh = 0; hh < 2; ++hh) {
            apply_exit4(code, base + 4u * hh, p0, p1, m0, m1, m2, m3);
            unsigned long long u;
            float w;
            u = p0; p0 = p2; p2 = u;
            u = p1; p1 = p3; p3 = u;
            w = m0; m0 = m4; m4 = w;
            w = m1; m1 = m5; m5 = w;
            w = m2; m2 = m6; m6 = w;
            w = m3; m3 = m7; m7 = w;
        }
    }
    const float2 a = pair_f2(p0), b = pair_f2(p1), c = pair_f2(p2), e = pair_f2(p3);
    top[0] = a.x; top[1] = a.y; top[2] = b.x; top[3] = b.y;
    top[4] = c.x; top[5] = c.y; top[6] = e.x; top[7] = e.y;
    bad[0] = !A::ok(m0); bad[1] = !A::ok(m1); bad[2] = !A::ok(m2); bad[3] = !A::ok(m3);
    bad[4] = !A::ok(m4); bad[5] = !A::ok(m5); bad[6] = !A::ok(m6); bad[7] = !A::ok(m7);
}

#undef BG8_UNPACK
#undef BG8_PACK
#undef BG8_TRK
#undef BG8_TRACK8
#undef BG8_PAIRS_TT
#undef BG8_PAIRS_TA
#undef BG8_PAIRS_AT
#undef BG8_PDIV2
#undef BG8_DISPATCH
#undef BG8_ROW
#undef BG8_XA
#undef BG8_C2
#undef BG8_STROW
#undef BG8_LDROW
#undef BG8_LDROW_A
#undef BG8_LDROW_T
#undef BG8_LDX_A
#undef BG8_LDX_T
#undef BG8_EXIT

}  // namespace beagle
