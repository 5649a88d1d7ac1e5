// Interpreter loop for the FP32 path with 4 cases per lane, written in inline PTX so that the
// token dispatch is one indexed branch (brx.idx over a .branchtargets table) instead of a
// compare-and-branch tree, and each handler dispatches the next token itself. Semantics are
// those of run_program in score.cuh, handler for handler: the same fp32 operations in the
// same order (.rn forms, so nothing is contracted), the same protected division and square
// root, the same validity decisions (the tracker skips the protected square root, sin, cos
// and the protected log, whose results are finite and at most 1e15 in magnitude whenever
// their operand is valid).
//
// The value arithmetic runs in Blackwell's paired FP32 instructions (add/mul/fma .rn.f32x2:
// two IEEE single-precision operations in one instruction, each half rounded to nearest like
// its scalar form, so the results are bit-identical to scalar code): the top of stack is two
// pairs, %0 = cases (4l, 4l+1) and %1 = (4l+2, 4l+3) of lane l.
//
// sin, cos and the protected log run in the loop (transcend.cuh's branch-free forms, the
// floating-point steps paired, with the same bits). exp, POW and the rest of Table 3's
// transcendentals, and sin and cos of arguments above 65536, leave the loop with their
// handler id; the caller applies them to the top of stack (CUDA's expf and the others) and
// re-enters.
#pragma once

#include "score.cuh"

namespace beagle {

#define BG4_UNPACK "mov.b64 {t0, t1}, %0;\n\tmov.b64 {t2, t3}, %1;\n\t"
#define BG4_PACK "mov.b64 %0, {t0, t1};\n\tmov.b64 %1, {t2, t3};\n\t"
// Validity tracker of one case: m = max.NaN(m, |t|).
#define BG4_TRK(T, M) "abs.f32 z, " T ";\n\tmax.NaN.f32 " M ", " M ", z;\n\t"
#define BG4_TRACK                                                                          \
    BG4_UNPACK BG4_TRK("t0", "%2") BG4_TRK("t1", "%3") BG4_TRK("t2", "%4") BG4_TRK("t3", "%5")
// Protected division of one pair, DST = |DEN| > 1e-3 ? NUM / DEN : 1 per half (Markstein's
// quotient, the steps of Arith<float>::pdiv): y = rcp.approx(den) refined by one Newton step
// to the correctly rounded 1/den, w = num y, then w + (num - den w) y with the remainder exact
// by FMA; the FMA steps paired.
#define BG4_PDIV2(DST, NUM, DEN)                                                           \
    "mov.b64 {d0, d1}, " DEN ";\n\t"                                                       \
    "abs.f32 z, d0;\n\tsetp.gt.f32 q0, z, 0f3A83126F;\n\t"                                 \
    "abs.f32 z, d1;\n\tsetp.gt.f32 q1, z, 0f3A83126F;\n\t"                                 \
    "rcp.approx.ftz.f32 d0, d0;\n\trcp.approx.ftz.f32 d1, d1;\n\tmov.b64 Y, {d0, d1};\n\t"  \
    "mov.b64 KA, " BG_PTX_PAIR(BG_K_NONE) ";\n\tmul.rn.f32x2 ND, " DEN ", KA;\n\t"             \
    "mov.b64 KA, " BG_PTX_PAIR(BG_K_ONE) ";\n\t"                                               \
    "fma.rn.f32x2 E, ND, Y, KA;\n\tfma.rn.f32x2 Y, E, Y, Y;\n\t"                            \
    "mul.rn.f32x2 Z, " NUM ", Y;\n\tfma.rn.f32x2 E, ND, Z, " NUM ";\n\t"                     \
    "fma.rn.f32x2 Z, E, Y, Z;\n\t"                                                          \
    "mov.b64 {d0, d1}, Z;\n\tselp.f32 d0, d0, 0f3F800000, q0;\n\t"                          \
    "selp.f32 d1, d1, 0f3F800000, q1;\n\tmov.b64 " DST ", {d0, d1};\n\t"

// sin or cos of one pair X (transcend.cuh's sincos_fast step for step, the floating-point
// steps paired): t = x 2/pi + 1.5 2^23, k = t - 1.5 2^23, r = x - k pi/2 in three parts,
// both polynomials in s = r^2, then per half the quadrant q = bits(t) - bits(1.5 2^23) + qo
// (qo in the register qoff with the magic subtracted): an odd q takes the cosine, bit 1 of q
// flips the sign.
#define BG4_SINCOS2(X)                                                                     \
    "mov.b64 KA, " BG_PTX_PAIR(BG_K_TWO_OVER_PI) ";\n\tmov.b64 KB, " BG_PTX_PAIR(BG_K_MAGIC) ";\n\t" \
    "fma.rn.f32x2 TQ, " X ", KA, KB;\n\t"                                                  \
    "mov.b64 KA, " BG_PTX_PAIR(BG_K_NMAGIC) ";\n\tadd.rn.f32x2 E, TQ, KA;\n\t"               \
    "mov.b64 KA, " BG_PTX_PAIR(BG_K_NPIO2_C1) ";\n\tfma.rn.f32x2 Z, E, KA, " X ";\n\t"        \
    "mov.b64 KA, " BG_PTX_PAIR(BG_K_NPIO2_C2) ";\n\tfma.rn.f32x2 Z, E, KA, Z;\n\t"            \
    "mov.b64 KA, " BG_PTX_PAIR(BG_K_NPIO2_C3) ";\n\tfma.rn.f32x2 Z, E, KA, Z;\n\t"            \
    "mul.rn.f32x2 Y, Z, Z;\n\t"                                                            \
    "mov.b64 KA, " BG_PTX_PAIR(BG_K_SIN_P3) ";\n\tmov.b64 KB, " BG_PTX_PAIR(BG_K_SIN_P2) ";\n\t" \
    "fma.rn.f32x2 A01, KA, Y, KB;\n\t"                                                     \
    "mov.b64 KB, " BG_PTX_PAIR(BG_K_SIN_P1) ";\n\tfma.rn.f32x2 A01, A01, Y, KB;\n\t"          \
    "mov.b64 KB, " BG_PTX_PAIR(BG_K_SIN_P0) ";\n\tfma.rn.f32x2 A01, A01, Y, KB;\n\t"          \
    "mov.b64 KA, " BG_PTX_PAIR(BG_K_COS_Q3) ";\n\tmov.b64 KB, " BG_PTX_PAIR(BG_K_COS_Q2) ";\n\t" \
    "fma.rn.f32x2 A23, KA, Y, KB;\n\t"                                                     \
    "mov.b64 KB, " BG_PTX_PAIR(BG_K_COS_Q1) ";\n\tfma.rn.f32x2 A23, A23, Y, KB;\n\t"          \
    "mov.b64 KB, " BG_PTX_PAIR(BG_K_COS_Q0) ";\n\tfma.rn.f32x2 A23, A23, Y, KB;\n\t"          \
    "mul.rn.f32x2 E, Z, Y;\n\tfma.rn.f32x2 A01, E, A01, Z;\n\t"                            \
    "mov.b64 KB, " BG_PTX_PAIR(BG_K_ONE) ";\n\tfma.rn.f32x2 A23, Y, A23, KB;\n\t"             \
    "mov.b64 {u0, u1}, TQ;\n\tmov.b64 {w0, w1}, A01;\n\tmov.b64 {w2, w3}, A23;\n\t"         \
    "add.s32 u0, u0, qoff;\n\tadd.s32 u1, u1, qoff;\n\t"                                   \
    "bfe.s32 v, u0, 0, 1;\n\tlop3.b32 w0, w0, w2, v, 0xD8;\n\t"                            \
    "bfe.s32 v, u1, 0, 1;\n\tlop3.b32 w1, w1, w3, v, 0xD8;\n\t"                            \
    "shl.b32 u0, u0, 30;\n\tlop3.b32 w0, w0, u0, 0x80000000, 0x78;\n\t"                    \
    "shl.b32 u1, u1, 30;\n\tlop3.b32 w1, w1, u1, 0x80000000, 0x78;\n\t"                    \
    "mov.b64 " X ", {w0, w1};\n\t"
// The protected log of one pair X (plog_dev step for step, the floating-point steps paired):
// |x| = m 2^e with m in [b, 2b), b just above sqrt(1/2), from integer arithmetic on the bits;
// f = m - 1; ln m = f + f^2 (-1/2 + f L(f)); plus e ln 2 in two parts; 0 where |x| <= 1e-3.
#define BG4_PLOG2(X)                                                                       \
    "mov.b64 {d0, d1}, " X ";\n\tabs.f32 d0, d0;\n\tabs.f32 d1, d1;\n\t"                    \
    "mov.b32 u0, d0;\n\tmov.b32 u1, d1;\n\t"                                               \
    "add.u32 u0, u0, 0x004AFB0C;\n\tadd.u32 u1, u1, 0x004AFB0C;\n\t"                       \
    "shr.u32 w0, u0, 23;\n\tadd.u32 w0, w0, 0x4B3FFF81;\n\t"                               \
    "shr.u32 w1, u1, 23;\n\tadd.u32 w1, w1, 0x4B3FFF81;\n\t"                               \
    "and.b32 u0, u0, 0x007FFFFF;\n\tadd.u32 u0, u0, 0x3F3504F4;\n\t"                       \
    "and.b32 u1, u1, 0x007FFFFF;\n\tadd.u32 u1, u1, 0x3F3504F4;\n\t"                       \
    "mov.b64 Z, {u0, u1};\n\tmov.b64 KA, " BG_PTX_PAIR(BG_K_NONE) ";\n\tadd.rn.f32x2 Z, Z, KA;\n\t" \
    "mov.b64 TQ, {w0, w1};\n\tmov.b64 KA, " BG_PTX_PAIR(BG_K_NMAGIC) ";\n\tadd.rn.f32x2 TQ, TQ, KA;\n\t" \
    "mov.b64 KA, " BG_PTX_PAIR(BG_K_LOG_L7) ";\n\tmov.b64 KB, " BG_PTX_PAIR(BG_K_LOG_L6) ";\n\t" \
    "fma.rn.f32x2 Y, KA, Z, KB;\n\t"                                                       \
    "mov.b64 KB, " BG_PTX_PAIR(BG_K_LOG_L5) ";\n\tfma.rn.f32x2 Y, Y, Z, KB;\n\t"              \
    "mov.b64 KB, " BG_PTX_PAIR(BG_K_LOG_L4) ";\n\tfma.rn.f32x2 Y, Y, Z, KB;\n\t"              \
    "mov.b64 KB, " BG_PTX_PAIR(BG_K_LOG_L3) ";\n\tfma.rn.f32x2 Y, Y, Z, KB;\n\t"              \
    "mov.b64 KB, " BG_PTX_PAIR(BG_K_LOG_L2) ";\n\tfma.rn.f32x2 Y, Y, Z, KB;\n\t"              \
    "mov.b64 KB, " BG_PTX_PAIR(BG_K_LOG_L1) ";\n\tfma.rn.f32x2 Y, Y, Z, KB;\n\t"              \
    "mov.b64 KB, " BG_PTX_PAIR(BG_K_LOG_L0) ";\n\tfma.rn.f32x2 Y, Y, Z, KB;\n\t"              \
    "mul.rn.f32x2 E, Z, Z;\n\t"                                                            \
    "mov.b64 KB, " BG_PTX_PAIR(BG_K_NHALF) ";\n\tfma.rn.f32x2 Y, Z, Y, KB;\n\t"               \
    "fma.rn.f32x2 Y, E, Y, Z;\n\t"                                                         \
    "mov.b64 KA, " BG_PTX_PAIR(BG_K_LN2_LO) ";\n\tfma.rn.f32x2 Y, TQ, KA, Y;\n\t"             \
    "mov.b64 KA, " BG_PTX_PAIR(BG_K_LN2_HI) ";\n\tfma.rn.f32x2 Y, TQ, KA, Y;\n\t"             \
    "mov.b64 {a0, a1}, Y;\n\t"                                                             \
    "setp.gt.f32 q0, d0, " BG_PTX_F32(BG_K_LOG_TINY) ";\n\tselp.f32 a0, a0, 0f00000000, q0;\n\t" \
    "setp.gt.f32 q1, d1, " BG_PTX_F32(BG_K_LOG_TINY) ";\n\tselp.f32 a1, a1, 0f00000000, q1;\n\t" \
    "mov.b64 " X ", {a0, a1};\n\t"

// Operands: %0/%1 top of stack (2 pairs), %2-%5 validity trackers, %6/%7 current token words,
// %8 shared address of the next token, %9 exit code (0 = program done, else the handler id of
// the operator the caller applies), %10 shared address of this lane's first case of input row
// 0, %11 tensor-memory address of the warp's stack row 0.
//
// The stack rows below the top live in tensor memory (TMEM), which this kernel has no other
// use for: row r of the warp is the 4 columns base + 4 r of its 32-lane quarter, lane l of the
// warp holding its 4 cases in TMEM lane quarter + l. Keeping them out of shared memory lets
// shared memory hold more warps. A row load waits for the warp's earlier row stores
// (tcgen05.wait::st) and for itself (tcgen05.wait::ld) before its values are used, so a value
// popped is always the one last pushed to that row.
// Threaded dispatch: every handler ends by loading the next token and branching through the
// table on that token's handler id, which the packer stores in bits 24-28 of the current token
// (so the branch does not wait for the load, whose latency the branch itself covers); the
// program's END token leaves the loop. The table has 32 entries (id 31 ends the program), so
// the 5-bit handler field needs no clamp before the indexed branch.
#define BG4_DISPATCH                                                                       \
    "shr.b32 h, %6, 24;\n\t"                                                               \
    "ld.shared.v2.u32 {%6, %7}, [%8];\n\t"                                                 \
    "add.u32 %8, %8, 8;\n\t"                                                               \
    "brx.idx.uni h, TBL_%=;\n"
#define BG4_ROW "bfe.u32 v, %6, 12, 8;\n\tmad.lo.u32 rp, v, 4, %11;\n\t"
#define BG4_XA "bfe.u32 v, %6, 8, 4;\n\tmad.lo.u32 xa, v, 1024, %10;\n\t"
#define BG4_STROW BG4_UNPACK "tcgen05.st.sync.aligned.32x32b.x4.b32 [rp], {t0, t1, t2, t3};\n\t"
#define BG4_LDROW(R)                                                                       \
    "tcgen05.wait::st.sync.aligned;\n\t"                                                   \
    "tcgen05.ld.sync.aligned.32x32b.x4.b32 {" R "0, " R "1, " R "2, " R "3}, [rp];\n\t"     \
    "tcgen05.wait::ld.sync.aligned;\n\t"
#define BG4_LDROW_A BG4_LDROW("a") "mov.b64 A01, {a0, a1};\n\tmov.b64 A23, {a2, a3};\n\t"
#define BG4_LDROW_T BG4_LDROW("t") BG4_PACK
#define BG4_LDX_A "ld.shared.v2.b64 {A01, A23}, [xa];\n\t"
#define BG4_EXIT(L, CODE) L "_%=:\n\tmov.u32 %9, " #CODE ";\n\tbra.uni OUT_%=;\n"

#define BG_PTX_INTERP4                                                                     \
    "{\n\t"                                                                                \
    ".reg .pred q0, q1;\n\t"                                                               \
    ".reg .b32 h, v, rp, xa;\n\t"                                                          \
    ".reg .b64 A01, A23, C2, Y, ND, E, Z, KA, KB, TQ;\n\t"                                  \
    ".reg .f32 t0, t1, t2, t3, a0, a1, a2, a3, z, d0, d1;\n\t"                             \
    ".reg .b32 u0, u1, w0, w1, w2, w3, qoff, sccode;\n\t"                                  \
    "TBL_%=: .branchtargets PUSHX_%=, PUSHC_%=, DUP_%=, SWAP_%=, DEL_%=, ADDSUB_%=, "      \
    "MUL_%=, PDIV_%=, SIN_%=, COS_%=, EXP_%=, PLOG_%=, PSQRT_%=, SQUARE_%=, ADDSUBX_%=, "   \
    "MULX_%=, PDIVX_%=, ADDC_%=, MULC_%=, PDIVC_%=, END_%=, POW_%=, SIGN_%=, CUBE_%=, "     \
    "CBRT_%=, TAN_%=, ASIN_%=, ACOS_%=, ATAN_%=, TANH_%=, PASTE_%=, END_%=;\n\t"           \
    BG4_DISPATCH                                                                           \
    /* The handlers the paper's operator set uses come first, in one block, and the rest   \
       (stack shuffles, the rest of Table 3, the exits) after it: the interpreter's speed   \
       depends on the instruction footprint of the code it runs. */                        \
    "PUSHX_%=:\n\t" BG4_ROW BG4_XA BG4_STROW "ld.shared.v2.b64 {%0, %1}, [xa];\n\t"         \
    BG4_DISPATCH                                                                           \
    "PUSHC_%=:\n\t" BG4_ROW BG4_STROW "mov.b64 %0, {%7, %7};\n\tmov.b64 %1, %0;\n\t"        \
    BG4_DISPATCH                                                                           \
    /* top = s top + a: a +- top with s = +-1, rounded once like an add or a subtraction */ \
    "ADDSUB_%=:\n\t" BG4_ROW "mov.b64 C2, {%7, %7};\n\t" BG4_LDROW_A                        \
    "fma.rn.f32x2 %0, C2, %0, A01;\n\tfma.rn.f32x2 %1, C2, %1, A23;\n\t"                   \
    BG4_TRACK BG4_DISPATCH                                                                 \
    "MUL_%=:\n\t" BG4_ROW BG4_LDROW_A                                                      \
    "mul.rn.f32x2 %0, A01, %0;\n\tmul.rn.f32x2 %1, A23, %1;\n\t" BG4_TRACK BG4_DISPATCH    \
    /* fused leaf + binary operator: top = s x + top; top + c (c negated for a subtraction); \
       each with its own copy of the arithmetic (sharing one copy through a branch measured \
       0.5 % slower) */                                                                    \
    "ADDSUBX_%=:\n\t" BG4_XA "mov.b64 C2, {%7, %7};\n\t" BG4_LDX_A                          \
    "fma.rn.f32x2 %0, C2, A01, %0;\n\tfma.rn.f32x2 %1, C2, A23, %1;\n\t"                   \
    BG4_TRACK BG4_DISPATCH                                                                 \
    "ADDC_%=:\n\t" "mov.b64 C2, {%7, %7};\n\t"                                             \
    "add.rn.f32x2 %0, %0, C2;\n\tadd.rn.f32x2 %1, %1, C2;\n\t" BG4_TRACK BG4_DISPATCH      \
    "MULX_%=:\n\t" BG4_XA BG4_LDX_A                                                        \
    "mul.rn.f32x2 %0, %0, A01;\n\tmul.rn.f32x2 %1, %1, A23;\n\t" BG4_TRACK BG4_DISPATCH    \
    "MULC_%=:\n\t" "mov.b64 C2, {%7, %7};\n\t"                                             \
    "mul.rn.f32x2 %0, %0, C2;\n\tmul.rn.f32x2 %1, %1, C2;\n\t" BG4_TRACK BG4_DISPATCH      \
    /* the divisions share one copy of the arithmetic, top = top / A: the stack division   \
       moves its operands there (the stack row to the top, the top to A), the fused ones    \
       load A from the input row or the constant word */                                   \
    "PDIV_%=:\n\t" BG4_ROW "mov.b64 A01, %0;\n\tmov.b64 A23, %1;\n\t" BG4_LDROW("a")       \
    "mov.b64 %0, {a0, a1};\n\tmov.b64 %1, {a2, a3};\n\tbra.uni DIVTA_%=;\n"                 \
    "PDIVX_%=:\n\t" BG4_XA BG4_LDX_A "bra.uni DIVTA_%=;\n"                                  \
    "PDIVC_%=:\n\t" "mov.b64 A01, {%7, %7};\n\tmov.b64 A23, A01;\n"                          \
    "DIVTA_%=:\n\t"                                                                         \
    BG4_PDIV2("%0", "%0", "A01") BG4_PDIV2("%1", "%1", "A23") BG4_TRACK BG4_DISPATCH       \
    "SQUARE_%=:\n\t" "mul.rn.f32x2 %0, %0, %0;\n\tmul.rn.f32x2 %1, %1, %1;\n\t"             \
    BG4_TRACK BG4_DISPATCH                                                                 \
    /* sin and cos: arguments above 65536 in magnitude or NaN on any lane leave the loop   \
       (the caller takes CUDA's sinf / cosf on those lanes); no tracking: the results of a    \
       valid operand are bounded */                                                        \
    "SIN_%=:\n\tmov.u32 qoff, 0xB4C00000;\n\tmov.u32 sccode, 8;\n\tbra.uni SC_%=;\n"          \
    "COS_%=:\n\tmov.u32 qoff, 0xB4C00001;\n\tmov.u32 sccode, 9;\n"                            \
    "SC_%=:\n\t" BG4_UNPACK                                                                 \
    "abs.f32 z, t0;\n\tabs.f32 d0, t1;\n\tmax.NaN.f32 z, z, d0;\n\t"                          \
    "abs.f32 d0, t2;\n\tmax.NaN.f32 z, z, d0;\n\tabs.f32 d0, t3;\n\tmax.NaN.f32 z, z, d0;\n\t"  \
    "setp.gtu.f32 q0, z, " BG_PTX_F32(BG_K_SINCOS_LIMIT) ";\n\t"                              \
    "vote.sync.any.pred q1, q0, 0xffffffff;\n\t@q1 bra.uni SCX_%=;\n\t"                      \
    BG4_SINCOS2("%0") BG4_SINCOS2("%1") BG4_DISPATCH                                       \
    /* the protected log: no tracking (|ln|v|| <= 69.1 for a valid operand) */              \
    "PLOG_%=:\n\t" BG4_PLOG2("%0") BG4_PLOG2("%1") BG4_DISPATCH                            \
    "PSQRT_%=:\n\t" BG4_UNPACK                                                             \
    "abs.f32 t0, t0;\n\tsqrt.rn.f32 t0, t0;\n\tabs.f32 t1, t1;\n\tsqrt.rn.f32 t1, t1;\n\t" \
    "abs.f32 t2, t2;\n\tsqrt.rn.f32 t2, t2;\n\tabs.f32 t3, t3;\n\tsqrt.rn.f32 t3, t3;\n\t" \
    BG4_PACK BG4_DISPATCH                                                                  \
    /* exp leaves the loop for CUDA's expf (an in-loop polynomial form measured slower:    \
       the loop's larger code costs more in instruction fetch than the exit) */             \
    BG4_EXIT("EXP", 10)                                                                    \
    "END_%=:\n\tmov.u32 %9, 0;\n\tbra.uni OUT_%=;\n"                                          \
    /* the rest: DUP, SWAP, DEL; SIGN (|v| unchanged, nothing to track), CUBE ((a a) a),     \
       PASTE (push the top, load the register's row, its index in the constant word); the   \
       operators that leave the loop */                                                    \
    "DUP_%=:\n\t" BG4_ROW BG4_STROW BG4_DISPATCH                                           \
    "SWAP_%=:\n\t" BG4_ROW BG4_LDROW_A BG4_STROW "mov.b64 %0, A01;\n\tmov.b64 %1, A23;\n\t"  \
    BG4_DISPATCH                                                                           \
    "DEL_%=:\n\t" BG4_ROW BG4_LDROW_T BG4_DISPATCH                                         \
    "SIGN_%=:\n\tmov.b64 KA, " BG_PTX_PAIR(BG_K_NONE) ";\n\t"                                 \
    "mul.rn.f32x2 %0, %0, KA;\n\tmul.rn.f32x2 %1, %1, KA;\n\t" BG4_DISPATCH                \
    "CUBE_%=:\n\t" "mul.rn.f32x2 A01, %0, %0;\n\tmul.rn.f32x2 A23, %1, %1;\n\t"             \
    "mul.rn.f32x2 %0, A01, %0;\n\tmul.rn.f32x2 %1, A23, %1;\n\t" BG4_TRACK BG4_DISPATCH    \
    "PASTE_%=:\n\t" BG4_ROW BG4_STROW "mad.lo.u32 rp, %7, 4, %11;\n\t" BG4_LDROW_T           \
    BG4_DISPATCH                                                                           \
    "SCX_%=:\n\tmov.u32 %9, sccode;\n\tbra.uni OUT_%=;\n"                                     \
    BG4_EXIT("POW", 21) BG4_EXIT("CBRT", 24) BG4_EXIT("TAN", 25) BG4_EXIT("ASIN", 26)      \
    BG4_EXIT("ACOS", 27) BG4_EXIT("ATAN", 28) BG4_EXIT("TANH", 29)                         \
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
static_assert(kBoxShift == 10, "the PTX loop hard-codes the input row shift");

// Four values of a tensor-memory stack row (the warp's earlier stores are waited for).
__device__ __forceinline__ void tmem_ld_row4(uint32_t addr, float &a0, float &a1, float &a2,
                                             float &a3) {
    asm volatile(
        "tcgen05.wait::st.sync.aligned;\n\t"
        "tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0, %1, %2, %3}, [%4];\n\t"
        "tcgen05.wait::ld.sync.aligned;"
        : "=f"(a0), "=f"(a1), "=f"(a2), "=f"(a3)
        : "r"(addr)
        : "memory");
}

// POW and the transcendentals of the rest of Table 3 on 4 values (b: POW's base operands, the
// 4 values of its stack row). Out of line: inlined, the code of these seven functions sits
// next to the interpreter loop and slows every program, the many that never use them too.
static __device__ __noinline__ float4 ext_values4(uint32_t code, float4 t, float4 b) {
    using A = Arith<float>;
    switch (code) {
    case H_POW: return make_float4(A::pow_(b.x, t.x), A::pow_(b.y, t.y), A::pow_(b.z, t.z), A::pow_(b.w, t.w));
    case H_CBRT: return make_float4(A::cbrt_(t.x), A::cbrt_(t.y), A::cbrt_(t.z), A::cbrt_(t.w));
    case H_TAN: return make_float4(A::tan_(t.x), A::tan_(t.y), A::tan_(t.z), A::tan_(t.w));
    case H_ASIN: return make_float4(A::asin_(t.x), A::asin_(t.y), A::asin_(t.z), A::asin_(t.w));
    case H_ACOS: return make_float4(A::acos_(t.x), A::acos_(t.y), A::acos_(t.z), A::acos_(t.w));
    case H_ATAN: return make_float4(A::atan_(t.x), A::atan_(t.y), A::atan_(t.z), A::atan_(t.w));
    default: return make_float4(A::tanh_(t.x), A::tanh_(t.y), A::tanh_(t.z), A::tanh_(t.w));
    }
}

__device__ __forceinline__ float2 pair_f2(unsigned long long p) {
    return make_float2(__uint_as_float(static_cast<uint32_t>(p)),
                       __uint_as_float(static_cast<uint32_t>(p >> 32)));
}
__device__ __forceinline__ unsigned long long f2_pair(float2 v) {
    return static_cast<unsigned long long>(__float_as_uint(v.x)) |
           (static_cast<unsigned long long>(__float_as_uint(v.y)) << 32);
}

// The operators that leave the loop, on 4 values of a lane (two pairs) and their 4 trackers:
// code is the handler id; base is the tensor-memory address of POW's base operands (the 4
// values of its stack row, read only for POW). exp, the one exit of the paper's operator set
// that every program may take, runs in line; the others (sin and cos of large arguments, the
// rest of Table 3, the 8-case loop's log) run out of line, so that their code does not take
// room in the instruction cache next to the loop.
struct Lane4 {
    unsigned long long pa, pb;
    float m0, m1, m2, m3;
};

static __device__ __noinline__ Lane4 exit_values4(uint32_t code, uint32_t base, Lane4 s) {
    using A = Arith<float>;
    float2 a = pair_f2(s.pa), b = pair_f2(s.pb);
    if (code >= H_POW) {   // the rest of Table 3
        float4 bv = make_float4(0.f, 0.f, 0.f, 0.f);
        if (code == H_POW) tmem_ld_row4(base, bv.x, bv.y, bv.z, bv.w);
        const float4 r = ext_values4(code, make_float4(a.x, a.y, b.x, b.y), bv);
        a = make_float2(r.x, r.y);
        b = make_float2(r.z, r.w);
        // cbrt, atan and tanh of a valid value are valid too; tracking them changes nothing
        s.m0 = A::track(s.m0, a.x);
        s.m1 = A::track(s.m1, a.y);
        s.m2 = A::track(s.m2, b.x);
        s.m3 = A::track(s.m3, b.y);
    } else if (code == H_PLOG) {
        a = plog2(a);
        b = plog2(b);
    } else {
        sincos4_paired(a, b, static_cast<int>(code) - H_SIN);
    }
    // sin, cos and the protected log of a valid value are finite and bounded (|ln|v|| <= 69.1
    // for |v| <= 1e30), and an invalid operand was recorded when it was pushed: no tracking.
    s.pa = f2_pair(a);
    s.pb = f2_pair(b);
    return s;
}

__device__ __forceinline__ void apply_exit4(uint32_t code, uint32_t base,
                                            unsigned long long &pa, unsigned long long &pb,
                                            float &m0, float &m1, float &m2, float &m3) {
    using A = Arith<float>;
    if (code == H_EXP) {
        float2 a = pair_f2(pa), b = pair_f2(pb);
        a = make_float2(A::exp_(a.x), A::exp_(a.y));
        b = make_float2(A::exp_(b.x), A::exp_(b.y));
        m0 = A::track(m0, a.x);
        m1 = A::track(m1, a.y);
        m2 = A::track(m2, b.x);
        m3 = A::track(m3, b.y);
        pa = f2_pair(a);
        pb = f2_pair(b);
        return;
    }
    const Lane4 s = exit_values4(code, base, Lane4{pa, pb, m0, m1, m2, m3});
    pa = s.pa;
    pb = s.pb;
    m0 = s.m0;
    m1 = s.m1;
    m2 = s.m2;
    m3 = s.m3;
}

// prog: shared address of the packed program (bits 24-28 of each token: the next token's
// handler id); xrow: shared address of this lane's first case of input row 0; tstk:
// tensor-memory address of the warp's stack row 0 (4 columns a row).
__device__ __forceinline__ void run_program_ptx4(uint32_t prog, uint32_t xrow, uint32_t tstk,
                                                 float (&top)[4], bool (&bad)[4]) {
    using A = Arith<float>;
    unsigned long long p0 = 0ull, p1 = 0ull;
    float m0 = 0.f, m1 = 0.f, m2 = 0.f, m3 = 0.f;
    // The loop's first dispatch loads token 0 and branches on the handler id in bits 24-28 of
    // the "current" token: start with token 0's id there.
    uint32_t cx = (lds_token(prog).x & 31u) << 24, cy = 0u, pa = prog;
    for (;;) {
        uint32_t code;
        asm volatile(BG_PTX_INTERP4
                     : "+l"(p0), "+l"(p1), "+f"(m0), "+f"(m1), "+f"(m2), "+f"(m3), "+r"(cx),
                       "+r"(cy), "+r"(pa), "=r"(code)
                     : "r"(xrow), "r"(tstk)
                     : "memory");
        if (code == 0) break;
        apply_exit4(code, tstk + 4u * ((cx >> 12) & 0xffu), p0, p1, m0, m1, m2, m3);
    }
    const float2 a = pair_f2(p0), b = pair_f2(p1);
    top[0] = a.x; top[1] = a.y; top[2] = b.x; top[3] = b.y;
    bad[0] = !A::ok(m0); bad[1] = !A::ok(m1); bad[2] = !A::ok(m2); bad[3] = !A::ok(m3);
}

#undef BG4_UNPACK
#undef BG4_PACK
#undef BG4_TRK
#undef BG4_TRACK
#undef BG4_PDIV2
#undef BG4_DISPATCH
#undef BG4_ROW
#undef BG4_XA
#undef BG4_STROW
#undef BG4_LDROW
#undef BG4_LDROW_A
#undef BG4_LDROW_T
#undef BG4_LDX_A
#undef BG4_EXIT
#undef BG4_SINCOS2
#undef BG4_PLOG2

}  // namespace beagle
