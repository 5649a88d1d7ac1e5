// Interpreter loop for the FP32 path with 8 cases per lane (one 256-case tile per pass): the
// inline-PTX threaded interpreter of interp_ptx.cuh, handler for handler, on twice the cases
// per dispatch. An indexed branch costs about a hundred cycles of a warp's time on this GPU
// whatever the handler does, so doubling the cases per dispatch halves that cost per case.
//
// Lane l holds cases 4l..4l+3 and 128+4l..128+4l+3 of the tile (the two halves of the same
// case-to-lane map the 4-case loop uses for its two passes over 256 cases). A stack row is
// 1 KB: half 0 (32 lanes x 4 cases, 512 bytes) then half 1; input row k of the staged box is
// kBox floats further, its half 1 128 floats into the row. Every access is one 16-byte load or
// store per half, 512 contiguous bytes across the warp.
//
// Semantics are those of run_program in score.cuh: the same fp32 operations in the same
// order (.rn forms), the same protected division and square root, the same validity decisions
// (results of psqrt, sin, cos and the protected log of valid operands are bounded, so they are
// not tracked). sin, cos, exp and the protected log leave the loop with their handler id; the
// caller applies transcend.cuh's forms (CUDA's expf) to the eight values and re-enters.
#pragma once

#include "score.cuh"

namespace beagle {

#define BG8_TRACK(T, M) "abs.f32 z, " T ";\n\tmax.NaN.f32 " M ", " M ", z;\n\t"
#define BG8_TRACK8                                                                         \
    BG8_TRACK("%0", "%8") BG8_TRACK("%1", "%9") BG8_TRACK("%2", "%10")                     \
    BG8_TRACK("%3", "%11") BG8_TRACK("%4", "%12") BG8_TRACK("%5", "%13")                   \
    BG8_TRACK("%6", "%14") BG8_TRACK("%7", "%15")
// Protected division, the quotient rounded to nearest by Markstein's method (the steps of
// Arith<float>::pdiv).
#define BG8_PDIV(DST, NUM, DEN)                                                            \
    "abs.f32 z, " DEN ";\n\tsetp.gt.f32 q, z, 0f3A83126F;\n\t"                             \
    "neg.f32 nd, " DEN ";\n\trcp.approx.ftz.f32 y, " DEN ";\n\t"                            \
    "fma.rn.f32 e, nd, y, 0f3F800000;\n\tfma.rn.f32 y, e, y, y;\n\t"                       \
    "mul.rn.f32 z, " NUM ", y;\n\tfma.rn.f32 e, nd, z, " NUM ";\n\t"                        \
    "fma.rn.f32 z, e, y, z;\n\tselp.f32 " DST ", z, 0f3F800000, q;\n\t"
#define BG8_TBLPAD                                                                         \
    ", POW_%=, SIGN_%=, CUBE_%=, CBRT_%=, TAN_%=, ASIN_%=, ACOS_%=, ATAN_%=, TANH_%=, "   \
    "PASTE_%=, END_%="
// %0-%7 top of stack (8 cases), %8-%15 validity trackers, %16/%17 current token words, %18/%19
// next token words (prefetched), %20 shared address of the token after that, %21 exit code,
// %22 shared address of this lane's first case of input row 0 (half 0), %23 shared address of
// this lane's slot in stack row 0 (half 0).
#define BG8_DISPATCH                                                                       \
    "and.b32 h, %18, 31;\n\t"                                                              \
    "mov.b32 %16, %18;\n\tmov.b32 %17, %19;\n\t"                                           \
    "ld.shared.v2.u32 {%18, %19}, [%20];\n\t"                                              \
    "add.u32 %20, %20, 8;\n\t"                                                             \
    "brx.idx.uni h, TBL_%=;\n"
#define BG8_ROW "bfe.u32 v, %16, 12, 8;\n\tmad.lo.u32 rp, v, 1024, %23;\n\t"
#define BG8_XA "bfe.u32 v, %16, 8, 4;\n\tmad.lo.u32 xa, v, 1024, %22;\n\t"
#define BG8_S "mov.b32 s, %17;\n\t"
#define BG8_ST_TOP(A)                                                                      \
    "st.shared.v4.f32 [" A "], {%0, %1, %2, %3};\n\t"                                      \
    "st.shared.v4.f32 [" A "+512], {%4, %5, %6, %7};\n\t"
#define BG8_LD_TOP(A)                                                                      \
    "ld.shared.v4.f32 {%0, %1, %2, %3}, [" A "];\n\t"                                      \
    "ld.shared.v4.f32 {%4, %5, %6, %7}, [" A "+512];\n\t"
#define BG8_LD_A(A)                                                                        \
    "ld.shared.v4.f32 {a0, a1, a2, a3}, [" A "];\n\t"                                      \
    "ld.shared.v4.f32 {a4, a5, a6, a7}, [" A "+512];\n\t"
// OP(D, L, R): D = L op R for the eight (D, L, R) triples given by the two lists
#define BG8_MAP(OPM, D, L, R)                                                              \
    OPM("%0", L##0, R##0) OPM("%1", L##1, R##1) OPM("%2", L##2, R##2) OPM("%3", L##3, R##3) \
    OPM("%4", L##4, R##4) OPM("%5", L##5, R##5) OPM("%6", L##6, R##6) OPM("%7", L##7, R##7)
#define BG8_T0 "%0"
#define BG8_T1 "%1"
#define BG8_T2 "%2"
#define BG8_T3 "%3"
#define BG8_T4 "%4"
#define BG8_T5 "%5"
#define BG8_T6 "%6"
#define BG8_T7 "%7"
#define BG8_A0 "a0"
#define BG8_A1 "a1"
#define BG8_A2 "a2"
#define BG8_A3 "a3"
#define BG8_A4 "a4"
#define BG8_A5 "a5"
#define BG8_A6 "a6"
#define BG8_A7 "a7"
#define BG8_SS0 "s"
#define BG8_SS1 "s"
#define BG8_SS2 "s"
#define BG8_SS3 "s"
#define BG8_SS4 "s"
#define BG8_SS5 "s"
#define BG8_SS6 "s"
#define BG8_SS7 "s"
// a0..a7 = s (a constant operand broadcast, so the fused-constant handlers share the code of
// the fused-input ones: the instruction footprint decides this interpreter's speed)
#define BG8_SET_A_S                                                                        \
    "mov.f32 a0, s;\n\tmov.f32 a1, s;\n\tmov.f32 a2, s;\n\tmov.f32 a3, s;\n\t"             \
    "mov.f32 a4, s;\n\tmov.f32 a5, s;\n\tmov.f32 a6, s;\n\tmov.f32 a7, s;\n\t"
#define BG8_OP_FMA_S_T_A(D, T, A) "fma.rn.f32 " D ", s, " T ", " A ";\n\t"   // D = s*T + A
#define BG8_OP_FMA_S_A_T(D, A, T) "fma.rn.f32 " D ", s, " A ", " T ";\n\t"   // D = s*A + T
#define BG8_OP_MUL(D, L, R) "mul.rn.f32 " D ", " L ", " R ";\n\t"
#define BG8_OP_ADD(D, L, R) "add.rn.f32 " D ", " L ", " R ";\n\t"
#define BG8_OP_PDIV(D, L, R) BG8_PDIV(D, L, R)

// The rest of Table 3 (as in interp_ptx.cuh): POW and the transcendentals leave the loop;
// SIGN, CUBE ((a a) a) and PASTE (push the top, load the register's row) run here.
#define BG8_EXT_BODY                                                                       \
    "POW_%=:\n\tmov.u32 %21, 21;\n\tbra.uni OUT_%=;\n"                                      \
    "CBRT_%=:\n\tmov.u32 %21, 24;\n\tbra.uni OUT_%=;\n"                                     \
    "TAN_%=:\n\tmov.u32 %21, 25;\n\tbra.uni OUT_%=;\n"                                      \
    "ASIN_%=:\n\tmov.u32 %21, 26;\n\tbra.uni OUT_%=;\n"                                     \
    "ACOS_%=:\n\tmov.u32 %21, 27;\n\tbra.uni OUT_%=;\n"                                     \
    "ATAN_%=:\n\tmov.u32 %21, 28;\n\tbra.uni OUT_%=;\n"                                     \
    "TANH_%=:\n\tmov.u32 %21, 29;\n\tbra.uni OUT_%=;\n"                                     \
    "SIGN_%=:\n\t"                                                                         \
    "neg.f32 %0, %0;\n\tneg.f32 %1, %1;\n\tneg.f32 %2, %2;\n\tneg.f32 %3, %3;\n\t"          \
    "neg.f32 %4, %4;\n\tneg.f32 %5, %5;\n\tneg.f32 %6, %6;\n\tneg.f32 %7, %7;\n\t"          \
    BG8_DISPATCH                                                                           \
    "CUBE_%=:\n\t"                                                                         \
    "mul.rn.f32 a0, %0, %0;\n\tmul.rn.f32 a1, %1, %1;\n\tmul.rn.f32 a2, %2, %2;\n\t"        \
    "mul.rn.f32 a3, %3, %3;\n\tmul.rn.f32 a4, %4, %4;\n\tmul.rn.f32 a5, %5, %5;\n\t"        \
    "mul.rn.f32 a6, %6, %6;\n\tmul.rn.f32 a7, %7, %7;\n\t"                                 \
    BG8_MAP(BG8_OP_MUL, , BG8_A, BG8_T) BG8_TRACK8 BG8_DISPATCH                            \
    "PASTE_%=:\n\t" BG8_ROW BG8_ST_TOP("rp")                                                \
    "mad.lo.u32 rp, %17, 1024, %23;\n\t" BG8_LD_TOP("rp") BG8_DISPATCH

#define BG_PTX_INTERP8                                                                     \
    "{\n\t"                                                                                \
    ".reg .pred q;\n\t"                                                                    \
    ".reg .b32 h, v, rp, xa;\n\t"                                                          \
    ".reg .f32 a0, a1, a2, a3, a4, a5, a6, a7, s, z, nd, y, e;\n\t"                                  \
    "TBL_%=: .branchtargets PUSHX_%=, PUSHC_%=, DUP_%=, SWAP_%=, DEL_%=, ADDSUB_%=, "      \
    "MUL_%=, PDIV_%=, SIN_%=, COS_%=, EXP_%=, PLOG_%=, PSQRT_%=, SQUARE_%=, ADDSUBX_%=, "   \
    "MULX_%=, PDIVX_%=, ADDC_%=, MULC_%=, PDIVC_%=, END_%=" BG8_TBLPAD ";\n\t"             \
    BG8_DISPATCH                                                                           \
    "PUSHX_%=:\n\t" BG8_ROW BG8_XA BG8_ST_TOP("rp") BG8_LD_TOP("xa") BG8_DISPATCH          \
    "PUSHC_%=:\n\t" BG8_ROW BG8_S BG8_ST_TOP("rp")                                          \
    "mov.f32 %0, s;\n\tmov.f32 %1, s;\n\tmov.f32 %2, s;\n\tmov.f32 %3, s;\n\t"             \
    "mov.f32 %4, s;\n\tmov.f32 %5, s;\n\tmov.f32 %6, s;\n\tmov.f32 %7, s;\n\t"             \
    BG8_DISPATCH                                                                           \
    "DUP_%=:\n\t" BG8_ROW BG8_ST_TOP("rp") BG8_DISPATCH                                     \
    "SWAP_%=:\n\t" BG8_ROW BG8_LD_A("rp") BG8_ST_TOP("rp")                                  \
    "mov.f32 %0, a0;\n\tmov.f32 %1, a1;\n\tmov.f32 %2, a2;\n\tmov.f32 %3, a3;\n\t"         \
    "mov.f32 %4, a4;\n\tmov.f32 %5, a5;\n\tmov.f32 %6, a6;\n\tmov.f32 %7, a7;\n\t"         \
    BG8_DISPATCH                                                                           \
    "DEL_%=:\n\t" BG8_ROW BG8_LD_TOP("rp") BG8_DISPATCH                                     \
    "ADDSUB_%=:\n\t" BG8_ROW BG8_S BG8_LD_A("rp")                                           \
    BG8_MAP(BG8_OP_FMA_S_T_A, , BG8_T, BG8_A) BG8_TRACK8 BG8_DISPATCH                     \
    "MUL_%=:\n\t" BG8_ROW BG8_LD_A("rp")                                                   \
    BG8_MAP(BG8_OP_MUL, , BG8_A, BG8_T) BG8_TRACK8 BG8_DISPATCH                            \
    "PDIV_%=:\n\t" BG8_ROW BG8_LD_A("rp")                                                  \
    BG8_MAP(BG8_OP_PDIV, , BG8_A, BG8_T) BG8_TRACK8 BG8_DISPATCH                           \
    "SIN_%=:\n\tmov.u32 %21, 8;\n\tbra.uni OUT_%=;\n"                                      \
    "COS_%=:\n\tmov.u32 %21, 9;\n\tbra.uni OUT_%=;\n"                                      \
    "EXP_%=:\n\tmov.u32 %21, 10;\n\tbra.uni OUT_%=;\n"                                     \
    "PLOG_%=:\n\tmov.u32 %21, 11;\n\tbra.uni OUT_%=;\n"                                    \
    "PSQRT_%=:\n\t"                                                                        \
    "abs.f32 %0, %0;\n\tsqrt.rn.f32 %0, %0;\n\tabs.f32 %1, %1;\n\tsqrt.rn.f32 %1, %1;\n\t" \
    "abs.f32 %2, %2;\n\tsqrt.rn.f32 %2, %2;\n\tabs.f32 %3, %3;\n\tsqrt.rn.f32 %3, %3;\n\t" \
    "abs.f32 %4, %4;\n\tsqrt.rn.f32 %4, %4;\n\tabs.f32 %5, %5;\n\tsqrt.rn.f32 %5, %5;\n\t" \
    "abs.f32 %6, %6;\n\tsqrt.rn.f32 %6, %6;\n\tabs.f32 %7, %7;\n\tsqrt.rn.f32 %7, %7;\n\t" \
    BG8_DISPATCH                                                                           \
    "SQUARE_%=:\n\t" BG8_MAP(BG8_OP_MUL, , BG8_T, BG8_T) BG8_TRACK8 BG8_DISPATCH           \
    "ADDSUBX_%=:\n\t" BG8_XA BG8_S BG8_LD_A("xa") "bra.uni ADDTA_%=;\n"                     \
    "ADDC_%=:\n\t" BG8_S BG8_SET_A_S "mov.f32 s, 0f3F800000;\n"                              \
    "ADDTA_%=:\n\t" BG8_MAP(BG8_OP_FMA_S_A_T, , BG8_A, BG8_T) BG8_TRACK8 BG8_DISPATCH       \
    "MULX_%=:\n\t" BG8_XA BG8_LD_A("xa") "bra.uni MULTA_%=;\n"                               \
    "MULC_%=:\n\t" BG8_S BG8_SET_A_S                                                       \
    "MULTA_%=:\n\t" BG8_MAP(BG8_OP_MUL, , BG8_T, BG8_A) BG8_TRACK8 BG8_DISPATCH            \
    "PDIVX_%=:\n\t" BG8_XA BG8_LD_A("xa") "bra.uni DIVTA_%=;\n"                              \
    "PDIVC_%=:\n\t" BG8_S BG8_SET_A_S                                                      \
    "DIVTA_%=:\n\t" BG8_MAP(BG8_OP_PDIV, , BG8_T, BG8_A) BG8_TRACK8 BG8_DISPATCH           \
    BG8_EXT_BODY                                                                           \
    "END_%=:\n\tmov.u32 %21, 0;\n"                                                         \
    "OUT_%=:\n\t"                                                                          \
    "}"

static_assert(H_PUSHX == 0 && H_PUSHC == 1 && H_DUP == 2 && H_SWAP == 3 && H_DEL == 4 &&
                  H_ADDSUB == 5 && H_MUL == 6 && H_PDIV == 7 && H_SIN == 8 && H_COS == 9 &&
                  H_EXP == 10 && H_PLOG == 11 && H_PSQRT == 12 && H_SQUARE == 13 &&
                  H_ADDSUBX == 14 && H_MULX == 15 && H_PDIVX == 16 && H_ADDC == 17 &&
                  H_MULC == 18 && H_PDIVC == 19 && H_END == 20,
              "the PTX jump table lists the handlers in this order");
static_assert(kBoxShift == 10, "the 8-case loop hard-codes 1 KB input rows");

// prog: shared address of the packed program; xrow: this lane's first input case (half 0 of
// row 0); stk: this lane's slot in stack row 0 (half 0). top[0..3] are cases 4l..4l+3 and
// top[4..7] cases 128+4l..128+4l+3 of the 256-case tile.
__device__ __forceinline__ void run_program_ptx8(uint32_t prog, uint32_t xrow, uint32_t stk,
                                                 float (&top)[8], bool (&bad)[8]) {
    using A = Arith<float>;
    float t0 = 0.f, t1 = 0.f, t2 = 0.f, t3 = 0.f, t4 = 0.f, t5 = 0.f, t6 = 0.f, t7 = 0.f;
    float m0 = 0.f, m1 = 0.f, m2 = 0.f, m3 = 0.f, m4 = 0.f, m5 = 0.f, m6 = 0.f, m7 = 0.f;
    const uint2 first = lds_token(prog);
    uint32_t cx = 0u, cy = 0u, nx = first.x, ny = first.y, pa = prog + 8u;
    for (;;) {
        uint32_t code;
        asm volatile(BG_PTX_INTERP8
                     : "+f"(t0), "+f"(t1), "+f"(t2), "+f"(t3), "+f"(t4), "+f"(t5), "+f"(t6),
                       "+f"(t7), "+f"(m0), "+f"(m1), "+f"(m2), "+f"(m3), "+f"(m4), "+f"(m5),
                       "+f"(m6), "+f"(m7), "+r"(cx), "+r"(cy), "+r"(nx), "+r"(ny), "+r"(pa),
                       "=r"(code)
                     : "r"(xrow), "r"(stk)
                     : "memory");
        if (code == 0) break;
        // The eight values in two rounds of four through one copy of each function (the
        // loop is kept rolled so that the code stays small).
#pragma unroll 1
        for (int hh = 0; hh < 2; ++hh) {
            float u0 = hh ? t4 : t0, u1 = hh ? t5 : t1, u2 = hh ? t6 : t2, u3 = hh ? t7 : t3;
            float n0 = hh ? m4 : m0, n1 = hh ? m5 : m1, n2 = hh ? m6 : m2, n3 = hh ? m7 : m3;
            if (code >= H_POW) {   // the rest of Table 3
                if (code == H_POW) {   // second operand: this half of the token's stack row
                    float a0, a1, a2, a3;
                    lds4(stk + ((cx >> 12) & 0xffu) * 1024u + 512u * hh, a0, a1, a2, a3);
                    u0 = A::pow_(a0, u0); u1 = A::pow_(a1, u1);
                    u2 = A::pow_(a2, u2); u3 = A::pow_(a3, u3);
                } else {
                    switch (code) {
                    case H_CBRT: u0 = A::cbrt_(u0); u1 = A::cbrt_(u1); u2 = A::cbrt_(u2); u3 = A::cbrt_(u3); break;
                    case H_TAN: u0 = A::tan_(u0); u1 = A::tan_(u1); u2 = A::tan_(u2); u3 = A::tan_(u3); break;
                    case H_ASIN: u0 = A::asin_(u0); u1 = A::asin_(u1); u2 = A::asin_(u2); u3 = A::asin_(u3); break;
                    case H_ACOS: u0 = A::acos_(u0); u1 = A::acos_(u1); u2 = A::acos_(u2); u3 = A::acos_(u3); break;
                    case H_ATAN: u0 = A::atan_(u0); u1 = A::atan_(u1); u2 = A::atan_(u2); u3 = A::atan_(u3); break;
                    default: u0 = A::tanh_(u0); u1 = A::tanh_(u1); u2 = A::tanh_(u2); u3 = A::tanh_(u3); break;
                    }
                }
                n0 = A::track(n0, u0); n1 = A::track(n1, u1);
                n2 = A::track(n2, u2); n3 = A::track(n3, u3);
            } else switch (code) {
            case H_SIN:
            case H_COS: sincos4(u0, u1, u2, u3, static_cast<int>(code) - H_SIN); break;
            case H_PLOG:
                u0 = A::plog(u0); u1 = A::plog(u1); u2 = A::plog(u2); u3 = A::plog(u3);
                break;
            default:
                u0 = A::exp_(u0); u1 = A::exp_(u1); u2 = A::exp_(u2); u3 = A::exp_(u3);
                n0 = A::track(n0, u0); n1 = A::track(n1, u1);
                n2 = A::track(n2, u2); n3 = A::track(n3, u3);
                break;
            }
            if (hh) { t4 = u0; t5 = u1; t6 = u2; t7 = u3; m4 = n0; m5 = n1; m6 = n2; m7 = n3; }
            else { t0 = u0; t1 = u1; t2 = u2; t3 = u3; m0 = n0; m1 = n1; m2 = n2; m3 = n3; }
        }
    }
    top[0] = t0; top[1] = t1; top[2] = t2; top[3] = t3;
    top[4] = t4; top[5] = t5; top[6] = t6; top[7] = t7;
    bad[0] = !A::ok(m0); bad[1] = !A::ok(m1); bad[2] = !A::ok(m2); bad[3] = !A::ok(m3);
    bad[4] = !A::ok(m4); bad[5] = !A::ok(m5); bad[6] = !A::ok(m6); bad[7] = !A::ok(m7);
}

#undef BG8_TRACK
#undef BG8_TRACK8
#undef BG8_PDIV
#undef BG8_TBLPAD
#undef BG8_DISPATCH
#undef BG8_ROW
#undef BG8_XA
#undef BG8_S
#undef BG8_ST_TOP
#undef BG8_LD_TOP
#undef BG8_LD_A
#undef BG8_MAP
#undef BG8_SET_A_S
#undef BG8_EXT_BODY

}  // namespace beagle
