// Interpreter loop for the FP32 path with 4 cases per lane, written in inline PTX so that the
// token dispatch is one indexed branch (brx.idx over a .branchtargets table) instead of a
// compare-and-branch tree, and each handler dispatches the next token itself. Semantics are
// those of run_program in score.cuh, handler for handler: the same fp32 operations in the
// same order (.rn forms, so nothing is contracted), the same protected division and square
// root, the same validity decisions (the tracker skips the protected square root, sin, cos
// and the protected log, whose results are finite and at most 1e15 in magnitude whenever
// their operand is valid). sin, cos, exp and the protected log leave the loop with their
// handler id; the caller applies them to the top of stack (transcend.cuh's branch-free sin,
// cos and log; CUDA's expf) and re-enters.
#pragma once

#include "score.cuh"

namespace beagle {

// One case of the validity tracker: m = max.NaN(m, |t|).
#define BG_PTX_TRACK(T, M) "abs.f32 z, " T ";\n\tmax.NaN.f32 " M ", " M ", z;\n\t"
#define BG_PTX_TRACK4                                                                      \
    BG_PTX_TRACK("%0", "%4") BG_PTX_TRACK("%1", "%5") BG_PTX_TRACK("%2", "%6")             \
    BG_PTX_TRACK("%3", "%7")
// dst = |den| > 1e-3 ? num / den : 1   (protected division, "Fitness Functions" reading). The
// quotient is rounded to nearest by Markstein's method, without branches: y = rcp.approx(den)
// refined by one Newton step to the correctly rounded 1/den, w = num y, then w + (num - den w) y
// with the remainder exact by FMA (the same steps as Arith<float>::pdiv).
#define BG_PTX_PDIV(DST, NUM, DEN)                                                         \
    "abs.f32 z, " DEN ";\n\tsetp.gt.f32 q, z, 0f3A83126F;\n\t"                             \
    "neg.f32 nd, " DEN ";\n\trcp.approx.ftz.f32 y, " DEN ";\n\t"                            \
    "fma.rn.f32 e, nd, y, 0f3F800000;\n\tfma.rn.f32 y, e, y, y;\n\t"                       \
    "mul.rn.f32 z, " NUM ", y;\n\tfma.rn.f32 e, nd, z, " NUM ";\n\t"                        \
    "fma.rn.f32 z, e, y, z;\n\tselp.f32 " DST ", z, 0f3F800000, q;\n\t"

// Operands: %0-%3 top of stack (4 cases), %4-%7 validity trackers, %8/%9 current token words,
// %10 shared address of the next token, %11 exit code (0 = program done, else the
// transcendental handler id), %12 shared address of this lane's first case of input row 0,
// %13 tensor-memory address of the warp's stack row 0.
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
// program's END token leaves the loop.
// The table has 32 entries (id 31 ends the program), so the 5-bit handler field needs no
// clamp before the indexed branch. Ids 21-30 are the rest of Table 3 (POW and the
// transcendentals leave the loop like sin; SIGN, CUBE and PASTE run here).
#define BG_PTX_TBLPAD \
    ", POW_%=, SIGN_%=, CUBE_%=, CBRT_%=, TAN_%=, ASIN_%=, ACOS_%=, ATAN_%=, TANH_%=, " \
    "PASTE_%=, END_%="
#define BG_PTX_DISPATCH                                                                    \
    "shr.b32 h, %8, 24;\n\t"                                                               \
    "ld.shared.v2.u32 {%8, %9}, [%10];\n\t"                                                \
    "add.u32 %10, %10, 8;\n\t"                                                             \
    "brx.idx.uni h, TBL_%=;\n"
#define BG_PTX_ROW "bfe.u32 v, %8, 12, 8;\n\tmad.lo.u32 rp, v, 4, %13;\n\t"
// push the top (4 cases) to stack row rp; load stack row rp into D0..D3
#define BG_PTX_STROW "tcgen05.st.sync.aligned.32x32b.x4.b32 [rp], {%0, %1, %2, %3};\n\t"
#define BG_PTX_LDROW(D0, D1, D2, D3)                                                       \
    "tcgen05.wait::st.sync.aligned;\n\t"                                                   \
    "tcgen05.ld.sync.aligned.32x32b.x4.b32 {" D0 ", " D1 ", " D2 ", " D3 "}, [rp];\n\t"       \
    "tcgen05.wait::ld.sync.aligned;\n\t"
#define BG_PTX_XA "bfe.u32 v, %8, 8, 4;\n\tmad.lo.u32 xa, v, 1024, %12;\n\t"
#define BG_PTX_S "mov.b32 s, %9;\n\t"

// Fused add/subtract and multiply by an input or a constant, each with its own copy of the
// arithmetic (sharing one copy through a branch measured 0.5 % slower): the input add is a
// fused multiply-add by the sign s = +-1, rounded exactly like an add or a subtraction; the
// constant add adds the token's constant, already negated for a subtraction.
#define BG_PTX_ADDMUL_BODY                                                                 \
    "ADDSUBX_%=:\n\t" BG_PTX_XA BG_PTX_S                                                   \
    "ld.shared.v4.f32 {a0, a1, a2, a3}, [xa];\n\t"                                         \
    "fma.rn.f32 %0, s, a0, %0;\n\tfma.rn.f32 %1, s, a1, %1;\n\t"                           \
    "fma.rn.f32 %2, s, a2, %2;\n\tfma.rn.f32 %3, s, a3, %3;\n\t"                           \
    BG_PTX_TRACK4 BG_PTX_DISPATCH                                                          \
    "ADDC_%=:\n\t" BG_PTX_S                                                                \
    "add.rn.f32 %0, %0, s;\n\tadd.rn.f32 %1, %1, s;\n\t"                                   \
    "add.rn.f32 %2, %2, s;\n\tadd.rn.f32 %3, %3, s;\n\t"                                   \
    BG_PTX_TRACK4 BG_PTX_DISPATCH                                                          \
    "MULX_%=:\n\t" BG_PTX_XA                                                               \
    "ld.shared.v4.f32 {a0, a1, a2, a3}, [xa];\n\t"                                         \
    "mul.rn.f32 %0, %0, a0;\n\tmul.rn.f32 %1, %1, a1;\n\t"                                 \
    "mul.rn.f32 %2, %2, a2;\n\tmul.rn.f32 %3, %3, a3;\n\t"                                 \
    BG_PTX_TRACK4 BG_PTX_DISPATCH                                                          \
    "MULC_%=:\n\t" BG_PTX_S                                                                \
    "mul.rn.f32 %0, %0, s;\n\tmul.rn.f32 %1, %1, s;\n\t"                                   \
    "mul.rn.f32 %2, %2, s;\n\tmul.rn.f32 %3, %3, s;\n\t"                                   \
    BG_PTX_TRACK4 BG_PTX_DISPATCH

// Fused division by an input or a constant: both load the divisor into a0..a3 and share one
// copy of the four divisions (the interpreter's speed depends on its instruction footprint).
#define BG_PTX_PDIVX_BODY                                                                  \
    "PDIVX_%=:\n\t" BG_PTX_XA                                                              \
    "ld.shared.v4.f32 {a0, a1, a2, a3}, [xa];\n\tbra.uni DIVTA_%=;\n"                       \
    "PDIVC_%=:\n\t" BG_PTX_S                                                               \
    "mov.f32 a0, s;\n\tmov.f32 a1, s;\n\tmov.f32 a2, s;\n\tmov.f32 a3, s;\n"              \
    "DIVTA_%=:\n\t"                                                                         \
    BG_PTX_PDIV("%0", "%0", "a0") BG_PTX_PDIV("%1", "%1", "a1")                            \
    BG_PTX_PDIV("%2", "%2", "a2") BG_PTX_PDIV("%3", "%3", "a3")                            \
    BG_PTX_TRACK4 BG_PTX_DISPATCH

// The rest of Table 3: SIGN flips the four signs (|v| unchanged: nothing to track); CUBE is
// (a a) a, each product rounded; PASTE pushes the top to its stack row, then loads the
// register's row (its index in the constant word); POW and the transcendentals leave the loop.
#define BG_PTX_EXT_BODY                                                                    \
    "POW_%=:\n\tmov.u32 %11, 21;\n\tbra.uni OUT_%=;\n"                                      \
    "CBRT_%=:\n\tmov.u32 %11, 24;\n\tbra.uni OUT_%=;\n"                                     \
    "TAN_%=:\n\tmov.u32 %11, 25;\n\tbra.uni OUT_%=;\n"                                      \
    "ASIN_%=:\n\tmov.u32 %11, 26;\n\tbra.uni OUT_%=;\n"                                     \
    "ACOS_%=:\n\tmov.u32 %11, 27;\n\tbra.uni OUT_%=;\n"                                     \
    "ATAN_%=:\n\tmov.u32 %11, 28;\n\tbra.uni OUT_%=;\n"                                     \
    "TANH_%=:\n\tmov.u32 %11, 29;\n\tbra.uni OUT_%=;\n"                                     \
    "SIGN_%=:\n\t"                                                                         \
    "neg.f32 %0, %0;\n\tneg.f32 %1, %1;\n\tneg.f32 %2, %2;\n\tneg.f32 %3, %3;\n\t"          \
    BG_PTX_DISPATCH                                                                        \
    "CUBE_%=:\n\t"                                                                         \
    "mul.rn.f32 a0, %0, %0;\n\tmul.rn.f32 a1, %1, %1;\n\t"                                 \
    "mul.rn.f32 a2, %2, %2;\n\tmul.rn.f32 a3, %3, %3;\n\t"                                 \
    "mul.rn.f32 %0, a0, %0;\n\tmul.rn.f32 %1, a1, %1;\n\t"                                 \
    "mul.rn.f32 %2, a2, %2;\n\tmul.rn.f32 %3, a3, %3;\n\t"                                 \
    BG_PTX_TRACK4 BG_PTX_DISPATCH                                                          \
    "PASTE_%=:\n\t" BG_PTX_ROW BG_PTX_STROW                                                 \
    "mad.lo.u32 rp, %9, 4, %13;\n\t" BG_PTX_LDROW("%0", "%1", "%2", "%3")                   \
    BG_PTX_DISPATCH

#define BG_PTX_INTERP4                                                                     \
    "{\n\t"                                                                                \
    ".reg .pred q;\n\t"                                                                    \
    ".reg .b32 h, v, rp, xa;\n\t"                                                          \
    ".reg .f32 a0, a1, a2, a3, s, z, nd, y, e;\n\t"                                                  \
    "TBL_%=: .branchtargets PUSHX_%=, PUSHC_%=, DUP_%=, SWAP_%=, DEL_%=, ADDSUB_%=, "      \
    "MUL_%=, PDIV_%=, SIN_%=, COS_%=, EXP_%=, PLOG_%=, PSQRT_%=, SQUARE_%=, ADDSUBX_%=, "   \
    "MULX_%=, PDIVX_%=, ADDC_%=, MULC_%=, PDIVC_%=, END_%=" BG_PTX_TBLPAD ";\n\t"          \
    BG_PTX_DISPATCH                                                                        \
    "PUSHX_%=:\n\t" BG_PTX_ROW BG_PTX_XA BG_PTX_STROW                                      \
    "ld.shared.v4.f32 {%0, %1, %2, %3}, [xa];\n\t"                                         \
    BG_PTX_DISPATCH                                                                        \
    "PUSHC_%=:\n\t" BG_PTX_ROW BG_PTX_S BG_PTX_STROW                                       \
    "mov.f32 %0, s;\n\tmov.f32 %1, s;\n\tmov.f32 %2, s;\n\tmov.f32 %3, s;\n\t"             \
    BG_PTX_DISPATCH                                                                        \
    "DUP_%=:\n\t" BG_PTX_ROW BG_PTX_STROW                                                  \
    BG_PTX_DISPATCH                                                                        \
    "SWAP_%=:\n\t" BG_PTX_ROW BG_PTX_LDROW("a0", "a1", "a2", "a3") BG_PTX_STROW            \
    "mov.f32 %0, a0;\n\tmov.f32 %1, a1;\n\tmov.f32 %2, a2;\n\tmov.f32 %3, a3;\n\t"         \
    BG_PTX_DISPATCH                                                                        \
    "DEL_%=:\n\t" BG_PTX_ROW BG_PTX_LDROW("%0", "%1", "%2", "%3")                          \
    BG_PTX_DISPATCH                                                                        \
    "ADDSUB_%=:\n\t" BG_PTX_ROW BG_PTX_S BG_PTX_LDROW("a0", "a1", "a2", "a3")              \
    "fma.rn.f32 %0, s, %0, a0;\n\tfma.rn.f32 %1, s, %1, a1;\n\t"                           \
    "fma.rn.f32 %2, s, %2, a2;\n\tfma.rn.f32 %3, s, %3, a3;\n\t"                           \
    BG_PTX_TRACK4 BG_PTX_DISPATCH                                                          \
    "MUL_%=:\n\t" BG_PTX_ROW BG_PTX_LDROW("a0", "a1", "a2", "a3")                          \
    "mul.rn.f32 %0, a0, %0;\n\tmul.rn.f32 %1, a1, %1;\n\t"                                 \
    "mul.rn.f32 %2, a2, %2;\n\tmul.rn.f32 %3, a3, %3;\n\t"                                 \
    BG_PTX_TRACK4 BG_PTX_DISPATCH                                                          \
    "PDIV_%=:\n\t" BG_PTX_ROW BG_PTX_LDROW("a0", "a1", "a2", "a3")                         \
    BG_PTX_PDIV("%0", "a0", "%0") BG_PTX_PDIV("%1", "a1", "%1")                            \
    BG_PTX_PDIV("%2", "a2", "%2") BG_PTX_PDIV("%3", "a3", "%3")                            \
    BG_PTX_TRACK4 BG_PTX_DISPATCH                                                          \
    "SIN_%=:\n\tmov.u32 %11, 8;\n\tbra.uni OUT_%=;\n"                                      \
    "COS_%=:\n\tmov.u32 %11, 9;\n\tbra.uni OUT_%=;\n"                                      \
    "EXP_%=:\n\tmov.u32 %11, 10;\n\tbra.uni OUT_%=;\n"                                     \
    "PLOG_%=:\n\tmov.u32 %11, 11;\n\tbra.uni OUT_%=;\n"                                    \
    "PSQRT_%=:\n\t"                                                                        \
    "abs.f32 %0, %0;\n\tsqrt.rn.f32 %0, %0;\n\tabs.f32 %1, %1;\n\tsqrt.rn.f32 %1, %1;\n\t" \
    "abs.f32 %2, %2;\n\tsqrt.rn.f32 %2, %2;\n\tabs.f32 %3, %3;\n\tsqrt.rn.f32 %3, %3;\n\t" \
    BG_PTX_DISPATCH                                                                        \
    "SQUARE_%=:\n\t"                                                                       \
    "mul.rn.f32 %0, %0, %0;\n\tmul.rn.f32 %1, %1, %1;\n\t"                                 \
    "mul.rn.f32 %2, %2, %2;\n\tmul.rn.f32 %3, %3, %3;\n\t"                                 \
    BG_PTX_TRACK4 BG_PTX_DISPATCH                                                          \
    BG_PTX_ADDMUL_BODY                                                                     \
    BG_PTX_PDIVX_BODY                                                                      \
    BG_PTX_EXT_BODY                                                                        \
    "END_%=:\n\tmov.u32 %11, 0;\n"                                                         \
    "OUT_%=:\n\t"                                                                          \
    "}"

static_assert(H_PUSHX == 0 && H_PUSHC == 1 && H_DUP == 2 && H_SWAP == 3 && H_DEL == 4 &&
                  H_ADDSUB == 5 && H_MUL == 6 && H_PDIV == 7 && H_SIN == 8 && H_COS == 9 &&
                  H_EXP == 10 && H_PLOG == 11 && H_PSQRT == 12 && H_SQUARE == 13 &&
                  H_ADDSUBX == 14 && H_MULX == 15 && H_PDIVX == 16 && H_ADDC == 17 &&
                  H_MULC == 18 && H_PDIVC == 19 && H_END == 20,
              "the PTX jump table lists the handlers in this order");
static_assert(H_POW == 21 && H_SIGN == 22 && H_CUBE == 23 && H_CBRT == 24 && H_TAN == 25 &&
                  H_ASIN == 26 && H_ACOS == 27 && H_ATAN == 28 && H_TANH == 29 &&
                  H_PASTE == 30 && kNumHandlers == 31,
              "the PTX jump table lists the rest of Table 3 in this order");
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

// POW and the transcendentals of the rest of Table 3 on the 4 top values; tok is the token
// that left the loop (POW's second operand is in its stack row).
__device__ __forceinline__ void run_ext4(uint32_t code, uint32_t tok, uint32_t tstk, float &t0,
                                         float &t1, float &t2, float &t3) {
    using A = Arith<float>;
    switch (code) {
    case H_POW: {
        float a0, a1, a2, a3;
        tmem_ld_row4(tstk + 4u * ((tok >> 12) & 0xffu), a0, a1, a2, a3);
        t0 = A::pow_(a0, t0); t1 = A::pow_(a1, t1); t2 = A::pow_(a2, t2); t3 = A::pow_(a3, t3);
    } break;
    case H_CBRT: t0 = A::cbrt_(t0); t1 = A::cbrt_(t1); t2 = A::cbrt_(t2); t3 = A::cbrt_(t3); break;
    case H_TAN: t0 = A::tan_(t0); t1 = A::tan_(t1); t2 = A::tan_(t2); t3 = A::tan_(t3); break;
    case H_ASIN: t0 = A::asin_(t0); t1 = A::asin_(t1); t2 = A::asin_(t2); t3 = A::asin_(t3); break;
    case H_ACOS: t0 = A::acos_(t0); t1 = A::acos_(t1); t2 = A::acos_(t2); t3 = A::acos_(t3); break;
    case H_ATAN: t0 = A::atan_(t0); t1 = A::atan_(t1); t2 = A::atan_(t2); t3 = A::atan_(t3); break;
    default: t0 = A::tanh_(t0); t1 = A::tanh_(t1); t2 = A::tanh_(t2); t3 = A::tanh_(t3); break;
    }
}

// prog: shared address of the packed program; xrow: shared address of this lane's first case
// of input row 0; tstk: tensor-memory address of the warp's stack row 0 (4 columns a row).
__device__ __forceinline__ void run_program_ptx4(uint32_t prog, uint32_t xrow, uint32_t tstk,
                                                 float (&top)[4], bool (&bad)[4]) {
    using A = Arith<float>;
    float t0 = 0.f, t1 = 0.f, t2 = 0.f, t3 = 0.f, m0 = 0.f, m1 = 0.f, m2 = 0.f, m3 = 0.f;
    // The loop's first dispatch loads token 0 and branches on the handler id in bits 24-28 of
    // the "current" token: start with token 0's id there.
    uint32_t cx = (lds_token(prog).x & 31u) << 24, cy = 0u, pa = prog;
    for (;;) {
        uint32_t code;
        asm volatile(BG_PTX_INTERP4
                     : "+f"(t0), "+f"(t1), "+f"(t2), "+f"(t3), "+f"(m0), "+f"(m1), "+f"(m2),
                       "+f"(m3), "+r"(cx), "+r"(cy), "+r"(pa), "=r"(code)
                     : "r"(xrow), "r"(tstk)
                     : "memory");
        if (code == 0) break;
        if (code >= H_POW) {   // the rest of Table 3
            run_ext4(code, cx, tstk, t0, t1, t2, t3);
            // cbrt, atan and tanh of a valid value are valid; pow, tan, asin, acos may not be
            if (code == H_CBRT || code == H_ATAN || code == H_TANH) continue;
        } else {
            switch (code) {
            case H_SIN:
            case H_COS: sincos4(t0, t1, t2, t3, static_cast<int>(code) - H_SIN); break;
            case H_EXP: t0 = A::exp_(t0); t1 = A::exp_(t1); t2 = A::exp_(t2); t3 = A::exp_(t3); break;
            default: t0 = A::plog(t0); t1 = A::plog(t1); t2 = A::plog(t2); t3 = A::plog(t3); break;
            }
            // sin, cos and the protected log of a valid value are finite and bounded (|ln|v||
            // <= 69.1 for |v| <= 1e30), and an invalid operand was recorded when it was
            // pushed, so only exp can produce a new invalid value here.
            if (code != H_EXP) continue;
        }
        m0 = A::track(m0, t0);
        m1 = A::track(m1, t1);
        m2 = A::track(m2, t2);
        m3 = A::track(m3, t3);
    }
    top[0] = t0; top[1] = t1; top[2] = t2; top[3] = t3;
    bad[0] = !A::ok(m0); bad[1] = !A::ok(m1); bad[2] = !A::ok(m2); bad[3] = !A::ok(m3);
}

#undef BG_PTX_TRACK
#undef BG_PTX_TRACK4
#undef BG_PTX_PDIV
#undef BG_PTX_DISPATCH
#undef BG_PTX_ROW
#undef BG_PTX_STROW
#undef BG_PTX_LDROW
#undef BG_PTX_XA
#undef BG_PTX_S
#undef BG_PTX_TBLPAD
#undef BG_PTX_PDIVX_BODY
#undef BG_PTX_ADDMUL_BODY
#undef BG_PTX_EXT_BODY

}  // namespace beagle
