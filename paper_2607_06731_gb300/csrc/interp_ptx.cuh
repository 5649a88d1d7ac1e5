// Interpreter loop for the FP32 path with 4 cases per lane, written in inline PTX so that the
// token dispatch is one indexed branch (brx.idx over a .branchtargets table) instead of a
// compare-and-branch tree, and each handler dispatches the next token itself. Semantics are
// those of run_program in score.cuh, handler for handler: the same fp32 operations in the
// same order (.rn forms, so nothing is contracted), the same protected division and square
// root. sin, cos, exp and the protected log leave the loop with their handler id; the caller
// applies them to the top of stack (CUDA's sinf, cosf, expf, logf) and re-enters.
//
// Validity: one pair of trackers per lane covers the lane's 4 cases, the running max and min of
// every value produced (three-operand max.NaN / min.NaN, so NaN sticks; four instructions per
// handler); a value is valid when min >= -1e30 and max <= 1e30. That is only used on chunks
// whose 4 x 32 cases all exist; a ragged last chunk runs the C++ loop with one tracker per
// case, so padding cases never affect the flag.
#pragma once

#include "score.cuh"

namespace beagle {

// Running max / min of three values; NaN in any operand gives NaN.
__device__ __forceinline__ float max3nan(float m, float a, float b) {
    float r;
    asm("max.NaN.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(m), "f"(a), "f"(b));
    return r;
}
__device__ __forceinline__ float min3nan(float m, float a, float b) {
    float r;
    asm("min.NaN.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(m), "f"(a), "f"(b));
    return r;
}

#define BG_PTX_TRACK4                                                                      \
    "max.NaN.f32 %4, %4, %0, %1;\n\tmax.NaN.f32 %4, %4, %2, %3;\n\t"                      \
    "min.NaN.f32 %5, %5, %0, %1;\n\tmin.NaN.f32 %5, %5, %2, %3;\n\t"
// dst = |den| > 1e-3 ? num / den : 1   (protected division reading)
#define BG_PTX_PDIV(DST, NUM, DEN)                                                         \
    "abs.f32 z, " DEN ";\n\tsetp.gt.f32 q, z, 0f3A83126F;\n\t"                             \
    "div.rn.f32 z, " NUM ", " DEN ";\n\tselp.f32 " DST ", z, 0f3F800000, q;\n\t"

// Operands: %0-%3 top of stack (4 cases), %4/%5 running max/min of the values, %6 operand word
// of the current token, %7/%8 next token (prefetched), %9 shared address of the token after
// that, %10 exit code (0 = program done, else the transcendental handler id), %11 shared
// address of this lane's first case of input row 0, %12 shared address of this lane's slot
// in stack row 0.
#define BG_PTX_DISPATCH                                                                    \
    "mov.b32 h, %7;\n\tmov.b32 %6, %8;\n\t"                                                \
    "ld.shared.v2.u32 {%7, %8}, [%9];\n\t"                                                 \
    "add.u32 %9, %9, 8;\n\t"                                                               \
    "brx.idx.uni h, TBL_%=;\n"
#define BG_PTX_ROW "and.b32 v, %6, 65535;\n\tadd.u32 rp, %12, v;\n\t"
#define BG_PTX_XA "shr.u32 v, %6, 16;\n\tadd.u32 xa, %11, v;\n\t"
#define BG_PTX_S "mov.b32 s, %6;\n\t"
#define BG_PTX_PUSHC(R, OFF)                                                               \
    "PUSHC" #R "_%=:\n\t" BG_PTX_S                                                         \
    "st.shared.v4.f32 [%12+" #OFF "], {%0, %1, %2, %3};\n\t"                               \
    "mov.f32 %0, s;\n\tmov.f32 %1, s;\n\tmov.f32 %2, s;\n\tmov.f32 %3, s;\n\t"             \
    BG_PTX_DISPATCH

#define BG_PTX_INTERP4                                                                     \
    "{\n\t"                                                                                \
    ".reg .pred q;\n\t"                                                                    \
    ".reg .b32 h, v, rp, xa;\n\t"                                                          \
    ".reg .f32 a0, a1, a2, a3, s, z;\n\t"                                                  \
    "TBL_%=: .branchtargets PUSHX_%=, DUP_%=, SWAP_%=, DEL_%=, ADD_%=, SUB_%=, MUL_%=, "   \
    "PDIV_%=, SIN_%=, COS_%=, EXP_%=, PLOG_%=, PSQRT_%=, SQUARE_%=, ADDX_%=, SUBX_%=, "     \
    "MULX_%=, PDIVX_%=, ADDC_%=, MULC_%=, PDIVC_%=, END_%=, PUSHC0_%=, PUSHC1_%=, "         \
    "PUSHC2_%=, PUSHC3_%=, PUSHC4_%=, PUSHC5_%=, PUSHC6_%=, PUSHC7_%=, PUSHC8_%=, "        \
    "PUSHC9_%=, PUSHC10_%=, PUSHC11_%=, PUSHC12_%=, PUSHC13_%=, PUSHC14_%=;\n\t"           \
    BG_PTX_DISPATCH                                                                        \
    "PUSHX_%=:\n\t" BG_PTX_ROW BG_PTX_XA                                                   \
    "st.shared.v4.f32 [rp], {%0, %1, %2, %3};\n\t"                                         \
    "ld.shared.v4.f32 {%0, %1, %2, %3}, [xa];\n\t"                                         \
    BG_PTX_DISPATCH                                                                        \
    "DUP_%=:\n\t" BG_PTX_ROW                                                               \
    "st.shared.v4.f32 [rp], {%0, %1, %2, %3};\n\t"                                         \
    BG_PTX_DISPATCH                                                                        \
    "SWAP_%=:\n\t" BG_PTX_ROW                                                              \
    "ld.shared.v4.f32 {a0, a1, a2, a3}, [rp];\n\t"                                         \
    "st.shared.v4.f32 [rp], {%0, %1, %2, %3};\n\t"                                         \
    "mov.f32 %0, a0;\n\tmov.f32 %1, a1;\n\tmov.f32 %2, a2;\n\tmov.f32 %3, a3;\n\t"         \
    BG_PTX_DISPATCH                                                                        \
    "DEL_%=:\n\t" BG_PTX_ROW                                                               \
    "ld.shared.v4.f32 {%0, %1, %2, %3}, [rp];\n\t"                                         \
    BG_PTX_DISPATCH                                                                        \
    "ADD_%=:\n\t" BG_PTX_ROW                                                               \
    "ld.shared.v4.f32 {a0, a1, a2, a3}, [rp];\n\t"                                         \
    "add.rn.f32 %0, a0, %0;\n\tadd.rn.f32 %1, a1, %1;\n\t"                                 \
    "add.rn.f32 %2, a2, %2;\n\tadd.rn.f32 %3, a3, %3;\n\t"                                 \
    BG_PTX_TRACK4 BG_PTX_DISPATCH                                                          \
    "SUB_%=:\n\t" BG_PTX_ROW                                                               \
    "ld.shared.v4.f32 {a0, a1, a2, a3}, [rp];\n\t"                                         \
    "sub.rn.f32 %0, a0, %0;\n\tsub.rn.f32 %1, a1, %1;\n\t"                                 \
    "sub.rn.f32 %2, a2, %2;\n\tsub.rn.f32 %3, a3, %3;\n\t"                                 \
    BG_PTX_TRACK4 BG_PTX_DISPATCH                                                          \
    "MUL_%=:\n\t" BG_PTX_ROW                                                               \
    "ld.shared.v4.f32 {a0, a1, a2, a3}, [rp];\n\t"                                         \
    "mul.rn.f32 %0, a0, %0;\n\tmul.rn.f32 %1, a1, %1;\n\t"                                 \
    "mul.rn.f32 %2, a2, %2;\n\tmul.rn.f32 %3, a3, %3;\n\t"                                 \
    BG_PTX_TRACK4 BG_PTX_DISPATCH                                                          \
    "PDIV_%=:\n\t" BG_PTX_ROW                                                              \
    "ld.shared.v4.f32 {a0, a1, a2, a3}, [rp];\n\t"                                         \
    BG_PTX_PDIV("%0", "a0", "%0") BG_PTX_PDIV("%1", "a1", "%1")                            \
    BG_PTX_PDIV("%2", "a2", "%2") BG_PTX_PDIV("%3", "a3", "%3")                            \
    BG_PTX_TRACK4 BG_PTX_DISPATCH                                                          \
    "SIN_%=:\n\tmov.u32 %10, 8;\n\tbra.uni OUT_%=;\n"                                       \
    "COS_%=:\n\tmov.u32 %10, 9;\n\tbra.uni OUT_%=;\n"                                       \
    "EXP_%=:\n\tmov.u32 %10, 10;\n\tbra.uni OUT_%=;\n"                                      \
    "PLOG_%=:\n\tmov.u32 %10, 11;\n\tbra.uni OUT_%=;\n"                                     \
    "PSQRT_%=:\n\t"                                                                        \
    "abs.f32 %0, %0;\n\tsqrt.rn.f32 %0, %0;\n\tabs.f32 %1, %1;\n\tsqrt.rn.f32 %1, %1;\n\t" \
    "abs.f32 %2, %2;\n\tsqrt.rn.f32 %2, %2;\n\tabs.f32 %3, %3;\n\tsqrt.rn.f32 %3, %3;\n\t" \
    BG_PTX_TRACK4 BG_PTX_DISPATCH                                                          \
    "SQUARE_%=:\n\t"                                                                       \
    "mul.rn.f32 %0, %0, %0;\n\tmul.rn.f32 %1, %1, %1;\n\t"                                 \
    "mul.rn.f32 %2, %2, %2;\n\tmul.rn.f32 %3, %3, %3;\n\t"                                 \
    BG_PTX_TRACK4 BG_PTX_DISPATCH                                                          \
    "ADDX_%=:\n\t" BG_PTX_XA                                                               \
    "ld.shared.v4.f32 {a0, a1, a2, a3}, [xa];\n\t"                                         \
    "add.rn.f32 %0, %0, a0;\n\tadd.rn.f32 %1, %1, a1;\n\t"                                 \
    "add.rn.f32 %2, %2, a2;\n\tadd.rn.f32 %3, %3, a3;\n\t"                                 \
    BG_PTX_TRACK4 BG_PTX_DISPATCH                                                          \
    "SUBX_%=:\n\t" BG_PTX_XA                                                               \
    "ld.shared.v4.f32 {a0, a1, a2, a3}, [xa];\n\t"                                         \
    "sub.rn.f32 %0, %0, a0;\n\tsub.rn.f32 %1, %1, a1;\n\t"                                 \
    "sub.rn.f32 %2, %2, a2;\n\tsub.rn.f32 %3, %3, a3;\n\t"                                 \
    BG_PTX_TRACK4 BG_PTX_DISPATCH                                                          \
    "MULX_%=:\n\t" BG_PTX_XA                                                               \
    "ld.shared.v4.f32 {a0, a1, a2, a3}, [xa];\n\t"                                         \
    "mul.rn.f32 %0, %0, a0;\n\tmul.rn.f32 %1, %1, a1;\n\t"                                 \
    "mul.rn.f32 %2, %2, a2;\n\tmul.rn.f32 %3, %3, a3;\n\t"                                 \
    BG_PTX_TRACK4 BG_PTX_DISPATCH                                                          \
    "PDIVX_%=:\n\t" BG_PTX_XA                                                              \
    "ld.shared.v4.f32 {a0, a1, a2, a3}, [xa];\n\t"                                         \
    BG_PTX_PDIV("%0", "%0", "a0") BG_PTX_PDIV("%1", "%1", "a1")                            \
    BG_PTX_PDIV("%2", "%2", "a2") BG_PTX_PDIV("%3", "%3", "a3")                            \
    BG_PTX_TRACK4 BG_PTX_DISPATCH                                                          \
    "ADDC_%=:\n\t" BG_PTX_S                                                                \
    "add.rn.f32 %0, %0, s;\n\tadd.rn.f32 %1, %1, s;\n\t"                                   \
    "add.rn.f32 %2, %2, s;\n\tadd.rn.f32 %3, %3, s;\n\t"                                   \
    BG_PTX_TRACK4 BG_PTX_DISPATCH                                                          \
    "MULC_%=:\n\t" BG_PTX_S                                                                \
    "mul.rn.f32 %0, %0, s;\n\tmul.rn.f32 %1, %1, s;\n\t"                                   \
    "mul.rn.f32 %2, %2, s;\n\tmul.rn.f32 %3, %3, s;\n\t"                                   \
    BG_PTX_TRACK4 BG_PTX_DISPATCH                                                          \
    "PDIVC_%=:\n\t" BG_PTX_S                                                               \
    BG_PTX_PDIV("%0", "%0", "s") BG_PTX_PDIV("%1", "%1", "s")                              \
    BG_PTX_PDIV("%2", "%2", "s") BG_PTX_PDIV("%3", "%3", "s")                              \
    BG_PTX_TRACK4 BG_PTX_DISPATCH                                                          \
    BG_PTX_PUSHC(0, 0) BG_PTX_PUSHC(1, 512) BG_PTX_PUSHC(2, 1024) BG_PTX_PUSHC(3, 1536)     \
    BG_PTX_PUSHC(4, 2048) BG_PTX_PUSHC(5, 2560) BG_PTX_PUSHC(6, 3072)                      \
    BG_PTX_PUSHC(7, 3584) BG_PTX_PUSHC(8, 4096) BG_PTX_PUSHC(9, 4608)                      \
    BG_PTX_PUSHC(10, 5120) BG_PTX_PUSHC(11, 5632) BG_PTX_PUSHC(12, 6144)                   \
    BG_PTX_PUSHC(13, 6656) BG_PTX_PUSHC(14, 7168)                                          \
    "END_%=:\n\tmov.u32 %10, 0;\n"                                                          \
    "OUT_%=:\n\t"                                                                          \
    "}"

static_assert(H_PUSHX == 0 && H_DUP == 1 && H_SWAP == 2 && H_DEL == 3 && H_ADD == 4 &&
                  H_SUB == 5 && H_MUL == 6 && H_PDIV == 7 && H_SIN == 8 && H_COS == 9 &&
                  H_EXP == 10 && H_PLOG == 11 && H_PSQRT == 12 && H_SQUARE == 13 &&
                  H_ADDX == 14 && H_SUBX == 15 && H_MULX == 16 && H_PDIVX == 17 &&
                  H_ADDC == 18 && H_MULC == 19 && H_PDIVC == 20 && H_END == 21 &&
                  H_PUSHC0 == 22 && H_COUNT == 37,
              "the PTX jump table lists the handlers in this order");
static_assert(StackGeom<float, 4>::kRowBytes == 512 && kMaxDepth == 16,
              "the PTX constant pushes hard-code 15 stack rows of 512 bytes");

// Run the packed program on a chunk whose 4 x 32 cases all exist; see run_program.
__device__ __forceinline__ void run_program_ptx4(uint32_t prog, uint32_t xrow, uint32_t stk,
                                                 float (&top)[4], bool (&bad)[4]) {
    using A = Arith<float>;
    float t0 = 0.f, t1 = 0.f, t2 = 0.f, t3 = 0.f, hi = 0.f, lo = 0.f;
    const uint2 first = lds_token(prog);
    // The loop's first step takes the "next" token: start with token 0 there.
    uint32_t cy = 0u, nx = first.x, ny = first.y, pa = prog + 8u;
    for (;;) {
        uint32_t code;
        asm volatile(BG_PTX_INTERP4
                     : "+f"(t0), "+f"(t1), "+f"(t2), "+f"(t3), "+f"(hi), "+f"(lo), "+r"(cy),
                       "+r"(nx), "+r"(ny), "+r"(pa), "=r"(code)
                     : "r"(xrow), "r"(stk)
                     : "memory");
        if (code == 0) break;
        switch (code) {
        case H_SIN: t0 = A::sin_(t0); t1 = A::sin_(t1); t2 = A::sin_(t2); t3 = A::sin_(t3); break;
        case H_COS: t0 = A::cos_(t0); t1 = A::cos_(t1); t2 = A::cos_(t2); t3 = A::cos_(t3); break;
        case H_EXP: t0 = A::exp_(t0); t1 = A::exp_(t1); t2 = A::exp_(t2); t3 = A::exp_(t3); break;
        default: t0 = A::plog(t0); t1 = A::plog(t1); t2 = A::plog(t2); t3 = A::plog(t3); break;
        }
        hi = max3nan(max3nan(hi, t0, t1), t2, t3);
        lo = min3nan(min3nan(lo, t0, t1), t2, t3);
    }
    top[0] = t0; top[1] = t1; top[2] = t2; top[3] = t3;
    const bool b = !(hi <= Arith<float>::kBig && lo >= -Arith<float>::kBig);
    bad[0] = bad[1] = bad[2] = bad[3] = b;
}

#undef BG_PTX_TRACK4
#undef BG_PTX_PDIV
#undef BG_PTX_DISPATCH
#undef BG_PTX_ROW
#undef BG_PTX_XA
#undef BG_PTX_S
#undef BG_PTX_PUSHC

}  // namespace beagle
