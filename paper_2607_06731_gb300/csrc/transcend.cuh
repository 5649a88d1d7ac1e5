// sin, cos and the protected log of the FP32 path (exp is CUDA's expf).
//
// The interpreter applies each of these to the 4 cases of a lane at once. CUDA's sinf, cosf
// and logf are written for one argument (sinf and cosf branch per call to a slow path for
// large arguments), so four calls run one after another. The forms here are branch-free in
// the common case, so the four evaluations interleave, and sin and cos share one body
// (CUDA's expf, built on the hardware exponential, stays faster than a polynomial form):
//
//   sin, cos  Cody and Waite's additive range reduction k = round(x 2/pi), r = x - k pi/2 with
//             pi/2 held as three fp32 parts (fused multiply-adds; the first step is exact since
//             x and k C1 share their low bits), |r| <= pi/4 (1 % more when the rounded quotient
//             is off by one). Quadrant q = k for sin and k + 1 for cos (cos x = sin(x + pi/2));
//             odd q takes the cosine polynomial and q & 2 flips the sign bit. sin r = r + r^3 P(s),
//             cos r = 1 + s Q(s), s = r^2. Arguments above 65536 in magnitude (and NaN) take
//             CUDA's sinf/cosf on the lanes that hold them.
//   plog      ln|x| for |x| > 1e-3, else 0: |x| = m 2^e with m in (sqrt(1/2), sqrt(2)],
//             ln m = f + f^2 (-1/2 + f L(f)), f = m - 1 (exact), plus e ln 2 in two parts.
//             Only valid operands matter (finite, |x| <= 1e30): the results for others are
//             never used, because the program is already invalid.
//
// sincos_fast2 and plog2 take two arguments at once with the paired FP32 instructions, with
// the same bits as the one-argument forms.
//
// P, Q and L are polynomials whose coefficients gen_poly.py (beside this file) fits to
// relative error and rounds to fp32; with exact evaluation their maximum relative errors are
// 3.6e-9, 3.9e-9 and 6.6e-9 (under 0.1 ulp). Each result is a function of its argument alone,
// so every path and launch shape gives the same bits.
#pragma once

namespace beagle {

constexpr float kTwoOverPi = 0x1.45f306p-1f;
constexpr float kPio2C1 = 0x1.921fb6p+0f;
constexpr float kPio2C2 = -0x1.777a5cp-25f;
constexpr float kPio2C3 = -0x1.ee59dap-50f;
constexpr float kSinP0 = -0x1.555556p-3f, kSinP1 = 0x1.111108p-7f, kSinP2 = -0x1.a00f12p-13f,
                kSinP3 = 0x1.6cb80cp-19f;
constexpr float kCosQ0 = -0x1.0p-1f, kCosQ1 = 0x1.55553ap-5f, kCosQ2 = -0x1.6c0756p-10f,
                kCosQ3 = 0x1.98f230p-16f;
constexpr float kSinCosFastLimit = 0x1.0p+16f;   // 65536

constexpr float kLn2Hi = 0x1.62e430p-1f;
constexpr float kLn2Lo = -0x1.05c610p-29f;
constexpr float kLogL0 = 0x1.555554p-2f, kLogL1 = -0x1.000226p-2f, kLogL2 = 0x1.99a01ep-3f,
                kLogL3 = -0x1.547254p-3f, kLogL4 = 0x1.22d8aep-3f, kLogL5 = -0x1.0d837cp-3f,
                kLogL6 = 0x1.0562e0p-3f, kLogL7 = -0x1.38ceaap-4f;
constexpr float kLogTiny = 1e-3f;

// The same constants as fp32 bit patterns (hex digits), for the inline-PTX interpreter loops:
// BG_PTX_F32 gives a PTX fp32 immediate, BG_PTX_PAIR the 64-bit immediate of the pair (c, c).
// Each is checked against its value above at compile time.
#define BG_K_TWO_OVER_PI 3F22F983
#define BG_K_PIO2_C1 3FC90FDB
#define BG_K_PIO2_C2 B33BBD2E
#define BG_K_PIO2_C3 A6F72CED
#define BG_K_NPIO2_C1 BFC90FDB
#define BG_K_NPIO2_C2 333BBD2E
#define BG_K_NPIO2_C3 26F72CED
#define BG_K_SIN_P0 BE2AAAAB
#define BG_K_SIN_P1 3C088884
#define BG_K_SIN_P2 B9500789
#define BG_K_SIN_P3 36365C06
#define BG_K_COS_Q0 BF000000
#define BG_K_COS_Q1 3D2AAA9D
#define BG_K_COS_Q2 BAB603AB
#define BG_K_COS_Q3 37CC7918
#define BG_K_SINCOS_LIMIT 47800000
#define BG_K_LN2_HI 3F317218
#define BG_K_LN2_LO B102E308
#define BG_K_LOG_L0 3EAAAAAA
#define BG_K_LOG_L1 BE800113
#define BG_K_LOG_L2 3E4CD00F
#define BG_K_LOG_L3 BE2A392A
#define BG_K_LOG_L4 3E116C57
#define BG_K_LOG_L5 BE06C1BE
#define BG_K_LOG_L6 3E02B170
#define BG_K_LOG_L7 BD9C6755
#define BG_K_LOG_TINY 3A83126F
#define BG_K_MAGIC 4B400000
#define BG_K_NMAGIC CB400000
#define BG_K_ONE 3F800000
#define BG_K_NONE BF800000
#define BG_K_NHALF BF000000
#define BG_STR_(x) #x
#define BG_STR(x) BG_STR_(x)
#define BG_HEX_(h) 0x##h##u
#define BG_HEX(h) BG_HEX_(h)
#define BG_PTX_F32(h) "0f" BG_STR(h)
#define BG_PTX_PAIR(h) "0x" BG_STR(h) BG_STR(h)
#define BG_CHECK_BITS(v, h) static_assert(__builtin_bit_cast(unsigned, v) == BG_HEX(h), #v)
BG_CHECK_BITS(kTwoOverPi, BG_K_TWO_OVER_PI);
BG_CHECK_BITS(kPio2C1, BG_K_PIO2_C1);
BG_CHECK_BITS(kPio2C2, BG_K_PIO2_C2);
BG_CHECK_BITS(kPio2C3, BG_K_PIO2_C3);
BG_CHECK_BITS(-kPio2C1, BG_K_NPIO2_C1);
BG_CHECK_BITS(-kPio2C2, BG_K_NPIO2_C2);
BG_CHECK_BITS(-kPio2C3, BG_K_NPIO2_C3);
BG_CHECK_BITS(kSinP0, BG_K_SIN_P0);
BG_CHECK_BITS(kSinP1, BG_K_SIN_P1);
BG_CHECK_BITS(kSinP2, BG_K_SIN_P2);
BG_CHECK_BITS(kSinP3, BG_K_SIN_P3);
BG_CHECK_BITS(kCosQ0, BG_K_COS_Q0);
BG_CHECK_BITS(kCosQ1, BG_K_COS_Q1);
BG_CHECK_BITS(kCosQ2, BG_K_COS_Q2);
BG_CHECK_BITS(kCosQ3, BG_K_COS_Q3);
BG_CHECK_BITS(kSinCosFastLimit, BG_K_SINCOS_LIMIT);
BG_CHECK_BITS(kLn2Hi, BG_K_LN2_HI);
BG_CHECK_BITS(kLn2Lo, BG_K_LN2_LO);
BG_CHECK_BITS(kLogL0, BG_K_LOG_L0);
BG_CHECK_BITS(kLogL1, BG_K_LOG_L1);
BG_CHECK_BITS(kLogL2, BG_K_LOG_L2);
BG_CHECK_BITS(kLogL3, BG_K_LOG_L3);
BG_CHECK_BITS(kLogL4, BG_K_LOG_L4);
BG_CHECK_BITS(kLogL5, BG_K_LOG_L5);
BG_CHECK_BITS(kLogL6, BG_K_LOG_L6);
BG_CHECK_BITS(kLogL7, BG_K_LOG_L7);
BG_CHECK_BITS(kLogTiny, BG_K_LOG_TINY);
BG_CHECK_BITS(1.0f, BG_K_ONE);
BG_CHECK_BITS(-1.0f, BG_K_NONE);
BG_CHECK_BITS(-0.5f, BG_K_NHALF);

// ---------------------------------------------------------------- sin, cos (qo = 0 / 1)
// Adding 1.5 * 2^23 rounds a float of magnitude below 2^22 to an integer held in the low
// mantissa bits: the rounding and the conversion to int without the conversion unit.
constexpr float kRoundMagic = 0x1.8p+23f;
constexpr int kRoundMagicBits = 0x4b400000;
BG_CHECK_BITS(kRoundMagic, BG_K_MAGIC);
BG_CHECK_BITS(-kRoundMagic, BG_K_NMAGIC);

__device__ __forceinline__ float sincos_fast(float x, int qo) {
    const float t = fmaf(x, kTwoOverPi, kRoundMagic);   // |x 2/pi| < 2^22 on this path
    const float kf = t - kRoundMagic;                    // k = x 2/pi rounded to nearest
    float r = fmaf(-kf, kPio2C1, x);
    r = fmaf(-kf, kPio2C2, r);
    r = fmaf(-kf, kPio2C3, r);
    const int q = (__float_as_int(t) - kRoundMagicBits) + qo;
    const float s = r * r;
    // Both polynomials, then a select: fewer instructions than selecting their coefficients.
    const float ps = fmaf(fmaf(fmaf(kSinP3, s, kSinP2), s, kSinP1), s, kSinP0);
    const float pc = fmaf(fmaf(fmaf(kCosQ3, s, kCosQ2), s, kCosQ1), s, kCosQ0);
    const float vs = fmaf(r * s, ps, r);
    const float vc = fmaf(s, pc, 1.0f);
    const float v = (q & 1) ? vc : vs;
    return __int_as_float(__float_as_int(v) ^ ((q & 2) << 30));
}

// Large arguments: one out-of-line copy of CUDA's functions, so that their long reduction
// code stays out of the interpreter's instruction stream.
static __device__ __noinline__ float sincos_slow(float x, int qo) { return qo ? cosf(x) : sinf(x); }

__device__ __forceinline__ float sincos_dev(float x, int qo) {
    if (fabsf(x) <= kSinCosFastLimit) return sincos_fast(x, qo);
    return sincos_slow(x, qo);
}

__device__ __forceinline__ void sincos4(float &t0, float &t1, float &t2, float &t3, int qo) {
    const float a0 = t0, a1 = t1, a2 = t2, a3 = t3;
    t0 = sincos_fast(a0, qo);
    t1 = sincos_fast(a1, qo);
    t2 = sincos_fast(a2, qo);
    t3 = sincos_fast(a3, qo);
    // One test for the four: their magnitudes' sum (additions, not compares) is at most the
    // limit only if each is; NaN fails it too. Each case then decides for itself.
    const float big = (fabsf(a0) + fabsf(a1)) + (fabsf(a2) + fabsf(a3));
    if (!(big <= kSinCosFastLimit)) {
        if (!(fabsf(a0) <= kSinCosFastLimit)) t0 = sincos_slow(a0, qo);
        if (!(fabsf(a1) <= kSinCosFastLimit)) t1 = sincos_slow(a1, qo);
        if (!(fabsf(a2) <= kSinCosFastLimit)) t2 = sincos_slow(a2, qo);
        if (!(fabsf(a3) <= kSinCosFastLimit)) t3 = sincos_slow(a3, qo);
    }
}

// The same on two arguments at once with the paired FP32 instructions (FFMA2, FADD2, FMUL2:
// each half rounded exactly like its scalar form), so each result has the bits sincos_fast
// gives it.
__device__ __forceinline__ float2 f2(float c) { return make_float2(c, c); }

__device__ __forceinline__ float2 sincos_fast2(float2 x, int qo) {
    const float2 t = __ffma2_rn(x, f2(kTwoOverPi), f2(kRoundMagic));
    const float2 kf = __fadd2_rn(t, f2(-kRoundMagic));
    float2 r = __ffma2_rn(kf, f2(-kPio2C1), x);
    r = __ffma2_rn(kf, f2(-kPio2C2), r);
    r = __ffma2_rn(kf, f2(-kPio2C3), r);
    const float2 s = __fmul2_rn(r, r);
    const float2 ps = __ffma2_rn(
        __ffma2_rn(__ffma2_rn(f2(kSinP3), s, f2(kSinP2)), s, f2(kSinP1)), s, f2(kSinP0));
    const float2 pc = __ffma2_rn(
        __ffma2_rn(__ffma2_rn(f2(kCosQ3), s, f2(kCosQ2)), s, f2(kCosQ1)), s, f2(kCosQ0));
    const float2 vs = __ffma2_rn(__fmul2_rn(r, s), ps, r);
    const float2 vc = __ffma2_rn(s, pc, f2(1.0f));
    const int qx = (__float_as_int(t.x) - kRoundMagicBits) + qo;
    const int qy = (__float_as_int(t.y) - kRoundMagicBits) + qo;
    const float vx = (qx & 1) ? vc.x : vs.x;
    const float vy = (qy & 1) ? vc.y : vs.y;
    return make_float2(__int_as_float(__float_as_int(vx) ^ ((qx & 2) << 30)),
                       __int_as_float(__float_as_int(vy) ^ ((qy & 2) << 30)));
}

// sin or cos of the four values of two pairs, large arguments as in sincos4.
__device__ __forceinline__ void sincos4_paired(float2 &a, float2 &b, int qo) {
    const float2 a0 = a, b0 = b;
    a = sincos_fast2(a0, qo);
    b = sincos_fast2(b0, qo);
    const float big = (fabsf(a0.x) + fabsf(a0.y)) + (fabsf(b0.x) + fabsf(b0.y));
    if (!(big <= kSinCosFastLimit)) {
        if (!(fabsf(a0.x) <= kSinCosFastLimit)) a.x = sincos_slow(a0.x, qo);
        if (!(fabsf(a0.y) <= kSinCosFastLimit)) a.y = sincos_slow(a0.y, qo);
        if (!(fabsf(b0.x) <= kSinCosFastLimit)) b.x = sincos_slow(b0.x, qo);
        if (!(fabsf(b0.y) <= kSinCosFastLimit)) b.y = sincos_slow(b0.y, qo);
    }
}

// ---------------------------------------------------------------- protected log
__device__ __forceinline__ float plog_dev(float x) {
    const float a = fabsf(x);
    // m in [b, 2b), b = 0x3f3504f4 (just above sqrt(1/2)): adding 1.0's bits minus b's to
    // |x|'s bits carries into the exponent field exactly when |x|'s mantissa is at least 2b, so
    // the exponent field gives e and the low 23 bits plus b give m (no compare, no select).
    const uint32_t ix = __float_as_uint(a) + (0x3f800000u - 0x3f3504f4u);
    const int e = static_cast<int>(ix >> 23) - 127;
    const float f = __uint_as_float((ix & 0x007fffffu) + 0x3f3504f4u) - 1.0f;
    float l = fmaf(fmaf(fmaf(kLogL7, f, kLogL6), f, kLogL5), f, kLogL4);
    l = fmaf(fmaf(fmaf(fmaf(l, f, kLogL3), f, kLogL2), f, kLogL1), f, kLogL0);
    const float lnm = fmaf(f * f, fmaf(f, l, -0.5f), f);
    const float ef = __int_as_float(kRoundMagicBits + e) - kRoundMagic;   // exact for |e| < 2^22
    const float v = fmaf(ef, kLn2Hi, fmaf(ef, kLn2Lo, lnm));
    return a > kLogTiny ? v : 0.0f;
}

// The protected log of two arguments at once, the floating-point steps of plog_dev paired.
__device__ __forceinline__ float2 plog2(float2 x) {
    const float ax = fabsf(x.x), ay = fabsf(x.y);
    const uint32_t ix = __float_as_uint(ax) + (0x3f800000u - 0x3f3504f4u);
    const uint32_t iy = __float_as_uint(ay) + (0x3f800000u - 0x3f3504f4u);
    const int ex = static_cast<int>(ix >> 23) - 127, ey = static_cast<int>(iy >> 23) - 127;
    const float2 f = __fadd2_rn(make_float2(__uint_as_float((ix & 0x007fffffu) + 0x3f3504f4u),
                                            __uint_as_float((iy & 0x007fffffu) + 0x3f3504f4u)),
                                f2(-1.0f));
    float2 l = __ffma2_rn(__ffma2_rn(__ffma2_rn(f2(kLogL7), f, f2(kLogL6)), f, f2(kLogL5)), f,
                          f2(kLogL4));
    l = __ffma2_rn(__ffma2_rn(__ffma2_rn(__ffma2_rn(l, f, f2(kLogL3)), f, f2(kLogL2)), f,
                              f2(kLogL1)), f, f2(kLogL0));
    const float2 lnm = __ffma2_rn(__fmul2_rn(f, f), __ffma2_rn(f, l, f2(-0.5f)), f);
    const float2 ef = __fadd2_rn(make_float2(__int_as_float(kRoundMagicBits + ex),
                                             __int_as_float(kRoundMagicBits + ey)),
                                 f2(-kRoundMagic));
    const float2 v = __ffma2_rn(ef, f2(kLn2Hi), __ffma2_rn(ef, f2(kLn2Lo), lnm));
    return make_float2(ax > kLogTiny ? v.x : 0.0f, ay > kLogTiny ? v.y : 0.0f);
}

}  // namespace beagle
