// interval.cuh -- rectangular complex intervals with directed rounding.
//
// Section 2.5 of Steinke & Sainudiin (CCA 2010): a real interval [lo, hi]
// is carried by its two bounds; every lower bound is computed with rounding
// toward -inf and every upper bound with rounding toward +inf, so the
// machine interval always contains the exact real result.  A complex
// interval is the rectangle [rl, rh] + i [il, ih].  Addition and subtraction
// act componentwise; multiplication expands (z1 w1 - z2 w2) + i (z1 w2 +
// z2 w1) into real interval products.
//
// Only the IEEE directed-rounding intrinsics are used (__dadd_rd, __dmul_ru,
// __fma_rd, ... and their binary32 counterparts).  They are never contracted
// or reassociated by the compiler.  A fused multiply-add is used only where
// its single rounding goes in the direction of the bound it produces:
//   lower bound of a*b - c*d  =  fma_rd(a, b, -RU(c*d))  <=  a*b - c*d
// with (a, b) the endpoint pair that minimises the first product and (c, d)
// the pair that maximises the second one.
#pragma once
#include <cstdint>

namespace ssm {

// aligned to its size (16 B for binary32, 32 B for binary64) so that global
// and shared memory accesses move it with 128-bit vector instructions
template <typename T>
struct alignas(4 * sizeof(T)) CI {
    T rl, rh, il, ih;   // [rl, rh] + i [il, ih]
};

// ---- directed rounding --------------------------------------------------------

// GB300 retires a binary64 fma at about 1.19 times the rate of a binary64
// add or product (625 against 527 G operations/s, ssmul_debug_pipe_rate).
// An add a + b written as fma(a, 1, b) and a product a b written as
// fma(a, b, z) round the same exact value once, so they give the same bits;
// z = +0 when rounding down and -0 when rounding up (and to nearest) keeps
// even the sign of an exact zero product: +0 + (+0) and (-0) + (+0) are +0
// and -0 under rounding down, (+0) + (-0) and (-0) + (-0) are +0 and -0
// otherwise.  The unit and the zeros are read from constant memory, so the
// compiler cannot turn the fmas back into adds and products.
#ifndef SSMUL_F64_VIA_FMA
#define SSMUL_F64_VIA_FMA 1
#endif
__constant__ double c_f64_unit[3] = {1.0, 0.0, -0.0};

__device__ __forceinline__ double add_dn(double a, double b) {
    return SSMUL_F64_VIA_FMA ? __fma_rd(a, c_f64_unit[0], b) : __dadd_rd(a, b);
}
__device__ __forceinline__ double add_up(double a, double b) {
    return SSMUL_F64_VIA_FMA ? __fma_ru(a, c_f64_unit[0], b) : __dadd_ru(a, b);
}
__device__ __forceinline__ double sub_dn(double a, double b) {
    return SSMUL_F64_VIA_FMA ? __fma_rd(-b, c_f64_unit[0], a) : __dsub_rd(a, b);
}
__device__ __forceinline__ double sub_up(double a, double b) {
    return SSMUL_F64_VIA_FMA ? __fma_ru(-b, c_f64_unit[0], a) : __dsub_ru(a, b);
}
__device__ __forceinline__ double mul_dn(double a, double b) {
    return SSMUL_F64_VIA_FMA ? __fma_rd(a, b, c_f64_unit[1]) : __dmul_rd(a, b);
}
__device__ __forceinline__ double mul_up(double a, double b) {
    return SSMUL_F64_VIA_FMA ? __fma_ru(a, b, c_f64_unit[2]) : __dmul_ru(a, b);
}
__device__ __forceinline__ double add_rn(double a, double b) {
    return SSMUL_F64_VIA_FMA ? __fma_rn(a, c_f64_unit[0], b) : __dadd_rn(a, b);
}
__device__ __forceinline__ double sub_rn(double a, double b) {
    return SSMUL_F64_VIA_FMA ? __fma_rn(-b, c_f64_unit[0], a) : __dsub_rn(a, b);
}
__device__ __forceinline__ double mul_rn(double a, double b) {
    return SSMUL_F64_VIA_FMA ? __fma_rn(a, b, c_f64_unit[2]) : __dmul_rn(a, b);
}
__device__ __forceinline__ double fma_dn(double a, double b, double c) { return __fma_rd(a, b, c); }
__device__ __forceinline__ double fma_up(double a, double b, double c) { return __fma_ru(a, b, c); }

__device__ __forceinline__ float add_dn(float a, float b) { return __fadd_rd(a, b); }
__device__ __forceinline__ float add_up(float a, float b) { return __fadd_ru(a, b); }
__device__ __forceinline__ float sub_dn(float a, float b) { return __fsub_rd(a, b); }
__device__ __forceinline__ float sub_up(float a, float b) { return __fsub_ru(a, b); }
__device__ __forceinline__ float mul_dn(float a, float b) { return __fmul_rd(a, b); }
__device__ __forceinline__ float mul_up(float a, float b) { return __fmul_ru(a, b); }
__device__ __forceinline__ float fma_dn(float a, float b, float c) { return __fmaf_rd(a, b, c); }
__device__ __forceinline__ float fma_up(float a, float b, float c) { return __fmaf_ru(a, b, c); }

// Sign bit tests on the integer pipe (a binary64 compare would occupy the
// narrow fp64 pipe).  -0.0 counts as negative; every use below stays correct
// for either sign of zero.
__device__ __forceinline__ bool neg(double x) { return __double2hiint(x) < 0; }
__device__ __forceinline__ bool neg(float x) { return __float_as_int(x) < 0; }

// Exact negation by flipping the sign bit on the integer pipe: for values
// that are selected or stored rather than fed straight into an arithmetic
// operation (where the compiler folds a negation into an operand modifier).
__device__ __forceinline__ double flip(double x) {
    return __hiloint2double(__double2hiint(x) ^ int(0x80000000), __double2loint(x));
}
__device__ __forceinline__ float flip(float x) { return __int_as_float(__float_as_int(x) ^ int(0x80000000)); }

// 2^-k for 0 <= k <= 1022, built from its exponent bits
__device__ __forceinline__ double pow2_neg(int k) {
    return __longlong_as_double(static_cast<long long>(1023 - k) << 52);
}

// Exact binary64 value of an integer |v| < 2^31 built from its bits on the
// integer pipe (an int-to-double conversion would occupy the binary64 pipe).
__device__ __forceinline__ double int_to_double(int v) {
    const unsigned int a = v < 0 ? 0u - unsigned(v) : unsigned(v);
    const int e = 31 - __clz(int(a | 1u));                 // floor(log2 a) for a >= 1
    const unsigned long long mant = (static_cast<unsigned long long>(a) << (52 - e)) &
                                    ((1ull << 52) - 1ull);
    const unsigned long long bits = (static_cast<unsigned long long>(1023 + e) << 52) | mant |
                                    (v < 0 ? (1ull << 63) : 0ull);
    return __longlong_as_double(a == 0u ? 0ll : static_cast<long long>(bits));
}

// ---- complex interval add / subtract (sharp, Section 2.5) --------------------

template <typename T>
__device__ __forceinline__ CI<T> operator+(const CI<T>& a, const CI<T>& b) {
    return {add_dn(a.rl, b.rl), add_up(a.rh, b.rh), add_dn(a.il, b.il), add_up(a.ih, b.ih)};
}

template <typename T>
__device__ __forceinline__ CI<T> operator-(const CI<T>& a, const CI<T>& b) {
    return {sub_dn(a.rl, b.rh), sub_up(a.rh, b.rl), sub_dn(a.il, b.ih), sub_up(a.ih, b.il)};
}

// multiplication by +i and -i and conjugation: exact
template <typename T>
__device__ __forceinline__ CI<T> mul_i(const CI<T>& a) { return {-a.ih, -a.il, a.rl, a.rh}; }
template <typename T>
__device__ __forceinline__ CI<T> mul_negi(const CI<T>& a) { return {a.il, a.ih, -a.rh, -a.rl}; }
template <typename T>
__device__ __forceinline__ CI<T> conj(const CI<T>& a) { return {a.rl, a.rh, -a.ih, -a.il}; }
// the same, with the negations on the integer pipe, for a value that is stored
template <typename T>
__device__ __forceinline__ CI<T> conj_flip(const CI<T>& a) {
    return {a.rl, a.rh, flip(a.ih), flip(a.il)};
}
template <typename T>
__device__ __forceinline__ CI<T> mul_negi_flip(const CI<T>& a) {
    return {a.il, a.ih, flip(a.rh), flip(a.rl)};
}

// ---- product by a twiddle ------------------------------------------------------
//
// Each component of a twiddle enclosure is either a point (0, +-1) or an
// interval that does not contain 0 (the enclosure of a nonzero cos or sin
// value is far narrower than its distance to 0 for every supported length).
// For such a w = [wl, wh] and any x = [xl, xh] the extremes of x*w are
//   w >= 0:  min = xl * (xl >= 0 ? wl : wh),  max = xh * (xh >= 0 ? wh : wl)
//   w <  0:  min = xh * (xh >= 0 ? wl : wh),  max = xl * (xl >= 0 ? wh : wl)
// so one product per bound suffices.

template <typename T>
struct Pair { T a, b; };

template <typename T>
__device__ __forceinline__ void pick_tw(T xl, T xh, T wl, T wh, Pair<T>& lo, Pair<T>& hi) {
    const bool wneg = neg(wl);
    lo.a = wneg ? xh : xl;
    lo.b = neg(lo.a) ? wh : wl;
    hi.a = wneg ? xl : xh;
    hi.b = neg(hi.a) ? wl : wh;
}

// x * w for a twiddle enclosure w: 4 directed products and 4 directed fmas
template <typename T>
__device__ __forceinline__ CI<T> mul_tw(const CI<T>& x, const CI<T>& w) {
    Pair<T> rr_lo, rr_hi, ii_lo, ii_hi, ri_lo, ri_hi, ir_lo, ir_hi;
    pick_tw(x.rl, x.rh, w.rl, w.rh, rr_lo, rr_hi);   // xr * wr
    pick_tw(x.il, x.ih, w.il, w.ih, ii_lo, ii_hi);   // xi * wi
    pick_tw(x.rl, x.rh, w.il, w.ih, ri_lo, ri_hi);   // xr * wi
    pick_tw(x.il, x.ih, w.rl, w.rh, ir_lo, ir_hi);   // xi * wr
    CI<T> r;
    r.rl = fma_dn(rr_lo.a, rr_lo.b, -mul_up(ii_hi.a, ii_hi.b));
    r.rh = fma_up(rr_hi.a, rr_hi.b, -mul_dn(ii_lo.a, ii_lo.b));
    r.il = fma_dn(ri_lo.a, ri_lo.b, mul_dn(ir_lo.a, ir_lo.b));
    r.ih = fma_up(ri_hi.a, ri_hi.b, mul_up(ir_hi.a, ir_hi.b));
    return r;
}

// x * w for a real twiddle w = [w.rl, w.rh] (w.il = w.ih = 0, the radix-3
// and radix-5 scalars cos(2 pi k / R)): 4 directed products.  The same
// bounds as mul_tw's, without its products by the zero imaginary part.
template <typename T>
__device__ __forceinline__ CI<T> mul_real(const CI<T>& x, const CI<T>& w) {
    Pair<T> r_lo, r_hi, i_lo, i_hi;
    pick_tw(x.rl, x.rh, w.rl, w.rh, r_lo, r_hi);     // xr * wr
    pick_tw(x.il, x.ih, w.rl, w.rh, i_lo, i_hi);     // xi * wr
    return {mul_dn(r_lo.a, r_lo.b), mul_up(r_hi.a, r_hi.b), mul_dn(i_lo.a, i_lo.b),
            mul_up(i_hi.a, i_hi.b)};
}

// x * w for a pure imaginary twiddle w = i [w.il, w.ih] (the scalars
// i sin(2 pi k / R)): x w = -xi wi + i xr wi, 4 directed products
template <typename T>
__device__ __forceinline__ CI<T> mul_imag(const CI<T>& x, const CI<T>& w) {
    Pair<T> a_lo, a_hi, b_lo, b_hi;
    pick_tw(x.il, x.ih, w.il, w.ih, a_lo, a_hi);     // xi * wi
    pick_tw(x.rl, x.rh, w.il, w.ih, b_lo, b_hi);     // xr * wi
    return {flip(mul_up(a_hi.a, a_hi.b)), flip(mul_dn(a_lo.a, a_lo.b)), mul_dn(b_lo.a, b_lo.b),
            mul_up(b_hi.a, b_hi.b)};
}

// ---- general real interval product (Section 2.5) -------------------------------
//
// [a][b] = [min, max] of the four endpoint products.  The sign classes of
// the operands select the endpoint pairs; only when both operands straddle
// zero are two candidates compared.  A class is taken from sign bits, so
// a bound of -0.0 may send an operand to the straddling class, whose
// formulas are also valid for it.

template <typename T>
__device__ __forceinline__ void ir_mul(T al, T ah, T bl, T bh, T& lo, T& hi) {
    const bool a_nn = !neg(al), a_np = neg(ah);   // a >= 0, a <= 0
    const bool b_nn = !neg(bl), b_np = neg(bh);
    T la, lb, ha, hb;
    if (a_nn) {
        la = b_nn ? al : ah;  lb = bl;
        ha = b_np ? al : ah;  hb = bh;
    } else if (a_np) {
        la = b_np ? ah : al;  lb = bh;
        ha = b_nn ? ah : al;  hb = bl;
    } else if (b_nn) {          // a straddles, b >= 0
        la = al; lb = bh; ha = ah; hb = bh;
    } else if (b_np) {          // a straddles, b <= 0
        la = ah; lb = bl; ha = al; hb = bl;
    } else {                    // both straddle zero
        lo = fmin(mul_dn(al, bh), mul_dn(ah, bl));
        hi = fmax(mul_up(al, bl), mul_up(ah, bh));
        return;
    }
    lo = mul_dn(la, lb);
    hi = mul_up(ha, hb);
}

// general complex interval product (pointwise step of Section 2.3)
template <typename T>
__device__ __forceinline__ CI<T> mul_ci(const CI<T>& a, const CI<T>& b) {
    T p1l, p1h, p2l, p2h, p3l, p3h, p4l, p4h;
    ir_mul(a.rl, a.rh, b.rl, b.rh, p1l, p1h);   // ar br
    ir_mul(a.il, a.ih, b.il, b.ih, p2l, p2h);   // ai bi
    ir_mul(a.rl, a.rh, b.il, b.ih, p3l, p3h);   // ar bi
    ir_mul(a.il, a.ih, b.rl, b.rh, p4l, p4h);   // ai br
    return {sub_dn(p1l, p2h), sub_up(p1h, p2l), add_dn(p3l, p4l), add_up(p3h, p4h)};
}

// scaling by a power of two (division by the transform length, Section
// 2.5): rounded outward, so it stays rigorous even if a bound underflows
template <typename T>
__device__ __forceinline__ CI<T> scale_out(const CI<T>& a, T s) {
    return {mul_dn(a.rl, s), mul_up(a.rh, s), mul_dn(a.il, s), mul_up(a.ih, s)};
}

}  // namespace ssm
