// disc.cuh -- circular (midpoint-radius) complex containment sets, and the
// unverified point arithmetic of a naive transform.
//
// The paper's conclusion (Section 4) proposes circular containment sets in
// place of rectangles: a multiplication by e^{i theta}, the only complex
// product the transform needs besides the pointwise one, maps a disc onto a
// disc of the same radius, so rotations cause no wrapping effect.
//
// A Disc is {z : |z - (x + i y)| <= r} with a binary64 centre and a binary32
// radius.  Centres are computed with round-to-nearest binary64 operations,
// whose error is at most half an ulp of the computed result (IEEE 754); that
// bound, and an upper bound on |x|, are read from the exponent and mantissa
// bits with integer operations, and the radius is accumulated with binary32
// operations rounded upward.  Every rule below therefore gives a disc that
// contains the exact result of the operation on any points of the operand
// discs.  Only the centre arithmetic uses the binary64 pipe: 2 operations
// for an addition and 4 for a product, half of what the inf-sup rectangles
// of interval.cuh need.
//
// Pt is the point arithmetic of the "naive" transform the paper uses as a
// speed reference (Section 3): round-to-nearest binary64 with no enclosure.
#pragma once
#include <cstdint>
#include "interval.cuh"

namespace ssm {

struct alignas(8) Disc {
    double x, y;     // centre
    float r;         // radius (rounded up)
    float pad;
};

struct alignas(16) Pt {
    double x, y;
};

// disc twiddle: centre and radius of an enclosure of omega^j, and an
// upper bound on the modulus of the centre (TW_MOD_UP for the roots of
// unity; smaller for the real and imaginary scalars of the radix-3 and
// radix-5 steps)
struct DiscTw {
    double c, s;
    float rho;
    float mod;
};

// ---- bounds from the bit patterns (integer pipe) ----------------------------------

// An upper bound (binary32) on half an ulp of the binary64 value x, i.e. on
// the error of a round-to-nearest operation whose result is x:
// 2^(e - 1076) for a normal x with biased exponent e; 2^-126 for values
// below the binary32 normal range (covers zero and subnormal results, whose
// error is at most 2^-1075); +inf for inf or NaN.
__device__ __forceinline__ float half_ulp_up(double x) {
    const int e = (__double2hiint(x) >> 20) & 0x7FF;
    int fe = e - 949;                         // 2^(e-1076) as a binary32 exponent field
    fe = fe < 1 ? 1 : (fe > 255 ? 255 : fe);  // 255: +inf
    return __int_as_float(fe << 23);
}

// An upper bound (binary32, rounded up) on |x|.
__device__ __forceinline__ float abs_up(double x) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(x) & 0x7FFFFFFFFFFFFFFFull;
    const int e = int(b >> 52);
    const int fe = e - 896;                   // binary32 exponent field of 2^(e-1023)
    if (fe <= 0) return __int_as_float(1 << 23);          // |x| < 2^-126
    if (fe >= 255) return __int_as_float(0x7F800000);     // +inf (and NaN)
    unsigned int fb = (unsigned int)(fe << 23) | (unsigned int)((b >> 29) & 0x7FFFFFu);
    fb += (b & ((1ull << 29) - 1ull)) != 0ull ? 1u : 0u;  // round the dropped bits up
    return __uint_as_float(fb);
}

__device__ __forceinline__ float err2(double a, double b) {
    return __fadd_ru(half_ulp_up(a), half_ulp_up(b));
}

// upper bound on the modulus of a centre: |x + i y| <= |x| + |y|
__device__ __forceinline__ float mod_up(double x, double y) {
    return __fadd_ru(abs_up(x), abs_up(y));
}

// |centre of a twiddle| <= 1 + 2^-23 (the centres are within a few ulps of
// points of the unit circle)
constexpr float TW_MOD_UP = 1.00000012f;

// ---- disc arithmetic ------------------------------------------------------------

__device__ __forceinline__ Disc operator+(const Disc& a, const Disc& b) {
    Disc z;
    z.x = add_rn(a.x, b.x);
    z.y = add_rn(a.y, b.y);
    z.r = __fadd_ru(__fadd_ru(a.r, b.r), err2(z.x, z.y));
    z.pad = 0.f;
    return z;
}

__device__ __forceinline__ Disc operator-(const Disc& a, const Disc& b) {
    Disc z;
    z.x = sub_rn(a.x, b.x);
    z.y = sub_rn(a.y, b.y);
    z.r = __fadd_ru(__fadd_ru(a.r, b.r), err2(z.x, z.y));
    z.pad = 0.f;
    return z;
}

__device__ __forceinline__ Disc mul_i(const Disc& a) { return {-a.y, a.x, a.r, 0.f}; }
__device__ __forceinline__ Disc mul_negi(const Disc& a) { return {a.y, -a.x, a.r, 0.f}; }
__device__ __forceinline__ Disc conj(const Disc& a) { return {a.x, -a.y, a.r, 0.f}; }
__device__ __forceinline__ Disc conj_flip(const Disc& a) { return {a.x, flip(a.y), a.r, 0.f}; }
__device__ __forceinline__ Disc mul_negi_flip(const Disc& a) { return {a.y, flip(a.x), a.r, 0.f}; }

// a * w for a twiddle disc w = D(c + i s, rho) with |w_c| <= w.mod:
// |a w - a_c w_c| <= r (|w_c| + rho) + |a_c| rho, plus the centre rounding:
// x = RN(fma(ax, c, -RN(ay s))) errs by <= hu(t1) + hu(x), likewise y.
__device__ __forceinline__ Disc mul_tw(const Disc& a, const DiscTw& w) {
    Disc z;
    const double t1 = mul_rn(a.y, w.s);
    z.x = __fma_rn(a.x, w.c, -t1);
    const double t2 = mul_rn(a.y, w.c);
    z.y = __fma_rn(a.x, w.s, t2);
    const float rnd = __fadd_ru(err2(t1, z.x), err2(t2, z.y));
    const float prop = __fmaf_ru(a.r, __fadd_ru(w.mod, w.rho), __fmul_ru(mod_up(a.x, a.y), w.rho));
    z.r = __fadd_ru(prop, rnd);
    z.pad = 0.f;
    return z;
}

// a * w for a real twiddle disc w = D(c, rho) (w.s = 0, |c| <= w.mod): the
// centre (RN(ax c), RN(ay c)) errs by hu(x) + hu(y); the propagation is
// mul_tw's
__device__ __forceinline__ Disc mul_real(const Disc& a, const DiscTw& w) {
    Disc z;
    z.x = mul_rn(a.x, w.c);
    z.y = mul_rn(a.y, w.c);
    const float prop = __fmaf_ru(a.r, __fadd_ru(w.mod, w.rho), __fmul_ru(mod_up(a.x, a.y), w.rho));
    z.r = __fadd_ru(prop, err2(z.x, z.y));
    z.pad = 0.f;
    return z;
}

// a * w for a pure imaginary twiddle disc w = D(i s, rho) (w.c = 0):
// (-RN(ay s), RN(ax s)), the same bounds
__device__ __forceinline__ Disc mul_imag(const Disc& a, const DiscTw& w) {
    Disc z;
    z.x = flip(mul_rn(a.y, w.s));
    z.y = mul_rn(a.x, w.s);
    const float prop = __fmaf_ru(a.r, __fadd_ru(w.mod, w.rho), __fmul_ru(mod_up(a.x, a.y), w.rho));
    z.r = __fadd_ru(prop, err2(z.x, z.y));
    z.pad = 0.f;
    return z;
}

// general product (pointwise step): |a b - a_c b_c| <= |a_c| rb + |b_c| ra + ra rb
__device__ __forceinline__ Disc mul_ci(const Disc& a, const Disc& b) {
    Disc z;
    const double t1 = mul_rn(a.y, b.y);
    z.x = __fma_rn(a.x, b.x, -t1);
    const double t2 = mul_rn(a.y, b.x);
    z.y = __fma_rn(a.x, b.y, t2);
    const float rnd = __fadd_ru(err2(t1, z.x), err2(t2, z.y));
    const float ma = mod_up(a.x, a.y), mb = mod_up(b.x, b.y);
    const float prop = __fmaf_ru(ma, b.r, __fmaf_ru(mb, a.r, __fmul_ru(a.r, b.r)));
    z.r = __fadd_ru(prop, rnd);
    z.pad = 0.f;
    return z;
}

// scaling by 2^-k (k >= 0): exact for normal results; the half-ulp terms
// cover a result that falls into the subnormal range
__device__ __forceinline__ Disc scale_pow2(const Disc& a, int k) {
    const double s = pow2_neg(k);
    Disc z;
    z.x = mul_rn(a.x, s);
    z.y = mul_rn(a.y, s);
    z.r = __fadd_ru(__fmul_ru(a.r, __int_as_float((127 - k) << 23)), err2(z.x, z.y));
    z.pad = 0.f;
    return z;
}

// ---- naive point arithmetic (unverified) -------------------------------------------

__device__ __forceinline__ Pt operator+(const Pt& a, const Pt& b) {
    return {add_rn(a.x, b.x), add_rn(a.y, b.y)};
}
__device__ __forceinline__ Pt operator-(const Pt& a, const Pt& b) {
    return {sub_rn(a.x, b.x), sub_rn(a.y, b.y)};
}
__device__ __forceinline__ Pt mul_i(const Pt& a) { return {-a.y, a.x}; }
__device__ __forceinline__ Pt mul_negi(const Pt& a) { return {a.y, -a.x}; }
__device__ __forceinline__ Pt conj(const Pt& a) { return {a.x, -a.y}; }
__device__ __forceinline__ Pt conj_flip(const Pt& a) { return {a.x, flip(a.y)}; }
__device__ __forceinline__ Pt mul_negi_flip(const Pt& a) { return {a.y, flip(a.x)}; }
__device__ __forceinline__ Pt mul_tw(const Pt& a, const DiscTw& w) {
    return {__fma_rn(a.x, w.c, -mul_rn(a.y, w.s)), __fma_rn(a.x, w.s, mul_rn(a.y, w.c))};
}
__device__ __forceinline__ Pt mul_real(const Pt& a, const DiscTw& w) {
    return {mul_rn(a.x, w.c), mul_rn(a.y, w.c)};
}
__device__ __forceinline__ Pt mul_imag(const Pt& a, const DiscTw& w) {
    return {flip(mul_rn(a.y, w.s)), mul_rn(a.x, w.s)};
}
__device__ __forceinline__ Pt mul_ci(const Pt& a, const Pt& b) {
    return {__fma_rn(a.x, b.x, -mul_rn(a.y, b.y)), __fma_rn(a.x, b.y, mul_rn(a.y, b.x))};
}
__device__ __forceinline__ Pt scale_pow2(const Pt& a, int k) {
    const double s = pow2_neg(k);
    return {mul_rn(a.x, s), mul_rn(a.y, s)};
}

}  // namespace ssm
