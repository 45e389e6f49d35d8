// ddisc.cuh -- circular containment sets with double-binary32 centres.
//
// On GB300 the binary32 pipe retires about 73 times as many operations as
// the binary64 pipe, so the cheapest way to carry ~48 significant bits is a
// pair of binary32 numbers x = h + l with |l| <= u |h| (u = 2^-24): the
// error-free transformations TwoSum (Knuth, TAOCP vol. 2, 4.2.2) and
// TwoProduct via a fused multiply-add give the exact error of a binary32 sum
// and product.  A DDisc is the disc {z : |z - (x + i y)| <= r} with such
// pair centres and a binary32 radius rounded upward, i.e. the circular sets
// of the paper's Section 4 in another machine format; the enclosure
// property holds because every operation adds to the radius a proved bound
// of its own rounding error (derivations beside each rule):
//
//   pair sum     (s, e) = TwoSum(xh, yh); v = RN(e + RN(xl + yl));
//                z = FastTwoSum(s, v).  |z - (x + y)| <= u |RN(xl + yl)| + u |v|
//                <= u^2 (|xh| + |yh|) (2 + u) + u^2 (1 + u) (|xh| + |yh|)
//                <= 3.0001 u^2 (|xh| + |yh|).  FastTwoSum is exact here
//                (Dekker: when s = 0 or exp(s) >= exp(v)) for normalised
//                operands, h = RN(h + l), so |l| <= ulp(h) / 2 <= u |h|:
//                without cancellation (|xh + yh| >= (|xh| + |yh|) / 3)
//                |v| <= 4.01 u |s|; with it (yh within a factor 2 of -xh)
//                Sterbenz makes s = xh + yh exact and e = 0, s is a nonzero
//                multiple of U = min(ulp(xh), ulp(yh)) or zero, and
//                |v| = |RN(xl + yl)| <= (ulp(xh) + ulp(yh)) / 2 <= 1.5 U, so
//                exp(v) <= exp(U) <= exp(s).  Every result is again
//                normalised (zh = RN(zh + zl)).
//   pair product p = RN(xh wh); pe = fma(xh, wh, -p) (exact);
//                r = RN(xl wh + RN(xh wl + pe)); z = FastTwoSum(p, r) (exact,
//                |r| <= 3u|p|).  The dropped xl wl and the two roundings give
//                |z - x w| <= 6.001 u^2 |xh| |wh|.
//   complex product: each component is two pair products and one pair sum:
//                error <= 9.01 u^2 (|axh| + |ayh|)(|bxh| + |byh|) for both
//                components together.
//
// Each bound also gets ETA = 2^-126, far above the error of any operation
// whose result falls into the binary32 subnormal range.  All arithmetic
// uses explicit round-to-nearest intrinsics, so nothing is contracted or
// reassociated.
#pragma once
#include <cstdint>
#include "interval.cuh"
#include "disc.cuh"

namespace ssm {

struct alignas(8) DDisc {
    float xh, xl, yh, yl;   // centre (xh + xl) + i (yh + yl)
    float r;                // radius (rounded up)
    float pad;
};

struct alignas(8) DDiscTw {
    float ch, cl, sh, sl;   // centre (ch + cl) + i (sh + sl)
    float rho;
    float mod;              // upper bound on |centre| (see DiscTw)
};

// twiddle table entry: the centre only.  Every entry of a table shares one
// radius, so that a scattered read moves 16 bytes; it costs nothing here, as
// the pair split's 2u^2 dominates every entry's radius.
struct alignas(16) DDiscC {
    float ch, cl, sh, sl;
};

constexpr float DD_U2 = 5.9604645e-8f * 5.9604645e-8f;      // u^2 = 2^-48 (exact)
constexpr float DD_ADD = 3.0001f * DD_U2;
constexpr float DD_MUL = 9.01f * DD_U2;
constexpr float DD_ETA = 1.17549435e-38f;                     // 2^-126
constexpr float DD_ONE_U = 1.00000024f;                      // >= 1 + 2u: |h + l| <= (1+u)|h|

__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// exact when |a| >= |b| or a == 0
__device__ __forceinline__ void fast_two_sum(float a, float b, float& s, float& e) {
    s = __fadd_rn(a, b);
    e = __fsub_rn(b, __fsub_rn(s, a));
}

__device__ __forceinline__ void pair_add(float xh, float xl, float yh, float yl, float& zh,
                                         float& zl) {
    float s, e;
    two_sum(xh, yh, s, e);
    const float v = __fadd_rn(e, __fadd_rn(xl, yl));
    fast_two_sum(s, v, zh, zl);
}

__device__ __forceinline__ void pair_mul(float xh, float xl, float wh, float wl, float& zh,
                                         float& zl) {
    const float p = __fmul_rn(xh, wh);
    const float pe = __fmaf_rn(xh, wh, -p);
    const float q = __fmaf_rn(xh, wl, pe);
    const float r = __fmaf_rn(xl, wh, q);
    fast_two_sum(p, r, zh, zl);
}

// upper bound on |centre| from the high parts: (|xh| + |yh|)(1 + 2u)
__device__ __forceinline__ float dd_mod_up(float xh, float yh) {
    return __fmul_ru(__fadd_ru(fabsf(xh), fabsf(yh)), DD_ONE_U);
}

__device__ __forceinline__ DDisc operator+(const DDisc& a, const DDisc& b) {
    DDisc z;
    pair_add(a.xh, a.xl, b.xh, b.xl, z.xh, z.xl);
    pair_add(a.yh, a.yl, b.yh, b.yl, z.yh, z.yl);
    const float m = __fadd_ru(__fadd_ru(fabsf(a.xh), fabsf(b.xh)),
                              __fadd_ru(fabsf(a.yh), fabsf(b.yh)));
    z.r = __fadd_ru(__fadd_ru(a.r, b.r), __fmaf_ru(DD_ADD, m, 2.f * DD_ETA));
    z.pad = 0.f;
    return z;
}

__device__ __forceinline__ DDisc operator-(const DDisc& a, const DDisc& b) {
    DDisc z;
    pair_add(a.xh, a.xl, -b.xh, -b.xl, z.xh, z.xl);
    pair_add(a.yh, a.yl, -b.yh, -b.yl, z.yh, z.yl);
    const float m = __fadd_ru(__fadd_ru(fabsf(a.xh), fabsf(b.xh)),
                              __fadd_ru(fabsf(a.yh), fabsf(b.yh)));
    z.r = __fadd_ru(__fadd_ru(a.r, b.r), __fmaf_ru(DD_ADD, m, 2.f * DD_ETA));
    z.pad = 0.f;
    return z;
}

// ---- radix-4 butterfly with one radius for its four outputs -----------------------
//
// The two levels of sums of a radix-4 butterfly (a +- c, b +- d, then their
// sums and differences, one of them times +-i) give every output the radius
// r_a + r_b + r_c + r_d plus the rounding of one first-level and one
// second-level sum of each component.  With M the sum of |xh| + |yh| over
// the four inputs: the first-level sums feeding an output err by at most
// DD_ADD (M_ac + M_bd) = DD_ADD M (+ 4 ETA); a first-level result z of, say,
// a.x + c.x has |z| <= (|a.xh| + |c.xh|)(1 + u + 3.0001 u^2) and its high
// part |zh| <= |z| / (1 - u), so the second-level operands' high parts sum
// to at most M (1 + 3u) and that sum errs by at most DD_ADD M (1 + 3u)
// (+ 2 ETA).  Every output therefore lies within
//   r = r_a + r_b + r_c + r_d + DD_ADD (2 + 3u) M + 6 ETA
// of its computed centre; DD_BFLY >= DD_ADD (2 + 3u).  One radius costs 13
// operations where eight per-sum radii cost 48.
constexpr float DD_BFLY = 6.0003f * DD_U2;

__device__ __forceinline__ DDisc centre_add(const DDisc& a, const DDisc& b) {
    DDisc z;
    pair_add(a.xh, a.xl, b.xh, b.xl, z.xh, z.xl);
    pair_add(a.yh, a.yl, b.yh, b.yl, z.yh, z.yl);
    z.r = 0.f;
    z.pad = 0.f;
    return z;
}

__device__ __forceinline__ DDisc centre_sub(const DDisc& a, const DDisc& b) {
    DDisc z;
    pair_add(a.xh, a.xl, -b.xh, -b.xl, z.xh, z.xl);
    pair_add(a.yh, a.yl, -b.yh, -b.yl, z.yh, z.yl);
    z.r = 0.f;
    z.pad = 0.f;
    return z;
}

template <int SIGN>
__device__ __forceinline__ void bfly4_dd(DDisc& a, DDisc& b, DDisc& c, DDisc& d) {
    const float mab = __fadd_ru(__fadd_ru(fabsf(a.xh), fabsf(a.yh)), __fadd_ru(fabsf(b.xh), fabsf(b.yh)));
    const float mcd = __fadd_ru(__fadd_ru(fabsf(c.xh), fabsf(c.yh)), __fadd_ru(fabsf(d.xh), fabsf(d.yh)));
    const float m = __fadd_ru(mab, mcd);
    const float rs = __fadd_ru(__fadd_ru(a.r, b.r), __fadd_ru(c.r, d.r));
    const float r = __fmaf_ru(DD_BFLY, m, __fadd_ru(rs, 6.f * DD_ETA));
    const DDisc apc = centre_add(a, c), amc = centre_sub(a, c);
    const DDisc bpd = centre_add(b, d), bmd = centre_sub(b, d);
    // jb = (SIGN i) bmd, exact
    const DDisc jb = SIGN > 0 ? DDisc{-bmd.yh, -bmd.yl, bmd.xh, bmd.xl, 0.f, 0.f}
                              : DDisc{bmd.yh, bmd.yl, -bmd.xh, -bmd.xl, 0.f, 0.f};
    a = centre_add(apc, bpd);
    c = centre_sub(apc, bpd);
    b = centre_add(amc, jb);
    d = centre_sub(amc, jb);
    a.r = r;
    b.r = r;
    c.r = r;
    d.r = r;
}

__device__ __forceinline__ DDisc mul_i(const DDisc& a) { return {-a.yh, -a.yl, a.xh, a.xl, a.r, 0.f}; }
__device__ __forceinline__ DDisc mul_negi(const DDisc& a) { return {a.yh, a.yl, -a.xh, -a.xl, a.r, 0.f}; }
__device__ __forceinline__ DDisc conj(const DDisc& a) { return {a.xh, a.xl, -a.yh, -a.yl, a.r, 0.f}; }
__device__ __forceinline__ DDisc conj_flip(const DDisc& a) {
    return {a.xh, a.xl, flip(a.yh), flip(a.yl), a.r, 0.f};
}
__device__ __forceinline__ DDisc mul_negi_flip(const DDisc& a) {
    return {a.yh, a.yl, flip(a.xh), flip(a.xl), a.r, 0.f};
}

// centre of a * b (its rounding error is at most DD_MUL ma mb + 6 ETA with
// ma = |axh| + |ayh|, mb = |bxh| + |byh|)
__device__ __forceinline__ void pair_cmul(float axh, float axl, float ayh, float ayl, float bxh,
                                          float bxl, float byh, float byl, DDisc& z) {
    float p1h, p1l, p2h, p2l, p3h, p3l, p4h, p4l;
    pair_mul(axh, axl, bxh, bxl, p1h, p1l);     // ax bx
    pair_mul(ayh, ayl, byh, byl, p2h, p2l);     // ay by
    pair_mul(axh, axl, byh, byl, p3h, p3l);     // ax by
    pair_mul(ayh, ayl, bxh, bxl, p4h, p4l);     // ay bx
    pair_add(p1h, p1l, -p2h, -p2l, z.xh, z.xl);
    pair_add(p3h, p3l, p4h, p4l, z.yh, z.yl);
}

// a * w for a twiddle disc: |a w - a_c w_c| <= r (|w_c| + rho) + |a_c| rho
// with |a_c| <= ma (1 + 2u), plus the centre's rounding DD_MUL ma mb + 6 ETA,
// gathered as r (mod + rho) + ma (DD_MUL mb + (1 + 2u) rho) + 6 ETA with
// |w_c| <= w.mod (the terms in rho and mod alone are the same for every
// twiddle of a table)
__device__ __forceinline__ DDisc mul_tw(const DDisc& a, const DDiscTw& w) {
    DDisc z;
    pair_cmul(a.xh, a.xl, a.yh, a.yl, w.ch, w.cl, w.sh, w.sl, z);
    const float ma = __fadd_ru(fabsf(a.xh), fabsf(a.yh));
    const float mb = __fadd_ru(fabsf(w.ch), fabsf(w.sh));
    const float k = __fmaf_ru(DD_MUL, mb, __fmul_ru(DD_ONE_U, w.rho));
    z.r = __fmaf_ru(a.r, __fadd_ru(w.mod, w.rho), __fmaf_ru(ma, k, 6.f * DD_ETA));
    z.pad = 0.f;
    return z;
}

// a * w for a real twiddle w = D(ch + cl, rho) (sh = sl = 0, |centre| <=
// w.mod): two pair products, whose rounding errs by at most
// DD_PMUL (|axh| + |ayh|) |ch| + 2 ETA; the propagation is mul_tw's
constexpr float DD_PMUL = 6.001f * DD_U2;

__device__ __forceinline__ DDisc mul_real(const DDisc& a, const DDiscTw& w) {
    DDisc z;
    pair_mul(a.xh, a.xl, w.ch, w.cl, z.xh, z.xl);
    pair_mul(a.yh, a.yl, w.ch, w.cl, z.yh, z.yl);
    const float ma = __fadd_ru(fabsf(a.xh), fabsf(a.yh));
    const float k = __fmaf_ru(DD_PMUL, fabsf(w.ch), __fmul_ru(DD_ONE_U, w.rho));
    z.r = __fmaf_ru(a.r, __fadd_ru(w.mod, w.rho), __fmaf_ru(ma, k, 4.f * DD_ETA));
    z.pad = 0.f;
    return z;
}

// a * w for a pure imaginary twiddle w = D(i (sh + sl), rho) (ch = cl = 0):
// (-ay s, ax s), the same bounds with |sh|
__device__ __forceinline__ DDisc mul_imag(const DDisc& a, const DDiscTw& w) {
    DDisc z;
    float th, tl;
    pair_mul(a.yh, a.yl, w.sh, w.sl, th, tl);
    z.xh = flip(th);
    z.xl = flip(tl);
    pair_mul(a.xh, a.xl, w.sh, w.sl, z.yh, z.yl);
    const float ma = __fadd_ru(fabsf(a.xh), fabsf(a.yh));
    const float k = __fmaf_ru(DD_PMUL, fabsf(w.sh), __fmul_ru(DD_ONE_U, w.rho));
    z.r = __fmaf_ru(a.r, __fadd_ru(w.mod, w.rho), __fmaf_ru(ma, k, 4.f * DD_ETA));
    z.pad = 0.f;
    return z;
}

// general product (pointwise step): |a b - a_c b_c| <= |a_c| rb + |b_c| ra + ra rb
__device__ __forceinline__ DDisc mul_ci(const DDisc& a, const DDisc& b) {
    DDisc z;
    pair_cmul(a.xh, a.xl, a.yh, a.yl, b.xh, b.xl, b.yh, b.yl, z);
    const float err = __fmaf_ru(__fmul_ru(DD_MUL, __fadd_ru(fabsf(a.xh), fabsf(a.yh))),
                                __fadd_ru(fabsf(b.xh), fabsf(b.yh)), 6.f * DD_ETA);
    const float ma = dd_mod_up(a.xh, a.yh), mb = dd_mod_up(b.xh, b.yh);
    const float prop = __fmaf_ru(ma, b.r, __fmaf_ru(mb, a.r, __fmul_ru(a.r, b.r)));
    z.r = __fadd_ru(prop, err);
    z.pad = 0.f;
    return z;
}

// scaling by 2^-k (0 <= k <= 126): exact unless a part becomes subnormal
__device__ __forceinline__ DDisc scale_pow2(const DDisc& a, int k) {
    const float s = __int_as_float((127 - k) << 23);
    DDisc z{__fmul_rn(a.xh, s), __fmul_rn(a.xl, s), __fmul_rn(a.yh, s), __fmul_rn(a.yl, s),
            0.f, 0.f};
    z.r = __fadd_ru(__fmul_ru(a.r, s), 4.f * DD_ETA);
    return z;
}

// twiddle discs from the binary64 disc table: c = ch + cl with
// ch = RN32(c), cl = RN32(c - ch) (c - ch exact in binary64), so
// |c - ch - cl| <= u |cl| <= 2^-48 for |c| <= 1; the radius grows by the
// two components' errors: rho[1] = rho[0] + 2u^2 + ETA, rounded up
__global__ void k_ddisc_tw_gen(const DiscTw* td, float* rho, DDiscC* tdd, int64_t count) {
    for (int64_t j = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; j < count;
         j += int64_t(gridDim.x) * blockDim.x) {
        const DiscTw e = td[j];
        const float ch = __double2float_rn(e.c);
        const float cl = __double2float_rn(e.c - double(ch));
        const float sh = __double2float_rn(e.s);
        const float sl = __double2float_rn(e.s - double(sh));
        tdd[j] = {ch, cl, sh, sl};
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) rho[1] = __fadd_ru(rho[0], 2.f * DD_U2 + DD_ETA);
}

}  // namespace ssm
