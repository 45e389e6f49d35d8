// twiddle.cuh -- rigorous enclosures of the roots of unity omega_N^j.
//
// The DFT of Section 2.2 uses omega = e^{2 pi i / N}; its inverse uses
// omega^-1.  The plan builds, once, tables of enclosures of
// cos(2 pi j / Ntab) and sin(2 pi j / Ntab) for the first octant
// j = 0 .. Ntab/8, for up to three families of lengths Ntab = R 2^K with
// R = 1, 3 or 5.  Every power of a root omega_N with N dividing
// Ntab is read from the table through exact symmetries of the circle
// (reflection about pi/4 swaps cos and sin; a quarter turn maps (c, s) to
// (-s, c); the inverse root conjugates).  These hold for every Ntab that
// is a multiple of 8.
//
// Each table entry comes from the device's sincospi(x), x = 2 j / Ntab.
// The CUDA Math API documents a maximum error of 2 ulp for the binary64
// sincospi.
//   R = 1: x is exact (Ntab is a power of two); each value is widened
//          outward by TW_WIDEN_ULPS = 4 steps of nextafter (the bound plus
//          margin for the change of ulp size at a power of two).
//   R = 3, 5: when R divides j the argument (2 j / R) 2^-K is exact and
//          the widening is TW_WIDEN_ULPS.  Otherwise x = q 2^-K with
//          q = RN(2 j / R); the remainder 2 j - R q is exact (one fma), so
//          the true argument is x + d with d = ((2 j - R q) / R) 2^-K,
//          |d| <= 2^-53 x.  The values at x + d are those at x corrected to
//          first order, s + pi d c and c - pi d s, each with one rounding
//          (1/2 ulp); the second-order term (pi d)^2 / 2 < 2^-104 and the
//          inputs' own errors times pi d are far below an ulp.  With
//          sincospi's 2 ulp each value is within 2.5 ulp; counted in steps
//          of a lower binade when the value sits just above a power of two,
//          5 steps.  The widening is TW3_WIDEN_ULPS = 6.
// The values are then clamped to what is known exactly on the first octant
// (cos in [0, 1], sin in [0, 1]); j = 0 is the exact point (1, 0).  The
// binary32 table is the binary64 one rounded outward.
//
// The binary64 table stores, per entry, only the two values before the
// widening (TwMid, 16 bytes); the bounds are rebuilt where they are read
// (tw_expand).  For the positive finite values of the first octant one
// nextafter step is one unit of the binary64 bit pattern, and the bit
// patterns of nonnegative doubles order like the integers, so the widening
// and the clamp are integer additions and min / max on the bit patterns:
// the rebuilt bounds are those the widening computes, bit for bit, from
// half the bytes (the per-element twiddles of the four-step and packing
// passes are read from L2 once per element).
#pragma once
#include <cstring>

#include "interval.cuh"
#include "disc.cuh"

namespace ssm {

constexpr int TW_WIDEN_ULPS = 4;
constexpr int TW3_WIDEN_ULPS = 6;

template <typename T>
struct TwEntry {
    T cl, ch, sl, sh;
};

// an entry of the binary64 table before its widening
struct alignas(16) TwMid {
    double c, s;
};

__host__ __device__ __forceinline__ long long tw_bits(double x) {
#ifdef __CUDA_ARCH__
    return __double_as_longlong(x);
#else
    long long b;
    memcpy(&b, &x, sizeof b);
    return b;
#endif
}
__host__ __device__ __forceinline__ double tw_from_bits(long long b) {
#ifdef __CUDA_ARCH__
    return __longlong_as_double(b);
#else
    double x;
    memcpy(&x, &b, sizeof x);
    return x;
#endif
}

// The widening steps of entry j of a table of family R: none at j = 0,
// TW_WIDEN_ULPS where the argument is exact, TW3_WIDEN_ULPS otherwise.
template <int R>
__host__ __device__ __forceinline__ int tw_widen(uint32_t j);

// Entry j's bounds from its values: each value moved w binary64 steps down
// and up (integer steps of the bit pattern), then clamped to [0, 1].
__host__ __device__ __forceinline__ TwEntry<double> tw_expand_w(TwMid m, int w) {
    constexpr long long ONE = 0x3FF0000000000000ll;          // the bit pattern of 1.0
    const long long bc = tw_bits(m.c), bs = tw_bits(m.s);
    const long long cl = bc - w, ch = bc + w, sl = bs - w, sh = bs + w;
    return {tw_from_bits(cl > 0 ? cl : 0), tw_from_bits(ch < ONE ? ch : ONE),
            tw_from_bits(sl > 0 ? sl : 0), tw_from_bits(sh < ONE ? sh : ONE)};
}

struct DDiscC;
struct ScalarSet;

// Step-ordered twiddles.  The radix-4 step of sub-length n multiplies by
// omega_n^{u p} for p < n/4 and u = 1, 2, 3; a step table holds that value
// of the forward transform at [(u - 1) STEP_TAB + n/4 + p], so the lanes
// of a warp, which work on consecutive p, read consecutive entries.  One
// set of tables serves n = 2^j (8 <= n <= 2^LOG_STEP_MAX), another, in a
// table of family R = 3 or 5, n = R 2^j (4 R <= n <= 4096); in both the
// ranges [n/4, n/2) of successive n are disjoint.  The entries are copies
// of the octant tables' values (moved by the same exact symmetries).
constexpr int LOG_STEP_MAX = 12;
constexpr int STEP_TAB = 1 << (LOG_STEP_MAX - 1);

struct TwTable {
    const TwMid* t64;             // Ntab/8 + 1 entries (values before the widening)
    const TwEntry<float>* t32;    // same, binary32
    int log_n;                    // Ntab = R 2^log_n (R: the kernel's family)
    const DiscTw* td;             // same, as discs (centre, radius)
    const DDiscC* tdd;            // same, as double-binary32 disc centres
    float rho_dd;                 // the radius of every entry of tdd
    // step-ordered copies (3 STEP_TAB entries each) for n = 2^j, or all
    // null: then the transforms read the octant tables
    const CI<double>* s64;
    const CI<float>* s32;
    const DiscTw* sd;
    const DDiscC* sdd;
    // the same for n = R 2^j (set in a table of family R = 3 or 5)
    const CI<double>* s64_r;
    const CI<float>* s32_r;
    const DiscTw* sd_r;
    const DDiscC* sdd_r;
    // the real and imaginary scalars of the radix-R step (family R = 3, 5)
    const ScalarSet* scal;
};

template <int R>
__host__ __device__ __forceinline__ int tw_widen(uint32_t j) {
    return j == 0 ? 0 : ((R == 1 || j % uint32_t(R) == 0) ? TW_WIDEN_ULPS : TW3_WIDEN_ULPS);
}

// tw_widen for a family R known at run time
__host__ __device__ __forceinline__ int tw_widen_r(uint32_t j, int R) {
    return R == 1 ? tw_widen<1>(j) : (R == 3 ? tw_widen<3>(j) : tw_widen<5>(j));
}

__global__ void k_twiddle_gen(TwMid* t64, TwEntry<float>* t32, int log_n, int R) {
    const int64_t ntab = int64_t(R) << log_n;
    const int64_t count = ntab / 8 + 1;
    for (int64_t j = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; j < count;
         j += int64_t(gridDim.x) * blockDim.x) {
        TwMid m;
        if (j == 0) {
            m = {1.0, 0.0};
        } else {
            // 2 j / ntab: exact for R = 1 and for j divisible by R
            const bool exact = R == 1 || j % R == 0;
            const double q = R == 1 ? double(2 * j) : __ddiv_rn(double(2 * j), double(R));
            const double x = ldexp(q, -log_n);
            double s, c;
            sincospi(x, &s, &c);
            if (!exact) {
                const double rem = __fma_rn(-double(R), q, double(2 * j));    // exact
                const double pd = __dmul_rn(3.141592653589793, ldexp(__ddiv_rn(rem, double(R)), -log_n));
                const double s0 = s;
                s = __fma_rn(pd, c, s);
                c = __fma_rn(-pd, s0, c);
            }
            m = {c, s};
        }
        // the widening and the clamp to the first octant (0 < sin <= cos <= 1)
        const TwEntry<double> e = tw_expand_w(m, tw_widen_r(uint32_t(j), R));
        t64[j] = m;
        t32[j] = {__double2float_rd(e.cl), __double2float_ru(e.ch),
                  __double2float_rd(e.sl), __double2float_ru(e.sh)};
    }
}

// The disc form of each enclosure: centre = the rounded midpoint of each
// component's interval, radius >= (distance of the centre to either end,
// rounded up) summed over the two components, which bounds the complex
// distance to any point of the rectangle.  *rho (zero on entry) becomes the
// largest of these radii (nonnegative binary32 values order like their bit
// patterns), the radius the double-binary32 table shares.
__global__ void k_disc_tw_gen(const TwMid* t64, int R, DiscTw* td, float* rho, int64_t count) {
    for (int64_t j = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; j < count;
         j += int64_t(gridDim.x) * blockDim.x) {
        const TwEntry<double> e = tw_expand_w(t64[j], tw_widen_r(uint32_t(j), R));
        const double c = __dadd_rn(0.5 * e.cl, 0.5 * e.ch);
        const double s = __dadd_rn(0.5 * e.sl, 0.5 * e.sh);
        const double ec = fmax(__dsub_ru(c, e.cl), __dsub_ru(e.ch, c));
        const double es = fmax(__dsub_ru(s, e.sl), __dsub_ru(e.sh, s));
        const float r = __double2float_ru(__dadd_ru(ec, es));
        td[j] = {c, s, r, TW_MOD_UP};
        atomicMax(reinterpret_cast<int*>(rho), __float_as_int(r));
    }
}

// Position of omega_Ntab^j (any j >= 0; Ntab = R 2^ln, ln >= 3) relative
// to the first octant: the quadrant (mod 4), and the octant entry jj, with
// refl set when the angle inside the quadrant is past pi/4 (then jj is
// measured back from the quadrant's end and cos and sin swap).
struct TwPos {
    uint32_t quad, jj;
    bool refl;
};

template <int R>
__device__ __forceinline__ TwPos tw_pos(int ln, uint32_t j) {
    const uint32_t q = uint32_t(R) << (ln - 2);       // a quarter turn
    uint32_t quad;
    if (R == 1) {
        j &= (1u << ln) - 1u;
        quad = j >> (ln - 2);
    } else {
        quad = (j >> (ln - 2)) / uint32_t(R);          // floor(j / q)
    }
    const uint32_t r = j - quad * q;
    const bool refl = r > (q >> 1);
    return {quad & 3u, refl ? q - r : r, refl};
}

// Disc enclosure of omega_Ntab^(sign * j): the same symmetries as twiddle();
// they move the centre exactly and keep the radius.
template <int SIGN, int R = 1>
__device__ __forceinline__ DiscTw twiddle_disc(const TwTable& tw, uint32_t j) {
    const TwPos ps = tw_pos<R>(tw.log_n, j);
    const DiscTw e = tw.td[ps.jj];
    const double c = ps.refl ? e.s : e.c, s = ps.refl ? e.c : e.s;
    const bool swap = ps.quad & 1u;
    const double wc = swap ? s : c, ws = swap ? c : s;
    const bool negr = ps.quad == 1u || ps.quad == 2u;
    const bool negi = (ps.quad >= 2u) != (SIGN < 0);
    return {negr ? flip(wc) : wc, negi ? flip(ws) : ws, e.rho, e.mod};
}

// entry jj of a family-R table, as bounds
template <typename T, int R>
__device__ __forceinline__ TwEntry<T> tw_entry(const TwTable& tw, uint32_t jj);
template <>
__device__ __forceinline__ TwEntry<float> tw_entry<float, 1>(const TwTable& tw, uint32_t jj) { return tw.t32[jj]; }
template <>
__device__ __forceinline__ TwEntry<float> tw_entry<float, 3>(const TwTable& tw, uint32_t jj) { return tw.t32[jj]; }
template <>
__device__ __forceinline__ TwEntry<float> tw_entry<float, 5>(const TwTable& tw, uint32_t jj) { return tw.t32[jj]; }
template <>
__device__ __forceinline__ TwEntry<double> tw_entry<double, 1>(const TwTable& tw, uint32_t jj) {
    return tw_expand_w(tw.t64[jj], tw_widen<1>(jj));
}
template <>
__device__ __forceinline__ TwEntry<double> tw_entry<double, 3>(const TwTable& tw, uint32_t jj) {
    return tw_expand_w(tw.t64[jj], tw_widen<3>(jj));
}
template <>
__device__ __forceinline__ TwEntry<double> tw_entry<double, 5>(const TwTable& tw, uint32_t jj) {
    return tw_expand_w(tw.t64[jj], tw_widen<5>(jj));
}

// Enclosure of omega_Ntab^(sign * j) for any integer j (taken mod Ntab).
template <typename T, int SIGN, int R = 1>
__device__ __forceinline__ CI<T> twiddle(const TwTable& tw, uint32_t j) {
    const TwPos ps = tw_pos<R>(tw.log_n, j);
    const TwEntry<T> e = tw_entry<T, R>(tw, ps.jj);
    const T cl = ps.refl ? e.sl : e.cl, ch = ps.refl ? e.sh : e.ch;
    const T sl = ps.refl ? e.cl : e.sl, sh = ps.refl ? e.ch : e.sh;
    // a quarter turn maps (c, s) to (-s, c); the negations are sign-bit
    // flips on the integer pipe (the interval -[l, h] is [-h, -l])
    const bool swap = ps.quad & 1u;                     // quadrants 1 and 3
    const bool negr = ps.quad == 1u || ps.quad == 2u;   // real part negated
    const bool negi = ps.quad >= 2u;                    // imaginary part negated
    T rl = swap ? sl : cl, rh = swap ? sh : ch;         // real part before sign
    T il = swap ? cl : sl, ih = swap ? ch : sh;         // imaginary part before sign
    CI<T> w;
    w.rl = negr ? flip(rh) : rl;
    w.rh = negr ? flip(rl) : rh;
    const bool ni = negi != (SIGN < 0);                 // the inverse conjugates
    w.il = ni ? flip(ih) : il;
    w.ih = ni ? flip(il) : ih;
    return w;
}

}  // namespace ssm
