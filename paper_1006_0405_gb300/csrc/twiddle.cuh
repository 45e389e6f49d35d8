// twiddle.cuh -- rigorous enclosures of the roots of unity omega_N^j.
//
// The DFT of Section 2.2 uses omega = e^{2 pi i / N}; its inverse uses
// omega^-1.  The plan builds, once, a table of enclosures of
// cos(2 pi j / Ntab) and sin(2 pi j / Ntab) for the first octant
// j = 0 .. Ntab/8; every other power of every root omega_N (N <= Ntab, both
// powers of two) is read from it through exact symmetries of the circle
// (reflection about pi/4 swaps cos and sin; a quarter turn maps (c, s) to
// (-s, c); the inverse root conjugates).
//
// Each table entry comes from the device's sincospi(2 j / Ntab), whose
// argument is exact because Ntab is a power of two.  The CUDA Math API
// documents a maximum error of 2 ulp for the binary64 sincospi; each value
// is widened outward by TW_WIDEN_ULPS = 4 steps of nextafter (the bound
// plus margin for the change of ulp size at a power of two), then clamped
// to what is known exactly on the first octant (cos in [0, 1], sin in
// [0, 1]).  j = 0 is the exact point (1, 0).  The binary32 table is the
// binary64 one rounded outward.
#pragma once
#include "interval.cuh"
#include "disc.cuh"

namespace ssm {

constexpr int TW_WIDEN_ULPS = 4;
constexpr int TW_DOC_ULPS = 2;

template <typename T>
struct TwEntry {
    T cl, ch, sl, sh;
};

struct DDiscC;

// Step-ordered twiddles.  The radix-4 step of sub-length n = 2^logn
// (3 <= logn <= LOG_STEP_MAX) multiplies by omega_n^{u p} for p < n/4 and
// u = 1, 2, 3; a step table holds that value of the forward transform at
// [(u - 1) STEP_TAB + n/4 + p], so the lanes of a warp, which work on
// consecutive p, read consecutive entries.  The entries are copies of the
// octant table's values (moved by the same exact symmetries).
constexpr int LOG_STEP_MAX = 12;
constexpr int STEP_TAB = 1 << (LOG_STEP_MAX - 1);

struct TwTable {
    const TwEntry<double>* t64;   // Ntab/8 + 1 entries
    const TwEntry<float>* t32;    // same, binary32
    int log_n;                    // log2 Ntab
    const DiscTw* td;             // same, as discs (centre, radius)
    const DDiscC* tdd;            // same, as double-binary32 disc centres
    float rho_dd;                 // the radius of every entry of tdd
    // step-ordered copies (3 STEP_TAB entries each), or all null: then the
    // transforms read the octant tables
    const CI<double>* s64;
    const CI<float>* s32;
    const DiscTw* sd;
    const DDiscC* sdd;
};

__global__ void k_twiddle_gen(TwEntry<double>* t64, TwEntry<float>* t32, int log_n) {
    const int64_t ntab = int64_t(1) << log_n;
    const int64_t count = ntab / 8 + 1;
    for (int64_t j = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; j < count;
         j += int64_t(gridDim.x) * blockDim.x) {
        TwEntry<double> e;
        if (j == 0) {
            e = {1.0, 1.0, 0.0, 0.0};
        } else {
            // 2 j / ntab is exact: a small integer times a power of two
            const double x = ldexp(double(2 * j), -log_n);
            double s, c;
            sincospi(x, &s, &c);
            double cl = c, ch = c, sl = s, sh = s;
            for (int k = 0; k < TW_WIDEN_ULPS; ++k) {
                cl = nextafter(cl, -1.0e300);
                ch = nextafter(ch, 1.0e300);
                sl = nextafter(sl, -1.0e300);
                sh = nextafter(sh, 1.0e300);
            }
            // first octant: 0 < sin <= cos <= 1
            e = {fmax(cl, 0.0), fmin(ch, 1.0), fmax(sl, 0.0), fmin(sh, 1.0)};
        }
        t64[j] = e;
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
__global__ void k_disc_tw_gen(const TwEntry<double>* t64, DiscTw* td, float* rho, int log_n) {
    const int64_t count = (int64_t(1) << log_n) / 8 + 1;
    for (int64_t j = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; j < count;
         j += int64_t(gridDim.x) * blockDim.x) {
        const TwEntry<double> e = t64[j];
        const double c = __dadd_rn(0.5 * e.cl, 0.5 * e.ch);
        const double s = __dadd_rn(0.5 * e.sl, 0.5 * e.sh);
        const double ec = fmax(__dsub_ru(c, e.cl), __dsub_ru(e.ch, c));
        const double es = fmax(__dsub_ru(s, e.sl), __dsub_ru(e.sh, s));
        const float r = __double2float_ru(__dadd_ru(ec, es));
        td[j] = {c, s, r, 0.f};
        atomicMax(reinterpret_cast<int*>(rho), __float_as_int(r));
    }
}

// Disc enclosure of omega_Ntab^(sign * j): the same symmetries as twiddle();
// they move the centre exactly and keep the radius.
template <int SIGN>
__device__ __forceinline__ DiscTw twiddle_disc(const TwTable& tw, uint32_t j) {
    const int ln = tw.log_n;
    j &= (1u << ln) - 1u;
    const uint32_t q = 1u << (ln - 2);
    const uint32_t quad = j >> (ln - 2);
    const uint32_t r = j & (q - 1u);
    const bool refl = r > (q >> 1);
    const DiscTw e = tw.td[refl ? q - r : r];
    const double c = refl ? e.s : e.c, s = refl ? e.c : e.s;
    const bool swap = quad & 1u;
    const double wc = swap ? s : c, ws = swap ? c : s;
    const bool negr = quad == 1u || quad == 2u;
    const bool negi = (quad >= 2u) != (SIGN < 0);
    return {negr ? flip(wc) : wc, negi ? flip(ws) : ws, e.rho, 0.f};
}

template <typename T>
__device__ __forceinline__ const TwEntry<T>* tw_ptr(const TwTable& tw);
template <>
__device__ __forceinline__ const TwEntry<double>* tw_ptr<double>(const TwTable& tw) { return tw.t64; }
template <>
__device__ __forceinline__ const TwEntry<float>* tw_ptr<float>(const TwTable& tw) { return tw.t32; }

// Enclosure of omega_Ntab^(sign * j) for any integer j (taken mod Ntab).
template <typename T, int SIGN>
__device__ __forceinline__ CI<T> twiddle(const TwTable& tw, uint32_t j) {
    const int ln = tw.log_n;
    const uint32_t mask = (1u << ln) - 1u;
    j &= mask;
    const uint32_t q = 1u << (ln - 2);               // a quarter turn
    const uint32_t quad = j >> (ln - 2);
    const uint32_t r = j & (q - 1u);
    const bool refl = r > (q >> 1);                  // past pi/4 inside the quadrant
    const uint32_t jj = refl ? q - r : r;
    const TwEntry<T> e = tw_ptr<T>(tw)[jj];
    const T cl = refl ? e.sl : e.cl, ch = refl ? e.sh : e.ch;
    const T sl = refl ? e.cl : e.sl, sh = refl ? e.ch : e.sh;
    // a quarter turn maps (c, s) to (-s, c); the negations are sign-bit
    // flips on the integer pipe (the interval -[l, h] is [-h, -l])
    const bool swap = quad & 1u;                       // quadrants 1 and 3
    const bool negr = quad == 1u || quad == 2u;        // real part negated
    const bool negi = quad >= 2u;                      // imaginary part negated
    T rl = swap ? sl : cl, rh = swap ? sh : ch;        // real part before sign
    T il = swap ? cl : sl, ih = swap ? ch : sh;        // imaginary part before sign
    CI<T> w;
    w.rl = negr ? flip(rh) : rl;
    w.rh = negr ? flip(rl) : rh;
    const bool ni = negi != (SIGN < 0);                // the inverse conjugates
    w.il = ni ? flip(ih) : il;
    w.ih = ni ? flip(il) : ih;
    return w;
}

}  // namespace ssm
