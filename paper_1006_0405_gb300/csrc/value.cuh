// value.cuh -- the value types the transform kernels are instantiated for.
//
//   CI<float>   rung 0: binary32 inf-sup rectangles (Section 2.5)
//   CI<double>  rung 1: binary64 inf-sup rectangles (Section 2.5)
//   Disc        rung 2: binary64 midpoint-radius discs (Section 4's
//               circular containment sets)
//   Pt          rung 3: unverified round-to-nearest binary64 points (the
//               naive transform of Section 3, a speed reference)
//   DDisc       rung 4: midpoint-radius discs with double-binary32 centres
//               (the circular sets on the binary32 pipe)
//
// Each type provides +, -, mul_i, mul_negi, conj, mul_tw (by its twiddle
// type), mul_ci, scale_pow2, make_point, get_twiddle and the isolation of
// its two components.
#pragma once
#include "interval.cuh"
#include "disc.cuh"
#include "ddisc.cuh"
#include "twiddle.cuh"

namespace ssm {

constexpr int RUNGS = 5;

// sw_src, sw_mask: the shared-memory swizzle of SBuf for the type's size;
// reg_rows, reg_cols: register caps of k_rows and of the column kernels,
// mostly chosen so that one more CTA shares an SM than the natural register
// count allows (an explicit cap for every type: a cap of 255 is not the
// same as none)
template <typename V> struct VTraits;
template <> struct VTraits<CI<float>> {
    using Tw = CI<float>;
    static constexpr int rung = 0, sw_src = 3, sw_mask = 3;
    static constexpr int reg_rows = 64, reg_cols = 72;
};
#ifndef SSMUL_REG_COLS5_F64
#define SSMUL_REG_COLS5_F64 96
#endif
template <> struct VTraits<CI<double>> {
    using Tw = CI<double>;
    static constexpr int rung = 1, sw_src = 2, sw_mask = 3;
    // k_rows: 128 registers hold its whole state (no spills, 4 CTAs of 4
    // warps per SM); at 96 (5 CTAs) it spilled 72 bytes per thread and
    // moved 1.6 times the L1 <-> L2 bytes in the same time
    static constexpr int reg_rows = 128, reg_cols = 80;
    // the columns of the lengths 5 2^k run 5-warp CTAs (160 threads for the
    // 320-point columns, four columns per CTA): at 96 registers four CTAs
    // still fit an SM (5 warps x 3072 registers per 16,384-register quarter),
    // as at 80, with fewer spills
    static constexpr int reg_cols5 = SSMUL_REG_COLS5_F64;
};
template <> struct VTraits<Disc> {
    using Tw = DiscTw;
    static constexpr int rung = 2, sw_src = 3, sw_mask = 7;
    static constexpr int reg_rows = 80, reg_cols = 80;
};
template <> struct VTraits<Pt> {
    using Tw = DiscTw;
    static constexpr int rung = 3, sw_src = 3, sw_mask = 3;
    static constexpr int reg_rows = 64, reg_cols = 72;
};
template <> struct VTraits<DDisc> {
    using Tw = DDiscTw;
    static constexpr int rung = 4, sw_src = 3, sw_mask = 7;
    static constexpr int reg_rows = 64, reg_cols = 64;
};

// The binary64 rectangles move Z and W between global memory and the
// registers of the transform steps that use them, with no pass through
// shared memory: the forward columns of lengths R 2^k twiddle and store Z
// from the radix-R step (block_fft_odd's epilogue), k_rows loads its first
// radix-4 step from Z and twiddles and stores W from its last step
// (block_fft's loader and epilogue).  Their 32-byte elements fill a sector
// per lane; the other types keep the passes (pair discs were 10% and discs
// 0.5% slower with the forward columns' epilogue).  The inverse columns
// isolate after the pass for every type: isolating from the registers made
// the binary64 kernel 9% slower.
template <typename V>
__host__ __device__ constexpr bool io_from_registers() {
    return std::is_same<V, CI<double>>::value;
}

// k_rows' register-fed first step (every type) and last step (every type
// whose inverse rows cannot end with the radix-8 step): there the lanes of a
// warp read and write consecutive elements, so elements of any size stay
// coalesced
template <typename V>
__host__ __device__ constexpr bool rows_load_from_registers() {
    return true;
}
template <typename V>
__host__ __device__ constexpr bool rows_store_from_registers() {
    return !std::is_same<V, DDisc>::value;
}

// register cap of the column kernels of family R
template <typename V, int R>
__host__ __device__ constexpr int cols_regs() {
    if constexpr (std::is_same<V, CI<double>>::value) return R == 5 ? VTraits<V>::reg_cols5 : VTraits<V>::reg_cols;
    else return VTraits<V>::reg_cols;
}

// A transform buffer in shared memory.  Element i lives in slot
// i ^ ((i >> sw_src) & sw_mask): the swizzle permutes each aligned group of
// sw_mask + 1 elements, so it maps [0, n) onto itself for every n that is a
// multiple of that group or smaller than 2^sw_src.  It spreads the strided
// accesses of the radix-4 steps (stride 4 s for s < 32) over more banks
// (16-, 24- and 32-byte elements each take the variant with the fewest
// shared-memory wavefronts over the steps of the transform lengths in use).
template <typename V>
struct SBuf {
    V* p;
    __device__ __forceinline__ V& operator[](int i) const {
        return p[i ^ ((i >> VTraits<V>::sw_src) & VTraits<V>::sw_mask)];
    }
};

// Enclosure of omega_Ntab^(SIGN j) in the twiddle type of V, from a table
// of family R (Ntab = R 2^tw.log_n).
template <typename V, int SIGN, int R> struct TwOf;
template <int SIGN, int R> struct TwOf<CI<float>, SIGN, R> {
    static __device__ __forceinline__ CI<float> get(const TwTable& tw, uint32_t j) {
        return twiddle<float, SIGN, R>(tw, j);
    }
};
template <int SIGN, int R> struct TwOf<CI<double>, SIGN, R> {
    static __device__ __forceinline__ CI<double> get(const TwTable& tw, uint32_t j) {
        return twiddle<double, SIGN, R>(tw, j);
    }
};
template <int SIGN, int R> struct TwOf<Disc, SIGN, R> {
    static __device__ __forceinline__ DiscTw get(const TwTable& tw, uint32_t j) {
        return twiddle_disc<SIGN, R>(tw, j);
    }
};
template <int SIGN, int R> struct TwOf<Pt, SIGN, R> : TwOf<Disc, SIGN, R> {};

// disc twiddle with double-binary32 centre: the symmetries of twiddle_disc
template <int SIGN, int R = 1>
__device__ __forceinline__ DDiscTw twiddle_ddisc(const TwTable& tw, uint32_t j) {
    const TwPos ps = tw_pos<R>(tw.log_n, j);
    const DDiscC e = tw.tdd[ps.jj];
    const float ch = ps.refl ? e.sh : e.ch, cl = ps.refl ? e.sl : e.cl;
    const float sh = ps.refl ? e.ch : e.sh, sl = ps.refl ? e.cl : e.sl;
    const bool swap = ps.quad & 1u;
    const float wch = swap ? sh : ch, wcl = swap ? sl : cl;
    const float wsh = swap ? ch : sh, wsl = swap ? cl : sl;
    const bool negr = ps.quad == 1u || ps.quad == 2u;
    const bool negi = (ps.quad >= 2u) != (SIGN < 0);
    return {negr ? flip(wch) : wch, negr ? flip(wcl) : wcl, negi ? flip(wsh) : wsh,
            negi ? flip(wsl) : wsl, tw.rho_dd, TW_MOD_UP};
}
template <int SIGN, int R> struct TwOf<DDisc, SIGN, R> {
    static __device__ __forceinline__ DDiscTw get(const TwTable& tw, uint32_t j) {
        return twiddle_ddisc<SIGN, R>(tw, j);
    }
};

template <typename V, int SIGN, int R = 1>
__device__ __forceinline__ typename VTraits<V>::Tw get_twiddle(const TwTable& tw, uint32_t j) {
    return TwOf<V, SIGN, R>::get(tw, j);
}

// ---- step-ordered twiddles -------------------------------------------------------
//
// omega_n^(SIGN u p) for the radix-4 step of sub-length n: the step table's
// entry (a forward twiddle; the inverse root is its conjugate, a sign-bit
// flip), or the octant table's when the plan has no step tables.  Both give
// the same bits.

__device__ __forceinline__ CI<double> tw_conj(const CI<double>& w) { return conj_flip(w); }
__device__ __forceinline__ CI<float> tw_conj(const CI<float>& w) { return conj_flip(w); }
__device__ __forceinline__ DiscTw tw_conj(const DiscTw& w) { return {w.c, flip(w.s), w.rho, w.mod}; }
__device__ __forceinline__ DDiscTw tw_conj(const DDiscTw& w) {
    return {w.ch, w.cl, flip(w.sh), flip(w.sl), w.rho, w.mod};
}

// table(tw, three): the step table of V for n = 2^j (three = false) or
// n = 3 2^j (three = true)
template <typename V> struct StepOf;
template <> struct StepOf<CI<double>> {
    static __device__ __forceinline__ const CI<double>* table(const TwTable& tw, bool three) {
        return three ? tw.s64_r : tw.s64;
    }
    static __device__ __forceinline__ CI<double> load(const CI<double>* t, int i, const TwTable&) {
        return t[i];
    }
};
template <> struct StepOf<CI<float>> {
    static __device__ __forceinline__ const CI<float>* table(const TwTable& tw, bool three) {
        return three ? tw.s32_r : tw.s32;
    }
    static __device__ __forceinline__ CI<float> load(const CI<float>* t, int i, const TwTable&) {
        return t[i];
    }
};
template <> struct StepOf<Disc> {
    static __device__ __forceinline__ const DiscTw* table(const TwTable& tw, bool three) {
        return three ? tw.sd_r : tw.sd;
    }
    static __device__ __forceinline__ DiscTw load(const DiscTw* t, int i, const TwTable&) {
        return t[i];
    }
};
template <> struct StepOf<Pt> : StepOf<Disc> {};
template <> struct StepOf<DDisc> {
    static __device__ __forceinline__ const DDiscC* table(const TwTable& tw, bool three) {
        return three ? tw.sdd_r : tw.sdd;
    }
    static __device__ __forceinline__ DDiscTw load(const DDiscC* t, int i, const TwTable& tw) {
        const DDiscC e = t[i];
        return {e.ch, e.cl, e.sh, e.sl, tw.rho_dd, TW_MOD_UP};
    }
};

// n = 2^logn, the table of family R
template <typename V, int SIGN, int R = 1>
__device__ __forceinline__ typename VTraits<V>::Tw step_twiddle(const TwTable& tw, int logn, int p,
                                                                int u) {
    const auto* t = StepOf<V>::table(tw, false);
    if (t == nullptr)        // Ntab / n = R 2^(log_n - logn)
        return get_twiddle<V, SIGN, R>(tw, uint32_t(R * u * p) << (tw.log_n - logn));
    const auto w = StepOf<V>::load(t, (u - 1) * STEP_TAB + (1 << (logn - 2)) + p, tw);
    return SIGN > 0 ? w : tw_conj(w);
}

// n = R 2^logn2 (R = 3 or 5), the table of family R
template <typename V, int SIGN, int R>
__device__ __forceinline__ typename VTraits<V>::Tw step_twiddle_r(const TwTable& tw, int logn2, int p,
                                                                  int u) {
    const auto* t = StepOf<V>::table(tw, true);
    if (t == nullptr)        // Ntab / n = 2^(log_n - logn2)
        return get_twiddle<V, SIGN, R>(tw, uint32_t(u * p) << (tw.log_n - logn2));
    const auto w = StepOf<V>::load(t, (u - 1) * STEP_TAB + (R << (logn2 - 2)) + p, tw);
    return SIGN > 0 ? w : tw_conj(w);
}

// Fills step tables from the octant tables of family R (the pair-disc step
// table holds centres: its radius is the table's).  R = 1: the tables for
// n = 2^j; R = 3, 5: those for n = R 2^j (n <= 4096).
template <int R>
__global__ void k_step_tw_gen(TwTable tw, CI<double>* s64, CI<float>* s32, DiscTw* sd,
                              DDiscC* sdd) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < 3 * STEP_TAB;
         i += gridDim.x * blockDim.x) {
        const int u = i / STEP_TAB + 1, pos = i % STEP_TAB;
        // n/4 = R 2^lq <= pos < R 2^(lq+1)
        const int lq = pos < R ? -1 : 31 - __clz(pos / R);
        const int logn = lq + 2;                                // n = R 2^logn
        if (lq < (R == 1 ? 1 : 0) || logn > tw.log_n || (R > 1 && (R << logn) > 4096)) {
            s64[i] = {};
            s32[i] = {};
            sd[i] = {};
            sdd[i] = {};
            continue;
        }
        const uint32_t j = uint32_t(u * (pos - (R << lq))) << (tw.log_n - logn);
        s64[i] = twiddle<double, 1, R>(tw, j);
        s32[i] = twiddle<float, 1, R>(tw, j);
        sd[i] = twiddle_disc<1, R>(tw, j);
        const DDiscTw dd = twiddle_ddisc<1, R>(tw, j);
        sdd[i] = {dd.ch, dd.cl, dd.sh, dd.sl};
    }
}

// The scalars of a radix-3 or radix-5 step in every twiddle type (see
// k_scalar_gen): R = 3 uses [0], R = 5 [0 .. 3].
struct ScalarSet {
    CI<double> d[4];
    CI<float> f[4];
    DiscTw disc[4];
    DDiscTw dd[4];
};

// a digit pair as an exact point (small integers are exact in every type)
template <typename V> __device__ __forceinline__ V make_point(int re, int im);
template <> __device__ __forceinline__ CI<float> make_point<CI<float>>(int re, int im) {
    return {float(re), float(re), float(im), float(im)};
}
template <> __device__ __forceinline__ CI<double> make_point<CI<double>>(int re, int im) {
    const double r = int_to_double(re), i = int_to_double(im);
    return {r, r, i, i};
}
template <> __device__ __forceinline__ Disc make_point<Disc>(int re, int im) {
    return {int_to_double(re), int_to_double(im), 0.f, 0.f};
}
template <> __device__ __forceinline__ Pt make_point<Pt>(int re, int im) {
    return {int_to_double(re), int_to_double(im)};
}
template <> __device__ __forceinline__ DDisc make_point<DDisc>(int re, int im) {
    return {float(re), 0.f, float(im), 0.f, 0.f, 0.f};
}

__device__ __forceinline__ CI<double> scale_pow2(const CI<double>& a, int k) {
    return scale_out(a, pow2_neg(k));
}
__device__ __forceinline__ CI<float> scale_pow2(const CI<float>& a, int k) {
    return scale_out(a, __int_as_float((127 - k) << 23));     // 2^-k, k <= 126
}

}  // namespace ssm
