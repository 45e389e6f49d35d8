// fft.cuh -- interval DFT of lines held in shared memory.
//
// Computes X_k = sum_j x_j omega_L^{SIGN j k} (the DFT of Section 2.2 for
// SIGN = +1, the unscaled inverse for SIGN = -1) for `nl` lines of length
// L = 2^logL, line l at buf[l * pitch ...], natural order in and out (the
// indices are SBuf's, before its swizzle).
//
// The paper's transform is the radix-2 Cooley-Tukey recursion.  Here the
// same DFT is evaluated by the Stockham autosort factorisation in radix 4
// (with one final radix-2 step when log2 L is odd): decimation in
// frequency with sub-length n and stride s,
//   y[q + s(4p + u)] = omega_n^{p u} * sum_t x[q + s(p + t n/4)] (SIGN i)^{t u},
// for p < n/4, q < s, u = 0..3, then n /= 4, s *= 4.  The 4-point sums use
// only exact multiplications by +-i, so a radix-4 step needs three twiddle
// products where two radix-2 steps need four, which also means fewer
// rectangular wrapping effects (Section 2.5) per element.
//
// The element type V is any of value.cuh's (inf-sup rectangles, discs or
// points); twiddles come from step_twiddle<V>.
//
// Each step reads all its inputs into registers, synchronises the block,
// then writes all its outputs in place: the block must hold every
// butterfly of a step at once, i.e. nl * L / 4 <= BPT * blockDim.x, with
// BPT butterflies per thread (1 or 2; with 1 a thread holds half the
// registers, so more warps can cover the binary64 pipe's latency).
#pragma once
#include <type_traits>
#include "value.cuh"

namespace ssm {

template <typename V, int SIGN>
__device__ __forceinline__ void bfly4(V& a, V& b, V& c, V& d) {
    if constexpr (std::is_same<V, DDisc>::value) {
        bfly4_dd<SIGN>(a, b, c, d);      // one radius bound for the four outputs
    } else {
        const V apc = a + c, amc = a - c, bpd = b + d, bmd = b - d;
        const V jb = (SIGN > 0) ? mul_i(bmd) : mul_negi(bmd);
        a = apc + bpd;   // u = 0
        c = apc - bpd;   // u = 2
        b = amc + jb;    // u = 1
        d = amc - jb;    // u = 3
    }
}

// The last step of a line of odd log2 length L >= 8 in radix 8 (n = 8,
// s = L/8, p = 0, so no step twiddles): y[q + s u] = sum_t x[q + s t]
// omega_8^{SIGN t u}, evaluated as the 4-point DFTs of a_t = x_t + x_{t+4}
// (outputs u = 0, 2, 4, 6) and of b_t = (x_t - x_{t+4}) omega_8^{SIGN t}
// (outputs u = 1, 3, 5, 7), omega_8^{2 SIGN} = SIGN i being exact.  It
// replaces the radix-4 step at n = 8 and the radix-2 step after it: one
// pass over shared memory instead of two.  Each thread owns the eight
// slots it reads and writes.
template <typename V, int SIGN, int R>
__device__ void radix8_last(SBuf<V> buf, int logL, int nl, int pitch, const TwTable& tw) {
    const int logs = logL - 3, s = 1 << logs;
    const int nbf = nl << logs;
    const uint32_t j8 = uint32_t(R) << (tw.log_n - 3);       // omega_Ntab^j8 = omega_8
    for (int b = threadIdx.x; b < nbf; b += blockDim.x) {
        const int x = (b >> logs) * pitch + (b & (s - 1));
        V a0 = buf[x], a1 = buf[x + s], a2 = buf[x + 2 * s], a3 = buf[x + 3 * s];
        V c0 = buf[x + 4 * s], c1 = buf[x + 5 * s], c2 = buf[x + 6 * s], c3 = buf[x + 7 * s];
        const V d0 = a0 - c0, d1 = a1 - c1, d2 = a2 - c2, d3 = a3 - c3;
        a0 = a0 + c0;
        a1 = a1 + c1;
        a2 = a2 + c2;
        a3 = a3 + c3;
        bfly4<V, SIGN>(a0, a1, a2, a3);
        buf[x] = a0;
        buf[x + 2 * s] = a1;
        buf[x + 4 * s] = a2;
        buf[x + 6 * s] = a3;
        c0 = d0;
        c1 = mul_tw(d1, get_twiddle<V, SIGN, R>(tw, j8));
        c2 = SIGN > 0 ? mul_i(d2) : mul_negi(d2);
        c3 = mul_tw(d3, get_twiddle<V, SIGN, R>(tw, 3u * j8));
        bfly4<V, SIGN>(c0, c1, c2, c3);
        buf[x + s] = c0;
        buf[x + 3 * s] = c1;
        buf[x + 5 * s] = c2;
        buf[x + 7 * s] = c3;
    }
    __syncthreads();
}

// the value types whose odd-length lines end with radix8_last (the pair
// discs, whose kernels are issue-bound: one pass less pays; the binary64
// types would spill the eight values under their register caps)
template <typename V>
__host__ __device__ constexpr bool last_radix8() { return std::is_same<V, DDisc>::value; }

// The first step's inputs come from buf (FromBuf), or, with a loader
// in(line, k) (element k of line `line`, from global memory), straight into
// the registers of the thread that combines them, with no staging pass; the
// last step's outputs go to buf (ToBuf, then a barrier), or to an epilogue
// out(line, k, y) from registers, with no barrier after.
struct FromBuf {};
struct ToBuf {};

// R: the family of the twiddle table tw (the line length is 2^logL either way).
// skip_first: the first radix-4 step (n = L) is done already
// (first_step_exact), so the steps start at n = L / 4, s = 4.  LAST8: an
// odd-length line of a last_radix8 type ends with radix8_last.  A loader
// (In) needs a first radix-4 step (logL >= 2, not skip_first); an epilogue
// (Out) a type without the radix-8 last step.  leave_radix2: an odd-length
// transform stops before its final radix-2 step (n = 2, s = L/2, no
// twiddle), which the caller then does itself, fused with what follows.
template <typename V, int SIGN, int BPT = 2, int R = 1, bool LAST8 = true,
          typename In = FromBuf, typename Out = ToBuf>
__device__ void block_fft(SBuf<V> buf, int logL, int nl, int pitch, const TwTable& tw,
                          bool skip_first = false, In in = In{}, Out out = Out{},
                          bool leave_radix2 = false) {
    constexpr bool FROM_BUF = std::is_same<In, FromBuf>::value;
    constexpr bool TO_BUF = std::is_same<Out, ToBuf>::value;
    static_assert(TO_BUF || !(LAST8 && last_radix8<V>()), "no epilogue after radix8_last");
    const int L = 1 << logL;
    const int quarter_log = logL - 2;
    int logn = skip_first ? logL - 2 : logL, logs = skip_first ? 2 : 0;
    const int stop = (LAST8 && last_radix8<V>() && (logL & 1) && logL >= 3) ? 3 : 1;
    bool first = !skip_first;
    while (logn > stop) {
        const int m = 1 << (logn - 2);          // n / 4
        const int s = 1 << logs;
        const int nbf = nl << (logL - 2);       // butterflies in this step
        const bool load = !FROM_BUF && first;   // inputs from the loader
        const bool emit = !TO_BUF && logn == 2; // the transform's last step: to the epilogue
        V v[BPT][4];
        int base[BPT], pp[BPT], ln[BPT], kq[BPT];
        bool act[BPT];
#pragma unroll
        for (int h = 0; h < BPT; ++h) {
            const int b = threadIdx.x + h * blockDim.x;
            act[h] = b < nbf;
            if (act[h]) {
                const int line = b >> quarter_log;
                const int bb = b & ((L >> 2) - 1);
                const int p = bb >> logs, q = bb & (s - 1);
                const int x = line * pitch + q;
                if constexpr (!FROM_BUF) {
                    if (load) {
#pragma unroll
                        for (int t = 0; t < 4; ++t) v[h][t] = in(line, q + s * (p + t * m));
                    } else {
#pragma unroll
                        for (int t = 0; t < 4; ++t) v[h][t] = buf[x + s * (p + t * m)];
                    }
                } else {
#pragma unroll
                    for (int t = 0; t < 4; ++t) v[h][t] = buf[x + s * (p + t * m)];
                }
                bfly4<V, SIGN>(v[h][0], v[h][1], v[h][2], v[h][3]);
                if (p != 0) {
                    // omega_n^{p u}
                    v[h][1] = mul_tw(v[h][1], step_twiddle<V, SIGN, R>(tw, logn, p, 1));
                    v[h][2] = mul_tw(v[h][2], step_twiddle<V, SIGN, R>(tw, logn, p, 2));
                    v[h][3] = mul_tw(v[h][3], step_twiddle<V, SIGN, R>(tw, logn, p, 3));
                }
                base[h] = line * pitch + q + s * 4 * p;
                pp[h] = s;
                ln[h] = line;
                kq[h] = q + s * 4 * p;
            }
        }
        if constexpr (!TO_BUF) {
            if (emit) {
                // the last step (n = 4, p = 0): element q + u s of each line
#pragma unroll
                for (int h = 0; h < BPT; ++h) {
                    if (act[h]) {
#pragma unroll
                        for (int u = 0; u < 4; ++u) out(ln[h], kq[h] + u * pp[h], v[h][u]);
                    }
                }
                return;
            }
        }
        // the writes wait for every read of this step (none when loaded)
        if (!load) __syncthreads();
#pragma unroll
        for (int h = 0; h < BPT; ++h) {
            if (act[h]) {
#pragma unroll
                for (int u = 0; u < 4; ++u) buf[base[h] + u * pp[h]] = v[h][u];
            }
        }
        __syncthreads();
        logn -= 2;
        logs += 2;
        first = false;
    }
    if (logn == 3 && stop == 3) {
        radix8_last<V, SIGN, R>(buf, logL, nl, pitch, tw);
    } else if (logn == 1 && !leave_radix2) {
        // final radix-2 step: n = 2, s = L/2, no twiddle
        const int half = L >> 1;
        const int nbf = nl * half;
        for (int b = threadIdx.x; b < nbf; b += blockDim.x) {
            const int line = b / half, q = b - line * half;
            const int x = line * pitch + q;
            const V a = buf[x], c = buf[x + half];
            if constexpr (TO_BUF) {
                buf[x] = a + c;
                buf[x + half] = a - c;
            } else {
                out(line, q, a + c);
                out(line, q + half, a - c);
            }
        }
        if constexpr (TO_BUF) __syncthreads();
    }
}

// ---- lines of length L = R 2^a, R = 3 or 5 ---------------------------------------
//
// The same Stockham factorisation with the radix-4 steps first (sub-lengths
// n = R 2^a, R 2^(a-2), ..., 4 R; a even, so s stays a power of two and the
// twiddles omega_n^{p u} come from the family-R tables) and one radix-R
// step last (n = R, s = L/R, no twiddle):
//   y[q + s u] = sum_t x[q + s t] omega_R^{SIGN t u},   u = 0 .. R-1.
// Radix 3, with S = x1 + x2, D = x1 - x2 and omega_3^{+-1} = -1/2 +- i sqrt(3)/2:
//   y0 = x0 + S,   y1 = T + U,   y2 = T - U,
//   T = x0 - S/2,  U = (SIGN i sqrt(3)/2) D.
// Radix 5, with S1 = x1 + x4, D1 = x1 - x4, S2 = x2 + x3, D2 = x2 - x3 and
// omega_5^{SIGN k} = c_k + i s_k (k = 1, 2):
//   y0 = x0 + S1 + S2,
//   y1, y4 = A +- U,  A = x0 + c1 S1 + c2 S2,  U = i (s1 D1 + s2 D2),
//   y2, y3 = B +- W,  B = x0 + c2 S1 + c1 S2,  W = i (s2 D1 - s1 D2).
// S/2 is an exact scaling (scale_pow2); the products by the real numbers c_k
// and the pure imaginary numbers i s_k use enclosures of those numbers alone
// (ScalarSet, computed once per plan from the family-R table), in half the
// operations of a general twiddle product (mul_real, mul_imag).
// Requires nl * L / 4 <= BPT * blockDim.x, like block_fft.

// The real number cos or the pure imaginary number i sin of the enclosure
// omega_Ntab^j (family R, forward sign) in the twiddle type of V, built
// from the one component of the rectangle table that it needs: a rectangle
// with the other part the point 0; a disc whose radius bounds that
// component's error alone (a twiddle disc's radius covers both components)
// and whose modulus bound is |centre|.
__device__ __forceinline__ void mid_rad(double lo, double hi, double& c, float& r) {
    c = __dadd_rn(0.5 * lo, 0.5 * hi);
    r = __double2float_ru(fmax(__dsub_ru(c, lo), __dsub_ru(hi, c)));
}

template <int R>
__device__ void scalar_entry(const TwTable& tw, uint32_t j, bool imag, int k, ScalarSet& out) {
    const CI<double> w = twiddle<double, 1, R>(tw, j);
    const CI<float> f = twiddle<float, 1, R>(tw, j);
    out.d[k] = imag ? CI<double>{0.0, 0.0, w.il, w.ih} : CI<double>{w.rl, w.rh, 0.0, 0.0};
    out.f[k] = imag ? CI<float>{0.f, 0.f, f.il, f.ih} : CI<float>{f.rl, f.rh, 0.f, 0.f};
    double c;
    float r;
    mid_rad(imag ? w.il : w.rl, imag ? w.ih : w.rh, c, r);
    const float m = abs_up(c);
    out.disc[k] = imag ? DiscTw{0.0, c, r, m} : DiscTw{c, 0.0, r, m};
    // the binary64 centre split into a pair as in k_ddisc_tw_gen (|c| <= 1)
    const float h = __double2float_rn(c), l = __double2float_rn(c - double(h));
    const float rr = __fadd_ru(r, 2.f * DD_U2 + DD_ETA);
    const float mm = dd_mod_up(h, 0.f);
    out.dd[k] = imag ? DDiscTw{0.f, 0.f, h, l, rr, mm} : DDiscTw{h, l, 0.f, 0.f, rr, mm};
}

// R = 3: [0] = i sin(2 pi/3).  R = 5: [0] = cos(2 pi/5), [1] = cos(4 pi/5),
// [2] = i sin(2 pi/5), [3] = i sin(4 pi/5).  Written by one thread.
template <int R>
__global__ void k_scalar_gen(TwTable tw, ScalarSet* out) {
    if (blockIdx.x != 0 || threadIdx.x != 0) return;
    ScalarSet s{};
    const uint32_t third = 1u << tw.log_n;                   // Ntab / R
    if (R == 3) {
        scalar_entry<R>(tw, third, true, 0, s);
    } else {
        scalar_entry<R>(tw, third, false, 0, s);
        scalar_entry<R>(tw, 2u * third, false, 1, s);
        scalar_entry<R>(tw, third, true, 2, s);
        scalar_entry<R>(tw, 2u * third, true, 3, s);
    }
    *out = s;
}

template <typename V> struct ScalarOf;
template <> struct ScalarOf<CI<double>> {
    static __device__ __forceinline__ CI<double> get(const ScalarSet* s, int k) { return s->d[k]; }
};
template <> struct ScalarOf<CI<float>> {
    static __device__ __forceinline__ CI<float> get(const ScalarSet* s, int k) { return s->f[k]; }
};
template <> struct ScalarOf<Disc> {
    static __device__ __forceinline__ DiscTw get(const ScalarSet* s, int k) { return s->disc[k]; }
};
template <> struct ScalarOf<Pt> : ScalarOf<Disc> {};
template <> struct ScalarOf<DDisc> {
    static __device__ __forceinline__ DDiscTw get(const ScalarSet* s, int k) { return s->dd[k]; }
};

// scalar k for the transform of sign SIGN: the inverse conjugates, which
// negates the imaginary scalars (a sign-bit flip) and keeps the real ones
template <typename V, int SIGN>
__device__ __forceinline__ typename VTraits<V>::Tw scalar_tw(const TwTable& tw, int k) {
    const auto w = ScalarOf<V>::get(tw.scal, k);
    return SIGN > 0 ? w : tw_conj(w);
}

// As in block_fft, the first radix-4 step may take its inputs from a
// loader in(line, k) instead of buf (not with skip_first; loga >= 2), and
// the radix-R step may hand its outputs to an epilogue out(line, k, y)
// from the registers of the thread that computed them, with no barrier
// after: the kernels whose next use of an element is per element (the
// forward columns' four-step twiddle and store) skip a round trip through
// shared memory.
template <typename V, int SIGN, int BPT = 2, int R = 3, typename In = FromBuf, typename Out = ToBuf>
__device__ void block_fft_odd(SBuf<V> buf, int loga, int nl, int pitch, const TwTable& tw,
                              bool skip_first = false, In in = In{}, Out out = Out{}) {
    constexpr bool FROM_BUF = std::is_same<In, FromBuf>::value;
    constexpr bool TO_BUF = std::is_same<Out, ToBuf>::value;
    static_assert(R == 3 || R == 5, "odd factor 3 or 5");
    const int L = R << loga;
    const int Lq = L >> 2;                      // butterflies per line in a radix-4 step
    int logn2 = skip_first ? loga - 2 : loga;   // n = R 2^logn2, s = 2^logs
    int logs = skip_first ? 2 : 0;
    bool first = !skip_first;
    while (logn2 >= 2) {
        const int m = R << (logn2 - 2);         // n / 4
        const int s = 1 << logs;
        const int nbf = nl * Lq;
        const bool load = !FROM_BUF && first;   // inputs from the loader
        V v[BPT][4];
        int base[BPT], pp[BPT];
        bool act[BPT];
#pragma unroll
        for (int h = 0; h < BPT; ++h) {
            const int b = threadIdx.x + h * blockDim.x;
            act[h] = b < nbf;
            if (act[h]) {
                const int line = b / Lq;
                const int bb = b - line * Lq;
                const int p = bb >> logs, q = bb & (s - 1);
                const int x = line * pitch + q;
                if constexpr (!FROM_BUF) {
                    if (load) {
#pragma unroll
                        for (int t = 0; t < 4; ++t) v[h][t] = in(line, q + s * (p + t * m));
                    } else {
#pragma unroll
                        for (int t = 0; t < 4; ++t) v[h][t] = buf[x + s * (p + t * m)];
                    }
                } else {
#pragma unroll
                    for (int t = 0; t < 4; ++t) v[h][t] = buf[x + s * (p + t * m)];
                }
                bfly4<V, SIGN>(v[h][0], v[h][1], v[h][2], v[h][3]);
                if (p != 0) {
                    v[h][1] = mul_tw(v[h][1], step_twiddle_r<V, SIGN, R>(tw, logn2, p, 1));
                    v[h][2] = mul_tw(v[h][2], step_twiddle_r<V, SIGN, R>(tw, logn2, p, 2));
                    v[h][3] = mul_tw(v[h][3], step_twiddle_r<V, SIGN, R>(tw, logn2, p, 3));
                }
                base[h] = line * pitch + q + s * 4 * p;
                pp[h] = s;
            }
        }
        // the writes wait for every read of this step (none when loaded)
        if (!load) __syncthreads();
#pragma unroll
        for (int h = 0; h < BPT; ++h) {
            if (act[h]) {
#pragma unroll
                for (int u = 0; u < 4; ++u) buf[base[h] + u * pp[h]] = v[h][u];
            }
        }
        __syncthreads();
        logn2 -= 2;
        logs += 2;
        first = false;
    }
    // radix-R step: n = R, s = 2^loga; each thread owns its R elements
    const int part = 1 << loga;
    // output u of the butterfly at (line, q): element q + u part of the line
    const auto put = [&](int line, int q, int u, const V& y) {
        if constexpr (TO_BUF) buf[line * pitch + q + u * part] = y;
        else out(line, q + u * part, y);
    };
    if (R == 3) {
        const auto w3 = scalar_tw<V, SIGN>(tw, 0);        // i Im omega_3^SIGN
        for (int b = threadIdx.x; b < nl * part; b += blockDim.x) {
            const int line = b >> loga, q = b & (part - 1);
            const int x = line * pitch + q;
            const V x0 = buf[x], x1 = buf[x + part], x2 = buf[x + 2 * part];
            const V S = x1 + x2, D = x1 - x2;
            const V T = x0 - scale_pow2(S, 1);
            const V U = mul_imag(D, w3);
            put(line, q, 0, x0 + S);
            put(line, q, 1, T + U);
            put(line, q, 2, T - U);
        }
    } else {
        // omega_5^(SIGN k) = c_k + i s_k, k = 1, 2
        const auto c1 = scalar_tw<V, SIGN>(tw, 0), c2 = scalar_tw<V, SIGN>(tw, 1);
        const auto s1 = scalar_tw<V, SIGN>(tw, 2), s2 = scalar_tw<V, SIGN>(tw, 3);
        for (int b = threadIdx.x; b < nl * part; b += blockDim.x) {
            const int line = b >> loga, q = b & (part - 1);
            const int x = line * pitch + q;
            const V x0 = buf[x], x1 = buf[x + part], x2 = buf[x + 2 * part];
            const V x3 = buf[x + 3 * part], x4 = buf[x + 4 * part];
            const V S1 = x1 + x4, D1 = x1 - x4, S2 = x2 + x3, D2 = x2 - x3;
            const V A = (x0 + mul_real(S1, c1)) + mul_real(S2, c2);
            const V B = (x0 + mul_real(S1, c2)) + mul_real(S2, c1);
            const V U = mul_imag(D1, s1) + mul_imag(D2, s2);
            const V W = mul_imag(D1, s2) - mul_imag(D2, s1);
            put(line, q, 0, (x0 + S1) + S2);
            put(line, q, 1, A + U);
            put(line, q, 4, A - U);
            put(line, q, 2, B + W);
            put(line, q, 3, B - W);
        }
    }
    if constexpr (TO_BUF) __syncthreads();
}

// ---- the first step of a forward transform of digits ---------------------------------
//
// The forward transform's inputs are the Gaussian integers a_j + i b_j of
// the digits (Section 2.3), so the first radix-4 step's 4-point sums (n = L,
// s = 1, p < L/4) are exact in integer arithmetic: only its twiddle
// products omega_L^{p u} round.  in[line * ipitch + j] holds the inputs;
// the step's outputs go to buf at block_fft's positions (line * pitch +
// 4 p + u), after every input has been read, so in may share memory with
// buf.  ODD: L = R 2^lg with the family-R step twiddles (block_fft_odd);
// otherwise L = 2^lg >= 4.  The remaining steps are block_fft(...,
// skip_first = true) or block_fft_odd(..., true).  Requires
// nl * L / 4 <= BPT * blockDim.x.
template <typename V, int BPT, int R, bool ODD>
__device__ void first_step_exact(const int2* in, int ipitch, SBuf<V> buf, int lg, int nl, int pitch,
                                 const TwTable& tw) {
    const int m = ODD ? (R << (lg - 2)) : (1 << (lg - 2));      // L / 4
    const int nbf = nl * m;
    V v[BPT][4];
    int base[BPT];
    bool act[BPT];
#pragma unroll
    for (int h = 0; h < BPT; ++h) {
        const int b = threadIdx.x + h * blockDim.x;
        act[h] = b < nbf;
        if (act[h]) {
            const int line = ODD ? b / m : b >> (lg - 2);
            const int p = b - line * m;
            const int2* x = in + line * ipitch + p;
            const int2 x0 = x[0], x1 = x[m], x2 = x[2 * m], x3 = x[3 * m];
            const int apr = x0.x + x2.x, api = x0.y + x2.y, amr = x0.x - x2.x, ami = x0.y - x2.y;
            const int bpr = x1.x + x3.x, bpi = x1.y + x3.y, bmr = x1.x - x3.x, bmi = x1.y - x3.y;
            v[h][0] = make_point<V>(apr + bpr, api + bpi);      // u = 0
            v[h][2] = make_point<V>(apr - bpr, api - bpi);      // u = 2
            v[h][1] = make_point<V>(amr - bmi, ami + bmr);      // u = 1: + i (x1 - x3)
            v[h][3] = make_point<V>(amr + bmi, ami - bmr);      // u = 3: - i (x1 - x3)
            if (p != 0) {
#pragma unroll
                for (int u = 1; u < 4; ++u) {
                    if constexpr (ODD) v[h][u] = mul_tw(v[h][u], step_twiddle_r<V, 1, R>(tw, lg, p, u));
                    else v[h][u] = mul_tw(v[h][u], step_twiddle<V, 1, R>(tw, lg, p, u));
                }
            }
            base[h] = line * pitch + 4 * p;
        }
    }
    __syncthreads();
#pragma unroll
    for (int h = 0; h < BPT; ++h) {
        if (act[h]) {
#pragma unroll
            for (int u = 0; u < 4; ++u) buf[base[h] + u] = v[h][u];
        }
    }
    __syncthreads();
}

}  // namespace ssm
