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

// R: the family of the twiddle table tw (the line length is 2^logL either way)
template <typename V, int SIGN, int BPT = 2, int R = 1>
__device__ void block_fft(SBuf<V> buf, int logL, int nl, int pitch, const TwTable& tw) {
    const int L = 1 << logL;
    const int quarter_log = logL - 2;
    int logn = logL, logs = 0;
    while (logn >= 2) {
        const int m = 1 << (logn - 2);          // n / 4
        const int s = 1 << logs;
        const int nbf = nl << (logL - 2);       // butterflies in this step
        V v[BPT][4];
        int base[BPT], pp[BPT];
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
#pragma unroll
                for (int t = 0; t < 4; ++t) v[h][t] = buf[x + s * (p + t * m)];
                bfly4<V, SIGN>(v[h][0], v[h][1], v[h][2], v[h][3]);
                if (p != 0) {
                    // omega_n^{p u}
                    v[h][1] = mul_tw(v[h][1], step_twiddle<V, SIGN, R>(tw, logn, p, 1));
                    v[h][2] = mul_tw(v[h][2], step_twiddle<V, SIGN, R>(tw, logn, p, 2));
                    v[h][3] = mul_tw(v[h][3], step_twiddle<V, SIGN, R>(tw, logn, p, 3));
                }
                base[h] = line * pitch + q + s * 4 * p;
                pp[h] = s;
            }
        }
        __syncthreads();
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
    }
    if (logn == 1) {
        // final radix-2 step: n = 2, s = L/2, no twiddle
        const int half = L >> 1;
        const int nbf = nl * half;
        for (int b = threadIdx.x; b < nbf; b += blockDim.x) {
            const int line = b / half, q = b - line * half;
            const int x = line * pitch + q;
            const V a = buf[x], c = buf[x + half];
            buf[x] = a + c;
            buf[x + half] = a - c;
        }
        __syncthreads();
    }
}

// ---- lines of length L = 3 2^a --------------------------------------------------
//
// The same Stockham factorisation with the radix-4 steps first (sub-lengths
// n = 3 2^a, 3 2^(a-2), ..., 12; a even, so s stays a power of two and the
// twiddles omega_n^{p u} come from the family-3 tables) and one radix-3
// step last (n = 3, s = L/3, no twiddle):
//   y[q + s u] = sum_t x[q + s t] omega_3^{SIGN t u},   u = 0, 1, 2.
// With S = x1 + x2, D = x1 - x2 and omega_3^{+-1} = -1/2 +- i sqrt(3)/2:
//   y0 = x0 + S,   y1 = T + U,   y2 = T - U,
//   T = x0 - S/2,  U = (SIGN i sqrt(3)/2) D,
// where S/2 is an exact scaling (scale_pow2) and U a product with the
// enclosure of SIGN i sqrt(3)/2: the imaginary part of the family-3 table's
// enclosure of omega_3^SIGN, its real part replaced by the point 0 (the
// rectangle or disc of that pure imaginary number lies inside).
// Requires nl * L / 4 <= BPT * blockDim.x, like block_fft.

template <typename V> __device__ __forceinline__ typename VTraits<V>::Tw imag_only(const typename VTraits<V>::Tw& w);
template <> __device__ __forceinline__ CI<double> imag_only<CI<double>>(const CI<double>& w) {
    return {0.0, 0.0, w.il, w.ih};
}
template <> __device__ __forceinline__ CI<float> imag_only<CI<float>>(const CI<float>& w) {
    return {0.f, 0.f, w.il, w.ih};
}
template <> __device__ __forceinline__ DiscTw imag_only<Disc>(const DiscTw& w) {
    return {0.0, w.s, w.rho, 0.f};
}
template <> __device__ __forceinline__ DiscTw imag_only<Pt>(const DiscTw& w) {
    return {0.0, w.s, w.rho, 0.f};
}
template <> __device__ __forceinline__ DDiscTw imag_only<DDisc>(const DDiscTw& w) {
    return {0.f, 0.f, w.sh, w.sl, w.rho, 0.f};
}

template <typename V, int SIGN, int BPT = 2>
__device__ void block_fft3(SBuf<V> buf, int loga, int nl, int pitch, const TwTable& tw) {
    const int L = 3 << loga;
    const int Lq = L >> 2;                      // butterflies per line in a radix-4 step
    int logn2 = loga, logs = 0;                 // n = 3 2^logn2, s = 2^logs
    while (logn2 >= 2) {
        const int m = 3 << (logn2 - 2);         // n / 4
        const int s = 1 << logs;
        const int nbf = nl * Lq;
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
#pragma unroll
                for (int t = 0; t < 4; ++t) v[h][t] = buf[x + s * (p + t * m)];
                bfly4<V, SIGN>(v[h][0], v[h][1], v[h][2], v[h][3]);
                if (p != 0) {
                    v[h][1] = mul_tw(v[h][1], step_twiddle3<V, SIGN>(tw, logn2, p, 1));
                    v[h][2] = mul_tw(v[h][2], step_twiddle3<V, SIGN>(tw, logn2, p, 2));
                    v[h][3] = mul_tw(v[h][3], step_twiddle3<V, SIGN>(tw, logn2, p, 3));
                }
                base[h] = line * pitch + q + s * 4 * p;
                pp[h] = s;
            }
        }
        __syncthreads();
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
    }
    // radix-3 step: n = 3, s = 2^loga; each thread owns its three elements
    const auto w3 = imag_only<V>(get_twiddle<V, SIGN, 3>(tw, 1u << tw.log_n));   // omega_3^SIGN
    const int third = 1 << loga;
    for (int b = threadIdx.x; b < nl * third; b += blockDim.x) {
        const int line = b >> loga, q = b & (third - 1);
        const int x = line * pitch + q;
        const V x0 = buf[x], x1 = buf[x + third], x2 = buf[x + 2 * third];
        const V S = x1 + x2, D = x1 - x2;
        const V T = x0 - scale_pow2(S, 1);
        const V U = mul_tw(D, w3);
        buf[x] = x0 + S;
        buf[x + third] = T + U;
        buf[x + 2 * third] = T - U;
    }
    __syncthreads();
}

}  // namespace ssm
