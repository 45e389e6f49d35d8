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

template <typename V, int SIGN, int BPT = 2>
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
                    v[h][1] = mul_tw(v[h][1], step_twiddle<V, SIGN>(tw, logn, p, 1));
                    v[h][2] = mul_tw(v[h][2], step_twiddle<V, SIGN>(tw, logn, p, 2));
                    v[h][3] = mul_tw(v[h][3], step_twiddle<V, SIGN>(tw, logn, p, 3));
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

}  // namespace ssm
