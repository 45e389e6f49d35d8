/*
 * oracle/exact.c -- exact integer reference for the interval
 * Schoenhage-Strassen multiplier.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously correct CPU
 * oracle that the tests, the smoke check and the CPU-baseline leg of the
 * benchmark compare the GPU path against.  Nothing in the product path
 * includes, links or calls it, and it shares no code with the GPU path.
 *
 * Every routine here computes an exact integer result written straight from
 * its definition in Steinke & Sainudiin, "A Rigorous Extension of the
 * Schoenhage-Strassen Integer Multiplication Algorithm Using Complex
 * Interval Arithmetic" (CCA 2010):
 *
 *   digits          x = sum_i x_i b^i, b = 256, digit 0 least significant
 *                   (Section 2, digit convention)
 *   long_mul        the long multiplication algorithm (Section 2.1)
 *   conv            the coefficients of the product polynomial,
 *                   c_i = sum_j x_j y_{i-j}  (Section 2.1, product identity)
 *   carry           evaluating f_{x*y}(b) as base-b digits (Section 2.4,
 *                   the Schoenhage-Strassen algorithm's carry loop)
 *   conv_ntt        the same c_i for sizes where O(n m) is too slow: a
 *                   number-theoretic transform modulo the prime
 *                   p = 2^64 - 2^32 + 1.  Exact because every c_i < p.
 *                   It is a library-style primitive (an exact convolution),
 *                   not part of the paper's method, and tests pin it to
 *                   `conv` and to Python's own big-integer product.
 *   residue         x mod p by Horner's rule, for product checks mod primes.
 *
 * Accumulators are uint64: c_i <= 255^2 * min(n, m) < 2^40 for n, m < 2^24.
 */
#include <stdint.h>
#include <stddef.h>
#include <string.h>
#include <stdlib.h>

#define BASE 256u

/* Section 2.1, long multiplication: for i = 0 .. n+m-1, s = sum over the
 * admissible j of x_j y_{i-j}; z_i = (s + c) mod b; c = floor((s + c) / b).
 * Written in the order of the algorithm, single threaded. */
int oracle_long_mul(const uint8_t* x, size_t n, const uint8_t* y, size_t m, uint8_t* z)
{
    if (n == 0 || m == 0) return -1;
    uint64_t c = 0;
    for (size_t i = 0; i < n + m; ++i) {
        uint64_t s = 0;
        size_t jlo = (i + 1 > m) ? i + 1 - m : 0;      /* max{0, i-m+1} */
        size_t jhi = (i < n - 1) ? i : n - 1;          /* min{n-1, i}   */
        for (size_t j = jlo; j <= jhi && j < n; ++j)
            s += (uint64_t)x[j] * (uint64_t)y[i - j];
        z[i] = (uint8_t)((s + c) % BASE);
        c = (s + c) / BASE;
    }
    return c == 0 ? 0 : -2;   /* the final carry is zero: x y < b^(n+m) */
}

/* Section 2.1, product identity: c_i = sum_{j=max(0,i-m+1)}^{min(n-1,i)} x_j y_{i-j},
 * for i = 0 .. n+m-2.  Each c_i is an independent sum, so the loop over i
 * runs in parallel; the sum itself is the plain definition. */
int oracle_conv(const uint8_t* x, size_t n, const uint8_t* y, size_t m, uint64_t* c)
{
    if (n == 0 || m == 0) return -1;
    long long L = (long long)(n + m - 1);
#pragma omp parallel for schedule(dynamic, 256)
    for (long long ii = 0; ii < L; ++ii) {
        size_t i = (size_t)ii;
        size_t jlo = (i + 1 > m) ? i + 1 - m : 0;
        size_t jhi = (i < n - 1) ? i : n - 1;
        uint64_t s = 0;
        for (size_t j = jlo; j <= jhi; ++j)
            s += (uint32_t)x[j] * (uint32_t)y[i - j];
        c[i] = s;
    }
    return 0;
}

/* Section 2.4, carry: z_i = (c_i + carry) mod b, carry = floor((c_i + carry)/b)
 * for i = 0 .. L-1, then the remaining carry fills the top digits.  Returns
 * 0 when the value fits in nz digits, -2 otherwise. */
int oracle_carry(const uint64_t* c, size_t L, uint8_t* z, size_t nz)
{
    unsigned __int128 carry = 0;
    size_t i = 0;
    for (; i < L; ++i) {
        unsigned __int128 t = (unsigned __int128)c[i] + carry;
        if (i < nz) z[i] = (uint8_t)(t % BASE);
        else if (t % BASE) return -2;
        carry = t / BASE;
    }
    for (; i < nz; ++i) {
        z[i] = (uint8_t)(carry % BASE);
        carry /= BASE;
    }
    return carry == 0 ? 0 : -2;
}

/* ---- number-theoretic transform over Z_p, p = 2^64 - 2^32 + 1 ---------- */

static const uint64_t P = 0xFFFFFFFF00000001ull;   /* 2^32 divides p - 1 */
static const uint64_t G = 7;                       /* generator of Z_p^* */

static uint64_t mulmod(uint64_t a, uint64_t b) {
    return (uint64_t)(((unsigned __int128)a * b) % P);
}
static uint64_t addmod(uint64_t a, uint64_t b) {
    unsigned __int128 s = (unsigned __int128)a + b;
    return (uint64_t)(s % P);
}
static uint64_t submod(uint64_t a, uint64_t b) {
    return a >= b ? a - b : (uint64_t)((unsigned __int128)a + P - b);
}
static uint64_t powmod(uint64_t a, uint64_t e) {
    uint64_t r = 1;
    while (e) { if (e & 1) r = mulmod(r, a); a = mulmod(a, a); e >>= 1; }
    return r;
}

uint64_t oracle_ntt_prime(void) { return P; }
uint64_t oracle_ntt_root(uint64_t n) { return powmod(G, (P - 1) / n); }

/* In-place iterative radix-2 transform of length n (a power of two),
 * X_k = sum_j x_j w^{jk} with w = root of unity of order n (inverse: w^-1). */
static void ntt(uint64_t* a, size_t n, int inverse)
{
    for (size_t i = 1, j = 0; i < n; ++i) {            /* bit reversal */
        size_t bit = n >> 1;
        for (; j & bit; bit >>= 1) j ^= bit;
        j ^= bit;
        if (i < j) { uint64_t t = a[i]; a[i] = a[j]; a[j] = t; }
    }
    for (size_t len = 2; len <= n; len <<= 1) {
        uint64_t w = powmod(G, (P - 1) / len);
        if (inverse) w = powmod(w, P - 2);
        long long groups = (long long)(n / len);
#pragma omp parallel for schedule(static) if (n >= 4096)
        for (long long g = 0; g < groups; ++g) {
            size_t i = (size_t)g * len;
            uint64_t wj = 1;
            for (size_t j = 0; j < len / 2; ++j) {
                uint64_t u = a[i + j], v = mulmod(a[i + j + len / 2], wj);
                a[i + j] = addmod(u, v);
                a[i + j + len / 2] = submod(u, v);
                wj = mulmod(wj, w);
            }
        }
    }
    if (inverse) {
        uint64_t ninv = powmod((uint64_t)n, P - 2);
        for (size_t i = 0; i < n; ++i) a[i] = mulmod(a[i], ninv);
    }
}

/* Exact convolution by the NTT: same output as oracle_conv. */
int oracle_conv_ntt(const uint8_t* x, size_t n, const uint8_t* y, size_t m, uint64_t* c)
{
    if (n == 0 || m == 0) return -1;
    size_t L = n + m - 1, N = 1;
    while (N < L) N <<= 1;
    if (N > ((size_t)1 << 32)) return -3;
    uint64_t* fa = (uint64_t*)calloc(N, sizeof(uint64_t));
    uint64_t* fb = (uint64_t*)calloc(N, sizeof(uint64_t));
    if (!fa || !fb) { free(fa); free(fb); return -4; }
    for (size_t i = 0; i < n; ++i) fa[i] = x[i];
    for (size_t i = 0; i < m; ++i) fb[i] = y[i];
    ntt(fa, N, 0);
    ntt(fb, N, 0);
    for (size_t i = 0; i < N; ++i) fa[i] = mulmod(fa[i], fb[i]);
    ntt(fa, N, 1);
    memcpy(c, fa, L * sizeof(uint64_t));
    free(fa);
    free(fb);
    return 0;
}

/* x mod p by Horner's rule from the top digit: x = (...(x_{n-1} b + x_{n-2}) b ...) + x_0. */
uint64_t oracle_residue(const uint8_t* x, size_t n, uint64_t p)
{
    unsigned __int128 r = 0;
    for (size_t i = n; i-- > 0;) r = (r * BASE + x[i]) % p;
    return (uint64_t)r;
}

/* Same for a coefficient vector: sum_i c_i b^i mod p. */
uint64_t oracle_residue_coeffs(const uint64_t* c, size_t L, uint64_t p)
{
    unsigned __int128 r = 0;
    for (size_t i = L; i-- > 0;) r = (r * BASE + (c[i] % p)) % p;
    return (uint64_t)r;
}

int oracle_num_threads(void)
{
#ifdef _OPENMP
    extern int omp_get_max_threads(void);
    return omp_get_max_threads();
#else
    return 1;
#endif
}
