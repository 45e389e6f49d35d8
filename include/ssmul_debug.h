/*
 * ssmul_debug.h -- inspection entry points of the ssmul library, used by its
 * tests.  They expose intermediate results of the method so that its rigor
 * (every interval contains the exact value) can be checked from outside.
 * Same conventions as ssmul.h: plain pointers, ssmul_status results, no
 * aborts.  They are not on the performance path.
 */
#ifndef SSMUL_DEBUG_H
#define SSMUL_DEBUG_H

#include "ssmul.h"

#ifdef __cplusplus
extern "C" {
#endif

/*
 * Copy one of the plan's twiddle tables to host memory: the enclosures of
 * cos(2 pi j / Ntab) and sin(2 pi j / Ntab) for j = 0 .. Ntab/8 (the roots
 * of unity of the DFT, Section 2.2), as 4 doubles per entry
 * (cos_lo, cos_hi, sin_lo, sin_hi).  f32 bit 0 selects the binary32 table
 * (values widened to double exactly); bit 1 the family Ntab = 3 * 2^K of
 * the lengths 3 * 2^k, bit 2 the family Ntab = 5 * 2^K of the lengths
 * 5 * 2^k (SSMUL_OPT_LENGTHS; SSMUL_INVALID_ARG when the plan has none or
 * both bits are set), else Ntab = 2^K.  *log_ntab receives K.  cap is the
 * capacity of h_out in doubles; SSMUL_INVALID_ARG when too small.
 */
ssmul_status ssmul_debug_twiddles(ssmul_plan_t plan, int f32, double* h_out, size_t cap,
                                  int* log_ntab);

/*
 * One product as ssmul_mul, forced to a single precision rung (prec is
 * SSMUL_PREC_FP64, _FP32, _DISC64, _DISC32X2 or _NAIVE64), that also writes the enclosure of
 * every convolution coefficient c_i = sum_j a_j b_{i-j} (Section 2.1) to
 * d_iv (device memory, 2 * (na + nb - 1) doubles: lo_i, hi_i) after the
 * inverse transform and the division by N (Sections 2.3, 2.5).  For
 * _NAIVE64 both values are the unverified point result.  _FP32 transforms
 * the bytes here whatever SSMUL_OPT_FP32_NIBBLES says.
 * prec = SSMUL_DEBUG_PREC_FP32_NIBBLES (na + nb <= 2048): binary32
 * rectangles on the 4-bit digits a'_j, b'_j (a = sum_j a'_j 16^j); d_iv
 * receives the enclosures of c'_i = sum_j a'_j b'_{i-j}, i < 2 (na + nb) - 1
 * (2 * (2 (na + nb) - 1) doubles): the enclosures of the centred digits'
 * coefficients plus their exact correction, rounded outwards.
 * SSMUL_INVALID_ARG when the plan's SSMUL_OPT_FP32_NIBBLES is 0.
 */
#define SSMUL_DEBUG_PREC_FP32_NIBBLES 100
ssmul_status ssmul_debug_mul_intervals(ssmul_plan_t plan, const uint8_t* d_a, size_t na,
                                       const uint8_t* d_b, size_t nb, uint8_t* d_z,
                                       ssmul_result* h_res, ssmul_precision prec,
                                       double* d_iv);

/*
 * Elementwise complex interval operation on n operands (Section 2.5), for
 * unit tests of the device arithmetic.  d_x, d_y, d_out: device arrays of
 * 4 doubles per operand (re_lo, re_hi, im_lo, im_hi).  op: 0 add, 1
 * subtract, 2 product by a twiddle enclosure d_y (components that do not
 * contain 0 unless they are the point 0), 3 general product, 4 product by
 * the real enclosure d_y (its real part, not containing 0; the imaginary
 * part is not read), 5 product by the pure imaginary enclosure d_y (its
 * imaginary part, not containing 0).  f32 != 0 runs the binary32
 * arithmetic on operands that must be binary32 values.
 */
ssmul_status ssmul_debug_ci_op(int op, int f32, const double* d_x, const double* d_y,
                               double* d_out, size_t n);

/*
 * Elementwise disc operation on n operands (the circular containment sets
 * of SSMUL_PREC_DISC64), for unit tests of the device arithmetic.  d_x,
 * d_y, d_out: device arrays of 3 doubles per operand (centre re, centre im,
 * radius; the radius is used as a binary32 value).  op: 0 add, 1 subtract,
 * 2 product by a twiddle disc d_y (|centre| <= 1), 3 general product,
 * 4 scaling by 2^-k with k = (int) d_y[3 i], 5 (6) product by the real
 * (pure imaginary) disc d_y: the disc's centre im (re) is taken as 0.
 */
ssmul_status ssmul_debug_disc_op(int op, const double* d_x, const double* d_y, double* d_out,
                                 size_t n);

/*
 * The same for discs with double-binary32 centres (SSMUL_PREC_DISC32X2):
 * 5 doubles per operand (centre re as hi, lo; centre im as hi, lo; radius),
 * every value a binary32 number, pairs normalised (|lo| <= 2^-24 |hi|).
 * op 2 takes d_y as a twiddle disc (|centre| <= 1); op 4 scales by 2^-k
 * with k = (int) d_y[5 i].  op 5 (6): the radix-4 butterfly of the
 * transform (the inverse's) on the four discs d_x[20 i .. 20 i + 20), its
 * four outputs at d_out[20 i ..] sharing one radius; d_y is not read and
 * may be NULL.  op 7 (8): product by the real (pure imaginary) disc d_y,
 * whose centre im (re) is taken as 0.
 */
ssmul_status ssmul_debug_ddisc_op(int op, const double* d_x, const double* d_y, double* d_out,
                                  size_t n);

/*
 * The isolation decision (Section 1: accept a coefficient only when its
 * enclosure holds exactly one integer) for one component of a
 * double-binary32 disc, n of them independently.  Row i of d_x (device,
 * 4 doubles, the first three binary32 values) is (h, l, r, pad): the
 * enclosure [h + l - r, h + l + r]; pad != 0 makes it a value past the
 * product's last coefficient, which must contain 0.  path 0: the rung's
 * decision on the binary32 and integer pipes; path 1: the same set bounded
 * in binary64 and decided there.  paths 2, 3 (4, 5): the same two for a
 * transform of length 3 2^k (5 2^k), where the set encloses 3 c (5 c) and
 * the decision is on the set divided by 3 (5).  Outputs (device): d_class[i] = 0
 * isolated (d_value[i] = the integer), 1 not isolated, 2 empty (no
 * integer, a negative one, NaN, a centre beyond 2^53, or for pad rows a
 * set that excludes 0); d_value[i] = 0 otherwise.
 */
ssmul_status ssmul_debug_isolate(int path, const double* d_x, int64_t* d_value, int* d_class,
                                 size_t n);

/*
 * The exact scaled conversion the isolation uses: d_out[2 i] =
 * floor(d_x[i] 2^-d_k[i]), d_out[2 i + 1] = ceil(d_x[i] 2^-d_k[i]) for
 * 0 <= d_k[i] <= 1023 (device arrays, n entries); magnitudes of 2^62 or
 * more are capped at +-2^62, a NaN gives INT64_MIN for both.
 */
ssmul_status ssmul_debug_floor_ceil(const double* d_x, const int* d_k, int64_t* d_out, size_t n);

/* Kernel kinds counted by ssmul_debug_kernel_stats (index into its arrays):
 * kernel * 5 + rung for the four transform kernels (rungs: 0 F32 and 1 F64
 * rectangles, 2 DISC binary64 discs, 3 NAIVE points, 4 DISC32X2 discs),
 * then the carry, the finalisation, the balanced-digit prefix sums and the
 * ladder's lists of the products a later rung still runs. */
enum {
    SSMUL_K_SMALL = 0, SSMUL_K_FWD_COLS = 5, SSMUL_K_ROWS = 10, SSMUL_K_INV_COLS = 15,
    SSMUL_K_CARRY = 20, SSMUL_K_FINALIZE = 21, SSMUL_K_PREFIX = 22, SSMUL_K_GATE = 23,
    SSMUL_KERNEL_KINDS = 24
};

/*
 * Per-kind kernel statistics of the plan since the previous call: launch
 * counts always; device time in milliseconds (CUDA events recorded on the
 * plan's stream around each launch) while timing is enabled.  The call waits
 * for the recorded events, copies min(cap, SSMUL_KERNEL_KINDS) entries to
 * ms and launches (host arrays, either may be NULL), resets the
 * accumulators and then sets timing on (enable != 0) or off.
 */
ssmul_status ssmul_debug_kernel_stats(ssmul_plan_t plan, int enable, double* ms,
                                      unsigned long long* launches, int cap);

/*
 * Faults for tests of the failure paths, set on the host; nothing faults
 * or traps the device.  kind 0: clear all.  kind 1: the enclosures rung
 * `value` produces (0 binary32 rectangles, 1 binary64 rectangles, 2 binary64
 * discs, 3 points, 4 double-binary32 discs) are widened by 4 before isolation, so that rung cannot isolate
 * and the ladder must escalate (the sets still contain the exact values).
 * kind 2: carry tile `value` (4096 digits each) of every product never
 * publishes its look-back word, so later tiles give up after their bounded
 * wait (about a second) and the product reports SSMUL_TIMEOUT with its
 * digits zero-filled.  kind 3 (not a fault): value != 0 makes the
 * transforms read every twiddle from the octant tables instead of the
 * step-ordered copies, which must give the same bits.  Applies to the
 * plan's later calls.
 */
ssmul_status ssmul_debug_set_fault(ssmul_plan_t plan, int kind, long long value);

/*
 * The launch geometry the plan uses for transform length 2^log_n: the
 * four-step split (log2 N1, log2 N2) and log2 of the elements a column CTA
 * holds; for single-CTA lengths (N <= 4096) *log_n1 = 0 and the others are
 * log_n.  log_n = 32 + k (11 <= k <= 21) asks for the length 3 * 2^k and
 * log_n = 64 + k (10 <= k <= 19) for 5 * 2^k, split as N1 = R * 2^(*log_n1),
 * N2 = 2^(*log_n2) (R = 3 or 5).
 */
ssmul_status ssmul_debug_geometry(ssmul_plan_t plan, int log_n, int* log_n1, int* log_n2,
                                  int* log_cta);

/*
 * Throughput of one arithmetic operation on this device, in operations per
 * second / 1e9 (*gops): every thread of 8 CTAs per SM runs 16 independent
 * chains of the operation on run-time operands near 1 (the legacy default
 * stream, timed with CUDA events, best of 3 after a warm-up).  op: 0 binary64
 * add rounded down, 1 binary64 product rounded up, 2 binary64 fma rounded
 * down, 3 binary64 add written as an fma by a run-time 1, 4 binary64 add
 * rounded to nearest, 5 binary32 add rounded down, 6 binary32 fma rounded
 * down.  The ceilings the transforms' operation mixes run against; the paper
 * has no counterpart.
 */
ssmul_status ssmul_debug_pipe_rate(int op, double* gops);

#ifdef __cplusplus
}
#endif

#endif /* SSMUL_DEBUG_H */
