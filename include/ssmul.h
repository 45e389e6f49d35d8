/*
 * ssmul.h -- verified integer multiplication by complex interval FFT
 * convolution (a rigorous Schoenhage-Strassen multiplier) on one GPU.
 *
 * The method is that of T. Steinke and R. Sainudiin, "A Rigorous Extension
 * of the Schoenhage-Strassen Integer Multiplication Algorithm Using Complex
 * Interval Arithmetic" (CCA 2010):
 *   - Section 2 (digit convention): an operand is a little-endian vector
 *     of base-256 digits, x = sum_i x_i 256^i, digit 0 least significant;
 *   - Section 2.3 (fast convolution): the digit vectors are zero padded to
 *     a power-of-two length N >= na + nb - 1, transformed, multiplied
 *     pointwise and transformed back;
 *   - Section 2.5: every complex number is replaced by a rectangular complex
 *     interval whose bounds are rounded outward (directed rounding), so each
 *     output interval provably contains the exact coefficient of x * y;
 *   - Section 1: the unique integer in each containment set is taken; a set
 *     holding several integers is reported as an error (more precision is
 *     needed), never rounded;
 *   - Section 2.4: the integer coefficients are carried into base-256 digits.
 *
 * Every function returns an ssmul_status and never aborts or exits.
 * Device pointers are CUDA device addresses in the current device's memory;
 * host pointers are ordinary host memory.  The caller owns every buffer it
 * passes; a plan owns its workspace, twiddle tables and stream state.
 * A plan is bound to the device that was current when it was created and
 * is not thread-safe: one host thread at a time may use it.
 */
#ifndef SSMUL_H
#define SSMUL_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    SSMUL_OK = 0,
    /* some coefficient's containment set holds two or more integers at the
     * last precision tried (Section 1: more precision is needed) */
    SSMUL_ISOLATION_FAILED = 1,
    /* a containment set holds no integer, or is not finite: an internal
     * rigor violation, reported and never rounded away */
    SSMUL_CONTAINMENT_FAILED = 2,
    SSMUL_INVALID_ARG = 3,
    SSMUL_TOO_LARGE = 4,        /* sizes beyond the plan's maxima */
    SSMUL_CUDA_ERROR = 5,
    SSMUL_OUT_OF_MEMORY = 6,
    SSMUL_TIMEOUT = 7,          /* a bounded device-side wait gave up */
    /* SSMUL_PREC_NAIVE64 only: digits of the unverified round-to-nearest
     * transform, returned without any proof of correctness */
    SSMUL_UNVERIFIED = 8
} ssmul_status;

typedef enum {
    SSMUL_PREC_FP64 = 0,        /* binary64 inf-sup intervals only */
    SSMUL_PREC_FP32 = 1,        /* binary32 inf-sup intervals only */
    SSMUL_PREC_LADDER = 2,      /* binary32 first; products that do not
                                 * isolate are redone in binary64 */
    /* circular containment sets (the paper's Section 4 proposal): discs with
     * a binary64 centre and a binary32 radius, every rounding error bounded;
     * half the binary64 work of SSMUL_PREC_FP64 and no wrapping effect */
    SSMUL_PREC_DISC64 = 3,
    /* the naive transform of the paper's Section 3: round-to-nearest
     * binary64 without enclosures, a speed reference; status
     * SSMUL_UNVERIFIED */
    SSMUL_PREC_NAIVE64 = 4,
    /* binary32 rectangles (small products), then binary64 discs, then
     * binary64 rectangles for what is still unisolated */
    SSMUL_PREC_LADDER_DISC = 5,
    /* circular containment sets whose centres are pairs of binary32 numbers
     * (about 48 bits) with every rounding error bounded: the binary32 pipe
     * does all the work; wider sets than SSMUL_PREC_DISC64 */
    SSMUL_PREC_DISC32X2 = 6,
    /* binary32 rectangles (small products), then double-binary32 discs,
     * then binary64 discs, then binary64 rectangles */
    SSMUL_PREC_LADDER_FAST = 7
} ssmul_precision;

/* Per-product outcome. */
typedef struct {
    int32_t  status;            /* ssmul_status of this product */
    int32_t  precision_used;    /* ssmul_precision of the deciding rung:
                                 * SSMUL_PREC_FP32, _FP64, _DISC64,
                                 * _DISC32X2 or _NAIVE64 */
    uint32_t fft_log2;          /* the deciding rung's transform length
                                 * is N = fft_odd << fft_log2 (binary32 on
                                 * 4-bit digits: >= 2 (na + nb) - 1) */
    uint32_t n_unisolated;      /* coefficients whose set holds >= 2 integers */
    uint32_t n_empty;           /* coefficients whose set holds no integer */
    uint32_t fft_odd;           /* 1, 3 or 5 (SSMUL_OPT_LENGTHS) */
    double   max_width;         /* largest coefficient interval width
                                 * (rounded up), in units of 1; for
                                 * SSMUL_PREC_NAIVE64 the largest distance
                                 * to the nearest integer */
} ssmul_result;

/* One product of a batch: digits a_pool[a_off .. a_off+na), b_pool[b_off ..
 * b_off+nb), result digits z_pool[z_off .. z_off+na+nb). */
typedef struct {
    uint64_t a_off, b_off, z_off;
    uint32_t na, nb;
} ssmul_desc;

typedef struct ssmul_plan_s* ssmul_plan_t;

/*
 * Create a plan for products with na <= max_na and nb <= max_nb digits.
 * Allocates the device workspace for one product of the largest size, and
 * builds the twiddle enclosures omega_N^j = e^{2 pi i j / N} (the DFT root
 * of Section 2.2) on the device for N up to the largest transform length.
 * max_products bounds the count of one ssmul_mul_batched call (0: batches
 * are not used); for batches the plan also allocates an arena of transform
 * workspaces, at most 4 GiB (lowered by the environment variable
 * SSMUL_ARENA_MB), and a batch that does not fit runs in chunks.  prec selects the precision rule.  cuda_stream is a
 * cudaStream_t (NULL: the legacy default stream) on which all work of the
 * plan is ordered.
 * Errors: SSMUL_INVALID_ARG (null out, zero sizes, unknown precision),
 * SSMUL_TOO_LARGE (transform length above 2^23), SSMUL_OUT_OF_MEMORY,
 * SSMUL_CUDA_ERROR.  On error *out is set to NULL.
 */
ssmul_status ssmul_plan(ssmul_plan_t* out, size_t max_na, size_t max_nb,
                        size_t max_products, ssmul_precision prec,
                        void* cuda_stream);

/* Plan options (ssmul_plan_set_option).  None of them changes a product's
 * digits; they change how the work of Sections 2.3-2.5 is scheduled or
 * represented. */
typedef enum {
    /* value != 0: ssmul_mul_batched captures its launches in a CUDA graph and
     * replays the graph when the next call describes the same batch (same
     * descriptors, pools and result array); needs a plan stream other than
     * the legacy default stream, and is ignored on that stream.  A schedule
     * of the batch's transforms (Section 2.3); the paper has none. */
    SSMUL_OPT_GRAPH = 0,
    /* value != 0: time every candidate four-step geometry (split N = N1 N2,
     * column tile size) for each transform length of the plan now, and
     * keep the fastest; results are cached in the file named by the
     * environment variable SSMUL_TUNE_CACHE when it is set.  0: defaults.
     * The factorisation of the DFT of Section 2.2 changes, not its value. */
    SSMUL_OPT_AUTOTUNE = 1,
    /* under the ladders, try binary32 only for products with
     * na + nb <= value digits (and N <= 4096); 0: never.  Default 512 with
     * SSMUL_OPT_FP32_NIBBLES (binary32 rectangles isolated every uniform
     * square product up to 256 x 256 digits), 32 without it (16 x 16).  The
     * first rung of Section 1's "more precision on failure". */
    SSMUL_OPT_FP32_MAX_DIGITS = 2,
    /* value != 0: balanced digits.  The transforms carry a_j - 128 and
     * b_j - 128 instead of the digits, so their values (and the widths of
     * the containment sets) are much smaller; the isolated coefficients are
     * corrected exactly with integer window sums of the digits.  The
     * product is the same.  Default 0 (the paper's digits 0..255). */
    SSMUL_OPT_BALANCED = 3,
    /* value m >= 1024: the product calls cut a product whose longer
     * operand has more than m digits into parts of at most m digits per
     * operand, run each part's interval convolution (which isolates at
     * sizes the whole product would not), and add the parts' exact integer
     * coefficients before one carry: the way past the isolation limit that
     * Section 1 names ("use a different algorithm").  The status is the
     * worst of the parts'.  0 (default): off.  Batched calls split too:
     * their products past m digits run after the batch's other products,
     * one after another, each in its parts (such a batch is not captured in
     * a CUDA graph, and ssmul_mul_batched_host runs its pieces on one
     * stream).  A call whose products have more parts than any call before
     * grows the plan's part arrays first, after waiting for the plan's
     * queued work. */
    SSMUL_OPT_SPLIT_DIGITS = 4,
    /* bit mask of the transform length families besides 2^k: bit 0 the
     * lengths 3 * 2^k, bit 1 the lengths 5 * 2^k (default 3: both).  A
     * product takes the shortest allowed length N >= na + nb - 1 (the zero
     * padding of Section 2.3; odd lengths only above 4096): 5 * 2^(k-3) =
     * 0.625 * 2^k or 3 * 2^(k-2) = 0.75 * 2^k instead of the next power of
     * two 2^k.  The column transforms then end with one radix-5 or radix-3
     * step, the roots of unity come from a table of Ntab = 5 * 2^K or
     * 3 * 2^K, and the 1/N scaling leaves a factor 1/5 or 1/3 that the
     * isolation applies exactly to the integer bounds.  0: powers of two
     * only (the paper's 2^k). */
    SSMUL_OPT_LENGTHS = 5,
    /* value 1 .. 64: ssmul_mul_batched_host runs its batch in this many
     * pieces (consecutive runs of the descriptors) on internal streams of
     * decreasing priority, so that later pieces' operands upload and
     * earlier pieces' digits download while a piece computes, and a later
     * piece's thread blocks fill an earlier one's last waves.  1: one
     * upload, the whole batch, one download.  Default 4.
     * Data movement only: the paper's method starts from digit vectors
     * (Section 2) and ends with the digits of the carry (Section 2.4). */
    SSMUL_OPT_HOST_PIECES = 6,
    /* value 1 .. 4: ssmul_mul_batched spreads the transform-length groups of
     * a batch (each a set of independent products, Section 2.3) over this
     * many streams, the plan's own and internal ones, so that one group's
     * partly filled last wave of thread blocks overlaps another group's
     * work; they join the plan's stream before the outcomes are written.
     * Default 4; 1 puts every launch on the plan's stream. */
    SSMUL_OPT_LANES = 7,
    /* value != 0: the binary32 rung transforms the operands' 4-bit digits
     * (a = sum_j a'_j 16^j, a'_j in 0..15) for products with na + nb <= 2048:
     * coefficients at most 225 min(2 na, 2 nb) instead of 65025 min(na, nb),
     * so narrower containment sets for twice the transform length.  The
     * isolated base-16 coefficients c'_i become the base-256 coefficients
     * c'_{2k} + 16 c'_{2k+1} exactly before the carry (the product identity
     * of Section 2.1 in base 16).  The transform carries the centred 4-bit
     * digits a'_j - ma and b'_j - mb, ma and mb the rounded means of each
     * operand's 4-bit digits (whatever SSMUL_OPT_BALANCED says, which is
     * about the bytes of the other rungs); the isolated coefficients are
     * corrected exactly with integer window sums of the 4-bit digits.
     * Default 1; 0: the binary32 rung transforms the bytes like the other
     * rungs. */
    SSMUL_OPT_FP32_NIBBLES = 8
} ssmul_option;

/*
 * Set a plan option (ssmul_option: how the work of Sections 2.3-2.5 is
 * scheduled and represented; the products are the same).  Waits for the
 * plan's queued work first.
 * Errors: SSMUL_INVALID_ARG (null plan, unknown option, negative value),
 * SSMUL_OUT_OF_MEMORY / SSMUL_CUDA_ERROR from the autotuner.
 */
ssmul_status ssmul_plan_set_option(ssmul_plan_t plan, ssmul_option option, long long value);

/*
 * z = a * b for one product (Sections 2.3-2.5 and the carry of Section 2.4).
 * d_a: na digits, d_b: nb digits, d_z: na+nb digits, all device memory,
 * little-endian base 256 (leading zero digits are allowed).  The work is
 * ordered on the plan's stream and the call waits for it: the return value
 * is the product's status, and *h_res (host memory, may be NULL) receives
 * the per-product outcome.  When the status is not SSMUL_OK, d_z is
 * zero-filled: no unverified digit is ever returned.
 * Errors: SSMUL_INVALID_ARG (null pointers, na or nb zero), SSMUL_TOO_LARGE
 * (na > max_na or nb > max_nb), SSMUL_CUDA_ERROR, and the product statuses.
 */
ssmul_status ssmul_mul(ssmul_plan_t plan, const uint8_t* d_a, size_t na,
                       const uint8_t* d_b, size_t nb, uint8_t* d_z,
                       ssmul_result* h_res);

/*
 * Same as ssmul_mul (Sections 2.3-2.5 and the carry of Section 2.4), with
 * a, b and z in host memory.  The host-device copies go through the plan's
 * device buffers on the plan's stream.  Errors: as ssmul_mul.
 */
ssmul_status ssmul_mul_host(ssmul_plan_t plan, const uint8_t* h_a, size_t na,
                            const uint8_t* h_b, size_t nb, uint8_t* h_z,
                            ssmul_result* h_res);

/*
 * count independent products z = a * b, each computed as ssmul_mul computes
 * one (the fast convolution of Section 2.3 in the interval arithmetic of
 * Section 2.5, the isolation of Section 1 and the carry of Section 2.4),
 * described by h_desc (host memory, count entries) over device digit
 * pools: a_pool[a_off .. a_off + na), b_pool[b_off .. b_off + nb) and
 * z_pool[z_off .. z_off + na + nb), little-endian base 256.  Every product
 * obeys the plan's size maxima and count <= max_products; the z ranges of
 * different products must not overlap.  The work is only enqueued on the
 * plan's stream: the return value covers argument and launch errors, and
 * the per-product outcomes land in d_res (device memory, count entries),
 * valid after the stream is synchronised.  Products whose status is not
 * SSMUL_OK have their digits zero-filled.  h_desc may be reused as soon as
 * the call returns.
 * Errors: SSMUL_INVALID_ARG (null plan or pointers with count > 0, na or nb
 * zero), SSMUL_TOO_LARGE (count > max_products, a size above the plan's
 * maxima), SSMUL_OUT_OF_MEMORY, SSMUL_CUDA_ERROR.
 */
ssmul_status ssmul_mul_batched(ssmul_plan_t plan, size_t count,
                               const ssmul_desc* h_desc,
                               const uint8_t* d_a_pool, const uint8_t* d_b_pool,
                               uint8_t* d_z_pool, ssmul_result* d_res);

/*
 * ssmul_mul_batched from host memory to host memory: the digit vectors in
 * (Section 2's digit convention), the digits of Section 2.4's carry out.
 * h_desc offsets index the host pools h_a_pool, h_b_pool and h_z_pool;
 * h_res (host memory, count entries) receives the per-product outcomes.
 * The plan copies the bytes its products read to device buffers of its
 * own, runs the batch and copies the products' digits (exactly the bytes
 * [z_off, z_off + na + nb) of each product; nothing else of h_z_pool is
 * written) and outcomes back.  The batch runs in SSMUL_OPT_HOST_PIECES
 * pieces so that copies overlap the computation.  The call waits: on return
 * h_z_pool and h_res hold the results, and the return value covers argument,
 * memory and launch errors (each product's status is in h_res; digits of a
 * product whose status is not SSMUL_OK are zero-filled).
 * Page-locked host memory (cudaMallocHost, cudaHostAlloc, cudaHostRegister)
 * lets every copy run asynchronously; pageable memory works too, but its
 * copies go through driver staging and hold the calling thread.
 * Device memory: the plan's copies of the pools grow, on the first call that
 * needs more, to the span of the bytes a call touches in each pool (a
 * cudaMalloc after waiting for the plan's queued work).  SSMUL_OPT_GRAPH
 * does not apply to this call.
 * Errors: as ssmul_mul_batched, and SSMUL_INVALID_ARG for a null h_res.
 */
ssmul_status ssmul_mul_batched_host(ssmul_plan_t plan, size_t count,
                                    const ssmul_desc* h_desc,
                                    const uint8_t* h_a_pool, const uint8_t* h_b_pool,
                                    uint8_t* h_z_pool, ssmul_result* h_res);

/*
 * z = a * b without any device allocation, for callers that cannot call
 * cudaMalloc: for example a process whose device memory is already fully
 * reserved by another allocator (a framework's caching pool), or a
 * latency-bound caller that cannot accept the implicit device
 * synchronisation an allocation may cause.  The paper has no counterpart;
 * this is a property of the library, not of the method.
 *
 * Products with na + nb <= SSMUL_NOALLOC_MAX_DIGITS run the binary64 path
 * of ssmul_mul with identical results; larger ones return SSMUL_TOO_LARGE.
 * All scratch memory (twiddle table, descriptor, accumulators, integer
 * coefficients, carry words, outcome: about 60 KB) is one static device
 * array of the library, held on every device that loads it until the
 * process exits.  The first call on a device sets that array up (finds its
 * address, builds the twiddle table, marks it built and waits for it); make
 * that first call before any stream capture.  Every call looks the array's
 * address up again and its first kernel checks the mark, so after a device
 * reset (which re-creates the array, zero-filled) the next call sets it up
 * again instead of transforming with a missing table.  Every call on a
 * device shares the one array, so calls that may overlap on the GPU race
 * and must be serialised by the caller (for example: one stream).  d_a, d_b, d_z: device memory
 * of the current device; h_res: host memory, may be NULL; cuda_stream: a
 * cudaStream_t (NULL: legacy default stream).  The call waits for the
 * product and returns its status; d_z is zero-filled unless SSMUL_OK.
 */
#define SSMUL_NOALLOC_MAX_DIGITS 4097
ssmul_status ssmul_mul_noalloc(const uint8_t* d_a, size_t na, const uint8_t* d_b, size_t nb,
                               uint8_t* d_z, ssmul_result* h_res, void* cuda_stream);

/* Release everything the plan owns.  NULL is allowed. */
void ssmul_plan_destroy(ssmul_plan_t plan);

/* A static string naming the status. */
const char* ssmul_status_string(ssmul_status s);

#ifdef __cplusplus
}
#endif

#endif /* SSMUL_H */
