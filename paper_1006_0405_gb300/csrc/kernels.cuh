// kernels.cuh -- the interval convolution pipeline and the carry scan.
//
// One product z = a * b (Section 2.4) runs as:
//
//   pack      z_j = a_j + i b_j as point intervals, zero padded to N
//             (N = 2^k >= na + nb - 1, Section 2.3).  Both operands are
//             real, so one complex transform carries both.
//   forward   Z = DFT_N(z) (Section 2.2), interval arithmetic (Section 2.5).
//   split +   A_k = (Z_k + conj Z_{N-k}) / 2, B_k = (Z_k - conj Z_{N-k}) / 2i
//   pointwise are the transforms of a and b, and C_k = A_k B_k is the
//             transform of the convolution (the convolution theorem,
//             Section 2.3).  C_{N-k} = conj C_k because c is real.
//   pack      D_k = (C_k + C_{k+N/2}) + i omega_N^{-k} (C_k - C_{k+N/2}),
//             k < N/2: the length-N/2 inverse of D is c_{2j} + i c_{2j+1}.
//   inverse   d = IDFT_{N/2}(D) scaled by 1/N (exact power of two).
//   isolate   each of c_{2j} = Re d_j and c_{2j+1} = Im d_j must hold exactly
//             one integer (Section 1); coefficients past na + nb - 2 must
//             contain 0.
//   carry     the integer coefficients become na + nb base-256 digits.
//
// For N <= 4096 one CTA does everything up to the isolation in shared
// memory (k_small).  Larger N use the four-step factorisation N = N1 * N2,
// with the spectrum kept in "transposed" order (index k1 + N1 k2 stored at
// row k1, column k2) so no reordering pass is needed:
//   k_fwd_cols  column DFTs of length N1 and the twiddles omega_N^{j2 k1}
//   k_rows      row DFTs of length N2 for the row pair (k1, N1 - k1), the
//               split / pointwise / pack steps, the inverse row DFTs of
//               length N2/2 and the twiddles omega_{N/2}^{-j2 k1}
//   k_inv_cols  inverse column DFTs of length N1, scaling and isolation
#pragma once
#include <cuda_runtime.h>
#include <climits>
#include <type_traits>
#include "../../include/ssmul.h"
#include "value.cuh"
#include "fft.cuh"

namespace ssm {

constexpr int LOG_SMALL = 12;          // k_small handles N <= 2^12
constexpr int LOG_N2_MAX = 11;         // four-step row length limit
constexpr int LOG_N1_MAX = 12;         // four-step column length limit
constexpr int LOG_N_MAX = LOG_N1_MAX + LOG_N2_MAX;   // 2^23
constexpr int LOG_CTA_ELEMS = 11;      // column kernels hold >= 2^11 elements
constexpr int CARRY_TILE = 4096;       // digits per carry CTA
constexpr int CARRY_THREADS = 256;
constexpr int CARRY_PER_THREAD = CARRY_TILE / CARRY_THREADS;
constexpr uint32_t SPIN_LIMIT = 1u << 20;   // bounded look-back polls (about a second)
// Transform length codes: c < LEN3 means N = 2^c; LEN3 <= c < LEN5 means
// N = 3 2^(c - LEN3); c >= LEN5 means N = 5 2^(c - LEN5).  The odd lengths
// are four-step only: columns R 2^a with a even and R 2^a <= 4096, rows 2^b
// with 2 <= b <= 11.
constexpr int LEN3 = 32;
constexpr int LEN5 = 64;
constexpr int LOG3_MIN = 11;           // 6144 = 3 2^11 > 4096, the single-CTA limit
constexpr int LOG3_MAX = 21;           // 3 2^10 columns x 2^11 rows
constexpr int LOG5_MIN = 10;           // 5120 = 5 2^10
constexpr int LOG5_MAX = 19;           // 5 2^8 columns x 2^11 rows

// Per-product accumulators of one call, zeroed before the call; one entry
// per rung (value.cuh: 0 binary32 rectangles, 1 binary64 rectangles,
// 2 binary64 discs, 3 unverified points, 4 double-binary32 discs).
struct ProdState {
    unsigned int ran[RUNGS];
    unsigned int unisolated[RUNGS];
    unsigned int empty[RUNGS];
    unsigned int timeout;
    unsigned int carry_ticket;
    unsigned long long maxw[RUNGS];    // bit pattern of a nonnegative double
    unsigned int forced;               // split products: worst status of a part
    unsigned int pad;
};

struct ProdDesc {
    const uint8_t* a;
    const uint8_t* b;
    uint8_t* z;
    uint32_t na, nb;
    int32_t log_n;                     // length code (see LEN3)
    int32_t balanced;                  // digits enter the transform as x_j - 128
    void* Z;                           // four-step workspace, N intervals
    void* W;                           // four-step workspace, N/2 intervals
    int64_t* coeff;                    // N integer coefficients
    uint32_t* flags;                   // carry look-back words, one per tile
    ProdState* st;
    ssmul_result* res;
    double* iv;                        // optional: coefficient enclosures (tests)
    uint32_t* pre_a;                   // balanced: prefix sums of a (see k_prefix)
    uint32_t* pre_b;                   // balanced: prefix sums of b
    // test faults set on the host (0: off): rung + 1 whose enclosures are
    // widened by 4 so it cannot isolate; carry tile + 1 that never publishes
    int32_t fault_widen;
    int32_t fault_stall;
    // the binary32 rung transforms the operands' 4-bit digits (see
    // isolate_nib_value); set only when na + nb <= NIB_MAX_DIGITS
    int32_t fp32_nib;
    // coeff holds na + nb coefficients whatever rung decides (products
    // assembled from split parts); the carry then reads index na + nb - 1 too
    int32_t coef_nz;
};

// ---- balanced digits --------------------------------------------------------
//
// With balanced digits a'_j = a_j - 128, b'_j = b_j - 128 (zero past the
// operands) the transforms carry far smaller values.  The product is
// unchanged: with u the all-ones vectors,
//   a * b = a' * b' + 128 (u_a * b + a * u_b) - 16384 u_a * u_b,
// so c_i = c'_i + 128 (Wa_i + Wb_i) - 16384 cnt_i, where Wa_i and Wb_i are
// the sums of the digits of a and b that meet in coefficient i and cnt_i
// the number of such pairs.  The window sums come from prefix sums of the
// digits: for tile size PRE_TILE, local[k] (k = 1 .. n) is the sum of the
// digits from the start of the tile of digit k-1 up to digit k-1, and
// off[t] the sum of all digits before tile t.

constexpr int PRE_LOG_TILE = 11;
constexpr int PRE_TILE = 1 << PRE_LOG_TILE;
constexpr int PRE_THREADS = 256;

__device__ __forceinline__ uint32_t prefix_at(const uint32_t* pre, uint32_t n, uint32_t k) {
    if (k == 0) return 0u;
    return pre[n + 1 + ((k - 1) >> PRE_LOG_TILE)] + pre[k];
}

// the exact term that turns c'_i into c_i
__device__ __forceinline__ int64_t balance_corr(const ProdDesc& d, int64_t i) {
    const int64_t na = d.na, nb = d.nb;
    const int64_t ja_lo = i - nb + 1 > 0 ? i - nb + 1 : 0, ja_hi = i < na - 1 ? i : na - 1;
    const int64_t jb_lo = i - na + 1 > 0 ? i - na + 1 : 0, jb_hi = i < nb - 1 ? i : nb - 1;
    const int64_t wa = int64_t(prefix_at(d.pre_a, d.na, uint32_t(ja_hi + 1))) -
                       int64_t(prefix_at(d.pre_a, d.na, uint32_t(ja_lo)));
    const int64_t wb = int64_t(prefix_at(d.pre_b, d.nb, uint32_t(jb_hi + 1))) -
                       int64_t(prefix_at(d.pre_b, d.nb, uint32_t(jb_lo)));
    return 128 * (wa + wb) - 16384 * (ja_hi - ja_lo + 1);
}

// tile-local inclusive sums and tile totals; blockIdx.z: 0 for a, 1 for b
__global__ void __launch_bounds__(PRE_THREADS) k_prefix(const ProdDesc* descs) {
    __shared__ uint32_t s_warp[PRE_THREADS / 32];
    const ProdDesc d = descs[blockIdx.y];
    if (!d.balanced) return;
    const bool isb = blockIdx.z != 0;
    const uint32_t n = isb ? d.nb : d.na;
    const uint8_t* x = isb ? d.b : d.a;
    uint32_t* pre = isb ? d.pre_b : d.pre_a;
    const uint32_t base = blockIdx.x << PRE_LOG_TILE;
    if (base >= n) return;
    constexpr int PER = PRE_TILE / PRE_THREADS;
    const uint32_t k0 = base + threadIdx.x * PER;
    uint32_t v[PER];
    uint32_t sum = 0;
#pragma unroll
    for (int q = 0; q < PER; ++q) {
        v[q] = (k0 + q < n) ? uint32_t(x[k0 + q]) : 0u;
        sum += v[q];
    }
    // exclusive scan of the per-thread sums
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t inc = sum;
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t t = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += t;
    }
    if (lane == 31) s_warp[warp] = inc;
    __syncthreads();
    uint32_t wbase = 0;
    for (int w = 0; w < warp; ++w) wbase += s_warp[w];
    uint32_t run = wbase + inc - sum;
#pragma unroll
    for (int q = 0; q < PER; ++q) {
        run += v[q];
        if (k0 + q < n) pre[k0 + q + 1] = run;
    }
    if (threadIdx.x == PRE_THREADS - 1) pre[n + 1 + blockIdx.x] = run;   // tile total
    if (blockIdx.x == 0 && threadIdx.x == 0) pre[0] = 0u;
}

// exclusive scan of the tile totals, in place; blockIdx.y: 0 for a, 1 for b
__global__ void k_prefix_tiles(const ProdDesc* descs) {
    const ProdDesc d = descs[blockIdx.x];
    if (!d.balanced || threadIdx.x != 0) return;
    const bool isb = blockIdx.y != 0;
    const uint32_t n = isb ? d.nb : d.na;
    uint32_t* off = (isb ? d.pre_b : d.pre_a) + n + 1;
    const uint32_t tiles = (n + PRE_TILE - 1) >> PRE_LOG_TILE;
    uint32_t acc = 0;
    for (uint32_t t = 0; t < tiles; ++t) {
        const uint32_t tot = off[t];
        off[t] = acc;
        acc += tot;
    }
}

// ---- the rung gate of the precision ladder ------------------------------------

// true when a rung in `mask` (bit r: rung r) already decided this product:
// it ran and either isolated every coefficient or found an empty set
__device__ __forceinline__ bool decided_by(const ProdState* st, int mask) {
    // every field read up front and combined without branches, so the loads
    // go out together (short-circuit tests through the pointer would chain
    // them, and a launch whose products are all decided pays that chain in
    // every one of its CTAs)
    unsigned int ran[RUNGS], uni[RUNGS], emp[RUNGS];
#pragma unroll
    for (int r = 0; r < RUNGS; ++r) {
        ran[r] = st->ran[r];
        uni[r] = st->unisolated[r];
        emp[r] = st->empty[r];
    }
    bool dec = false;
#pragma unroll
    for (int r = 0; r < RUNGS; ++r)
        dec |= (((mask >> r) & 1) != 0) & (ran[r] != 0u) & ((uni[r] == 0u) | (emp[r] != 0u));
    return dec;
}

// The products of a batch that a later rung of the ladder still has to run:
// list[0] = n, list[1 .. n] their indices into descs (any order).  CTA row
// y of the rung's kernels runs product list[1 + y]; rows y >= n end after
// reading list[0], one load that every CTA shares, where a test of the
// product's own state would take two dependent loads.  One CTA.
__global__ void k_gate_list(const ProdDesc* descs, int count, int mask, int* list) {
    __shared__ int s_n;
    if (threadIdx.x == 0) s_n = 0;
    __syncthreads();
    for (int i = threadIdx.x; i < count; i += blockDim.x)
        if (!decided_by(descs[i].st, mask)) list[1 + atomicAdd(&s_n, 1)] = i;
    __syncthreads();
    if (threadIdx.x == 0) list[0] = s_n;
}

// kernel template argument -> value type: float and double name the inf-sup
// rectangles, Disc and Pt themselves
template <typename W> struct ValOf { using type = W; };
template <> struct ValOf<float> { using type = CI<float>; };
template <> struct ValOf<double> { using type = CI<double>; };

// ---- shared-memory stages common to k_small and k_rows -----------------------

// Pointwise product on the pairs (k, N - k).  Line l of `sm` holds the
// forward transform of row rows[l]; the partner of (row r, column k2) is
// row (N1 - r) mod N1, column (N2 - k2) mod N2 for r = 0 and N2 - 1 - k2
// otherwise.  With two lines the rows are partners of each other; with
// one line the row is its own partner.
template <typename V>
__device__ void pair_products(SBuf<V> sm, int nl, int row0, int logN2) {
    const int N2 = 1 << logN2;
    for (int k2 = threadIdx.x; k2 < N2; k2 += blockDim.x) {
        const int pc = (row0 == 0) ? ((N2 - k2) & (N2 - 1)) : (N2 - 1 - k2);
        if (nl == 1 && k2 > pc) continue;
        const int pi = (nl == 2 ? N2 : 0) + pc;
        const V zk = sm[k2];
        const V czp = conj(sm[pi]);
        const V a2 = zk + czp;                     // 2 A_k
        const V b2 = mul_negi_flip(zk - czp);      // 2 B_k
        const V c4 = mul_ci(a2, b2);               // 4 C_k
        sm[k2] = c4;
        if (pi != k2) sm[pi] = conj_flip(c4);      // 4 C_{N-k}
    }
}

// D_k for k2 < N2/2 of each line, written over the first half of the line
// (N1 = R 2^logN1, N = N1 N2; the twiddle table is of family R).
template <typename V, int R = 1>
__device__ void pack_half(SBuf<V> sm, int nl, int row0, int row1, int logN1, int logN2,
                          const TwTable& tw) {
    const int N2 = 1 << logN2, M2 = N2 >> 1;
    const uint32_t N1 = uint32_t(R) << logN1;
    const int logN = logN1 + logN2;
    for (int t = threadIdx.x; t < nl * M2; t += blockDim.x) {
        const int l = t >> (logN2 - 1), k2 = t & (M2 - 1);
        const int x = l * N2 + k2;
        const V c0 = sm[x], c1 = sm[x + M2];
        const uint32_t k = uint32_t(l ? row1 : row0) + uint32_t(k2) * N1;
        const auto w = get_twiddle<V, -1, R>(tw, k << (tw.log_n - logN));
        sm[x] = (c0 + c1) + mul_i(mul_tw(c0 - c1, w));
    }
}

// pair_products and pack_half of a row pair (two lines, rows row0 != 0 and
// row1 = N1 - row0) in one pass.  For k < N2/2 the elements line 0 at k and
// k + M2 and line 1 at M2 - 1 - k and N2 - 1 - k hold both partners of two
// pair products (k with N2 - 1 - k, k + M2 with M2 - 1 - k) and both inputs
// of the packed outputs line 0 at k and line 1 at M2 - 1 - k, so one thread
// computes them with the same operations as the two passes and writes only
// elements it read: no barrier between the steps.  R2: the forward
// transform left its final radix-2 step (odd log2 N2), whose butterflies for
// line 0 at k and line 1 at M2 - 1 - k produce exactly those four elements;
// the thread does them first, from the step's inputs at the same places.
template <typename V, int R = 1, bool R2 = false>
__device__ void pair_pack2(SBuf<V> sm, int row0, int row1, int logN1, int logN2,
                           const TwTable& tw) {
    const int N2 = 1 << logN2, M2 = N2 >> 1;
    const uint32_t N1 = uint32_t(R) << logN1;
    const int logN = logN1 + logN2;
    const auto prod = [](const V& zk, const V& zp) {       // 4 C_k from Z_k and its partner
        const V czp = conj(zp);
        const V a2 = zk + czp;                     // 2 A_k
        const V b2 = mul_negi_flip(zk - czp);      // 2 B_k
        return mul_ci(a2, b2);                     // 4 C_k
    };
    const auto pack = [&](const V& c0, const V& c1, int row, int k2) {
        const uint32_t k = uint32_t(row) + uint32_t(k2) * N1;
        const auto w = get_twiddle<V, -1, R>(tw, k << (tw.log_n - logN));
        return (c0 + c1) + mul_i(mul_tw(c0 - c1, w));
    };
    for (int k2 = threadIdx.x; k2 < M2; k2 += blockDim.x) {
        const int kb = M2 - 1 - k2;
        V z0lo, z0hi, z1lo, z1hi;       // line 0 at k2, k2 + M2; line 1 at kb, kb + M2
        if constexpr (R2) {
            const V a0 = sm[k2], b0 = sm[k2 + M2], a1 = sm[N2 + kb], b1 = sm[N2 + kb + M2];
            z0lo = a0 + b0;
            z0hi = a0 - b0;
            z1lo = a1 + b1;
            z1hi = a1 - b1;
        } else {
            z0lo = sm[k2];
            z0hi = sm[k2 + M2];
            z1lo = sm[N2 + kb];
            z1hi = sm[N2 + kb + M2];
        }
        const V c_lo = prod(z0lo, z1hi);        // line 0 at k2 (partner N2 - 1 - k2)
        const V c_hi = prod(z0hi, z1lo);        // line 0 at k2 + M2 (partner kb)
        // line 1 at kb and kb + M2 = N2 - 1 - k2: the conjugate-flipped partners
        sm[k2] = pack(c_lo, c_hi, row0, k2);
        sm[N2 + kb] = pack(conj_flip(c_hi), conj_flip(c_lo), row1, kb);
    }
}

// ---- isolation (Section 1) --------------------------------------------------

struct IsoAcc {
    unsigned int unisolated = 0, empty = 0;
    unsigned long long maxw_bits = 0;   // bit pattern of the largest width (>= 0)
    unsigned int maxw_f32 = 0;          // the same for widths held in binary32
    int wscale = 0;                     // maxw_bits is of sets 2^wscale times the coefficients'
};

// floor(x 2^-k) and ceil(x 2^-k) for a binary64 x and 0 <= k <= 1023, exact,
// on the integer pipe (the scaling by the transform length folded into the
// conversion, so neither takes a binary64 operation).  Results of magnitude
// 2^62 or more are capped at +-2^62 (past every value the isolation
// accepts); a NaN gives INT64_MIN for both.
__device__ __forceinline__ void floor_ceil_scaled(double x, int k, long long& fl, long long& ce) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const bool neg = (b >> 63) != 0;
    const int e = int((b >> 52) & 0x7FF);
    unsigned long long m = b & 0xFFFFFFFFFFFFFull;
    if (e == 0x7FF) {
        fl = ce = m ? LLONG_MIN : (neg ? -(1ll << 62) : (1ll << 62));
        return;
    }
    if (e) m |= 1ull << 52;
    const int sh = (e ? e : 1) - 1075 - k;       // |x| 2^-k = m 2^sh
    unsigned long long q;
    bool frac;
    if (sh >= 0) {
        q = sh > 9 ? (1ull << 62) : (m << sh);     // m < 2^53
        frac = false;
    } else if (sh > -64) {
        q = m >> -sh;
        frac = (m & ((1ull << -sh) - 1ull)) != 0ull;
    } else {
        q = 0;
        frac = m != 0ull;
    }
    const long long qi = (long long)q, f = frac ? 1 : 0;
    fl = neg ? -qi - f : qi;
    ce = neg ? -qi : qi + f;
}

// 2^k for 0 <= k <= 1023
__device__ __forceinline__ double pow2_pos(int k) {
    return __longlong_as_double((long long)(1023 + k) << 52);
}

// Integer division by R rounded up / down (exact, no overflow).
template <int R>
__device__ __forceinline__ long long ceil_div(long long x) { return x / R + (x % R > 0 ? 1 : 0); }
template <int R>
__device__ __forceinline__ long long floor_div(long long x) { return x / R - (x % R < 0 ? 1 : 0); }
template <int R>
__device__ __forceinline__ int floor_div32(int x) { return x / R - (x % R < 0 ? 1 : 0); }

// RU(1/R) for R = 1, 3, 5 (bit patterns: 1, the successor of RN(1/3), RN(1/5) > 1/5)
template <int R>
__device__ __forceinline__ double inv_up() {
    return R == 1 ? 1.0 : __longlong_as_double(R == 3 ? 0x3FD5555555555556ll : 0x3FC999999999999All);
}

// Decide coefficient idx from the enclosure [lo, hi] of c_idx (of c'_idx
// with balanced digits, corrected here to c_idx); L = na + nb - 1.  The
// decision is integer arithmetic on kl = ceil(lo) and kh = floor(hi),
// obtained by conversions to int64 that round up / round down and saturate:
// one integer lies in [lo, hi] iff kl == kh.  A NaN converts to the most
// negative value, and |k| >= 2^53 (an overflowed or infinite bound) is
// never accepted.  The exact coefficient is a nonnegative integer: an
// isolated negative value is a containment failure like an empty set.
//
// R = 3 or 5 (transform length R 2^k): [lo, hi] encloses R c_idx (the 1/N
// scaling applied only its power of two).  The integers of [lo/R, hi/R] are
// those of [ceil(kl'/R), floor(kh'/R)] with kl' = ceil(lo), kh' = floor(hi),
// so the same decision takes two exact integer divisions and no rounding.
//
// [lo, hi] 2^-k is the set (k: the power of two of the 1/N scaling, applied
// here exactly by floor_ceil_scaled; the widths are scaled at flush_acc).
template <int R = 1, typename T>
__device__ __forceinline__ void isolate_one(T lo, T hi, int k, int64_t idx, const ProdDesc& d,
                                            IsoAcc& acc, int rung) {
    const int64_t L = int64_t(d.na) + d.nb - 1;
    double dl = double(lo), dh = double(hi);          // exact widening
    if (d.fault_widen == rung + 1) {                  // test fault: still an enclosure
        const double f = 4.0 * R * pow2_pos(k);       // 4 in units of c (the set is of R c)
        dl = __dsub_rd(dl, f);
        dh = __dadd_ru(dh, f);
    }
    const unsigned long long wb = (unsigned long long)__double_as_longlong(__dsub_ru(dh, dl));
    acc.maxw_bits = wb > acc.maxw_bits ? wb : acc.maxw_bits;   // widths are >= 0 (or NaN)
    acc.wscale = k;
    long long kl, kh, unused;
    floor_ceil_scaled(dl, k, unused, kl);
    floor_ceil_scaled(dh, k, kh, unused);
    if (R != 1) {
        // [ceil(kl / R), floor(kh / R)]; a narrow set of moderate bounds (the
        // usual case) takes one 64-bit division: kl = q R + rm (0 <= rm < R),
        // kh = kl + span.  Capped, NaN or wide bounds take two.
        const bool narrow = kl > -(1ll << 61) && kl < (1ll << 61) && kh >= kl &&
                            kh - kl < (1ll << 30);
        const long long span = narrow ? kh - kl : 0;
        if (narrow) {
            const long long q = floor_div<R>(kl);
            const int rm = int(kl - q * R);
            kh = q + floor_div32<R>(rm + int(span));
            kl = q + (rm > 0 ? 1 : 0);
        } else {
            kl = ceil_div<R>(kl);
            kh = floor_div<R>(kh);
        }
    }
    constexpr long long KMAX = 1ll << 53;
    if (idx < L) {
        const int64_t corr = d.balanced ? balance_corr(d, idx) : 0;
        if (d.iv != nullptr) {
            const double sl = __dmul_rd(dl, pow2_neg(k)), sh = __dmul_ru(dh, pow2_neg(k));
            d.iv[2 * idx] = __dadd_rd(R != 1 ? __ddiv_rd(sl, double(R)) : sl, double(corr));
            d.iv[2 * idx + 1] = __dadd_ru(R != 1 ? __ddiv_ru(sh, double(R)) : sh, double(corr));
        }
        int64_t v = 0;
        if (kl == kh && kl > -KMAX && kl < KMAX && kl + corr >= 0) {
            v = kl + corr;
        } else if (kl < kh) {
            acc.unisolated++;
        } else {
            acc.empty++;           // no integer, a negative one, NaN or overflow
        }
        d.coeff[idx] = v;
    } else {
        if (!(kl <= 0 && kh >= 0)) acc.empty++;      // the exact value is 0
    }
}

// R = 3, 5: the widths were those of R c; the largest is scaled by RU(1/R)
template <int R = 1>
__device__ __forceinline__ void flush_acc(IsoAcc acc, ProdState* st, int rung) {
    if (acc.wscale && acc.maxw_bits)
        acc.maxw_bits = (unsigned long long)__double_as_longlong(
            __dmul_ru(__longlong_as_double((long long)acc.maxw_bits), pow2_neg(acc.wscale)));
    if (acc.maxw_f32) {
        // binary32 -> binary64 is exact and keeps the order (NaN stays the largest)
        const unsigned long long w =
            (unsigned long long)__double_as_longlong(double(__uint_as_float(acc.maxw_f32)));
        acc.maxw_bits = w > acc.maxw_bits ? w : acc.maxw_bits;
    }
    if (R != 1 && acc.maxw_bits)
        acc.maxw_bits = (unsigned long long)__double_as_longlong(
            __dmul_ru(__longlong_as_double((long long)acc.maxw_bits), inv_up<R>()));
    for (int o = 16; o > 0; o >>= 1) {
        acc.unisolated += __shfl_xor_sync(0xffffffffu, acc.unisolated, o);
        acc.empty += __shfl_xor_sync(0xffffffffu, acc.empty, o);
        const unsigned long long w = __shfl_xor_sync(0xffffffffu, acc.maxw_bits, o);
        acc.maxw_bits = w > acc.maxw_bits ? w : acc.maxw_bits;
    }
    if ((threadIdx.x & 31) == 0) {
        if (acc.unisolated) atomicAdd(&st->unisolated[rung], acc.unisolated);
        if (acc.empty) atomicAdd(&st->empty[rung], acc.empty);
        atomicMax(&st->maxw[rung], acc.maxw_bits);
    }
}

// Both coefficients carried by one complex value: c_{2j} (real part) and
// c_{2j+1} (imaginary part).
// v 2^-k (k: the 1/N scaling's power of two) for the binary64 and binary32
// rectangles and the binary64 discs, whose bounds are scaled exactly inside
// the integer conversion
template <int R = 1, typename T>
__device__ __forceinline__ void isolate_value(const CI<T>& v, int k, int64_t j, const ProdDesc& d,
                                              IsoAcc& acc) {
    constexpr int RUNG = VTraits<CI<T>>::rung;
    isolate_one<R>(v.rl, v.rh, k, 2 * j, d, acc, RUNG);
    isolate_one<R>(v.il, v.ih, k, 2 * j + 1, d, acc, RUNG);
}

template <int R = 1>
__device__ __forceinline__ void isolate_value(const Disc& v, int k, int64_t j, const ProdDesc& d,
                                              IsoAcc& acc) {
    const double r = double(v.r);
    isolate_one<R>(__dsub_rd(v.x, r), __dadd_ru(v.x, r), k, 2 * j, d, acc, 2);
    isolate_one<R>(__dsub_rd(v.y, r), __dadd_ru(v.y, r), k, 2 * j + 1, d, acc, 2);
}

// The decision of isolate_one for a component held as a double-binary32
// centre h + l and a binary32 radius r, without binary64 arithmetic (k0
// and k1 become integers by the conversion instructions, which take fewer
// issue slots than the same conversions done with integer operations).
// With k0 = rint(h), k1 = rint(l) (exact) the remainders t = h - k0
// and t' = l - k1 are exact and |t + t'| <= 1, so the component lies in
// [k0 + k1 + lo, k0 + k1 + hi] with lo = RD(RD(t + t') - r) and
// hi = RU(RU(t + t') + r).  While |lo|, |hi| < 2^22, ceil(lo) and floor(hi)
// are read off RU(lo + 1.5 2^23) and RD(hi + 1.5 2^23), whose ulp is 1.
// Beyond that r > 2^21 (the set holds many integers) unless a part is NaN
// or infinite (no integer: empty); a centre with |h| >= 2^53 cannot hold a
// coefficient (they are below 2^53) and is empty unless it is wide.
// R = 3, 5: the set encloses R c (see isolate_one); the integer bounds are
// divided by R exactly.
template <int R = 1>
__device__ __forceinline__ void isolate_pair(float h, float l, float r, int64_t idx,
                                             const ProdDesc& d, IsoAcc& acc, int rung) {
    const int64_t L = int64_t(d.na) + d.nb - 1;
    if (d.fault_widen == rung + 1) r = __fadd_ru(r, 4.f * R); // test fault: 4 in units of c
    const float k0 = rintf(h), k1 = rintf(l);
    const float t = __fsub_rn(h, k0), t2 = __fsub_rn(l, k1);
    const float lo = __fsub_rd(__fadd_rd(t, t2), r);
    const float hi = __fadd_ru(__fadd_ru(t, t2), r);
    const unsigned int wb = __float_as_uint(__fsub_ru(hi, lo));
    acc.maxw_f32 = wb > acc.maxw_f32 ? wb : acc.maxw_f32;
    constexpr float M = 12582912.f;                            // 1.5 2^23
    const bool fits = fabsf(lo) < 4194304.f && fabsf(hi) < 4194304.f;   // false for NaN
    const bool bad = (__float_as_int(h) & 0x7F800000) == 0x7F800000 ||
                     (__float_as_int(l) & 0x7F800000) == 0x7F800000 || r != r;
    const bool big = fabsf(h) >= 9007199254740992.f;            // 2^53
    const int cl = __float_as_int(__fadd_ru(lo, M)) - __float_as_int(M);
    const int fh = __float_as_int(__fadd_rd(hi, M)) - __float_as_int(M);
    // k0 and k1 are integers (|k0| < 2^53, |k1| < 2^30) unless a part is
    // large, infinite or NaN, when K plays no part in the decision
    const long long K = (big || bad) ? 0ll : __float2ll_rz(k0) + (long long)__float2int_rz(k1);
    long long kl = K + cl, kh = K + fh;
    if (R != 1) {
        // [ceil(kl / R), floor(kh / R)] with one 64-bit division: kl = q R + rm
        // (0 <= rm < R) and kh = kl + (fh - cl), a difference below 2^23 + 2
        // whenever the set fits (kl and kh decide nothing otherwise)
        const long long q = floor_div<R>(kl);
        const int rm = int(kl - q * R);
        kl = q + (rm > 0 ? 1 : 0);
        kh = q + floor_div32<R>(rm + (fits ? fh - cl : 0));
    }
    if (idx < L) {
        const int64_t corr = d.balanced ? balance_corr(d, idx) : 0;
        if (d.iv != nullptr) {
            // the enclosure as binary64 bounds (test output)
            const double dr = double(r);
            const double dl = __dsub_rd(__dadd_rd(double(h), double(l)), dr);
            const double dh = __dadd_ru(__dadd_ru(double(h), double(l)), dr);
            d.iv[2 * idx] = __dadd_rd(R != 1 ? __ddiv_rd(dl, double(R)) : dl, double(corr));
            d.iv[2 * idx + 1] = __dadd_ru(R != 1 ? __ddiv_ru(dh, double(R)) : dh, double(corr));
        }
        int64_t v = 0;
        if (bad) {
            acc.empty++;
        } else if (!fits) {
            acc.unisolated++;
        } else if (kl == kh && !big && kl + corr >= 0) {
            v = kl + corr;
        } else if (kl < kh) {
            acc.unisolated++;
        } else {
            acc.empty++;           // no integer, a negative one or overflow
        }
        d.coeff[idx] = v;
    } else {
        // the exact value is 0; for a wide or far centre, 0 is outside when
        // |h| - |l| > r (a lower bound on |h + l| exceeds the radius)
        const bool excl = (fits && !big) ? !(kl <= 0 && kh >= 0)
                                         : __fsub_rd(__fsub_rd(fabsf(h), fabsf(l)), r) > 0.f;
        if (bad || excl) acc.empty++;
    }
}

template <int R = 1>
__device__ __forceinline__ void isolate_value(const DDisc& v, int64_t j, const ProdDesc& d,
                                              IsoAcc& acc) {
    isolate_pair<R>(v.xh, v.xl, v.r, 2 * j, d, acc, 4);
    isolate_pair<R>(v.yh, v.yl, v.r, 2 * j + 1, d, acc, 4);
}

// ---- binary32 rectangles on 4-bit digits ------------------------------------------
//
// With d.fp32_nib the binary32 rung transforms the operands' base-16 digits
// a'_j = (a_{j/2} >> 4 (j mod 2)) & 15 (j < 2 na; likewise b'), whose
// coefficients c'_i = sum_j a'_j b'_{i-j} (i < 2 (na + nb) - 1, the product
// identity of Section 2.1 in base 16) are at most 225 min(2 na, 2 nb) instead
// of 65025 min(na, nb): narrower sets for twice the transform length.  Since
//   sum_i c'_i 16^i = sum_k (c'_{2k} + 16 c'_{2k+1}) 256^k,
// the base-256 carry of Section 2.4 takes C_k = c'_{2k} + 16 c'_{2k+1} for
// k < na + nb (one coefficient more than the na + nb - 1 of the bytes).  The
// packed inverse hands one thread c'_{2k} (real part) and c'_{2k+1}
// (imaginary part), so each thread isolates both (Section 1) and writes C_k,
// an exact integer sum.
//
// The transform carries the centred 4-bit digits e_j = a'_j - ma and
// f_j = b'_j - mb (zero past the operands), ma and mb the rounded means of
// a's and b's 4-bit digits: with J_i the pairs (j, i - j) that meet in
// coefficient i,
//   c'_i = sum_J (e_j + ma) (f_{i-j} + mb) = c''_i + mb Wa_i + ma Wb_i - ma mb |J_i|,
// Wa_i and Wb_i the sums of the 4-bit digits of a and b over J_i, which
// come from prefix sums Q of the 4-bit digits (a's, then b's) that the CTA
// builds in shared memory (nib_prefix_scan); c''_i is what the transform
// encloses.  Like the balanced bytes of the other rungs (balance_corr), this
// makes the transformed values and so the sets smaller without changing the
// product; the mean (8 for uniform digits, 0 for sparse operands, 15 for
// all-0xFF ones) is the constant that makes the digits' sum of squares least.

constexpr int NIB_MAX_DIGITS = 2048;      // na + nb: 2 (na + nb) - 1 <= 4096 = k_small's N

__device__ __forceinline__ int nib_log_n(const ProdDesc& d) {
    const int64_t lp = 2 * (int64_t(d.na) + d.nb) - 1;
    int k = 2;
    while ((int64_t(1) << k) < lp) ++k;
    return k;
}

// the centred base-16 digit j of the n-digit operand x: its 4-bit digit
// (x_{j/2} >> 4 (j mod 2)) & 15 minus m, and 0 past its 2 n digits
__device__ __forceinline__ int nibble_c(const uint8_t* x, uint32_t n, int j, int m) {
    return uint32_t(j) < 2u * n ? ((x[j >> 1] >> ((j & 1) * 4)) & 15) - m : 0;
}

// the prefix sums of the 4-bit digits and the two means they are centred on
struct NibCentre {
    const uint16_t* Q;
    int ma, mb;
};

// Shared-memory room of the prefix sums Q (uint16: sums of at most 4096
// digits of 15) and the scan's warp totals, after a transform buffer of n
// elements (2 (na + nb) - 1 <= n)
__host__ __device__ constexpr int nib_prefix_bytes(int n) { return 2 * n + 256; }

// Q[m] = the sum of the first m of the M = 2 (na + nb) 4-bit digits a'_0 ..
// a'_{2na-1}, b'_0 .. b'_{2nb-1} (m <= M), by one block scan: thread t sums
// a contiguous run of digits, the runs' totals are scanned across the warps
__device__ void nib_prefix_scan(const ProdDesc& d, uint16_t* Q, int* warp_tot) {
    const int na2 = 2 * int(d.na), M = na2 + 2 * int(d.nb);
    const auto digit = [&](int i) -> int {
        const uint8_t* x = i < na2 ? d.a : d.b;
        const int j = i < na2 ? i : i - na2;
        return (x[j >> 1] >> ((j & 1) * 4)) & 15;
    };
    const int T = blockDim.x, per = (M + T - 1) / T;
    const int i0 = threadIdx.x * per, lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int s = 0;
    for (int q = 0; q < per; ++q)
        if (i0 + q < M) s += digit(i0 + q);
    int x = s;                                      // inclusive scan within the warp
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, off);
        if (lane >= off) x += y;
    }
    if (lane == 31) warp_tot[warp] = x;
    __syncthreads();
    if (warp == 0) {
        int w = lane < (T >> 5) ? warp_tot[lane] : 0;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, w, off);
            if (lane >= off) w += y;
        }
        if (lane < (T >> 5)) warp_tot[lane] = w;
    }
    __syncthreads();
    int run = x - s + (warp > 0 ? warp_tot[warp - 1] : 0);
    if (threadIdx.x == 0) Q[0] = 0;
    for (int q = 0; q < per; ++q) {
        if (i0 + q < M) {
            run += digit(i0 + q);
            Q[i0 + q + 1] = uint16_t(run);
        }
    }
    __syncthreads();
}

// the rounded means of a's 2 na and b's 2 nb 4-bit digits, from Q
__device__ __forceinline__ NibCentre nib_centre(const ProdDesc& d, const uint16_t* Q) {
    const int na2 = 2 * int(d.na), nb2 = 2 * int(d.nb);
    const int sa = Q[na2], sb = int(Q[na2 + nb2]) - sa;
    return NibCentre{Q, (2 * sa + na2) / (2 * na2), (2 * sb + nb2) / (2 * nb2)};
}

// the exact term that turns c''_i into c'_i (i < 2 (na + nb) - 1), from Q
__device__ __forceinline__ int64_t nib_centre_corr(const ProdDesc& d, const NibCentre& c,
                                                   int64_t i) {
    const int64_t na2 = 2 * int64_t(d.na), nb2 = 2 * int64_t(d.nb);
    const int64_t ja_lo = i - nb2 + 1 > 0 ? i - nb2 + 1 : 0, ja_hi = i < na2 - 1 ? i : na2 - 1;
    const int64_t jb_lo = i - na2 + 1 > 0 ? i - na2 + 1 : 0, jb_hi = i < nb2 - 1 ? i : nb2 - 1;
    const int64_t wa = int64_t(c.Q[ja_hi + 1]) - int64_t(c.Q[ja_lo]);
    const int64_t wb = int64_t(c.Q[na2 + jb_hi + 1]) - int64_t(c.Q[na2 + jb_lo]);
    return int64_t(c.mb) * wa + int64_t(c.ma) * wb -
           int64_t(c.ma) * c.mb * (ja_hi - ja_lo + 1);
}

// The decision of isolate_one for nibble coefficient idx (lp of them) from
// the set [lo, hi] 2^-k of c''_idx; returns the isolated integer c'_idx
// (0 otherwise).
__device__ __forceinline__ int64_t isolate_nib_one(float lo, float hi, int k, int64_t idx,
                                                   int64_t lp, const ProdDesc& d,
                                                   const NibCentre& c, IsoAcc& acc) {
    double dl = double(lo), dh = double(hi);          // exact widening
    if (d.fault_widen == 1) {                         // test fault of the binary32 rung
        const double f = 4.0 * pow2_pos(k);
        dl = __dsub_rd(dl, f);
        dh = __dadd_ru(dh, f);
    }
    const unsigned long long wb = (unsigned long long)__double_as_longlong(__dsub_ru(dh, dl));
    acc.maxw_bits = wb > acc.maxw_bits ? wb : acc.maxw_bits;
    acc.wscale = k;
    long long kl, kh, unused;
    floor_ceil_scaled(dl, k, unused, kl);
    floor_ceil_scaled(dh, k, kh, unused);
    constexpr long long KMAX = 1ll << 53;
    if (idx < lp) {
        const int64_t corr = nib_centre_corr(d, c, idx);
        if (d.iv != nullptr) {                        // the set of c'_idx (tests)
            d.iv[2 * idx] = __dadd_rd(__dmul_rd(dl, pow2_neg(k)), double(corr));
            d.iv[2 * idx + 1] = __dadd_ru(__dmul_ru(dh, pow2_neg(k)), double(corr));
        }
        if (kl == kh && kl > -KMAX && kl < KMAX && kl + corr >= 0) return kl + corr;
        if (kl < kh) acc.unisolated++;
        else acc.empty++;              // no integer, a negative one, NaN or overflow
        return 0;
    }
    if (!(kl <= 0 && kh >= 0)) acc.empty++;          // the exact value is 0
    return 0;
}

__device__ __forceinline__ void isolate_nib_value(const CI<float>& v, int k, int64_t j,
                                                  const ProdDesc& d, const NibCentre& c,
                                                  IsoAcc& acc) {
    const int64_t nz = int64_t(d.na) + d.nb, lp = 2 * nz - 1;
    const int64_t c0 = isolate_nib_one(v.rl, v.rh, k, 2 * j, lp, d, c, acc);
    const int64_t c1 = isolate_nib_one(v.il, v.ih, k, 2 * j + 1, lp, d, c, acc);
    if (j < nz) d.coeff[j] = c0 + 16 * c1;
}

// the naive transform rounds to the nearest integer without any proof; its
// "width" statistic is the largest distance to that integer (R = 3, 5: v
// approximates R c; the distance is kept for R c like the enclosures' widths)
template <int R = 1>
__device__ __forceinline__ void naive_one(double v, int64_t idx, const ProdDesc& d,
                                          IsoAcc& acc) {
    const int64_t L = int64_t(d.na) + d.nb - 1;
    const double vv = R != 1 ? v * (1.0 / R) : v;
    const double k = rint(vv);
    const double dist = fabs(v - double(R) * k);
    const unsigned long long db = (unsigned long long)__double_as_longlong(dist);
    acc.maxw_bits = db > acc.maxw_bits ? db : acc.maxw_bits;
    if (idx < L) {
        const int64_t corr = d.balanced ? balance_corr(d, idx) : 0;
        if (d.iv != nullptr) {
            d.iv[2 * idx] = vv + double(corr);
            d.iv[2 * idx + 1] = vv + double(corr);
        }
        if (fabs(k) < 4.0e15 && int64_t(k) + corr >= 0) d.coeff[idx] = int64_t(k) + corr;
        else { d.coeff[idx] = 0; acc.empty++; }
    }
}

template <int R = 1>
__device__ __forceinline__ void isolate_value(const Pt& v, int64_t j, const ProdDesc& d,
                                              IsoAcc& acc) {
    naive_one<R>(v.x, 2 * j, d, acc);
    naive_one<R>(v.y, 2 * j + 1, d, acc);
}

// v 2^-k isolated: the rectangles and binary64 discs scale inside the
// integer conversion, the other types by scale_pow2 first
template <int R, typename V>
__device__ __forceinline__ void isolate_scaled(const V& v, int k, int64_t j, const ProdDesc& d,
                                               IsoAcc& acc) {
    if constexpr (std::is_same<V, CI<double>>::value || std::is_same<V, CI<float>>::value ||
                  std::is_same<V, Disc>::value)
        isolate_value<R>(v, k, j, d, acc);
    else
        isolate_value<R>(scale_pow2(v, k), j, d, acc);
}

// Global -> shared staging of `total` elements: a thread issues all of its
// (up to EPT) loads before its first store, so their latencies overlap.
template <int EPT, typename T, typename Load, typename Store>
__device__ __forceinline__ void stage(int total, Load load, Store store) {
    T v[EPT];
#pragma unroll
    for (int k = 0; k < EPT; ++k) {
        const int i = threadIdx.x + k * blockDim.x;
        if (i < total) v[k] = load(i);
    }
#pragma unroll
    for (int k = 0; k < EPT; ++k) {
        const int i = threadIdx.x + k * blockDim.x;
        if (i < total) store(i, v[k]);
    }
    for (int i = threadIdx.x + EPT * blockDim.x; i < total; i += blockDim.x) store(i, load(i));
}

// ---- k_small: the whole interval convolution of one product in one CTA -----

// One product per CTA (descs[blockIdx.x]), or with LIST the CTA's entry of
// the products a later rung of the ladder still runs (k_gate_list).  BPT:
// radix-4 butterflies per thread in block_fft (the launch gives
// nl * L / (4 BPT) threads)
template <typename Tag, int BPT>
__device__ __forceinline__ void small_one(const ProdDesc d, const TwTable& tw) {
    using V = typename ValOf<Tag>::type;
    constexpr int RUNG = VTraits<V>::rung;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const SBuf<V> sm{reinterpret_cast<V*>(smem_raw)};
    // binary32 rectangles may take the 4-bit digits (isolate_nib_value): the
    // transform length then covers 2 (na + nb) - 1 coefficients
    constexpr bool F32 = std::is_same<V, CI<float>>::value;
    const bool nib = F32 && d.fp32_nib != 0;
    const int logN = nib ? nib_log_n(d) : d.log_n, N = 1 << logN;
    const int bias = (d.balanced && !nib) ? 128 : 0;
    // 4-bit digits: their prefix sums after the transform buffer (the launch
    // adds nib_prefix_bytes to its N sizeof(V) bytes), then their means
    uint16_t* const Q = reinterpret_cast<uint16_t*>(smem_raw + size_t(N) * sizeof(V));
    if (nib) nib_prefix_scan(d, Q, reinterpret_cast<int*>(smem_raw + size_t(N) * sizeof(V) +
                                                          ((2 * N + 4 + 15) & ~15)));
    const NibCentre cen = nib ? nib_centre(d, Q) : NibCentre{Q, 0, 0};
    // the digit pairs as integers (8 bytes each, inside the buffer), then the
    // forward transform's exact first step (logN >= 2 for every plan length)
    int2* const si = reinterpret_cast<int2*>(smem_raw);
    stage<4 * BPT, int2>(
        N,
        [&](int j) {
            if (nib) return make_int2(nibble_c(d.a, d.na, j, cen.ma), nibble_c(d.b, d.nb, j, cen.mb));
            return make_int2(j < int(d.na) ? int(d.a[j]) - bias : 0,
                             j < int(d.nb) ? int(d.b[j]) - bias : 0);
        },
        [&](int j, int2 v) { si[j] = v; });
    __syncthreads();
    first_step_exact<V, BPT, 1, false>(si, N, sm, logN, 1, N, tw);
    // no radix-8 last step here: with one butterfly per thread a block
    // reaches 1024 threads at N = 4096, and its registers must stay <= 64
    block_fft<V, +1, BPT, 1, false>(sm, logN, 1, N, tw, true);
    pair_products(sm, 1, 0, logN);
    __syncthreads();
    pack_half(sm, 1, 0, 0, 0, logN, tw);
    __syncthreads();
    block_fft<V, -1, BPT, 1, false>(sm, logN - 1, 1, N, tw);
    IsoAcc acc;
    for (int j = threadIdx.x; j < (N >> 1); j += blockDim.x) {
        if constexpr (F32) {
            if (nib) {
                isolate_nib_value(sm[j], logN + 2, j, d, cen, acc);
                continue;
            }
        }
        isolate_scaled<1>(sm[j], logN + 2, j, d, acc);
    }
    flush_acc(acc, d.st, RUNG);
    if (threadIdx.x == 0) atomicOr(&d.st->ran[RUNG], 1u);
}

template <typename Tag, int BPT = 2, bool LIST = false>
__global__ void k_small(const ProdDesc* descs, TwTable tw, const int* list) {
    if constexpr (LIST) {
        // rows past the list's length have nothing to do: they end after one load
        if (int(blockIdx.x) < list[0]) small_one<Tag, BPT>(descs[list[1 + blockIdx.x]], tw);
    } else {
        small_one<Tag, BPT>(descs[blockIdx.x], tw);
    }
}

// ---- four-step kernels --------------------------------------------------------

// R: 1, 3 or 5 for N = R 2^k; N1 = R 2^logN1 (logN1 even when R > 1),
// N2 = 2^logN2, and tw is the twiddle table of family R.
// One element of Z or W to or from global memory.  A binary64 rectangle
// (32 bytes, 32-byte aligned: Z and W start on 256-byte boundaries) moves
// as one 256-bit access, so that a lane's element is one full sector even
// where the lanes of a warp touch addresses far apart.
template <typename V>
__device__ __forceinline__ void store_z(V* p, const V& v) { *p = v; }
template <>
__device__ __forceinline__ void store_z<CI<double>>(CI<double>* p, const CI<double>& v) {
    asm volatile("st.global.v4.f64 [%0], {%1, %2, %3, %4};"
                 :: "l"(p), "d"(v.rl), "d"(v.rh), "d"(v.il), "d"(v.ih) : "memory");
}
template <typename V>
__device__ __forceinline__ V load_z(const V* p) { return *p; }
template <>
__device__ __forceinline__ CI<double> load_z<CI<double>>(const CI<double>* p) {
    CI<double> v;
    asm volatile("ld.global.v4.f64 {%0, %1, %2, %3}, [%4];"
                 : "=d"(v.rl), "=d"(v.rh), "=d"(v.il), "=d"(v.ih) : "l"(p));
    return v;
}

template <typename Tag, int BPT, int R>
__device__ __forceinline__ void fwd_cols_one(const ProdDesc d, const TwTable& tw, int logN1,
                                             int logN2, int logC) {
    using V = typename ValOf<Tag>::type;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const SBuf<V> sm{reinterpret_cast<V*>(smem_raw)};
    const int N1 = R << logN1, C = 1 << logC;
    const uint32_t j2_0 = blockIdx.x << logC;
    V* Z = reinterpret_cast<V*>(d.Z);
    const int bias = d.balanced ? 128 : 0;
    const auto digits = [&](int idx) {
        const uint32_t j = (uint32_t(idx >> logC) << logN2) + j2_0 + (idx & (C - 1));
        return make_int2(j < d.na ? int(d.a[j]) - bias : 0, j < d.nb ? int(d.b[j]) - bias : 0);
    };
    const int logN = logN1 + logN2;
    // element k1 of column c: times the four-step twiddle omega_N^{j2 k1}, to Z
    const auto to_z = [&](int c, int k1, V v) {
        const uint32_t j2 = j2_0 + c;
        const uint32_t e = j2 * uint32_t(k1);             // < N
        if (e) v = mul_tw(v, get_twiddle<V, +1, R>(tw, e << (tw.log_n - logN)));
        store_z(Z + ((size_t(k1) << logN2) + j2), v);
    };
    if (R > 1 || logN1 >= 2) {
        // the digit pairs as integers, column c at c (N1 + 1) (the odd pitch
        // spreads the staging stores over the banks; C (N1 + 1) 8 bytes fit
        // in the buffer), then the exact first radix-4 step
        int2* const si = reinterpret_cast<int2*>(smem_raw);
        const int ip = N1 + 1;
        stage<4 * BPT, int2>(C * N1, digits,
                             [&](int idx, int2 v) { si[(idx & (C - 1)) * ip + (idx >> logC)] = v; });
        __syncthreads();
        first_step_exact<V, BPT, R, (R > 1)>(si, ip, sm, logN1, C, N1, tw);
        if constexpr (R == 1) {
            if constexpr (io_from_registers<V>()) {
                if (logN1 >= 3) {
                    // the last radix-4 or radix-2 step hands its outputs to
                    // to_z (N1 >= 8: a step remains after the exact first one)
                    block_fft<V, +1, BPT>(sm, logN1, C, N1, tw, true, FromBuf{}, to_z);
                    return;
                }
            }
            block_fft<V, +1, BPT>(sm, logN1, C, N1, tw, true);
        } else if constexpr (io_from_registers<V>()) {
            // the last (radix-R) step hands its outputs to to_z from registers
            block_fft_odd<V, +1, BPT, R>(sm, logN1, C, N1, tw, true, FromBuf{}, to_z);
            return;
        } else {
            block_fft_odd<V, +1, BPT, R>(sm, logN1, C, N1, tw, true);
        }
    } else {
        stage<4 * BPT, int2>(C * N1, digits, [&](int idx, int2 v) {
            sm[(idx & (C - 1)) * N1 + (idx >> logC)] = make_point<V>(v.x, v.y);
        });
        __syncthreads();
        block_fft<V, +1, BPT>(sm, logN1, C, N1, tw);
    }
    for (int idx = threadIdx.x; idx < C * N1; idx += blockDim.x) {
        const int c = idx & (C - 1), k1 = idx >> logC;
        to_z(c, k1, sm[c * N1 + k1]);
    }
}

template <typename Tag, int BPT = 2, int R = 1, bool LIST = false>
__global__ void __maxnreg__((cols_regs<typename ValOf<Tag>::type, R>()))
k_fwd_cols(const ProdDesc* descs, TwTable tw, int logN1, int logN2, int logC, const int* list) {
    if constexpr (LIST) {
        // rows past the list's length have nothing to do: they end after one load
        if (int(blockIdx.y) < list[0])
            fwd_cols_one<Tag, BPT, R>(descs[list[1 + blockIdx.y]], tw, logN1, logN2, logC);
    } else {
        fwd_cols_one<Tag, BPT, R>(descs[blockIdx.y], tw, logN1, logN2, logC);
    }
}

template <typename Tag, int BPT, int R>
__device__ __forceinline__ void rows_one(const ProdDesc d, const TwTable& tw, int logN1,
                                         int logN2) {
    using V = typename ValOf<Tag>::type;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const SBuf<V> sm{reinterpret_cast<V*>(smem_raw)};
    const int N1 = R << logN1, N2 = 1 << logN2, M2 = N2 >> 1;
    const int k1 = blockIdx.x;                              // 0 .. N1/2
    const int k1b = k1 ? N1 - k1 : 0;
    const int nl = (k1 == k1b) ? 1 : 2;
    const V* Z = reinterpret_cast<const V*>(d.Z);
    V* W = reinterpret_cast<V*>(d.W);
    const int logM = logN1 + logN2 - 1;
    // element j2 of line l: times the four-step twiddle omega_M^{-row j2}, to W
    const auto to_w = [&](int l, int j2, V v) {
        const int row = l ? k1b : k1;
        const uint32_t e = uint32_t(row) * uint32_t(j2);        // < N/2
        if (e) v = mul_tw(v, get_twiddle<V, -1, R>(tw, e << (tw.log_n - logM)));
        store_z(W + ((size_t(row) << (logN2 - 1)) + j2), v);
    };
    // a row pair with an odd log2 N2 leaves the forward transform's final
    // radix-2 step to pair_pack2
    const bool r2 = nl == 2 && (logN2 & 1) && !(last_radix8<V>() && logN2 >= 3);
    if constexpr (rows_load_from_registers<V>()) {
        // the forward transform's first step reads Z itself
        const auto from_z = [&](int l, int k) {
            return load_z(Z + ((size_t(l ? k1b : k1) << logN2) + k));
        };
        block_fft<V, +1, BPT, R>(sm, logN2, nl, N2, tw, false, from_z, ToBuf{}, r2);
    } else {
        stage<4 * BPT, V>(
            nl * N2,
            [&](int t) { return Z[(size_t((t >> logN2) ? k1b : k1) << logN2) + (t & (N2 - 1))]; },
            [&](int t, const V& v) { sm[t] = v; });
        __syncthreads();
        block_fft<V, +1, BPT, R>(sm, logN2, nl, N2, tw, false, FromBuf{}, ToBuf{}, r2);
    }
    if (r2) {
        pair_pack2<V, R, true>(sm, k1, k1b, logN1, logN2, tw);
    } else if (nl == 2) {
        pair_pack2<V, R>(sm, k1, k1b, logN1, logN2, tw);
    } else {
        pair_products(sm, nl, k1, logN2);
        __syncthreads();
        pack_half<V, R>(sm, nl, k1, k1b, logN1, logN2, tw);
    }
    __syncthreads();
    if constexpr (rows_store_from_registers<V>()) {
        // the inverse transform's last step hands its outputs to to_w
        block_fft<V, -1, BPT, R>(sm, logN2 - 1, nl, N2, tw, false, FromBuf{}, to_w);
    } else {
        block_fft<V, -1, BPT, R>(sm, logN2 - 1, nl, N2, tw);
        for (int t = threadIdx.x; t < nl * M2; t += blockDim.x) {
            const int l = t >> (logN2 - 1), j2 = t & (M2 - 1);
            to_w(l, j2, sm[l * N2 + j2]);
        }
    }
}

template <typename Tag, int BPT = 2, int R = 1, bool LIST = false>
__global__ void __maxnreg__(VTraits<typename ValOf<Tag>::type>::reg_rows)
k_rows(const ProdDesc* descs, TwTable tw, int logN1, int logN2, const int* list) {
    if constexpr (LIST) {
        // rows past the list's length have nothing to do: they end after one load
        if (int(blockIdx.y) < list[0]) rows_one<Tag, BPT, R>(descs[list[1 + blockIdx.y]], tw, logN1, logN2);
    } else {
        rows_one<Tag, BPT, R>(descs[blockIdx.y], tw, logN1, logN2);
    }
}

template <typename Tag, int BPT, int R>
__device__ __forceinline__ void inv_cols_one(const ProdDesc d, const TwTable& tw, int logN1,
                                             int logN2, int logC) {
    using V = typename ValOf<Tag>::type;
    constexpr int RUNG = VTraits<V>::rung;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const SBuf<V> sm{reinterpret_cast<V*>(smem_raw)};
    const int N1 = R << logN1, C = 1 << logC;
    const int logM2 = logN2 - 1;
    const uint32_t j2_0 = blockIdx.x << logC;
    const V* W = reinterpret_cast<const V*>(d.W);
    bool staged = true;
    if constexpr (io_from_registers<V>()) {
        // the first radix-4 step reads element j1 of column c from W itself
        // (columns of length N1 >= 4 for the lengths 2^k)
        const auto from_w = [&](int c, int j1) {
            return load_z(W + ((size_t(j1) << logM2) + j2_0 + c));
        };
        if (R > 1 || logN1 >= 2) {
            if constexpr (R == 1) block_fft<V, -1, BPT>(sm, logN1, C, N1, tw, false, from_w);
            else block_fft_odd<V, -1, BPT, R>(sm, logN1, C, N1, tw, false, from_w);
            staged = false;
        }
    }
    if (staged) {
        stage<4 * BPT, V>(
            C * N1,
            [&](int idx) { return W[(size_t(idx >> logC) << logM2) + j2_0 + (idx & (C - 1))]; },
            [&](int idx, const V& v) { sm[(idx & (C - 1)) * N1 + (idx >> logC)] = v; });
        __syncthreads();
        if constexpr (R == 1) block_fft<V, -1, BPT>(sm, logN1, C, N1, tw);
        else block_fft_odd<V, -1, BPT, R>(sm, logN1, C, N1, tw);
    }
    const int logN = logN1 + logN2;
    IsoAcc acc;
    for (int idx = threadIdx.x; idx < C * N1; idx += blockDim.x) {
        const int c = idx & (C - 1), j1 = idx >> logC;
        const int64_t j = (int64_t(j1) << logM2) + j2_0 + c;
        // 1 / (4 N) up to the factor 1/R, which the isolation applies exactly
        isolate_scaled<R>(sm[c * N1 + j1], logN + 2, j, d, acc);
    }
    flush_acc<R>(acc, d.st, RUNG);
    if (threadIdx.x == 0) atomicOr(&d.st->ran[RUNG], 1u);
}

template <typename Tag, int BPT = 2, int R = 1, bool LIST = false>
__global__ void __maxnreg__((cols_regs<typename ValOf<Tag>::type, R>()))
k_inv_cols(const ProdDesc* descs, TwTable tw, int logN1, int logN2, int logC, const int* list) {
    if constexpr (LIST) {
        // rows past the list's length have nothing to do: they end after one load
        if (int(blockIdx.y) < list[0])
            inv_cols_one<Tag, BPT, R>(descs[list[1 + blockIdx.y]], tw, logN1, logN2, logC);
    } else {
        inv_cols_one<Tag, BPT, R>(descs[blockIdx.y], tw, logN1, logN2, logC);
    }
}

// ---- the decision of a product ---------------------------------------------

// The rungs that ran are read in ladder order (binary32 rectangles,
// double-binary32 discs, binary64 discs, binary64 rectangles, unverified
// points): the first that isolated
// every coefficient, or found an empty set, decides; otherwise the last one
// that ran reports its isolation failure.
__device__ __forceinline__ int decide(const ProdState* stp, int* rung) {
    // one copy of the state: its loads are independent and go out together
    // (a walk over the rungs through the pointer would chain them)
    const ProdState st = *stp;
    const int order[RUNGS] = {0, 4, 2, 1, 3};
    int last = -1;
    int status = SSMUL_ISOLATION_FAILED;
    for (int k = 0; k < RUNGS; ++k) {
        const int r = order[k];
        if (!st.ran[r]) continue;
        last = r;
        if (r == 3) { status = SSMUL_UNVERIFIED; break; }
        if (st.empty[r]) { status = SSMUL_CONTAINMENT_FAILED; break; }
        if (st.unisolated[r] == 0) { status = SSMUL_OK; break; }
    }
    *rung = last < 0 ? 1 : last;
    if (st.forced) status = int(st.forced);
    return st.timeout ? SSMUL_TIMEOUT : status;
}

__device__ __forceinline__ int rung_precision(int rung) {
    switch (rung) {
        case 0: return SSMUL_PREC_FP32;
        case 2: return SSMUL_PREC_DISC64;
        case 3: return SSMUL_PREC_NAIVE64;
        case 4: return SSMUL_PREC_DISC32X2;
        default: return SSMUL_PREC_FP64;
    }
}

// ---- carry (Section 2.4) as a parallel carry-lookahead scan ------------------
//
// The coefficients c_i (0 <= c_i < 2^48) are split into bytes; the bytes
// that land on digit position k sum to u_k <= 6 * 255, and
// v_k = (u_k mod 256) + floor(u_{k-1} / 256) <= 260 satisfies
// sum_k v_k 256^k = sum_i c_i 256^i.  What remains is one carry bit per
// position: position k generates a carry when v_k >= 256 and propagates
// an incoming one when v_k = 255.  Within a warp the 32 (generate,
// propagate) pairs are evaluated by one binary addition of the bit masks
// A = generate|propagate and B = generate (the carry into lane i is bit i
// of (A + B + carry_in) ^ A ^ B); warps combine through shared memory and
// CTAs through a decoupled look-back whose waits are bounded.

__device__ __forceinline__ uint32_t ld_acquire(const uint32_t* p) {
    uint32_t v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release(uint32_t* p, uint32_t v) {
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// look-back word: bit 0 aggregate ready, bit 1 inclusive ready,
// bit 2 generate / carry-out, bit 3 propagate, bit 4 timed out upstream
constexpr uint32_t LB_AGG = 1u, LB_INC = 2u, LB_G = 4u, LB_P = 8u, LB_ERR = 16u;

// byte sum u_k of digit position k from the coefficients staged in shared
// memory: sc[i] holds c[k0_tile - CARRY_HALO + i]
constexpr int CARRY_HALO = 8;

__device__ __forceinline__ uint32_t digit_byte_sum_s(const int64_t* sc, int rel) {
    uint32_t u = 0;
#pragma unroll
    for (int t = 0; t < 6; ++t)
        u += uint32_t((uint64_t(sc[CARRY_HALO + rel - t]) >> (8 * t)) & 0xFFu);
    return u;
}

__global__ void __launch_bounds__(CARRY_THREADS, 4) k_carry(const ProdDesc* descs) {
    // coefficients of the tile (later reused for its output digits) and the
    // byte sums u_k, padded by one entry per 16 so that a thread's 16
    // consecutive entries fall into distinct banks
    __shared__ int64_t s_c[CARRY_TILE + CARRY_HALO];
    __shared__ uint16_t s_u[CARRY_TILE + CARRY_TILE / 16];
    __shared__ uint32_t s_uprev;
    __shared__ uint32_t s_tile, s_status, s_wA[CARRY_THREADS / 32], s_wB[CARRY_THREADS / 32];
    __shared__ uint32_t s_warp_cin[CARRY_THREADS / 32];
    __shared__ uint32_t s_ncoef;
    const ProdDesc d = descs[blockIdx.y];
    const int64_t nz = int64_t(d.na) + d.nb;
    if (threadIdx.x == 0) {
        s_tile = atomicAdd(&d.st->carry_ticket, 1u);   // tiles in start order
        int rung;
        s_status = decide(d.st, &rung);
        // na + nb - 1 coefficients of the digits, or na + nb when they came
        // from 4-bit digits (isolate_nib_value) or from split parts
        s_ncoef = (d.coef_nz || (rung == 0 && d.fp32_nib)) ? 1u : 0u;
    }
    __syncthreads();
    const int64_t L = nz - 1 + int64_t(s_ncoef);
    const uint32_t tile = s_tile;
    const int64_t k0 = int64_t(tile) * CARRY_TILE + int64_t(threadIdx.x) * CARRY_PER_THREAD;
    if (s_status != SSMUL_OK && s_status != SSMUL_UNVERIFIED) {
        // no unverified digit escapes: zero fill, publish a zero carry
        for (int q = 0; q < CARRY_PER_THREAD; ++q)
            if (k0 + q < nz) d.z[k0 + q] = 0;
        if (threadIdx.x == 0 && d.fault_stall != int32_t(tile) + 1)
            st_release(&d.flags[tile], LB_AGG | LB_INC);
        return;
    }
    const bool publish = d.fault_stall != int32_t(tile) + 1;   // test fault
    // stage c[tile start - CARRY_HALO .. tile end) with coalesced loads, all
    // of a thread's loads issued before its first shared store
    const int64_t kt = int64_t(tile) * CARRY_TILE;
    stage<(CARRY_TILE + CARRY_HALO + CARRY_THREADS - 1) / CARRY_THREADS, int64_t>(
        CARRY_TILE + CARRY_HALO,
        [&](int i) {
            const int64_t idx = kt - CARRY_HALO + i;
            return (idx >= 0 && idx < L) ? d.coeff[idx] : int64_t(0);
        },
        [&](int i, int64_t c) { s_c[i] = c; });
    __syncthreads();
    // byte sums u_k, one position per thread at a time (consecutive lanes,
    // consecutive coefficients)
    for (int kr = threadIdx.x; kr < CARRY_TILE; kr += CARRY_THREADS)
        s_u[kr + (kr >> 4)] = uint16_t((kt + kr < nz) ? digit_byte_sum_s(s_c, kr) : 0u);
    if (threadIdx.x == 0) s_uprev = (kt > 0) ? digit_byte_sum_s(s_c, -1) : 0u;
    __syncthreads();
    // v_k for this thread's positions, and its (generate, propagate) summary
    const int rel0 = int(k0 - kt);
    uint32_t v[CARRY_PER_THREAD];
    uint32_t prev_hi = (rel0 == 0) ? (s_uprev >> 8)
                                   : (uint32_t(s_u[(rel0 - 1) + ((rel0 - 1) >> 4)]) >> 8);
    bool G = false, P = true;
#pragma unroll
    for (int q = 0; q < CARRY_PER_THREAD; ++q) {
        const uint32_t u = s_u[(rel0 + q) + ((rel0 + q) >> 4)];
        v[q] = (u & 0xFFu) + prev_hi;
        prev_hi = u >> 8;
        const bool g = v[q] >= 256u, p = v[q] == 255u;
        G = g || (p && G);
        P = P && p;
    }
    // warp: carries into each lane with carry-in 0
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t A = __ballot_sync(0xffffffffu, G || P);
    const uint32_t B = __ballot_sync(0xffffffffu, G);
    if (lane == 0) { s_wA[warp] = A; s_wB[warp] = B; }
    __syncthreads();
    if (warp == 0) {
        // warp summaries: generate = carry out with carry-in 0,
        // propagate = every lane propagates
        constexpr int NW = CARRY_THREADS / 32;
        bool wg = false, wp = false;
        if (lane < NW) {
            const uint64_t s = uint64_t(s_wA[lane]) + uint64_t(s_wB[lane]);
            wg = (s >> 32) != 0;
            wp = (s_wA[lane] == 0xffffffffu) && (s_wB[lane] == 0u);
        }
        const uint32_t WA = __ballot_sync(0xffffffffu, wg || wp) & ((1u << NW) - 1u);
        const uint32_t WB = __ballot_sync(0xffffffffu, wg) & ((1u << NW) - 1u);
        // tile summary
        const uint64_t ts = uint64_t(WA) + uint64_t(WB);
        const bool tg = (ts >> NW) & 1u;
        const bool tp = WA == ((1u << NW) - 1u) && WB == 0u;
        uint32_t cin = 0, err = 0;
        if (tile == 0) {
            if (lane == 0 && publish) st_release(&d.flags[0], LB_INC | (tg ? LB_G : 0u));
        } else {
            if (lane == 0 && publish)
                st_release(&d.flags[tile], LB_AGG | (tg ? LB_G : 0u) | (tp ? LB_P : 0u));
            // warp-wide look-back: lane i polls tile (base - i); the closest
            // tile with an inclusive carry ends the walk, and the aggregates
            // of the tiles before it (nearest first) fold into (rg, rp)
            bool rg = false, rp = true;
            int64_t base = int64_t(tile) - 1;
            bool done = false;
            while (!done) {
                const int64_t t = base - lane;
                uint32_t f = LB_INC;                  // before tile 0: carry 0
                if (t >= 0) {
                    uint32_t it = 0;
                    for (; it < SPIN_LIMIT; ++it) {
                        f = ld_acquire(&d.flags[t]);
                        if (f & (LB_AGG | LB_INC)) break;
                        __nanosleep(64);
                    }
                    if (it == SPIN_LIMIT) {
                        f = LB_INC | LB_ERR;          // gave up: carry 0, flagged
                        atomicExch(&d.st->timeout, 1u);
                    }
                }
                const uint32_t inc = __ballot_sync(0xffffffffu, (f & LB_INC) != 0u);
                const uint32_t gm = __ballot_sync(0xffffffffu, (f & LB_G) != 0u);
                const uint32_t pm = __ballot_sync(0xffffffffu, (f & LB_P) != 0u);
                const uint32_t em = __ballot_sync(0xffffffffu, (f & LB_ERR) != 0u);
                const int j = inc ? __ffs(int(inc)) - 1 : 32;
                for (int i = 0; i < j; ++i) {
                    const bool pg = (gm >> i) & 1u, pp = (pm >> i) & 1u;
                    rg = rg || (rp && pg);
                    rp = rp && pp;
                }
                if (j < 32) {
                    cin = (rg || (rp && ((gm >> j) & 1u))) ? 1u : 0u;
                    err |= (em & ((2u << j) - 1u)) ? LB_ERR : 0u;
                    done = true;
                } else {
                    err |= em ? LB_ERR : 0u;
                    base -= 32;
                }
            }
            const bool cout = tg || (tp && cin);
            if (lane == 0 && publish)
                st_release(&d.flags[tile], LB_AGG | LB_INC | (cout ? LB_G : 0u) | err);
        }
        __syncwarp();
        cin = __shfl_sync(0xffffffffu, cin, 0);
        // carry into each warp of the tile
        const uint32_t carries = uint32_t((uint64_t(WA) + uint64_t(WB) + cin) ^ WA ^ WB);
        if (lane < NW) s_warp_cin[lane] = (carries >> lane) & 1u;
    }
    __syncthreads();
    const uint32_t wcin = s_warp_cin[warp];
    const uint32_t carries = uint32_t((uint64_t(A) + uint64_t(B) + wcin) ^ A ^ B);
    uint32_t c = (carries >> lane) & 1u;
    // digits staged in shared memory (the coefficients are no longer
    // needed), then written with consecutive lanes on consecutive bytes
    uint8_t* s_z = reinterpret_cast<uint8_t*>(s_c);
#pragma unroll
    for (int q = 0; q < CARRY_PER_THREAD; ++q) {
        const uint32_t t = v[q] + c;
        s_z[rel0 + q] = uint8_t(t & 0xFFu);
        c = t >> 8;
    }
    __syncthreads();
    for (int kr = threadIdx.x; kr < CARRY_TILE; kr += CARRY_THREADS)
        if (kt + kr < nz) d.z[kt + kr] = s_z[kr];
}

// ---- products split into parts (past the isolation limit) -------------------
//
// A product whose operands are cut into parts a = sum_k a_k 256^{k m},
// b = sum_l b_l 256^{l m} has the coefficients
//   c_i = sum_{k,l} c(a_k, b_l)_{i - (k + l) m},
// exact integer sums of the parts' isolated coefficients (Section 2.1's
// product identity applied block-wise).  Each part runs the interval
// convolution on its own; this kernel adds its coefficients into the
// parent's array at offset (k + l) m and folds its outcome into the
// parent's accumulators (the parts run one after another on one stream).
__global__ void k_split_accumulate(const ProdDesc* part, int64_t* total, uint64_t shift,
                                   ProdState* parent) {
    const ProdDesc d = *part;
    // the part's coefficients: na + nb of them when its binary32 rung took
    // 4-bit digits and decided (isolate_nib_value), else na + nb - 1
    int rung;
    const int status = decide(d.st, &rung);
    const int64_t L = int64_t(d.na) + d.nb - ((rung == 0 && d.fp32_nib) ? 0 : 1);
    for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < L;
         i += int64_t(gridDim.x) * blockDim.x)
        total[shift + i] += d.coeff[i];
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        parent->ran[rung] = 1u;
        parent->unisolated[rung] += d.st->unisolated[rung];
        parent->empty[rung] += d.st->empty[rung];
        if (d.st->maxw[rung] > parent->maxw[rung]) parent->maxw[rung] = d.st->maxw[rung];
        if (status != SSMUL_OK && unsigned(status) > parent->forced) parent->forced = unsigned(status);
        if (d.st->timeout) parent->timeout = 1u;
    }
}

// Final per-product outcome; zero-fills the digits of a product whose carry
// scan gave up waiting (the carry kernel already zero-filled the others).
__global__ void k_finalize(const ProdDesc* descs) {
    const ProdDesc d = descs[blockIdx.x];
    __shared__ int s_status;
    if (threadIdx.x == 0) {
        int rung;
        const int status = decide(d.st, &rung);
        ssmul_result r;
        r.status = status;
        r.precision_used = rung_precision(rung);
        // the deciding rung's transform: 4-bit digits double the bytes' length
        const bool nib = rung == 0 && d.fp32_nib;
        r.fft_log2 = nib ? uint32_t(nib_log_n(d)) : uint32_t(d.log_n % LEN3);
        r.n_unisolated = d.st->unisolated[rung];
        r.n_empty = d.st->empty[rung];
        r.fft_odd = nib ? 1u : (d.log_n >= LEN5 ? 5u : (d.log_n >= LEN3 ? 3u : 1u));
        r.max_width = __longlong_as_double((long long)d.st->maxw[rung]);
        *d.res = r;
        s_status = status;
    }
    __syncthreads();
    if (s_status == SSMUL_TIMEOUT) {
        const int64_t nz = int64_t(d.na) + d.nb;
        for (int64_t k = threadIdx.x; k < nz; k += blockDim.x) d.z[k] = 0;
    }
}

}  // namespace ssm
