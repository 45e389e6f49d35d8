// api.cu -- the C ABI of include/ssmul.h and include/ssmul_debug.h.
//
// Host-side orchestration only: argument checks, plan workspace, launch
// geometry (default or autotuned), the precision ladder, batching (grouped
// launches over a workspace arena, optionally captured in a CUDA graph).
// Every arithmetic step of the method runs in the kernels of kernels.cuh.
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <algorithm>
#include <cmath>
#include <mutex>
#include <string>
#include <type_traits>
#include <vector>

#include "kernels.cuh"
#include "../../include/ssmul_debug.h"

using namespace ssm;

namespace {

// the binary32 rung is tried when the product has at most this many digits
// in total (na + nb, a plan option; the default follows the digits the rung
// transforms): binary32 rectangles were measured to isolate every uniform
// square product up to 16 x 16 bytes (all-0xFF: 8 x 8), and up to 256 x 256
// digits on 4-bit digits centred on their means (all-0xFF: 1024 x 1024, all
// the 4-bit digits take); the width grows with the transform length
constexpr int FP32_MAX_LOG_N = LOG_SMALL;
constexpr size_t FP32_MAX_DIGITS = 32;          // bytes
constexpr size_t FP32_MAX_DIGITS_NIB = 512;     // 4-bit digits

// largest batch arena a plan allocates (the batch runs in chunks beyond it)
constexpr size_t ARENA_CAP = size_t(4) << 30;

// pieces of a host-buffer batch (ssmul_mul_batched_host): later pieces'
// operands upload and earlier pieces' digits download while a piece
// computes.  256 products of 75,000 x 75,000 digits took 16.72 / 16.60 /
// 16.55 / 16.60 ms in 1 / 2 / 4 / 8 pieces (16.31 ms on device buffers)
constexpr int HOST_PIECES = 4;

// compute lanes of a plan (streams that run independent work concurrently)
constexpr int LANES = 4;
// streams of the pieces of a host-buffer call
constexpr int PIECE_LANES = 4;
// lanes over which a batched call spreads the transform-length groups of a
// chunk (SSMUL_OPT_LANES): on 20,000 products of log-uniform sizes (64 to
// 131,072 digits, about 30 groups) four lanes took 0.8-1.1% less time than one
constexpr int GROUP_LANES = 4;

struct Geom {
    int log_n;       // transform length code (see LEN3)
    bool small;      // whole product in one CTA
    int r;           // 1, or 3 or 5: columns of r 2^log_n1 (four-step only)
    int log_n1, log_n2;
    int log_c1, log_c3;
    int log_cta;     // log2 of the elements a column CTA holds (at least N1)
};

constexpr int GEOM_CODES = LEN5 + LOG5_MAX + 1;

// the odd factor and the power of two of a length code
int odd_of(int code) { return code >= LEN5 ? 5 : (code >= LEN3 ? 3 : 1); }
int log2_of(int code) { return code % LEN3; }

// the transform length of a length code
size_t len_of(int code) { return size_t(odd_of(code)) << log2_of(code); }

int log_n_for(size_t na, size_t nb) {
    const size_t L = na + nb - 1;
    int k = 2;                          // N >= 4: the half-length inverse needs N/2 >= 2
    while ((size_t(1) << k) < L) ++k;
    return k;
}

// The length code of a product: the shortest allowed length >= na + nb - 1
// among the next power of two 2^k, 5 2^(k-3) = 0.625 2^k (lengths bit 1)
// and 3 2^(k-2) = 0.75 2^k (lengths bit 0), the only lengths of those
// families between 2^(k-1) and 2^k.
int length_code(size_t na, size_t nb, int lengths) {
    const int k = log_n_for(na, nb);
    const size_t L = na + nb - 1;
    const int j5 = k - 3, j3 = k - 2;
    if ((lengths & 2) && j5 >= LOG5_MIN && j5 <= LOG5_MAX && (size_t(5) << j5) >= L)
        return LEN5 + j5;
    if ((lengths & 1) && j3 >= LOG3_MIN && j3 <= LOG3_MAX && (size_t(3) << j3) >= L)
        return LEN3 + j3;
    return k;
}

int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

bool geom_valid(int log_n, int log_n2) {
    const int log_n1 = log_n - log_n2;
    return log_n2 >= 2 && log_n2 <= LOG_N2_MAX && log_n1 >= 1 && log_n1 <= LOG_N1_MAX;
}

// four-step split N = N1 * N2 with column CTAs of 2^log_cta elements
Geom make_geom(int log_n, int log_n2, int log_cta) {
    Geom g{};
    g.log_n = log_n;
    g.r = 1;
    g.small = log_n <= LOG_SMALL;
    if (!g.small) {
        g.log_n2 = log_n2;
        g.log_n1 = log_n - log_n2;
        g.log_cta = log_cta;
        const int c = log_cta - g.log_n1;
        g.log_c1 = clampi(c, 0, g.log_n2);
        g.log_c3 = clampi(c, 0, g.log_n2 - 1);
    }
    return g;
}

Geom default_geom(int log_n) {
    int log_n2 = (log_n + 1) / 2;
    if (log_n2 > LOG_N2_MAX) log_n2 = LOG_N2_MAX;
    return make_geom(log_n, log_n2, LOG_CTA_ELEMS);
}

// N = R 2^j = N1 N2 (R = 3 or 5) with N1 = R 2^a (a even: the radix-4 steps
// of a column end at length R; N1 <= 4096), N2 = 2^log_n2
bool geom_odd_valid(int R, int j, int log_n2) {
    const int a = j - log_n2;
    const bool jok = R == 3 ? (j >= LOG3_MIN && j <= LOG3_MAX) : (j >= LOG5_MIN && j <= LOG5_MAX);
    return jok && log_n2 >= 2 && log_n2 <= LOG_N2_MAX && a >= 2 && (R << a) <= 4096 &&
           (a & 1) == 0;
}

// column CTAs hold C R 2^a elements, between 2^(log_cta-1) and 1.5 2^(log_cta-1)
Geom make_geom_odd(int R, int j, int log_n2, int log_cta) {
    Geom g{};
    g.log_n = (R == 3 ? LEN3 : LEN5) + j;
    g.r = R;
    g.small = false;
    g.log_n2 = log_n2;
    g.log_n1 = j - log_n2;
    g.log_cta = log_cta;
    const int c = log_cta - g.log_n1 - (R == 3 ? 1 : 2);
    g.log_c1 = clampi(c, 0, g.log_n2);
    g.log_c3 = clampi(c, 0, g.log_n2 - 1);
    return g;
}

Geom default_geom_odd(int R, int j) {
    const int amax = R == 3 ? 10 : 8;           // R 2^a <= 4096, a even
    int b = (j + 1) / 2, a = j - b;
    if (a & 1) { --a; ++b; }
    while (b > LOG_N2_MAX) { b -= 2; a += 2; }
    while (a > amax) { a -= 2; b += 2; }
    // column CTAs of about 2^10 elements: the autotuner's choice at 3 2^16
    // (against 3 2^10: 2-3% faster for every rung)
    return make_geom_odd(R, j, b, LOG_CTA_ELEMS - 1);
}

Geom default_geom_code(int code) {
    return code >= LEN3 ? default_geom_odd(odd_of(code), log2_of(code)) : default_geom(code);
}

int threads_for(int elems) {          // block_fft with 2 butterflies per thread
    int t = elems / 8;
    if (t < 32) t = 32;
    return t;
}

// radix-4 butterflies per thread the plan's launches use: two for the
// binary64 types (one halves the registers but measured 6% slower on GB300),
// one for the double-binary32 discs (twice the warps for the issue-bound
// binary32 kernels: 5% faster at 75k digits)
template <typename V> constexpr int plan_bpt() { return std::is_same<V, DDisc>::value ? 1 : 2; }

template <typename V>
int fft_threads(int elems) {          // block_fft: nl * L / (4 BPT) threads
    int t = elems / (4 * plan_bpt<V>());
    if (t < 32) t = 32;
    return t;
}

size_t carry_tiles(size_t nz) { return (nz + CARRY_TILE - 1) / CARRY_TILE; }

// words of a balanced-digit prefix array (see k_prefix): local sums and tile offsets
size_t pre_words(size_t n) { return n + 1 + (n + PRE_TILE - 1) / PRE_TILE; }
size_t pre_bytes(size_t na, size_t nb) {
    return ((pre_words(na) + pre_words(nb)) * sizeof(uint32_t) + 255) & ~size_t(255);
}

ssmul_status cuda_status(cudaError_t e) {
    if (e == cudaSuccess) return SSMUL_OK;
    if (e == cudaErrorMemoryAllocation) return SSMUL_OUT_OF_MEMORY;
    return SSMUL_CUDA_ERROR;
}

#define SS_TRY(x)                                             \
    do {                                                      \
        cudaError_t e_ = (x);                                 \
        if (e_ != cudaSuccess) return cuda_status(e_);        \
    } while (0)

// ---- a prepared batch: launch structure computed on the host -------------------

struct BatchGroup {
    size_t g0, g1;      // descriptor range of one transform length
    size_t e1;          // [g0, e1) are binary32-eligible
    int log_n;
    size_t max_nz;
};

struct BatchChunk {
    size_t k0, k1;      // descriptors packed into the arena together
    std::vector<BatchGroup> groups;
};

struct GraphEntry {
    bool valid = false;
    std::vector<ssmul_desc> key;
    const void *a = nullptr, *b = nullptr, *z = nullptr, *res = nullptr;
    std::vector<ProdDesc> prepared;
    cudaGraphExec_t exec = nullptr;
    unsigned long long launches[SSMUL_KERNEL_KINDS] = {};
};

}  // namespace

// One family of twiddle tables, Ntab = R 2^log_tab (log_tab 0: none).
// The step tables hold n = R 2^j (for R = 1, n = 2^j).
struct TwFamily {
    int R = 1;
    int log_tab = 0;
    TwMid* t64 = nullptr;                 // values before the widening (tw_expand_w)
    TwEntry<float>* t32 = nullptr;
    DiscTw* td = nullptr;
    DDiscC* tdd = nullptr;
    float rho_dd = 0.f;                 // the radius of every entry of tdd
    CI<double>* s64 = nullptr;          // step-ordered twiddles (STEP_TAB x 3 each)
    CI<float>* s32 = nullptr;
    DiscTw* sd = nullptr;
    DDiscC* sdd = nullptr;
    ScalarSet* scal = nullptr;          // radix-3 / radix-5 scalars (R > 1)
    size_t entries() const { return log_tab ? (size_t(R) << log_tab) / 8 + 1 : 0; }
};

constexpr int FAMILIES = 3;             // R = 1, 3, 5
constexpr int FAMILY_R[FAMILIES] = {1, 3, 5};

struct ssmul_plan_s {
    int device = 0;
    cudaStream_t stream = nullptr;
    ssmul_precision prec = SSMUL_PREC_FP64;
    size_t max_na = 0, max_nb = 0, max_products = 0;
    int log_n_max = 0;
    TwFamily fam[FAMILIES];             // R = 1 always; R = 3, 5 when the plan reaches them
    float* rho = nullptr;               // device, 2 per family: largest td radius, tdd radius
    Geom geom[GEOM_CODES] = {};           // by length code
    int lengths = 3;                    // SSMUL_OPT_LENGTHS
    size_t fp32_max_digits = 0;         // SSMUL_OPT_FP32_MAX_DIGITS; 0: the default
    bool fp32_max_zero = false;         // the option was set to 0: never binary32 (ladders)
    bool fp32_nibbles = true;           // SSMUL_OPT_FP32_NIBBLES
    bool balanced = false;
    uint32_t* pre = nullptr;            // balanced: digit prefix sums of one product
    int fault_widen = 0, fault_stall = 0;   // ssmul_debug_set_fault
    bool octant_only = false;           // transforms read the octant tables (a test)
    // split products (SSMUL_OPT_SPLIT_DIGITS)
    size_t split_digits = 0;
    size_t split_slots = 0;
    int64_t* coeff_total = nullptr;     // max_na + max_nb coefficients
    ProdState* split_st = nullptr;      // split_slots entries
    ProdDesc* d_split = nullptr;        // split_slots entries
    ProdDesc* h_split = nullptr;        // pinned
    // single-product workspace
    void* Z = nullptr;
    void* W = nullptr;
    int64_t* coeff = nullptr;
    uint32_t* flags = nullptr;          // carry look-back words
    size_t flags_per_product = 0;
    ProdState* st = nullptr;            // max(1, max_products) entries
    ProdDesc* d_desc = nullptr;         // max(1, max_products) entries
    int* gate_list = nullptr;           // 1 + max(1, max_products) entries (k_gate_list)
    // compute lanes: lane 0 is the plan's stream, lanes 1 .. LANES-1 are
    // internal streams (created on first use) on which independent parts of
    // a batch run concurrently, each with a gate list of its own.  cur and
    // cur_gate are what the enqueue functions launch on: lane 0's, except
    // while a batch issues work on another lane.
    cudaStream_t lane_stream[LANES] = {};
    int* lane_gate[LANES] = {};
    cudaEvent_t lane_ev[LANES] = {};    // fork / join marks
    cudaStream_t cur = nullptr;
    int* cur_gate = nullptr;
    // host-buffer pieces (ssmul_mul_batched_host): internal streams of
    // decreasing priority, piece k on stream k mod PIECE_LANES, each with a
    // gate list of its own; piece_ev[0] marks the call's start on the plan's
    // stream, piece_ev[1 + l] the end of stream l's pieces
    cudaStream_t piece_stream[PIECE_LANES] = {};
    int* piece_gate[PIECE_LANES] = {};
    cudaEvent_t piece_ev[PIECE_LANES + 1] = {};
    int piece_lanes = 0;                // streams created (limited by the priority levels)
    int sms = 1;                        // streaming multiprocessors of the device
    ssmul_result* d_res = nullptr;
    ProdDesc* h_desc = nullptr;         // pinned
    ssmul_result* h_res = nullptr;      // pinned
    cudaEvent_t desc_free = nullptr;    // h_desc may be rewritten once this fired
    uint8_t* stage = nullptr;           // device staging for ssmul_mul_host
    // batch workspace: per-product transform buffers are carved from the
    // arena; a batch larger than the arena runs in stream-ordered chunks
    unsigned char* arena = nullptr;
    size_t arena_bytes = 0;
    std::vector<int> order;             // host scratch of a batched call
    std::vector<BatchChunk> chunks;
    size_t batch_nreg = 0;              // products of the prepared batch that are not split
    size_t split_cursor = 0;            // next free part entry of the current batched call
    // host-buffer batches (ssmul_mul_batched_host): device copies of the
    // pools and outcomes (grown on demand), two copy streams and the events
    // that order the pieces of a call
    uint8_t* hb_a = nullptr;
    uint8_t* hb_b = nullptr;
    uint8_t* hb_z = nullptr;
    size_t hb_a_cap = 0, hb_b_cap = 0, hb_z_cap = 0;
    ssmul_result* hb_res = nullptr;     // max(1, max_products) entries
    cudaStream_t up = nullptr, down = nullptr;
    std::vector<cudaEvent_t> hb_ev;     // two per piece
    int host_pieces = HOST_PIECES;      // SSMUL_OPT_HOST_PIECES
    int group_lanes = GROUP_LANES;      // SSMUL_OPT_LANES
    // CUDA graph of the last batched call (SSMUL_OPT_GRAPH)
    bool graph = false;
    bool capturing = false;
    GraphEntry cached;
    unsigned long long cap_launches[SSMUL_KERNEL_KINDS] = {};
    // optional per-kernel timing (ssmul_debug_kernel_stats)
    bool timing = false;
    std::vector<cudaEvent_t> ev_pool;
    std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> pending;
    double kt_ms[SSMUL_KERNEL_KINDS] = {};
    unsigned long long kt_launches[SSMUL_KERNEL_KINDS] = {};
    // the twiddle table of family f (0: R = 1; 1: R = 3; 2: R = 5).  Its
    // power-of-two step tables are family 0's (the same enclosed values).
    TwTable tw(int f = 0) const {
        const TwFamily& F = fam[f];
        const TwFamily& P = fam[0];
        const bool st = !octant_only;
        return TwTable{F.t64, F.t32, F.log_tab, F.td, F.tdd, F.rho_dd,
                       st ? P.s64 : nullptr, st ? P.s32 : nullptr, st ? P.sd : nullptr,
                       st ? P.sdd : nullptr,
                       st && f ? F.s64 : nullptr, st && f ? F.s32 : nullptr,
                       st && f ? F.sd : nullptr, st && f ? F.sdd : nullptr,
                       f ? F.scal : nullptr};
    }
};

namespace {

cudaEvent_t take_event(ssmul_plan_t p) {
    if (!p->ev_pool.empty()) {
        cudaEvent_t e = p->ev_pool.back();
        p->ev_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

// Launch bookkeeping around every kernel: a launch count always, and a
// pair of events on the plan's stream when timing is on (not inside a
// graph capture, whose launches are counted per replay).
struct LaunchScope {
    ssmul_plan_t p;
    int kind;
    cudaEvent_t e0 = nullptr;
    LaunchScope(ssmul_plan_t p_, int kind_) : p(p_), kind(kind_) {
        if (p->capturing) {
            p->cap_launches[kind]++;
            return;
        }
        p->kt_launches[kind]++;
        if (p->timing) {
            e0 = take_event(p);
            cudaEventRecord(e0, p->cur);
        }
    }
    ~LaunchScope() {
        if (e0) {
            cudaEvent_t e1 = take_event(p);
            cudaEventRecord(e1, p->cur);
            p->pending.push_back({kind, {e0, e1}});
        }
    }
};

// Lanes 1 .. n-1 (streams, gate lists) and the fork / join events of
// lanes 0 .. n-1, created on first use.
ssmul_status ensure_lanes(ssmul_plan_t p, int n) {
    const size_t slots = p->max_products ? p->max_products : 1;
    for (int l = 1; l < n; ++l) {
        if (!p->lane_stream[l])
            SS_TRY(cudaStreamCreateWithFlags(&p->lane_stream[l], cudaStreamNonBlocking));
        if (!p->lane_gate[l]) SS_TRY(cudaMalloc(&p->lane_gate[l], (slots + 1) * sizeof(int)));
    }
    for (int l = 0; l < n; ++l)
        if (!p->lane_ev[l]) SS_TRY(cudaEventCreateWithFlags(&p->lane_ev[l], cudaEventDisableTiming));
    return SSMUL_OK;
}

// Streams for the pieces of host-buffer calls, of decreasing priority
// (piece stream l at the device's greatest priority + l, while there are
// that many levels), created on first use; returns how many exist.
int ensure_piece_lanes(ssmul_plan_t p, int n, ssmul_status* err) {
    *err = SSMUL_OK;
    int least = 0, greatest = 0;
    if (cudaDeviceGetStreamPriorityRange(&least, &greatest) != cudaSuccess) least = greatest = 0;
    const int levels = least - greatest + 1;
    n = std::min(n, std::min(PIECE_LANES, levels < 1 ? 1 : levels));
    const size_t slots = p->max_products ? p->max_products : 1;
    for (int l = p->piece_lanes; l < n; ++l) {
        cudaError_t e = cudaStreamCreateWithPriority(&p->piece_stream[l], cudaStreamNonBlocking,
                                                     greatest + l);
        if (e == cudaSuccess) e = cudaMalloc(&p->piece_gate[l], (slots + 1) * sizeof(int));
        if (e != cudaSuccess) {
            *err = cuda_status(e);
            return 0;
        }
        p->piece_lanes = l + 1;
    }
    for (int l = 0; l <= n; ++l) {
        if (!p->piece_ev[l] &&
            cudaEventCreateWithFlags(&p->piece_ev[l], cudaEventDisableTiming) != cudaSuccess) {
            *err = SSMUL_CUDA_ERROR;
            return 0;
        }
    }
    return n;
}

// The enqueue functions launch on `stream` with gate list `gate` while this
// lives; the lane that was current before is restored after.
struct OnLane {
    ssmul_plan_t p;
    cudaStream_t prev;
    int* prev_gate;
    OnLane(ssmul_plan_t p_, cudaStream_t stream, int* gate)
        : p(p_), prev(p_->cur), prev_gate(p_->cur_gate) {
        p->cur = stream;
        p->cur_gate = gate;
    }
    ~OnLane() {
        p->cur = prev;
        p->cur_gate = prev_gate;
    }
};

template <typename W> constexpr int kind_off() { return VTraits<typename ValOf<W>::type>::rung; }

// the rungs a ladder can run after another one (binary32 rectangles and
// the naive points are only ever first), which also get the LIST kernels
template <typename T>
constexpr bool gateable() {
    return !std::is_same<T, float>::value && !std::is_same<T, Pt>::value;
}

template <typename T, bool LIST>
ssmul_status set_smem_attrs_as() {
    constexpr int B = plan_bpt<typename ValOf<T>::type>();
    const int big = 160 * 1024;
    const auto a = cudaFuncAttributeMaxDynamicSharedMemorySize;
    SS_TRY(cudaFuncSetAttribute(k_small<T, B, LIST>, a, big));
    SS_TRY(cudaFuncSetAttribute(k_fwd_cols<T, B, 1, LIST>, a, big));
    SS_TRY(cudaFuncSetAttribute(k_rows<T, B, 1, LIST>, a, big));
    SS_TRY(cudaFuncSetAttribute(k_inv_cols<T, B, 1, LIST>, a, big));
    SS_TRY(cudaFuncSetAttribute(k_fwd_cols<T, B, 3, LIST>, a, big));
    SS_TRY(cudaFuncSetAttribute(k_rows<T, B, 3, LIST>, a, big));
    SS_TRY(cudaFuncSetAttribute(k_inv_cols<T, B, 3, LIST>, a, big));
    SS_TRY(cudaFuncSetAttribute(k_fwd_cols<T, B, 5, LIST>, a, big));
    SS_TRY(cudaFuncSetAttribute(k_rows<T, B, 5, LIST>, a, big));
    SS_TRY(cudaFuncSetAttribute(k_inv_cols<T, B, 5, LIST>, a, big));
    return SSMUL_OK;
}

template <typename T>
ssmul_status set_smem_attrs() {
    ssmul_status s = set_smem_attrs_as<T, false>();
    if constexpr (gateable<T>()) {
        if (s == SSMUL_OK) s = set_smem_attrs_as<T, true>();
    }
    return s;
}


// The three four-step launches of one transform length of family R, one CTA
// row per product (LIST: per entry of list, a gated rung's products).
template <typename T, int R, bool LIST>
void enqueue_four_step(ssmul_plan_t p, const ProdDesc* d_desc, int count, const Geom& g,
                       const int* list, const TwTable& tw) {
    using V = typename ValOf<T>::type;
    constexpr int B = plan_bpt<V>();
    const int ko = kind_off<T>();
    const int n1 = R << g.log_n1, n2 = 1 << g.log_n2;
    const int e1 = n1 << g.log_c1, e3 = n1 << g.log_c3;
    const int t1 = n2 >> g.log_c1, t2 = n1 / 2 + 1, t3 = (n2 / 2) >> g.log_c3;
    {
        LaunchScope ls(p, SSMUL_K_FWD_COLS + ko);
        k_fwd_cols<T, B, R, LIST><<<dim3(t1, count),
                                    fft_threads<V>(e1), e1 * sizeof(V), p->cur>>>(
            d_desc, tw, g.log_n1, g.log_n2, g.log_c1, list);
    }
    {
        LaunchScope ls(p, SSMUL_K_ROWS + ko);
        k_rows<T, B, R, LIST><<<dim3(t2, count),
                                fft_threads<V>(2 * n2), 2 * n2 * sizeof(V), p->cur>>>(
            d_desc, tw, g.log_n1, g.log_n2, list);
    }
    {
        LaunchScope ls(p, SSMUL_K_INV_COLS + ko);
        k_inv_cols<T, B, R, LIST><<<dim3(t3, count),
                                    fft_threads<V>(e3), e3 * sizeof(V), p->cur>>>(
            d_desc, tw, g.log_n1, g.log_n2, g.log_c3, list);
    }
}

template <typename T, bool LIST>
ssmul_status enqueue_rung_as(ssmul_plan_t p, const ProdDesc* d_desc, int count, const Geom& g,
                             const int* list) {
    using V = typename ValOf<T>::type;
    constexpr int B = plan_bpt<V>();
    const int ko = kind_off<T>();
    if (g.small) {
        // binary32 rectangles on 4-bit digits need up to 4 times the length
        // of the bytes' transform (2 (na + nb) - 1 <= 4096 coefficients) and
        // room for the prefix sums of their centring (nib_prefix_scan)
        const bool nib = std::is_same<T, float>::value && p->fp32_nibbles;
        const int n = nib ? std::min(1 << LOG_SMALL, 4 << g.log_n) : 1 << g.log_n;
        const size_t smem = n * sizeof(V) + (nib ? size_t(nib_prefix_bytes(n)) : 0);
        LaunchScope ls(p, SSMUL_K_SMALL + ko);
        k_small<T, B, LIST><<<count, fft_threads<V>(n), smem, p->cur>>>(d_desc, p->tw(), list);
    } else if (g.r == 3) {
        enqueue_four_step<T, 3, LIST>(p, d_desc, count, g, list, p->tw(1));
    } else if (g.r == 5) {
        enqueue_four_step<T, 5, LIST>(p, d_desc, count, g, list, p->tw(2));
    } else {
        enqueue_four_step<T, 1, LIST>(p, d_desc, count, g, list, p->tw());
    }
    return cuda_status(cudaGetLastError());
}

// Enqueue the interval convolution of `count` products that share one
// transform length, described by d_desc[0 .. count).  gate: skip products
// an earlier rung in this bit mask already decided (k_gate_list lists the
// others, and the rung's kernels run over that list).
template <typename T>
ssmul_status enqueue_rung(ssmul_plan_t p, const ProdDesc* d_desc, int count, const Geom& g,
                          int gate) {
    if (!gate) return enqueue_rung_as<T, false>(p, d_desc, count, g, nullptr);
    if constexpr (gateable<T>()) {
        {
            LaunchScope ls(p, SSMUL_K_GATE);
            k_gate_list<<<1, 256, 0, p->cur>>>(d_desc, count, gate, p->cur_gate);
        }
        return enqueue_rung_as<T, true>(p, d_desc, count, g, p->cur_gate);
    } else {
        return SSMUL_INVALID_ARG;          // never gated (see gateable)
    }
}

bool fp32_eligible(ssmul_plan_t p, size_t na, size_t nb, int log_n) {
    if (p->fp32_max_zero) return false;
    const size_t limit = p->fp32_max_digits ? p->fp32_max_digits
                         : (p->fp32_nibbles ? FP32_MAX_DIGITS_NIB : FP32_MAX_DIGITS);
    return log_n <= FP32_MAX_LOG_N && na + nb <= limit;
}

bool uses_fp32(ssmul_precision prec) {
    return prec == SSMUL_PREC_FP32 || prec == SSMUL_PREC_LADDER ||
           prec == SSMUL_PREC_LADDER_DISC || prec == SSMUL_PREC_LADDER_FAST;
}

ssmul_status enqueue_rung_idx(ssmul_plan_t p, int rung, const ProdDesc* d_desc, int count,
                              const Geom& g, int gate) {
    switch (rung) {
        case 0: return enqueue_rung<float>(p, d_desc, count, g, gate);
        case 1: return enqueue_rung<double>(p, d_desc, count, g, gate);
        case 2: return enqueue_rung<Disc>(p, d_desc, count, g, gate);
        case 4: return enqueue_rung<DDisc>(p, d_desc, count, g, gate);
        default: return enqueue_rung<Pt>(p, d_desc, count, g, gate);
    }
}

// The rungs after the binary32 one, in order, for a precision rule.
int later_rungs(ssmul_precision prec, int* out) {
    switch (prec) {
        case SSMUL_PREC_FP32: return 0;
        case SSMUL_PREC_DISC64: out[0] = 2; return 1;
        case SSMUL_PREC_NAIVE64: out[0] = 3; return 1;
        case SSMUL_PREC_LADDER_DISC: out[0] = 2; out[1] = 1; return 2;
        case SSMUL_PREC_DISC32X2: out[0] = 4; return 1;
        case SSMUL_PREC_LADDER_FAST: out[0] = 4; out[1] = 2; out[2] = 1; return 3;
        default: out[0] = 1; return 1;                 // FP64, LADDER
    }
}

// Enqueue the rungs of `count` products of one transform length; the first
// n32 of them try binary32 first.  Each later rung skips the products an
// earlier rung decided.
ssmul_status enqueue_rungs(ssmul_plan_t p, ssmul_precision prec, const ProdDesc* d_desc,
                           int count, int n32, const Geom& g) {
    int mask = 0;
    if (n32 > 0) {
        ssmul_status s = enqueue_rung_idx(p, 0, d_desc, n32, g, 0);
        if (s != SSMUL_OK) return s;
        mask |= 1;
    }
    int rungs[4];
    const int nr = later_rungs(prec, rungs);
    for (int k = 0; k < nr; ++k) {
        ssmul_status s = enqueue_rung_idx(p, rungs[k], d_desc, count, g, mask);
        if (s != SSMUL_OK) return s;
        mask |= 1 << rungs[k];
    }
    return SSMUL_OK;
}

// Digit prefix sums of `count` products (balanced digits only).
ssmul_status enqueue_prefix(ssmul_plan_t p, const ProdDesc* d_desc, int count, size_t max_n) {
    if (!p->balanced) return SSMUL_OK;
    {
        LaunchScope ls(p, SSMUL_K_PREFIX);
        k_prefix<<<dim3(unsigned((max_n + PRE_TILE - 1) / PRE_TILE), unsigned(count), 2),
                   PRE_THREADS, 0, p->cur>>>(d_desc);
    }
    {
        LaunchScope ls(p, SSMUL_K_PREFIX);
        k_prefix_tiles<<<dim3(unsigned(count), 2), 32, 0, p->cur>>>(d_desc);
    }
    return cuda_status(cudaGetLastError());
}

// Enqueue one complete product (rungs, carry, outcome) for d_desc[0].
ssmul_status enqueue_product(ssmul_plan_t p, const ProdDesc* d_desc, size_t na, size_t nb,
                             ssmul_precision prec) {
    const Geom& g = p->geom[length_code(na, nb, p->lengths)];
    {
        ssmul_status s0 = enqueue_prefix(p, d_desc, 1, na > nb ? na : nb);
        if (s0 != SSMUL_OK) return s0;
    }
    const bool try32 = prec == SSMUL_PREC_FP32 ||
                       (uses_fp32(prec) && fp32_eligible(p, na, nb, g.log_n));
    ssmul_status s = enqueue_rungs(p, prec, d_desc, 1, try32 ? 1 : 0, g);
    if (s != SSMUL_OK) return s;
    const size_t tiles = carry_tiles(na + nb);
    {
        LaunchScope ls(p, SSMUL_K_CARRY);
        k_carry<<<dim3(unsigned(tiles), 1), CARRY_THREADS, 0, p->stream>>>(d_desc);
    }
    {
        LaunchScope ls(p, SSMUL_K_FINALIZE);
        k_finalize<<<1, 256, 0, p->stream>>>(d_desc);
    }
    return cuda_status(cudaGetLastError());
}

ssmul_status check_device(ssmul_plan_t p) {
    int cur = -1;
    SS_TRY(cudaGetDevice(&cur));
    if (cur != p->device) SS_TRY(cudaSetDevice(p->device));
    return SSMUL_OK;
}

ProdDesc single_desc(ssmul_plan_t p, const uint8_t* a, size_t na, const uint8_t* b, size_t nb,
                     uint8_t* z, size_t slot) {
    ProdDesc d{};
    d.a = a;
    d.b = b;
    d.z = z;
    d.na = uint32_t(na);
    d.nb = uint32_t(nb);
    d.log_n = length_code(na, nb, p->lengths);
    d.Z = p->Z;
    d.W = p->W;
    d.coeff = p->coeff;
    d.flags = p->flags + slot * p->flags_per_product;
    d.st = p->st + slot;
    d.res = p->d_res + slot;
    d.iv = nullptr;
    d.balanced = p->balanced ? 1 : 0;
    d.fault_widen = p->fault_widen;
    d.fault_stall = p->fault_stall;
    d.fp32_nib = (p->fp32_nibbles && na + nb <= size_t(NIB_MAX_DIGITS)) ? 1 : 0;
    d.coef_nz = 0;
    d.pre_a = p->pre;
    d.pre_b = p->pre + pre_words(p->max_na);
    return d;
}

// The parts of a product of na x nb digits cut into at most m digits per
// operand: ceil(na / m) ceil(nb / m).
size_t split_parts(size_t na, size_t nb, size_t m) { return ((na + m - 1) / m) * ((nb + m - 1) / m); }

// Room for `parts` part descriptors and states (grown after waiting for the
// plan's queued work).
ssmul_status ensure_split_capacity(ssmul_plan_t p, size_t parts) {
    if (parts <= p->split_slots) return SSMUL_OK;
    SS_TRY(cudaStreamSynchronize(p->stream));
    cudaFree(p->split_st);
    cudaFree(p->d_split);
    cudaFreeHost(p->h_split);
    p->split_st = nullptr;
    p->d_split = nullptr;
    p->h_split = nullptr;
    p->split_slots = 0;
    SS_TRY(cudaMalloc(&p->split_st, parts * sizeof(ProdState)));
    SS_TRY(cudaMalloc(&p->d_split, parts * sizeof(ProdDesc)));
    SS_TRY(cudaMallocHost(&p->h_split, parts * sizeof(ProdDesc)));
    p->split_slots = parts;
    return SSMUL_OK;
}

// Enqueue one product cut into parts of at most m = split_digits digits per
// operand (see k_split_accumulate) on the current lane: parent (host copy)
// and d_parent (its descriptor on the device, uploaded by the caller, whose
// state and look-back words the caller cleared); the parts take entries
// [off, off + parts) of the part arrays.  The parts run one after another
// in the plan's single-product workspace, add their exact coefficients into
// coeff_total, and the parent's carry and outcome follow.
ssmul_status enqueue_split(ssmul_plan_t p, const ProdDesc& parent, const ProdDesc* d_parent,
                           size_t off, ssmul_precision prec) {
    const size_t m = p->split_digits;
    const size_t na = parent.na, nb = parent.nb;
    const size_t ka = (na + m - 1) / m, kb = (nb + m - 1) / m;
    ProdDesc* const hs = p->h_split + off;
    size_t np = 0;
    for (size_t k = 0; k < ka; ++k) {
        for (size_t l = 0; l < kb; ++l, ++np) {
            const size_t la = (k + 1) * m <= na ? m : na - k * m;
            const size_t lb = (l + 1) * m <= nb ? m : nb - l * m;
            ProdDesc d = single_desc(p, parent.a + k * m, la, parent.b + l * m, lb, nullptr, 0);
            d.st = p->split_st + off + np;
            d.res = nullptr;
            d.flags = nullptr;
            hs[np] = d;
        }
    }
    SS_TRY(cudaMemsetAsync(p->split_st + off, 0, np * sizeof(ProdState), p->cur));
    SS_TRY(cudaMemsetAsync(p->coeff_total, 0, (na + nb) * sizeof(int64_t), p->cur));
    SS_TRY(cudaMemcpyAsync(p->d_split + off, hs, np * sizeof(ProdDesc), cudaMemcpyHostToDevice,
                           p->cur));
    ssmul_status s = SSMUL_OK;
    np = 0;
    for (size_t k = 0; k < ka; ++k) {
        for (size_t l = 0; l < kb; ++l, ++np) {
            const ProdDesc& hd = hs[np];
            const ProdDesc* dd = p->d_split + off + np;
            const Geom& g = p->geom[hd.log_n];
            s = enqueue_prefix(p, dd, 1, hd.na > hd.nb ? hd.na : hd.nb);
            if (s != SSMUL_OK) return s;
            const bool try32 = prec == SSMUL_PREC_FP32 ||
                               (uses_fp32(prec) && fp32_eligible(p, hd.na, hd.nb, g.log_n));
            s = enqueue_rungs(p, prec, dd, 1, try32 ? 1 : 0, g);
            if (s != SSMUL_OK) return s;
            const size_t L = size_t(hd.na) + hd.nb;
            k_split_accumulate<<<unsigned((L + 255) / 256 < 1024 ? (L + 255) / 256 : 1024), 256, 0,
                                 p->cur>>>(dd, p->coeff_total, (k + l) * m, parent.st);
            SS_TRY(cudaGetLastError());
        }
    }
    {
        LaunchScope ls(p, SSMUL_K_CARRY);
        k_carry<<<dim3(unsigned(carry_tiles(na + nb)), 1), CARRY_THREADS, 0, p->cur>>>(d_parent);
    }
    {
        LaunchScope ls(p, SSMUL_K_FINALIZE);
        k_finalize<<<1, 256, 0, p->cur>>>(d_parent);
    }
    return cuda_status(cudaGetLastError());
}

// The parent descriptor of a split product in slot `slot`: its
// coefficients are the parts' sums in coeff_total (na + nb of them).
ProdDesc split_parent(ssmul_plan_t p, const uint8_t* a, size_t na, const uint8_t* b, size_t nb,
                      uint8_t* z, size_t slot) {
    ProdDesc d = single_desc(p, a, na, b, nb, z, slot);
    d.coeff = p->coeff_total;
    d.coef_nz = 1;
    d.Z = nullptr;
    d.W = nullptr;
    return d;
}

// One product cut into parts; waits for the result.
ssmul_status run_split(ssmul_plan_t p, const uint8_t* d_a, size_t na, const uint8_t* d_b,
                       size_t nb, uint8_t* d_z, ssmul_result* h_res, ssmul_precision prec) {
    SS_TRY(cudaEventSynchronize(p->desc_free));
    ssmul_status s = ensure_split_capacity(p, split_parts(na, nb, p->split_digits));
    if (s != SSMUL_OK) return s;
    p->h_desc[0] = split_parent(p, d_a, na, d_b, nb, d_z, 0);
    SS_TRY(cudaMemsetAsync(p->st, 0, sizeof(ProdState), p->stream));
    SS_TRY(cudaMemsetAsync(p->flags, 0, carry_tiles(na + nb) * sizeof(uint32_t), p->stream));
    SS_TRY(cudaMemcpyAsync(p->d_desc, p->h_desc, sizeof(ProdDesc), cudaMemcpyHostToDevice,
                           p->stream));
    s = enqueue_split(p, p->h_desc[0], p->d_desc, 0, prec);
    if (s != SSMUL_OK) return s;
    SS_TRY(cudaEventRecord(p->desc_free, p->stream));
    SS_TRY(cudaMemcpyAsync(p->h_res, p->d_res, sizeof(ssmul_result), cudaMemcpyDeviceToHost,
                           p->stream));
    SS_TRY(cudaStreamSynchronize(p->stream));
    if (h_res) *h_res = p->h_res[0];
    return ssmul_status(p->h_res[0].status);
}

// one product on device buffers; fills h_res; waits for the result
ssmul_status run_single(ssmul_plan_t p, const uint8_t* d_a, size_t na, const uint8_t* d_b,
                        size_t nb, uint8_t* d_z, ssmul_result* h_res, ssmul_precision prec,
                        double* d_iv, bool iv_nibbles = false) {
    if (!d_a || !d_b || !d_z || na == 0 || nb == 0) return SSMUL_INVALID_ARG;
    if (na > p->max_na || nb > p->max_nb) return SSMUL_TOO_LARGE;
    ssmul_status s = check_device(p);
    if (s != SSMUL_OK) return s;
    if (p->split_digits && d_iv == nullptr && (na > p->split_digits || nb > p->split_digits))
        return run_split(p, d_a, na, d_b, nb, d_z, h_res, prec);
    SS_TRY(cudaEventSynchronize(p->desc_free));
    p->h_desc[0] = single_desc(p, d_a, na, d_b, nb, d_z, 0);
    p->h_desc[0].iv = d_iv;
    // the exported sets are those of the digits' coefficients, or with
    // iv_nibbles those of the 4-bit digits' (binary32 only)
    if (d_iv) p->h_desc[0].fp32_nib = iv_nibbles ? 1 : 0;
    SS_TRY(cudaMemsetAsync(p->st, 0, sizeof(ProdState), p->stream));
    SS_TRY(cudaMemsetAsync(p->flags, 0, carry_tiles(na + nb) * sizeof(uint32_t), p->stream));
    SS_TRY(cudaMemcpyAsync(p->d_desc, p->h_desc, sizeof(ProdDesc), cudaMemcpyHostToDevice,
                           p->stream));
    SS_TRY(cudaEventRecord(p->desc_free, p->stream));
    s = enqueue_product(p, p->d_desc, na, nb, prec);
    if (s != SSMUL_OK) return s;
    SS_TRY(cudaMemcpyAsync(p->h_res, p->d_res, sizeof(ssmul_result), cudaMemcpyDeviceToHost,
                           p->stream));
    SS_TRY(cudaStreamSynchronize(p->stream));
    if (h_res) *h_res = p->h_res[0];
    return ssmul_status(p->h_res[0].status);
}

// Bytes of arena one product needs (256-byte aligned pieces): the forward
// spectrum Z (N intervals; the integer coefficients reuse it once it is
// consumed) and the half-length inverse W (N/2 intervals) for four-step
// products, the coefficients alone for single-CTA products (N + 1: the 4-bit
// digits of the binary32 rung give na + nb <= N + 1 coefficients).
size_t arena_need(int log_n) {
    const size_t n = len_of(log_n);
    if (log_n <= LOG_SMALL) return ((n + 1) * sizeof(int64_t) + 255) & ~size_t(255);
    return ((n * sizeof(CI<double>) + 255) & ~size_t(255)) +
           (((n / 2) * sizeof(CI<double>) + 255) & ~size_t(255));
}

// Arena bytes of one product of a batch (its workspace at its transform
// length, and its digit prefix sums when the digits are balanced); 0 for a
// product that runs split, outside the arena.
size_t product_arena_bytes(ssmul_plan_t p, const ssmul_desc& hd) {
    const size_t m = p->split_digits;
    if (m && (hd.na > m || hd.nb > m)) return 0;
    return arena_need(length_code(hd.na, hd.nb, p->lengths)) +
           (p->balanced ? pre_bytes(hd.na, hd.nb) : 0);
}

// Host half of a batch: products sorted by transform length (longest
// first) and, inside one length, binary32-eligible products first, so that
// every launch covers a contiguous run of descriptors; descriptors written
// to the pinned array; products packed into the arena in that order, each
// full arena one chunk of launches.
// The batch occupies slots [base, base + count) of the plan's per-product
// arrays (descriptors, states, look-back words), so that the pieces of one
// host-buffer call can be prepared while earlier pieces still wait for
// their descriptor uploads, and bytes [arena_off, arena_off + arena_len) of
// the arena (pieces that run concurrently take disjoint windows).
ssmul_status prepare_batch(ssmul_plan_t p, size_t base, size_t count, const ssmul_desc* h_desc,
                           const uint8_t* d_a_pool, const uint8_t* d_b_pool, uint8_t* d_z_pool,
                           ssmul_result* d_res, size_t arena_off, size_t arena_len) {
    std::vector<int>& order = p->order;
    order.resize(count);
    std::vector<int> logn(count);
    std::vector<char> elig(count), cut(count);
    const size_t m = p->split_digits;
    size_t nsplit = 0;
    for (size_t i = 0; i < count; ++i) {
        order[i] = int(i);
        logn[i] = length_code(h_desc[i].na, h_desc[i].nb, p->lengths);
        elig[i] = p->prec == SSMUL_PREC_FP32 ||
                  (uses_fp32(p->prec) && fp32_eligible(p, h_desc[i].na, h_desc[i].nb, logn[i]));
        cut[i] = m && (h_desc[i].na > m || h_desc[i].nb > m);
        nsplit += cut[i];
    }
    // products past SSMUL_OPT_SPLIT_DIGITS go last: they run in parts after
    // the others (issue_batch), outside the length groups and the arena
    std::sort(order.begin(), order.end(), [&](int x, int y) {
        if (cut[x] != cut[y]) return cut[x] < cut[y];
        if (logn[x] != logn[y]) return logn[x] > logn[y];
        if (elig[x] != elig[y]) return elig[x] > elig[y];
        return x < y;
    });
    const size_t nreg = count - nsplit;
    for (size_t k = 0; k < count; ++k) {
        const int i = order[k];
        const ssmul_desc& h = h_desc[i];
        ProdDesc d = k < nreg ? single_desc(p, d_a_pool + h.a_off, h.na, d_b_pool + h.b_off, h.nb,
                                            d_z_pool + h.z_off, base + k)
                              : split_parent(p, d_a_pool + h.a_off, h.na, d_b_pool + h.b_off, h.nb,
                                             d_z_pool + h.z_off, base + k);
        d.res = d_res + i;
        p->h_desc[base + k] = d;
    }
    p->batch_nreg = nreg;
    p->chunks.clear();
    size_t k0 = 0;
    while (k0 < nreg) {
        BatchChunk c;
        c.k0 = k0;
        size_t used = 0, k1 = k0;
        while (k1 < nreg) {
            const int ln = logn[order[k1]];
            const ssmul_desc& hd = h_desc[order[k1]];
            const size_t pb = p->balanced ? pre_bytes(hd.na, hd.nb) : 0;
            const size_t need = product_arena_bytes(p, hd);
            if (used + need > arena_len) break;
            ProdDesc& d = p->h_desc[base + k1];
            unsigned char* const ws = p->arena + arena_off + used;   // this product's workspace
            if (pb) {
                d.pre_a = reinterpret_cast<uint32_t*>(ws + arena_need(ln));
                d.pre_b = d.pre_a + pre_words(hd.na);
            }
            if (ln <= LOG_SMALL) {
                d.Z = nullptr;
                d.W = nullptr;
            } else {
                const size_t zb = (len_of(ln) * sizeof(CI<double>) + 255) & ~size_t(255);
                d.Z = ws;
                d.W = ws + zb;
            }
            d.coeff = reinterpret_cast<int64_t*>(ws);
            used += need;
            ++k1;
        }
        if (k1 == k0) return SSMUL_OUT_OF_MEMORY;
        c.k1 = k1;
        size_t g0 = k0;
        while (g0 < k1) {
            BatchGroup g;
            g.g0 = g0;
            g.log_n = logn[order[g0]];
            g.e1 = g0;
            g.max_nz = 0;
            size_t g1 = g0;
            while (g1 < k1 && logn[order[g1]] == g.log_n) {
                if (elig[order[g1]]) g.e1 = g1 + 1;
                const size_t nz = size_t(h_desc[order[g1]].na) + h_desc[order[g1]].nb;
                if (nz > g.max_nz) g.max_nz = nz;
                ++g1;
            }
            g.g1 = g1;
            c.groups.push_back(g);
            g0 = g1;
        }
        p->chunks.push_back(std::move(c));
        k0 = k1;
    }
    return SSMUL_OK;
}

// Device half of a batch: every stream operation of the batch prepared in
// slots [base, base + count).  With fork_groups and more than one group
// lane, the length groups of a chunk (independent until the chunk's
// outcomes) run on up to group_lanes lanes: each group goes to the lane
// with the least work so far (the groups come longest first), the lanes
// fork from the plan's stream after the chunk's descriptor upload and join
// it before the chunk's outcomes are written.
ssmul_status issue_batch(ssmul_plan_t p, size_t base, size_t count, bool fork_groups = false) {
    ssmul_status s = SSMUL_OK;
    ProdDesc* const dd = p->d_desc + base;
    // the stream and gate list the batch was issued on (a host-buffer
    // piece's own); group lane 0 is that stream
    cudaStream_t const origin = p->cur;
    int* const origin_gate = p->cur_gate;
    const int lanes = fork_groups && origin == p->stream ? p->group_lanes : 1;
    SS_TRY(cudaMemsetAsync(p->st + base, 0, count * sizeof(ProdState), p->cur));
    SS_TRY(cudaMemsetAsync(p->flags + base * p->flags_per_product, 0,
                           count * p->flags_per_product * sizeof(uint32_t), p->cur));
    for (const BatchChunk& c : p->chunks) {
        SS_TRY(cudaMemcpyAsync(dd + c.k0, p->h_desc + base + c.k0,
                               (c.k1 - c.k0) * sizeof(ProdDesc), cudaMemcpyHostToDevice,
                               p->cur));
        s = enqueue_prefix(p, dd + c.k0, int(c.k1 - c.k0),
                           p->max_na > p->max_nb ? p->max_na : p->max_nb);
        if (s != SSMUL_OK) return s;
        const int nl = std::min<int>(lanes, int(c.groups.size()));
        if (nl > 1) {
            SS_TRY(cudaEventRecord(p->lane_ev[0], origin));
            for (int l = 1; l < nl; ++l) SS_TRY(cudaStreamWaitEvent(p->lane_stream[l], p->lane_ev[0], 0));
        }
        double load[LANES] = {};
        for (const BatchGroup& g : c.groups) {
            int lane = 0;
            for (int l = 1; l < nl; ++l)
                if (load[l] < load[lane]) lane = l;
            const double n = double(len_of(g.log_n));
            load[lane] += double(g.g1 - g.g0) * n * std::log2(n);
            OnLane on(p, lane ? p->lane_stream[lane] : origin, lane ? p->lane_gate[lane] : origin_gate);
            const Geom& geo = p->geom[g.log_n];
            s = enqueue_rungs(p, p->prec, dd + g.g0, int(g.g1 - g.g0), int(g.e1 - g.g0), geo);
            if (s != SSMUL_OK) return s;
            {
                LaunchScope ls(p, SSMUL_K_CARRY);
                k_carry<<<dim3(unsigned(carry_tiles(g.max_nz)), unsigned(g.g1 - g.g0)),
                          CARRY_THREADS, 0, p->cur>>>(dd + g.g0);
            }
            SS_TRY(cudaGetLastError());
        }
        for (int l = 1; l < nl; ++l) {
            SS_TRY(cudaEventRecord(p->lane_ev[l], p->lane_stream[l]));
            SS_TRY(cudaStreamWaitEvent(origin, p->lane_ev[l], 0));
        }
        {
            LaunchScope ls(p, SSMUL_K_FINALIZE);
            k_finalize<<<unsigned(c.k1 - c.k0), 256, 0, p->cur>>>(dd + c.k0);
        }
        SS_TRY(cudaGetLastError());
    }
    // products past the split size, one after another in parts (Section 1's
    // "different algorithm"); their part entries follow the call's cursor
    const size_t nreg = p->batch_nreg;
    if (nreg < count) {
        SS_TRY(cudaMemcpyAsync(dd + nreg, p->h_desc + base + nreg, (count - nreg) * sizeof(ProdDesc),
                               cudaMemcpyHostToDevice, p->cur));
        for (size_t k = nreg; k < count; ++k) {
            const ProdDesc& hd = p->h_desc[base + k];
            s = enqueue_split(p, hd, dd + k, p->split_cursor, p->prec);
            if (s != SSMUL_OK) return s;
            p->split_cursor += split_parts(hd.na, hd.nb, p->split_digits);
        }
    }
    return SSMUL_OK;
}

bool graph_key_matches(const GraphEntry& e, size_t count, const ssmul_desc* h_desc,
                       const void* a, const void* b, const void* z, const void* res) {
    return e.valid && e.key.size() == count && e.a == a && e.b == b && e.z == z &&
           e.res == res && std::memcmp(e.key.data(), h_desc, count * sizeof(ssmul_desc)) == 0;
}

void graph_drop(GraphEntry& e) {
    if (e.exec) cudaGraphExecDestroy(e.exec);
    e = GraphEntry();
}

// Part entries the products of a batched call past SSMUL_OPT_SPLIT_DIGITS
// need (they take consecutive entries from the call's cursor).
size_t batch_split_parts(ssmul_plan_t p, size_t count, const ssmul_desc* h_desc) {
    const size_t m = p->split_digits;
    size_t parts = 0;
    for (size_t i = 0; m && i < count; ++i)
        if (h_desc[i].na > m || h_desc[i].nb > m) parts += split_parts(h_desc[i].na, h_desc[i].nb, m);
    return parts;
}

ssmul_status enqueue_batch(ssmul_plan_t p, size_t count, const ssmul_desc* h_desc,
                           const uint8_t* d_a_pool, const uint8_t* d_b_pool, uint8_t* d_z_pool,
                           ssmul_result* d_res) {
    SS_TRY(cudaEventSynchronize(p->desc_free));
    const size_t parts = batch_split_parts(p, count, h_desc);
    if (parts) {
        const ssmul_status sc = ensure_split_capacity(p, parts);
        if (sc != SSMUL_OK) return sc;
    }
    p->split_cursor = 0;
    // a stream capture needs a stream other than the legacy default stream;
    // batches with split products run their parts' descriptors from the
    // host arrays of this call, so they are not captured
    const bool use_graph = p->graph && p->stream != nullptr && parts == 0;
    if (use_graph &&
        graph_key_matches(p->cached, count, h_desc, d_a_pool, d_b_pool, d_z_pool, d_res)) {
        std::memcpy(p->h_desc, p->cached.prepared.data(), count * sizeof(ProdDesc));
        SS_TRY(cudaGraphLaunch(p->cached.exec, p->stream));
        for (int k = 0; k < SSMUL_KERNEL_KINDS; ++k) p->kt_launches[k] += p->cached.launches[k];
        SS_TRY(cudaEventRecord(p->desc_free, p->stream));
        return SSMUL_OK;
    }
    ssmul_status s = prepare_batch(p, 0, count, h_desc, d_a_pool, d_b_pool, d_z_pool, d_res, 0,
                                   p->arena_bytes);
    if (s != SSMUL_OK) return s;
    if ((s = ensure_lanes(p, p->group_lanes)) != SSMUL_OK) return s;
    if (!use_graph) {
        s = issue_batch(p, 0, count, true);
        if (s != SSMUL_OK) return s;
        SS_TRY(cudaEventRecord(p->desc_free, p->stream));
        return SSMUL_OK;
    }
    graph_drop(p->cached);
    std::memset(p->cap_launches, 0, sizeof(p->cap_launches));
    SS_TRY(cudaStreamBeginCapture(p->stream, cudaStreamCaptureModeThreadLocal));
    p->capturing = true;
    s = issue_batch(p, 0, count, true);
    p->capturing = false;
    cudaGraph_t graph = nullptr;
    const cudaError_t ec = cudaStreamEndCapture(p->stream, &graph);
    if (s != SSMUL_OK) {
        if (graph) cudaGraphDestroy(graph);
        return s;
    }
    SS_TRY(ec);
    cudaGraphExec_t exec = nullptr;
    const cudaError_t ei = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    SS_TRY(ei);
    GraphEntry& e = p->cached;
    e.valid = true;
    e.key.assign(h_desc, h_desc + count);
    e.a = d_a_pool;
    e.b = d_b_pool;
    e.z = d_z_pool;
    e.res = d_res;
    e.prepared.assign(p->h_desc, p->h_desc + count);
    e.exec = exec;
    std::memcpy(e.launches, p->cap_launches, sizeof(e.launches));
    SS_TRY(cudaGraphLaunch(exec, p->stream));
    for (int k = 0; k < SSMUL_KERNEL_KINDS; ++k) p->kt_launches[k] += e.launches[k];
    SS_TRY(cudaEventRecord(p->desc_free, p->stream));
    return SSMUL_OK;
}

// ---- autotuner ------------------------------------------------------------------
//
// For every four-step length of the plan the tuner times the binary64 rung
// of a synthetic batch (all digits 0xA7, count = clamp(2^23 / N, 1, 64))
// under every candidate geometry: the split log2 N2 in {h-1, h, h+1}
// (h = ceil(log2 N / 2), where valid) and column CTAs of 2^9, 2^10 or 2^11
// elements.  The fastest (minimum of 3 timed runs after one warm-up)
// becomes the plan's geometry.  Results are cached in the text file named
// by SSMUL_TUNE_CACHE (device name, log2 N, log2 N2, log2 CTA elements).

std::string device_name(int dev) {
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, dev) != cudaSuccess) return "unknown";
    std::string s(prop.name);
    for (char& c : s)
        if (c == '\t' || c == '\n') c = ' ';
    return s;
}

void tune_cache_read(const std::string& dev, std::vector<Geom>& found) {
    const char* path = std::getenv("SSMUL_TUNE_CACHE");
    if (!path) return;
    FILE* f = std::fopen(path, "r");
    if (!f) return;
    char line[512];
    while (std::fgets(line, sizeof(line), f)) {
        char* tab = std::strchr(line, '\t');
        if (!tab) continue;
        *tab = 0;
        int ln, ln2, cta;
        if (dev == line && std::sscanf(tab + 1, "%d %d %d", &ln, &ln2, &cta) == 3 &&
            cta >= 9 && cta <= 12) {
            if (ln > LOG_SMALL && ln <= LOG_N_MAX && geom_valid(ln, ln2))
                found.push_back(make_geom(ln, ln2, cta));
            else if (ln >= LEN3 && ln < GEOM_CODES && geom_odd_valid(odd_of(ln), log2_of(ln), ln2))
                found.push_back(make_geom_odd(odd_of(ln), log2_of(ln), ln2, cta));
        }
    }
    std::fclose(f);
}

void tune_cache_append(const std::string& dev, const Geom& g) {
    const char* path = std::getenv("SSMUL_TUNE_CACHE");
    if (!path) return;
    FILE* f = std::fopen(path, "a");
    if (!f) return;
    std::fprintf(f, "%s\t%d %d %d\n", dev.c_str(), g.log_n, g.log_n2, g.log_cta);
    std::fclose(f);
}

ssmul_status autotune(ssmul_plan_t p) {
    const std::string dev = device_name(p->device);
    std::vector<Geom> cached;
    tune_cache_read(dev, cached);
    // the length codes the plan can use
    std::vector<int> codes;
    for (int ln = LOG_SMALL + 1; ln <= p->log_n_max; ++ln) codes.push_back(ln);
    for (int j = LOG3_MIN; p->fam[1].log_tab && j <= p->fam[1].log_tab; ++j) codes.push_back(LEN3 + j);
    for (int j = LOG5_MIN; p->fam[2].log_tab && j <= p->fam[2].log_tab; ++j) codes.push_back(LEN5 + j);
    std::vector<int> todo;
    for (int ln : codes) {
        bool have = false;
        for (const Geom& g : cached) {
            if (g.log_n == ln) {
                p->geom[ln] = g;
                have = true;
            }
        }
        if (!have) todo.push_back(ln);
    }
    if (todo.empty()) return SSMUL_OK;
    auto batch_count = [](int ln) { return clampi(int((size_t(1) << 23) / len_of(ln)), 1, 64); };
    size_t ws_bytes = 0, n_max = 0;
    for (int ln : todo) {
        const size_t b = arena_need(ln) * size_t(batch_count(ln));
        if (b > ws_bytes) ws_bytes = b;
        if (len_of(ln) > n_max) n_max = len_of(ln);
    }
    void* ws = nullptr;
    uint8_t* digits = nullptr;
    ProdDesc* dd = nullptr;
    ProdState* ds = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    ssmul_status s = SSMUL_OK;
    auto done = [&](ssmul_status r) {
        cudaStreamSynchronize(p->stream);
        cudaFree(ws);
        cudaFree(digits);
        cudaFree(dd);
        cudaFree(ds);
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
        return r;
    };
    if (cudaMalloc(&ws, ws_bytes) != cudaSuccess ||
        cudaMalloc(&digits, n_max / 2 + 1) != cudaSuccess ||
        cudaMalloc(&dd, 64 * sizeof(ProdDesc)) != cudaSuccess ||
        cudaMalloc(&ds, 64 * sizeof(ProdState)) != cudaSuccess)
        return done(SSMUL_OUT_OF_MEMORY);
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
        return done(SSMUL_CUDA_ERROR);
    if (cudaMemsetAsync(digits, 0xA7, n_max / 2 + 1, p->stream) != cudaSuccess)
        return done(SSMUL_CUDA_ERROR);
    const bool was_timing = p->timing;
    p->timing = false;
    for (int ln : todo) {
        const size_t n = len_of(ln);
        const int cnt = batch_count(ln);
        std::vector<ProdDesc> hd(cnt);
        for (int i = 0; i < cnt; ++i) {
            ProdDesc d{};
            d.a = digits;
            d.b = digits;
            d.na = d.nb = uint32_t(n / 2);
            d.log_n = ln;
            unsigned char* base = static_cast<unsigned char*>(ws) + size_t(i) * arena_need(ln);
            d.Z = base;
            d.W = base + (((n * sizeof(CI<double>)) + 255) & ~size_t(255));
            d.coeff = reinterpret_cast<int64_t*>(base);
            d.st = ds + i;
            hd[i] = d;
        }
        if (cudaMemcpy(dd, hd.data(), cnt * sizeof(ProdDesc), cudaMemcpyHostToDevice) !=
            cudaSuccess)
            return done(SSMUL_CUDA_ERROR);
        const bool three = ln >= LEN3;                // an odd family (3 or 5)
        const int k = log2_of(ln), R = odd_of(ln);
        const int h = (k + 1) / 2;
        float best = 1e30f;
        Geom best_g = p->geom[ln];
        // family 3: the column exponent must stay even, so try two steps either way
        for (int ln2 = h - (three ? 2 : 1); ln2 <= h + (three ? 2 : 1); ++ln2) {
            if (three ? !geom_odd_valid(R, k, ln2) : !geom_valid(ln, ln2)) continue;
            for (int cta = 9; cta <= 11; ++cta) {
                const Geom g = three ? make_geom_odd(R, k, ln2, cta) : make_geom(ln, ln2, cta);
                float t_min = 1e30f;
                for (int rep = 0; rep < 4; ++rep) {
                    if (cudaMemsetAsync(ds, 0, cnt * sizeof(ProdState), p->stream) != cudaSuccess)
                        return done(SSMUL_CUDA_ERROR);
                    cudaEventRecord(e0, p->stream);
                    s = enqueue_rung<double>(p, dd, cnt, g, 0);
                    cudaEventRecord(e1, p->stream);
                    if (s != SSMUL_OK) return done(s);
                    if (cudaEventSynchronize(e1) != cudaSuccess) return done(SSMUL_CUDA_ERROR);
                    float t = 0.f;
                    cudaEventElapsedTime(&t, e0, e1);
                    if (rep > 0 && t < t_min) t_min = t;
                }
                if (t_min < best) {
                    best = t_min;
                    best_g = g;
                }
            }
        }
        p->geom[ln] = best_g;
        tune_cache_append(dev, best_g);
    }
    p->timing = was_timing;
    return done(SSMUL_OK);
}

// ---- host-buffer batches --------------------------------------------------------

// Grows a device buffer to hold at least `need` bytes (waits for the plan's
// queued work before the old buffer is released).
template <typename T>
ssmul_status grow_device(ssmul_plan_t p, T*& buf, size_t& cap, size_t need) {
    if (need <= cap && buf) return SSMUL_OK;
    SS_TRY(cudaStreamSynchronize(p->stream));
    cudaFree(buf);
    buf = nullptr;
    cap = 0;
    const size_t bytes = (need + (size_t(1) << 20) - 1) & ~((size_t(1) << 20) - 1);
    SS_TRY(cudaMalloc(reinterpret_cast<void**>(&buf), bytes));
    cap = bytes;
    return SSMUL_OK;
}

// Byte ranges [lo, hi) merged where they overlap or touch, in ascending order.
void merge_ranges(std::vector<std::pair<uint64_t, uint64_t>>& r) {
    std::sort(r.begin(), r.end());
    size_t w = 0;
    for (size_t i = 0; i < r.size(); ++i) {
        if (w && r[i].first <= r[w - 1].second) {
            if (r[i].second > r[w - 1].second) r[w - 1].second = r[i].second;
        } else {
            r[w++] = r[i];
        }
    }
    r.resize(w);
}

// Uploads of one operand pool in ascending offset order: upload(end) copies
// every byte of the pool's merged ranges below `end` not copied yet.
struct PoolUpload {
    std::vector<std::pair<uint64_t, uint64_t>> ranges;
    size_t next = 0;
    uint64_t pos = 0;
    ssmul_status upload(uint64_t end, uint8_t* dev, uint64_t lo, const uint8_t* host,
                        cudaStream_t st) {
        while (next < ranges.size() && ranges[next].first < end) {
            const uint64_t a = ranges[next].first > pos ? ranges[next].first : pos;
            const uint64_t b = ranges[next].second < end ? ranges[next].second : end;
            if (b > a) SS_TRY(cudaMemcpyAsync(dev + (a - lo), host + a, b - a,
                                              cudaMemcpyHostToDevice, st));
            if (ranges[next].second <= end) {
                pos = ranges[next].second;
                ++next;
            } else {
                pos = end;
                break;
            }
        }
        return SSMUL_OK;
    }
};

// First descriptor of piece k of a host-buffer batch cut into `pieces`
// pieces (k = pieces: count).  With three or more pieces the first and the
// last take about a sixteenth of the batch each (at least one product): the
// first piece's upload and the last one's download are the copies no
// computation hides.
size_t piece_start(size_t count, size_t pieces, size_t k) {
    if (k == 0) return 0;
    if (k >= pieces) return count;
    if (pieces < 3) return count * k / pieces;
    const size_t edge = std::max<size_t>(1, count / 16);
    if (count < 2 * edge + (pieces - 2)) return count * k / pieces;
    const size_t mid = count - 2 * edge;
    return edge + mid * (k - 1) / (pieces - 2);
}

// The pieces of a host-buffer batch, in the caller's descriptor order:
// piece k waits for the uploads that reach its operands' last byte, runs
// as a batch in slots [i0, i1) of the plan's arrays, and its digits and
// outcomes are copied back once it is done.  Every compute piece is
// enqueued before the first download, so pageable destination memory
// (whose copies hold the calling thread) leaves no gap on the GPU.
ssmul_status run_batched_host(ssmul_plan_t p, size_t count, const ssmul_desc* h_desc,
                              const uint8_t* h_a, const uint8_t* h_b, uint8_t* h_z,
                              ssmul_result* h_res) {
    uint64_t a_lo = UINT64_MAX, a_hi = 0, b_lo = UINT64_MAX, b_hi = 0, z_lo = UINT64_MAX, z_hi = 0;
    for (size_t i = 0; i < count; ++i) {
        const ssmul_desc& d = h_desc[i];
        a_lo = std::min(a_lo, d.a_off);
        a_hi = std::max(a_hi, d.a_off + d.na);
        b_lo = std::min(b_lo, d.b_off);
        b_hi = std::max(b_hi, d.b_off + d.nb);
        z_lo = std::min(z_lo, d.z_off);
        z_hi = std::max(z_hi, d.z_off + d.na + d.nb);
    }
    ssmul_status s = SSMUL_OK;
    if ((s = grow_device(p, p->hb_a, p->hb_a_cap, a_hi - a_lo)) != SSMUL_OK) return s;
    if ((s = grow_device(p, p->hb_b, p->hb_b_cap, b_hi - b_lo)) != SSMUL_OK) return s;
    if ((s = grow_device(p, p->hb_z, p->hb_z_cap, z_hi - z_lo)) != SSMUL_OK) return s;
    if (!p->hb_res) {
        SS_TRY(cudaMalloc(&p->hb_res, (p->max_products ? p->max_products : 1) * sizeof(ssmul_result)));
    }
    if (!p->up) SS_TRY(cudaStreamCreateWithFlags(&p->up, cudaStreamNonBlocking));
    if (!p->down) SS_TRY(cudaStreamCreateWithFlags(&p->down, cudaStreamNonBlocking));
    const size_t pieces = std::min(count, size_t(p->host_pieces));
    // The pieces run on internal streams of decreasing priority with
    // disjoint windows of the arena: the block scheduler starts a later
    // piece's thread blocks only where an earlier piece leaves SMs idle (its
    // last waves), so the pieces finish in order, each download overlaps the
    // next pieces' work, and no piece waits for another's tail.  Fewer
    // streams when a window could not hold a product of the plan's largest
    // size (a piece reuses a stream, and its window, after the piece before).
    const size_t one = arena_need(p->log_n_max) + pre_bytes(p->max_na, p->max_nb);
    int lanes = ensure_piece_lanes(p, int(pieces), &s);
    if (s != SSMUL_OK) return s;
    while (lanes > 1 && ((p->arena_bytes / lanes) & ~size_t(255)) < one) --lanes;
    // split products share the plan's single-product workspace: their pieces
    // run on one stream
    const size_t parts = batch_split_parts(p, count, h_desc);
    if (parts) {
        lanes = 1;
        if ((s = ensure_split_capacity(p, parts)) != SSMUL_OK) return s;
    }
    p->split_cursor = 0;
    // each lane's window of the arena: what its largest piece needs (at
    // least one product of the plan's largest size), when those fit the
    // arena together, so that no piece is cut into chunks; else equal shares
    std::vector<size_t> win_off(lanes, 0), win_len(lanes, p->arena_bytes);
    if (lanes > 1) {
        const size_t eq = (p->arena_bytes / lanes) & ~size_t(255);
        std::vector<size_t> need(lanes, (one + 255) & ~size_t(255));
        for (size_t k = 0; k < pieces; ++k) {
            size_t b = 0;
            for (size_t i = piece_start(count, pieces, k); i < piece_start(count, pieces, k + 1); ++i)
                b += product_arena_bytes(p, h_desc[i]);
            b = (b + 255) & ~size_t(255);
            need[k % lanes] = std::max(need[k % lanes], b);
        }
        size_t total = 0;
        for (int l = 0; l < lanes; ++l) total += need[l];
        const bool fit = total <= p->arena_bytes;
        for (int l = 0; l < lanes; ++l) {
            win_len[l] = fit ? need[l] : eq;
            win_off[l] = fit ? (l ? win_off[l - 1] + win_len[l - 1] : 0) : size_t(l) * eq;
        }
    }
    while (p->hb_ev.size() < 2 * pieces) {
        cudaEvent_t e = nullptr;
        SS_TRY(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
        p->hb_ev.push_back(e);
    }
    // descriptors rebased onto the device copies of the pools
    std::vector<ssmul_desc> rd(h_desc, h_desc + count);
    PoolUpload ua, ub;
    ua.ranges.resize(count);
    ub.ranges.resize(count);
    for (size_t i = 0; i < count; ++i) {
        ua.ranges[i] = {h_desc[i].a_off, h_desc[i].a_off + h_desc[i].na};
        ub.ranges[i] = {h_desc[i].b_off, h_desc[i].b_off + h_desc[i].nb};
        rd[i].a_off -= a_lo;
        rd[i].b_off -= b_lo;
        rd[i].z_off -= z_lo;
    }
    merge_ranges(ua.ranges);
    merge_ranges(ub.ranges);
    SS_TRY(cudaEventSynchronize(p->desc_free));
    // on an error after the first copy, wait for everything queued before
    // returning, so no copy into the caller's memory outlives the call
    auto drain = [&](ssmul_status e) {
        cudaStreamSynchronize(p->up);
        cudaStreamSynchronize(p->stream);
        for (int l = 0; l < lanes; ++l) cudaStreamSynchronize(p->piece_stream[l]);
        cudaStreamSynchronize(p->down);
        return e;
    };
    // the pieces follow the work already queued on the plan's stream
    SS_TRY(cudaEventRecord(p->piece_ev[0], p->stream));
    for (int l = 0; l < lanes; ++l)
        if (cudaStreamWaitEvent(p->piece_stream[l], p->piece_ev[0], 0) != cudaSuccess)
            return drain(SSMUL_CUDA_ERROR);
    for (size_t k = 0; k < pieces; ++k) {
        const size_t i0 = piece_start(count, pieces, k), i1 = piece_start(count, pieces, k + 1);
        uint64_t ea = 0, eb = 0;
        for (size_t i = i0; i < i1; ++i) {
            ea = std::max(ea, h_desc[i].a_off + h_desc[i].na);
            eb = std::max(eb, h_desc[i].b_off + h_desc[i].nb);
        }
        if ((s = ua.upload(ea, p->hb_a, a_lo, h_a, p->up)) != SSMUL_OK) return drain(s);
        if ((s = ub.upload(eb, p->hb_b, b_lo, h_b, p->up)) != SSMUL_OK) return drain(s);
        cudaEvent_t in = p->hb_ev[2 * k], done = p->hb_ev[2 * k + 1];
        const int lane = int(k % lanes);
        OnLane on(p, p->piece_stream[lane], p->piece_gate[lane]);
        if (cudaEventRecord(in, p->up) != cudaSuccess ||
            cudaStreamWaitEvent(p->cur, in, 0) != cudaSuccess)
            return drain(SSMUL_CUDA_ERROR);
        s = prepare_batch(p, i0, i1 - i0, rd.data() + i0, p->hb_a, p->hb_b, p->hb_z,
                          p->hb_res + i0, win_off[lane], win_len[lane]);
        if (s == SSMUL_OK) s = issue_batch(p, i0, i1 - i0);
        if (s != SSMUL_OK) return drain(s);
        if (cudaEventRecord(done, p->cur) != cudaSuccess) return drain(SSMUL_CUDA_ERROR);
    }
    // the plan's stream joins the pieces' streams, so later work on it
    // follows the call
    for (int l = 0; l < lanes; ++l) {
        if (cudaEventRecord(p->piece_ev[1 + l], p->piece_stream[l]) != cudaSuccess ||
            cudaStreamWaitEvent(p->stream, p->piece_ev[1 + l], 0) != cudaSuccess)
            return drain(SSMUL_CUDA_ERROR);
    }
    if (cudaEventRecord(p->desc_free, p->stream) != cudaSuccess) return drain(SSMUL_CUDA_ERROR);
    std::vector<std::pair<uint64_t, uint64_t>> zr;
    for (size_t k = 0; k < pieces; ++k) {
        const size_t i0 = piece_start(count, pieces, k), i1 = piece_start(count, pieces, k + 1);
        if (cudaStreamWaitEvent(p->down, p->hb_ev[2 * k + 1], 0) != cudaSuccess)
            return drain(SSMUL_CUDA_ERROR);
        zr.clear();
        for (size_t i = i0; i < i1; ++i)
            zr.push_back({h_desc[i].z_off, h_desc[i].z_off + h_desc[i].na + h_desc[i].nb});
        merge_ranges(zr);
        for (const auto& r : zr) {
            if (cudaMemcpyAsync(h_z + r.first, p->hb_z + (r.first - z_lo), r.second - r.first,
                                cudaMemcpyDeviceToHost, p->down) != cudaSuccess)
                return drain(SSMUL_CUDA_ERROR);
        }
        if (cudaMemcpyAsync(h_res + i0, p->hb_res + i0, (i1 - i0) * sizeof(ssmul_result),
                            cudaMemcpyDeviceToHost, p->down) != cudaSuccess)
            return drain(SSMUL_CUDA_ERROR);
    }
    const cudaError_t e = cudaStreamSynchronize(p->down);
    if (e != cudaSuccess) return drain(cuda_status(e));
    return drain(SSMUL_OK);
}

}  // namespace

extern "C" {

const char* ssmul_status_string(ssmul_status s) {
    switch (s) {
        case SSMUL_OK: return "SSMUL_OK";
        case SSMUL_ISOLATION_FAILED: return "SSMUL_ISOLATION_FAILED";
        case SSMUL_CONTAINMENT_FAILED: return "SSMUL_CONTAINMENT_FAILED";
        case SSMUL_INVALID_ARG: return "SSMUL_INVALID_ARG";
        case SSMUL_TOO_LARGE: return "SSMUL_TOO_LARGE";
        case SSMUL_CUDA_ERROR: return "SSMUL_CUDA_ERROR";
        case SSMUL_OUT_OF_MEMORY: return "SSMUL_OUT_OF_MEMORY";
        case SSMUL_TIMEOUT: return "SSMUL_TIMEOUT";
        case SSMUL_UNVERIFIED: return "SSMUL_UNVERIFIED";
    }
    return "SSMUL_UNKNOWN_STATUS";
}

void ssmul_plan_destroy(ssmul_plan_t p) {
    if (!p) return;
    int cur = -1;
    cudaGetDevice(&cur);
    if (cur != p->device) cudaSetDevice(p->device);
    if (p->stream) cudaStreamSynchronize(p->stream);
    else cudaDeviceSynchronize();
    graph_drop(p->cached);
    for (TwFamily& F : p->fam) {
        cudaFree(F.t64);
        cudaFree(F.t32);
        cudaFree(F.td);
        cudaFree(F.tdd);
        cudaFree(F.s64);
        cudaFree(F.s32);
        cudaFree(F.sd);
        cudaFree(F.sdd);
        cudaFree(F.scal);
    }
    cudaFree(p->rho);
    cudaFree(p->Z);
    cudaFree(p->W);
    cudaFree(p->coeff);
    cudaFree(p->flags);
    cudaFree(p->st);
    cudaFree(p->d_desc);
    cudaFree(p->gate_list);
    cudaFree(p->d_res);
    cudaFree(p->stage);
    cudaFree(p->pre);
    cudaFree(p->arena);
    cudaFree(p->hb_a);
    cudaFree(p->hb_b);
    cudaFree(p->hb_z);
    cudaFree(p->hb_res);
    for (int l = 1; l < LANES; ++l) {
        if (p->lane_stream[l]) cudaStreamSynchronize(p->lane_stream[l]);
        if (p->lane_stream[l]) cudaStreamDestroy(p->lane_stream[l]);
        cudaFree(p->lane_gate[l]);
    }
    for (cudaEvent_t e : p->lane_ev)
        if (e) cudaEventDestroy(e);
    for (int l = 0; l < p->piece_lanes; ++l) {
        cudaStreamSynchronize(p->piece_stream[l]);
        cudaStreamDestroy(p->piece_stream[l]);
        cudaFree(p->piece_gate[l]);
    }
    for (cudaEvent_t e : p->piece_ev)
        if (e) cudaEventDestroy(e);
    if (p->up) cudaStreamDestroy(p->up);
    if (p->down) cudaStreamDestroy(p->down);
    for (cudaEvent_t e : p->hb_ev) cudaEventDestroy(e);
    cudaFree(p->coeff_total);
    cudaFree(p->split_st);
    cudaFree(p->d_split);
    cudaFreeHost(p->h_split);
    cudaFreeHost(p->h_desc);
    cudaFreeHost(p->h_res);
    if (p->desc_free) cudaEventDestroy(p->desc_free);
    for (auto& pe : p->pending) {
        cudaEventDestroy(pe.second.first);
        cudaEventDestroy(pe.second.second);
    }
    for (cudaEvent_t e : p->ev_pool) cudaEventDestroy(e);
    if (cur >= 0 && cur != p->device) cudaSetDevice(cur);
    delete p;
}

ssmul_status ssmul_plan(ssmul_plan_t* out, size_t max_na, size_t max_nb, size_t max_products,
                        ssmul_precision prec, void* cuda_stream) {
    if (!out) return SSMUL_INVALID_ARG;
    *out = nullptr;
    if (max_na == 0 || max_nb == 0) return SSMUL_INVALID_ARG;
    if (int(prec) < SSMUL_PREC_FP64 || int(prec) > SSMUL_PREC_LADDER_FAST)
        return SSMUL_INVALID_ARG;
    if (max_na > (size_t(1) << LOG_N_MAX) || max_nb > (size_t(1) << LOG_N_MAX))
        return SSMUL_TOO_LARGE;
    const int log_n = log_n_for(max_na, max_nb);
    if (log_n > LOG_N_MAX) return SSMUL_TOO_LARGE;

    ssmul_plan_s* p = new (std::nothrow) ssmul_plan_s();
    if (!p) return SSMUL_OUT_OF_MEMORY;
    ssmul_status s = SSMUL_OK;
    auto fail = [&](ssmul_status e) {
        ssmul_plan_destroy(p);
        return e;
    };
    if (cudaGetDevice(&p->device) != cudaSuccess) return fail(SSMUL_CUDA_ERROR);
    if (cudaDeviceGetAttribute(&p->sms, cudaDevAttrMultiProcessorCount, p->device) != cudaSuccess)
        return fail(SSMUL_CUDA_ERROR);
    p->stream = static_cast<cudaStream_t>(cuda_stream);
    p->cur = p->stream;
    p->prec = prec;
    p->max_na = max_na;
    p->max_nb = max_nb;
    p->max_products = max_products;
    p->log_n_max = log_n;
    // families: Ntab = 2^log_n; 3 2^(log_n - 2) and 5 2^(log_n - 3) hold every
    // odd length R 2^j the plan's products can take (R 2^j < 2^log_n)
    for (int f = 0; f < FAMILIES; ++f) p->fam[f].R = FAMILY_R[f];
    // the power-of-two table also serves the binary32 rung's 4-bit digits,
    // whose transforms are up to 4 times longer (at most 2^LOG_SMALL)
    p->fam[0].log_tab = std::max(log_n < 4 ? 4 : log_n, std::min(LOG_SMALL, log_n + 2));
    p->fam[1].log_tab = log_n - 2 >= LOG3_MIN ? (log_n - 2 > LOG3_MAX ? LOG3_MAX : log_n - 2) : 0;
    p->fam[2].log_tab = log_n - 3 >= LOG5_MIN ? (log_n - 3 > LOG5_MAX ? LOG5_MAX : log_n - 3) : 0;
    for (int c = 0; c < GEOM_CODES; ++c) p->geom[c] = default_geom_code(c);

    const size_t n = size_t(1) << log_n;
    const size_t slots = max_products ? max_products : 1;
    const size_t tab = p->fam[0].entries();
    p->flags_per_product = carry_tiles(max_na + max_nb);
    cudaError_t e = cudaSuccess;
    if (e == cudaSuccess) e = cudaMalloc(&p->rho, 2 * FAMILIES * sizeof(float));
    for (TwFamily& F : p->fam) {
        const size_t t = F.entries();
        if (!t) continue;
        if (e == cudaSuccess) e = cudaMalloc(&F.t64, t * sizeof(TwMid));
        if (e == cudaSuccess) e = cudaMalloc(&F.t32, t * sizeof(TwEntry<float>));
        if (e == cudaSuccess) e = cudaMalloc(&F.td, t * sizeof(DiscTw));
        if (e == cudaSuccess) e = cudaMalloc(&F.tdd, t * sizeof(DDiscC));
        if (e == cudaSuccess) e = cudaMalloc(&F.s64, 3 * STEP_TAB * sizeof(CI<double>));
        if (e == cudaSuccess) e = cudaMalloc(&F.s32, 3 * STEP_TAB * sizeof(CI<float>));
        if (e == cudaSuccess) e = cudaMalloc(&F.sd, 3 * STEP_TAB * sizeof(DiscTw));
        if (e == cudaSuccess) e = cudaMalloc(&F.sdd, 3 * STEP_TAB * sizeof(DDiscC));
        if (F.R > 1 && e == cudaSuccess) e = cudaMalloc(&F.scal, sizeof(ScalarSet));
    }
    if (e == cudaSuccess) e = cudaMalloc(&p->Z, n * sizeof(CI<double>));
    if (e == cudaSuccess) e = cudaMalloc(&p->W, (n / 2) * sizeof(CI<double>));
    if (e == cudaSuccess) e = cudaMalloc(&p->coeff, (n + 1) * sizeof(int64_t));
    if (e == cudaSuccess) e = cudaMalloc(&p->flags, slots * p->flags_per_product * sizeof(uint32_t));
    if (e == cudaSuccess) e = cudaMalloc(&p->st, slots * sizeof(ProdState));
    if (e == cudaSuccess) e = cudaMalloc(&p->d_desc, slots * sizeof(ProdDesc));
    if (e == cudaSuccess) e = cudaMalloc(&p->gate_list, (slots + 1) * sizeof(int));
    p->cur_gate = p->gate_list;
    if (e == cudaSuccess) e = cudaMalloc(&p->d_res, slots * sizeof(ssmul_result));
    if (e == cudaSuccess) e = cudaMalloc(&p->stage, 2 * (max_na + max_nb));
    if (e == cudaSuccess) e = cudaMalloc(&p->pre, pre_bytes(max_na, max_nb));
    if (e == cudaSuccess) e = cudaMallocHost(&p->h_desc, slots * sizeof(ProdDesc));
    if (e == cudaSuccess) e = cudaMallocHost(&p->h_res, slots * sizeof(ssmul_result));
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&p->desc_free, cudaEventDisableTiming);
    if (e == cudaSuccess && max_products) {
        // room for every product at the largest size, capped at ARENA_CAP
        // bytes (at least one product of the largest size)
        // (the environment variable SSMUL_ARENA_MB lowers the cap)
        size_t cap = ARENA_CAP;
        if (const char* env = std::getenv("SSMUL_ARENA_MB")) {
            const long long mb = std::atoll(env);
            if (mb > 0 && size_t(mb) << 20 < cap) cap = size_t(mb) << 20;
        }
        const size_t one = arena_need(log_n) + pre_bytes(max_na, max_nb);
        size_t want = one * max_products;
        if (want > cap) want = cap > one ? cap : one;
        p->arena_bytes = want;
        e = cudaMalloc(&p->arena, want);
    }
    if (e != cudaSuccess) return fail(cuda_status(e));

    if ((s = set_smem_attrs<double>()) != SSMUL_OK) return fail(s);
    if ((s = set_smem_attrs<float>()) != SSMUL_OK) return fail(s);
    if ((s = set_smem_attrs<Disc>()) != SSMUL_OK) return fail(s);
    if ((s = set_smem_attrs<Pt>()) != SSMUL_OK) return fail(s);
    if ((s = set_smem_attrs<DDisc>()) != SSMUL_OK) return fail(s);

    const int threads = 256;
    if ((e = cudaMemsetAsync(p->rho, 0, 2 * FAMILIES * sizeof(float), p->stream)) != cudaSuccess)
        return fail(cuda_status(e));
    for (int f = 0; f < FAMILIES; ++f) {
        TwFamily& F = p->fam[f];
        const size_t t = F.entries();
        if (!t) continue;
        const int blocks = int((t + threads - 1) / threads);
        k_twiddle_gen<<<blocks, threads, 0, p->stream>>>(F.t64, F.t32, F.log_tab, F.R);
        k_disc_tw_gen<<<blocks, threads, 0, p->stream>>>(F.t64, F.R, F.td, p->rho + 2 * f, int64_t(t));
        k_ddisc_tw_gen<<<blocks, threads, 0, p->stream>>>(F.td, p->rho + 2 * f, F.tdd, int64_t(t));
    }
    {
        p->octant_only = true;
        const TwTable oct[FAMILIES] = {p->tw(0), p->tw(1), p->tw(2)};
        p->octant_only = false;
        const int sb = (3 * STEP_TAB + threads - 1) / threads;
        k_step_tw_gen<1><<<sb, threads, 0, p->stream>>>(oct[0], p->fam[0].s64, p->fam[0].s32,
                                                        p->fam[0].sd, p->fam[0].sdd);
        if (p->fam[1].entries())
            k_step_tw_gen<3><<<sb, threads, 0, p->stream>>>(oct[1], p->fam[1].s64, p->fam[1].s32,
                                                            p->fam[1].sd, p->fam[1].sdd);
        if (p->fam[2].entries())
            k_step_tw_gen<5><<<sb, threads, 0, p->stream>>>(oct[2], p->fam[2].s64, p->fam[2].s32,
                                                            p->fam[2].sd, p->fam[2].sdd);
        if (p->fam[1].entries()) k_scalar_gen<3><<<1, 32, 0, p->stream>>>(oct[1], p->fam[1].scal);
        if (p->fam[2].entries()) k_scalar_gen<5><<<1, 32, 0, p->stream>>>(oct[2], p->fam[2].scal);
    }
    if ((e = cudaGetLastError()) != cudaSuccess) return fail(cuda_status(e));
    float h_rho[2 * FAMILIES] = {};
    if ((e = cudaMemcpyAsync(h_rho, p->rho, sizeof(h_rho), cudaMemcpyDeviceToHost, p->stream)) !=
        cudaSuccess)
        return fail(cuda_status(e));
    if ((e = cudaEventRecord(p->desc_free, p->stream)) != cudaSuccess) return fail(cuda_status(e));
    if ((e = cudaStreamSynchronize(p->stream)) != cudaSuccess) return fail(cuda_status(e));
    for (int f = 0; f < FAMILIES; ++f) p->fam[f].rho_dd = h_rho[2 * f + 1];
    *out = p;
    return SSMUL_OK;
}

ssmul_status ssmul_plan_set_option(ssmul_plan_t p, ssmul_option option, long long value) {
    if (!p) return SSMUL_INVALID_ARG;
    ssmul_status s = check_device(p);
    if (s != SSMUL_OK) return s;
    switch (option) {
        case SSMUL_OPT_GRAPH:
            SS_TRY(cudaStreamSynchronize(p->stream));
            p->graph = value != 0;
            graph_drop(p->cached);
            return SSMUL_OK;
        case SSMUL_OPT_AUTOTUNE:
            SS_TRY(cudaStreamSynchronize(p->stream));
            graph_drop(p->cached);
            if (value == 0) {
                for (int c = 0; c < GEOM_CODES; ++c) p->geom[c] = default_geom_code(c);
                return SSMUL_OK;
            }
            return autotune(p);
        case SSMUL_OPT_FP32_MAX_DIGITS:
            if (value < 0) return SSMUL_INVALID_ARG;
            graph_drop(p->cached);
            p->fp32_max_digits = value ? size_t(value) : 0;
            p->fp32_max_zero = value == 0;
            return SSMUL_OK;
        case SSMUL_OPT_FP32_NIBBLES:
            SS_TRY(cudaStreamSynchronize(p->stream));
            graph_drop(p->cached);
            p->fp32_nibbles = value != 0;
            return SSMUL_OK;
        case SSMUL_OPT_BALANCED:
            SS_TRY(cudaStreamSynchronize(p->stream));
            graph_drop(p->cached);
            p->balanced = value != 0;
            return SSMUL_OK;
        case SSMUL_OPT_LANES:
            if (value < 1 || value > LANES) return SSMUL_INVALID_ARG;
            SS_TRY(cudaStreamSynchronize(p->stream));
            graph_drop(p->cached);
            p->group_lanes = int(value);
            return SSMUL_OK;
        case SSMUL_OPT_HOST_PIECES:
            if (value < 1 || value > 64) return SSMUL_INVALID_ARG;
            p->host_pieces = int(value);
            return SSMUL_OK;
        case SSMUL_OPT_LENGTHS:
            if (value < 0 || value > 3) return SSMUL_INVALID_ARG;
            SS_TRY(cudaStreamSynchronize(p->stream));
            graph_drop(p->cached);
            p->lengths = int(value);
            return SSMUL_OK;
        case SSMUL_OPT_SPLIT_DIGITS: {
            if (value < 0 || (value > 0 && value < 1024)) return SSMUL_INVALID_ARG;
            SS_TRY(cudaStreamSynchronize(p->stream));
            cudaFree(p->coeff_total);
            cudaFree(p->split_st);
            cudaFree(p->d_split);
            cudaFreeHost(p->h_split);
            p->coeff_total = nullptr;
            p->split_st = nullptr;
            p->d_split = nullptr;
            p->h_split = nullptr;
            p->split_digits = 0;
            p->split_slots = 0;
            if (value == 0) return SSMUL_OK;
            const size_t m = size_t(value);
            const size_t slots = ((p->max_na + m - 1) / m) * ((p->max_nb + m - 1) / m);
            cudaError_t e = cudaMalloc(&p->coeff_total, (p->max_na + p->max_nb) * sizeof(int64_t));
            if (e == cudaSuccess) e = cudaMalloc(&p->split_st, slots * sizeof(ProdState));
            if (e == cudaSuccess) e = cudaMalloc(&p->d_split, slots * sizeof(ProdDesc));
            if (e == cudaSuccess) e = cudaMallocHost(&p->h_split, slots * sizeof(ProdDesc));
            if (e != cudaSuccess) return cuda_status(e);
            p->split_digits = m;
            p->split_slots = slots;
            return SSMUL_OK;
        }
    }
    return SSMUL_INVALID_ARG;
}

ssmul_status ssmul_mul(ssmul_plan_t p, const uint8_t* d_a, size_t na, const uint8_t* d_b,
                       size_t nb, uint8_t* d_z, ssmul_result* h_res) {
    if (!p) return SSMUL_INVALID_ARG;
    return run_single(p, d_a, na, d_b, nb, d_z, h_res, p->prec, nullptr);
}

ssmul_status ssmul_mul_host(ssmul_plan_t p, const uint8_t* h_a, size_t na, const uint8_t* h_b,
                            size_t nb, uint8_t* h_z, ssmul_result* h_res) {
    if (!p || !h_a || !h_b || !h_z || na == 0 || nb == 0) return SSMUL_INVALID_ARG;
    if (na > p->max_na || nb > p->max_nb) return SSMUL_TOO_LARGE;
    ssmul_status s = check_device(p);
    if (s != SSMUL_OK) return s;
    uint8_t* da = p->stage;
    uint8_t* db = da + na;
    uint8_t* dz = db + nb;
    SS_TRY(cudaMemcpyAsync(da, h_a, na, cudaMemcpyHostToDevice, p->stream));
    SS_TRY(cudaMemcpyAsync(db, h_b, nb, cudaMemcpyHostToDevice, p->stream));
    s = run_single(p, da, na, db, nb, dz, h_res, p->prec, nullptr);
    if (s != SSMUL_OK && s != SSMUL_ISOLATION_FAILED && s != SSMUL_CONTAINMENT_FAILED &&
        s != SSMUL_TIMEOUT && s != SSMUL_UNVERIFIED)
        return s;
    SS_TRY(cudaMemcpyAsync(h_z, dz, na + nb, cudaMemcpyDeviceToHost, p->stream));
    SS_TRY(cudaStreamSynchronize(p->stream));
    return s;
}

ssmul_status ssmul_mul_batched(ssmul_plan_t p, size_t count, const ssmul_desc* h_desc,
                               const uint8_t* d_a_pool, const uint8_t* d_b_pool,
                               uint8_t* d_z_pool, ssmul_result* d_res) {
    if (!p || (count && (!h_desc || !d_a_pool || !d_b_pool || !d_z_pool || !d_res)))
        return SSMUL_INVALID_ARG;
    if (count > p->max_products) return SSMUL_TOO_LARGE;
    for (size_t i = 0; i < count; ++i) {
        if (h_desc[i].na == 0 || h_desc[i].nb == 0) return SSMUL_INVALID_ARG;
        if (h_desc[i].na > p->max_na || h_desc[i].nb > p->max_nb) return SSMUL_TOO_LARGE;
    }
    if (count == 0) return SSMUL_OK;
    ssmul_status s = check_device(p);
    if (s != SSMUL_OK) return s;
    return enqueue_batch(p, count, h_desc, d_a_pool, d_b_pool, d_z_pool, d_res);
}

ssmul_status ssmul_mul_batched_host(ssmul_plan_t p, size_t count, const ssmul_desc* h_desc,
                                    const uint8_t* h_a_pool, const uint8_t* h_b_pool,
                                    uint8_t* h_z_pool, ssmul_result* h_res) {
    if (!p || (count && (!h_desc || !h_a_pool || !h_b_pool || !h_z_pool || !h_res)))
        return SSMUL_INVALID_ARG;
    if (count > p->max_products) return SSMUL_TOO_LARGE;
    for (size_t i = 0; i < count; ++i) {
        const ssmul_desc& d = h_desc[i];
        if (d.na == 0 || d.nb == 0) return SSMUL_INVALID_ARG;
        if (d.na > p->max_na || d.nb > p->max_nb) return SSMUL_TOO_LARGE;
        if (d.a_off > UINT64_MAX - d.na || d.b_off > UINT64_MAX - d.nb ||
            d.z_off > UINT64_MAX - d.na - d.nb)
            return SSMUL_INVALID_ARG;
    }
    if (count == 0) return SSMUL_OK;
    ssmul_status s = check_device(p);
    if (s != SSMUL_OK) return s;
    return run_batched_host(p, count, h_desc, h_a_pool, h_b_pool, h_z_pool, h_res);
}

// ---- inspection entry points (include/ssmul_debug.h) ----------------------------

ssmul_status ssmul_debug_kernel_stats(ssmul_plan_t p, int enable, double* ms,
                                      unsigned long long* launches, int cap) {
    if (!p) return SSMUL_INVALID_ARG;
    ssmul_status s = check_device(p);
    if (s != SSMUL_OK) return s;
    for (auto& pe : p->pending) {
        SS_TRY(cudaEventSynchronize(pe.second.second));
        float t = 0.f;
        SS_TRY(cudaEventElapsedTime(&t, pe.second.first, pe.second.second));
        p->kt_ms[pe.first] += t;
        p->ev_pool.push_back(pe.second.first);
        p->ev_pool.push_back(pe.second.second);
    }
    p->pending.clear();
    for (int k = 0; k < SSMUL_KERNEL_KINDS && k < cap; ++k) {
        if (ms) ms[k] = p->kt_ms[k];
        if (launches) launches[k] = p->kt_launches[k];
        p->kt_ms[k] = 0.0;
        p->kt_launches[k] = 0;
    }
    p->timing = enable != 0;
    return SSMUL_OK;
}

ssmul_status ssmul_debug_set_fault(ssmul_plan_t p, int kind, long long value) {
    if (!p) return SSMUL_INVALID_ARG;
    graph_drop(p->cached);
    switch (kind) {
        case 0:
            p->fault_widen = 0;
            p->fault_stall = 0;
            p->octant_only = false;
            return SSMUL_OK;
        case 3:
            p->octant_only = value != 0;
            return SSMUL_OK;
        case 1:
            if (value < 0 || value >= RUNGS) return SSMUL_INVALID_ARG;
            p->fault_widen = int(value) + 1;
            return SSMUL_OK;
        case 2:
            if (value < 0) return SSMUL_INVALID_ARG;
            p->fault_stall = int(value) + 1;
            return SSMUL_OK;
    }
    return SSMUL_INVALID_ARG;
}

ssmul_status ssmul_debug_geometry(ssmul_plan_t p, int log_n, int* log_n1, int* log_n2,
                                  int* log_cta) {
    if (!p || !log_n1 || !log_n2 || !log_cta) return SSMUL_INVALID_ARG;
    if (!((log_n >= 2 && log_n <= LOG_N_MAX) ||
          (log_n >= LEN3 + LOG3_MIN && log_n <= LEN3 + LOG3_MAX) ||
          (log_n >= LEN5 + LOG5_MIN && log_n <= LEN5 + LOG5_MAX)))
        return SSMUL_INVALID_ARG;
    const Geom& g = p->geom[log_n];
    *log_n1 = g.small ? 0 : g.log_n1;
    *log_n2 = g.small ? log_n : g.log_n2;
    *log_cta = g.small ? log_n : g.log_cta;
    return SSMUL_OK;
}

ssmul_status ssmul_debug_twiddles(ssmul_plan_t p, int f32, double* h_out, size_t cap,
                                  int* log_ntab) {
    if (!p || !h_out || !log_ntab || f32 < 0 || f32 > 5 || (f32 & 6) == 6) return SSMUL_INVALID_ARG;
    const TwFamily& F = p->fam[(f32 & 2) ? 1 : ((f32 & 4) ? 2 : 0)];
    const size_t tab = F.entries();
    if (!tab || cap < 4 * tab) return SSMUL_INVALID_ARG;
    ssmul_status s = check_device(p);
    if (s != SSMUL_OK) return s;
    *log_ntab = F.log_tab;
    if (!(f32 & 1)) {
        // the bounds the kernels rebuild from the stored values
        std::vector<TwMid> t(tab);
        SS_TRY(cudaMemcpy(t.data(), F.t64, tab * sizeof(TwMid), cudaMemcpyDeviceToHost));
        for (size_t j = 0; j < tab; ++j) {
            const TwEntry<double> e = tw_expand_w(t[j], tw_widen_r(uint32_t(j), F.R));
            h_out[4 * j] = e.cl;
            h_out[4 * j + 1] = e.ch;
            h_out[4 * j + 2] = e.sl;
            h_out[4 * j + 3] = e.sh;
        }
    } else {
        std::vector<TwEntry<float>> t(tab);
        SS_TRY(cudaMemcpy(t.data(), F.t32, tab * sizeof(TwEntry<float>), cudaMemcpyDeviceToHost));
        for (size_t j = 0; j < tab; ++j) {
            h_out[4 * j] = t[j].cl;
            h_out[4 * j + 1] = t[j].ch;
            h_out[4 * j + 2] = t[j].sl;
            h_out[4 * j + 3] = t[j].sh;
        }
    }
    return SSMUL_OK;
}

ssmul_status ssmul_debug_mul_intervals(ssmul_plan_t p, const uint8_t* d_a, size_t na,
                                       const uint8_t* d_b, size_t nb, uint8_t* d_z,
                                       ssmul_result* h_res, ssmul_precision prec,
                                       double* d_iv) {
    if (!p || !d_iv) return SSMUL_INVALID_ARG;
    if (int(prec) == SSMUL_DEBUG_PREC_FP32_NIBBLES) {
        // the binary32 launches are sized for 4-bit digits only while the
        // plan's SSMUL_OPT_FP32_NIBBLES is on
        if (na + nb > size_t(NIB_MAX_DIGITS) || !p->fp32_nibbles) return SSMUL_INVALID_ARG;
        return run_single(p, d_a, na, d_b, nb, d_z, h_res, SSMUL_PREC_FP32, d_iv, true);
    }
    if (prec != SSMUL_PREC_FP64 && prec != SSMUL_PREC_FP32 && prec != SSMUL_PREC_DISC64 &&
        prec != SSMUL_PREC_NAIVE64 && prec != SSMUL_PREC_DISC32X2)
        return SSMUL_INVALID_ARG;
    return run_single(p, d_a, na, d_b, nb, d_z, h_res, prec, d_iv);
}

}  // extern "C"

namespace {

template <typename T>
__global__ void k_ci_op(int op, const double* x, const double* y, double* out, size_t n) {
    for (size_t i = blockIdx.x * size_t(blockDim.x) + threadIdx.x; i < n;
         i += size_t(gridDim.x) * blockDim.x) {
        const CI<T> a{T(x[4 * i]), T(x[4 * i + 1]), T(x[4 * i + 2]), T(x[4 * i + 3])};
        const CI<T> b{T(y[4 * i]), T(y[4 * i + 1]), T(y[4 * i + 2]), T(y[4 * i + 3])};
        CI<T> r;
        switch (op) {
            case 0: r = a + b; break;
            case 1: r = a - b; break;
            case 2: r = mul_tw(a, b); break;
            case 3: r = mul_ci(a, b); break;
            case 4: r = mul_real(a, b); break;
            default: r = mul_imag(a, b); break;
        }
        out[4 * i] = r.rl;
        out[4 * i + 1] = r.rh;
        out[4 * i + 2] = r.il;
        out[4 * i + 3] = r.ih;
    }
}

__global__ void k_disc_op(int op, const double* x, const double* y, double* out, size_t n) {
    for (size_t i = blockIdx.x * size_t(blockDim.x) + threadIdx.x; i < n;
         i += size_t(gridDim.x) * blockDim.x) {
        const Disc a{x[3 * i], x[3 * i + 1], float(x[3 * i + 2]), 0.f};
        const Disc b{y[3 * i], y[3 * i + 1], float(y[3 * i + 2]), 0.f};
        Disc r;
        switch (op) {
            case 0: r = a + b; break;
            case 1: r = a - b; break;
            case 2: r = mul_tw(a, DiscTw{b.x, b.y, b.r, TW_MOD_UP}); break;
            case 3: r = mul_ci(a, b); break;
            case 4: r = scale_pow2(a, int(y[3 * i])); break;
            case 5: r = mul_real(a, DiscTw{b.x, 0.0, b.r, abs_up(b.x)}); break;
            default: r = mul_imag(a, DiscTw{0.0, b.y, b.r, abs_up(b.y)}); break;
        }
        out[3 * i] = r.x;
        out[3 * i + 1] = r.y;
        out[3 * i + 2] = r.r;
    }
}

__global__ void k_ddisc_op(int op, const double* x, const double* y, double* out, size_t n) {
    for (size_t i = blockIdx.x * size_t(blockDim.x) + threadIdx.x; i < n;
         i += size_t(gridDim.x) * blockDim.x) {
        if (op == 5 || op == 6) {
            // radix-4 butterfly of the four discs x[20 i ..] (SIGN +1 for op 5, -1 for op 6)
            DDisc v[4];
            for (int t = 0; t < 4; ++t) {
                const double* e = x + 20 * i + 5 * t;
                v[t] = {float(e[0]), float(e[1]), float(e[2]), float(e[3]), float(e[4]), 0.f};
            }
            if (op == 5) bfly4_dd<1>(v[0], v[1], v[2], v[3]);
            else bfly4_dd<-1>(v[0], v[1], v[2], v[3]);
            for (int t = 0; t < 4; ++t) {
                double* o = out + 20 * i + 5 * t;
                o[0] = v[t].xh;
                o[1] = v[t].xl;
                o[2] = v[t].yh;
                o[3] = v[t].yl;
                o[4] = v[t].r;
            }
            continue;
        }
        const double* a5 = x + 5 * i;
        const double* b5 = y + 5 * i;
        const DDisc a{float(a5[0]), float(a5[1]), float(a5[2]), float(a5[3]), float(a5[4]), 0.f};
        const DDisc b{float(b5[0]), float(b5[1]), float(b5[2]), float(b5[3]), float(b5[4]), 0.f};
        DDisc r;
        switch (op) {
            case 0: r = a + b; break;
            case 1: r = a - b; break;
            case 2: r = mul_tw(a, DDiscTw{b.xh, b.xl, b.yh, b.yl, b.r, TW_MOD_UP}); break;
            case 3: r = mul_ci(a, b); break;
            case 4: r = scale_pow2(a, int(b5[0])); break;
            case 7: r = mul_real(a, DDiscTw{b.xh, b.xl, 0.f, 0.f, b.r, dd_mod_up(b.xh, 0.f)}); break;
            default: r = mul_imag(a, DDiscTw{0.f, 0.f, b.yh, b.yl, b.r, dd_mod_up(0.f, b.yh)}); break;
        }
        double* o = out + 5 * i;
        o[0] = r.xh;
        o[1] = r.xl;
        o[2] = r.yh;
        o[3] = r.yl;
        o[4] = r.r;
    }
}

// one coefficient per thread: row i of x is (h, l, r, pad); pad != 0 puts
// the value past the product's last coefficient (it must contain 0)
__global__ void k_iso_op(int path, const double* x, int64_t* value, int* cls, size_t n) {
    for (size_t i = blockIdx.x * size_t(blockDim.x) + threadIdx.x; i < n;
         i += size_t(gridDim.x) * blockDim.x) {
        const double* r4 = x + 4 * i;
        const float h = float(r4[0]), l = float(r4[1]), r = float(r4[2]);
        ProdDesc d{};
        d.na = 1;
        d.nb = 1;                           // one coefficient: index 0
        d.coeff = value + i;
        const int64_t idx = r4[3] != 0.0 ? 1 : 0;
        value[i] = 0;
        IsoAcc acc;
        const double dr = double(r);
        const double lo = __dsub_rd(__dadd_rd(double(h), double(l)), dr);
        const double hi = __dadd_ru(__dadd_ru(double(h), double(l)), dr);
        switch (path) {
            case 0: isolate_pair<1>(h, l, r, idx, d, acc, 4); break;
            case 1: isolate_one<1>(lo, hi, 0, idx, d, acc, 4); break;
            case 2: isolate_pair<3>(h, l, r, idx, d, acc, 4); break;
            case 3: isolate_one<3>(lo, hi, 0, idx, d, acc, 4); break;
            case 4: isolate_pair<5>(h, l, r, idx, d, acc, 4); break;
            default: isolate_one<5>(lo, hi, 0, idx, d, acc, 4); break;
        }
        cls[i] = acc.empty ? 2 : (acc.unisolated ? 1 : 0);
    }
}

}  // namespace

namespace {
__global__ void k_floor_ceil(const double* x, const int* k, long long* out, size_t n) {
    for (size_t i = blockIdx.x * size_t(blockDim.x) + threadIdx.x; i < n;
         i += size_t(gridDim.x) * blockDim.x)
        floor_ceil_scaled(x[i], k[i], out[2 * i], out[2 * i + 1]);
}
}  // namespace

extern "C" ssmul_status ssmul_debug_floor_ceil(const double* d_x, const int* d_k, int64_t* d_out,
                                               size_t n) {
    if (n && (!d_x || !d_k || !d_out)) return SSMUL_INVALID_ARG;
    if (n == 0) return SSMUL_OK;
    const int threads = 256;
    const int blocks = int((n + threads - 1) / threads < 1024 ? (n + threads - 1) / threads : 1024);
    k_floor_ceil<<<blocks, threads>>>(d_x, d_k, reinterpret_cast<long long*>(d_out), n);
    SS_TRY(cudaGetLastError());
    SS_TRY(cudaDeviceSynchronize());
    return SSMUL_OK;
}

extern "C" ssmul_status ssmul_debug_isolate(int path, const double* d_x, int64_t* d_value,
                                            int* d_class, size_t n) {
    if (path < 0 || path > 5 || (n && (!d_x || !d_value || !d_class))) return SSMUL_INVALID_ARG;
    if (n == 0) return SSMUL_OK;
    const int threads = 256;
    const int blocks = int((n + threads - 1) / threads < 1024 ? (n + threads - 1) / threads : 1024);
    k_iso_op<<<blocks, threads>>>(path, d_x, d_value, d_class, n);
    SS_TRY(cudaGetLastError());
    SS_TRY(cudaDeviceSynchronize());
    return SSMUL_OK;
}

extern "C" ssmul_status ssmul_debug_ddisc_op(int op, const double* d_x, const double* d_y,
                                             double* d_out, size_t n) {
    if (op < 0 || op > 8 || (n && (!d_x || !d_out || ((op < 5 || op > 6) && !d_y)))) return SSMUL_INVALID_ARG;
    if (n == 0) return SSMUL_OK;
    const int threads = 256;
    const int blocks = int((n + threads - 1) / threads < 1024 ? (n + threads - 1) / threads : 1024);
    k_ddisc_op<<<blocks, threads>>>(op, d_x, d_y, d_out, n);
    SS_TRY(cudaGetLastError());
    SS_TRY(cudaDeviceSynchronize());
    return SSMUL_OK;
}

extern "C" ssmul_status ssmul_debug_disc_op(int op, const double* d_x, const double* d_y,
                                            double* d_out, size_t n) {
    if (op < 0 || op > 6 || (n && (!d_x || !d_y || !d_out))) return SSMUL_INVALID_ARG;
    if (n == 0) return SSMUL_OK;
    const int threads = 256;
    const int blocks = int((n + threads - 1) / threads < 1024 ? (n + threads - 1) / threads : 1024);
    k_disc_op<<<blocks, threads>>>(op, d_x, d_y, d_out, n);
    SS_TRY(cudaGetLastError());
    SS_TRY(cudaDeviceSynchronize());
    return SSMUL_OK;
}

extern "C" ssmul_status ssmul_debug_ci_op(int op, int f32, const double* d_x, const double* d_y,
                                          double* d_out, size_t n) {
    if (op < 0 || op > 5 || (n && (!d_x || !d_y || !d_out))) return SSMUL_INVALID_ARG;
    if (n == 0) return SSMUL_OK;
    const int threads = 256;
    const int blocks = int((n + threads - 1) / threads < 1024 ? (n + threads - 1) / threads : 1024);
    if (f32)
        k_ci_op<float><<<blocks, threads>>>(op, d_x, d_y, d_out, n);
    else
        k_ci_op<double><<<blocks, threads>>>(op, d_x, d_y, d_out, n);
    SS_TRY(cudaGetLastError());
    SS_TRY(cudaDeviceSynchronize());
    return SSMUL_OK;
}

// ---- arithmetic pipe rates (ssmul_debug_pipe_rate) ---------------------------------
//
// Each thread runs PROBE_CHAINS independent dependency chains of one
// operation for `iters` rounds; the operands are run-time values near 1, so
// the chains stay normal and the compiler cannot fold them.

namespace {

constexpr int PROBE_CHAINS = 16;
constexpr int PROBE_THREADS = 256;

template <int OP>
__global__ void __launch_bounds__(PROBE_THREADS) k_pipe_probe(double* sink, double seed, int iters) {
    const double a = 1.0 + seed * 0x1p-40, b = seed * 0x1p-30, one = 1.0 + seed * 0.0;
    const float af = float(a), bf = float(b);
    double x[PROBE_CHAINS];
    float y[PROBE_CHAINS];
#pragma unroll
    for (int i = 0; i < PROBE_CHAINS; ++i) {
        x[i] = 1.0 + (threadIdx.x * PROBE_CHAINS + i) * 0x1p-20;
        y[i] = float(x[i]);
    }
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int i = 0; i < PROBE_CHAINS; ++i) {
            if (OP == 0) x[i] = __dadd_rd(x[i], b);            // directed add
            if (OP == 1) x[i] = __dmul_ru(x[i], a);            // directed product
            if (OP == 2) x[i] = __fma_rd(x[i], a, -b);         // directed fma
            if (OP == 3) x[i] = __fma_rd(x[i], one, b);        // an add written as an fma
            if (OP == 4) x[i] = __dadd_rn(x[i], b);            // round-to-nearest add
            if (OP == 5) y[i] = __fadd_rd(y[i], bf);           // binary32 directed add
            if (OP == 6) y[i] = __fmaf_rd(y[i], af, -bf);      // binary32 directed fma
        }
    }
    double acc = 0.0;
#pragma unroll
    for (int i = 0; i < PROBE_CHAINS; ++i) acc += x[i] + double(y[i]);
    if (acc == seed) sink[0] = acc;                            // never true; keeps the chains
}

}  // namespace

extern "C" ssmul_status ssmul_debug_pipe_rate(int op, double* gops) {
    if (op < 0 || op > 6 || !gops) return SSMUL_INVALID_ARG;
    int dev = 0, sms = 0;
    SS_TRY(cudaGetDevice(&dev));
    SS_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    double* sink = nullptr;
    SS_TRY(cudaMalloc(&sink, sizeof(double)));
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const int blocks = sms * 8, iters = 2048;
    float best = 1e30f;
    cudaError_t e = cudaSuccess;
    for (int rep = 0; rep < 4 && e == cudaSuccess; ++rep) {
        cudaEventRecord(e0, 0);
        switch (op) {
            case 0: k_pipe_probe<0><<<blocks, PROBE_THREADS>>>(sink, 0.5, iters); break;
            case 1: k_pipe_probe<1><<<blocks, PROBE_THREADS>>>(sink, 0.5, iters); break;
            case 2: k_pipe_probe<2><<<blocks, PROBE_THREADS>>>(sink, 0.5, iters); break;
            case 3: k_pipe_probe<3><<<blocks, PROBE_THREADS>>>(sink, 0.5, iters); break;
            case 4: k_pipe_probe<4><<<blocks, PROBE_THREADS>>>(sink, 0.5, iters); break;
            case 5: k_pipe_probe<5><<<blocks, PROBE_THREADS>>>(sink, 0.5, iters); break;
            default: k_pipe_probe<6><<<blocks, PROBE_THREADS>>>(sink, 0.5, iters); break;
        }
        cudaEventRecord(e1, 0);
        e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0.f;
        if (e == cudaSuccess && rep > 0 && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess && ms < best)
            best = ms;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(sink);
    if (e != cudaSuccess) return cuda_status(e);
    *gops = double(blocks) * PROBE_THREADS * PROBE_CHAINS * iters / (best * 1e-3) / 1e9;
    return SSMUL_OK;
}

// ---- allocation-free entry point (ssmul_mul_noalloc) -----------------------------
//
// Everything the one-CTA binary64 path needs beyond the caller's inputs and
// outputs lives in one file-scope device array: the twiddle table for
// N <= 4096, the product descriptor, the per-call accumulators, the integer
// coefficients, the carry look-back words, the outcome and a word that
// marks the table as built.  Host code must not use the array's name as an
// address; each device's address comes from cudaGetSymbolAddress in
// noalloc_setup.

namespace {

constexpr int NOALLOC_LOG_N = LOG_SMALL;                         // N <= 4096
constexpr size_t NOALLOC_N = size_t(1) << NOALLOC_LOG_N;
constexpr size_t NOALLOC_TAB = NOALLOC_N / 8 + 1;
constexpr size_t NOALLOC_TILES = (NOALLOC_N + 1 + CARRY_TILE - 1) / CARRY_TILE;

constexpr size_t na_align(size_t x) { return (x + 255) & ~size_t(255); }
constexpr size_t NA_OFF_T64 = 0;
constexpr size_t NA_OFF_T32 = na_align(NA_OFF_T64 + NOALLOC_TAB * sizeof(TwMid));
constexpr size_t NA_OFF_DESC = na_align(NA_OFF_T32 + NOALLOC_TAB * sizeof(TwEntry<float>));
constexpr size_t NA_OFF_ST = na_align(NA_OFF_DESC + sizeof(ProdDesc));
constexpr size_t NA_OFF_RES = na_align(NA_OFF_ST + sizeof(ProdState));
constexpr size_t NA_OFF_FLAGS = na_align(NA_OFF_RES + sizeof(ssmul_result));
constexpr size_t NA_OFF_COEFF = na_align(NA_OFF_FLAGS + NOALLOC_TILES * sizeof(uint32_t));
constexpr size_t NA_OFF_MAGIC = na_align(NA_OFF_COEFF + NOALLOC_N * sizeof(int64_t));
constexpr size_t NOALLOC_BYTES = na_align(NA_OFF_MAGIC + sizeof(unsigned long long));
// written after the twiddle table is built; a device reset re-creates the
// array zero-filled, and a call that finds the word missing builds again
constexpr unsigned long long NOALLOC_MAGIC = 0x5353'4D55'4C54'5742ull;

static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_BYTES];

constexpr int NOALLOC_MAX_DEVICES = 64;
std::mutex g_noalloc_mu;
unsigned char* g_noalloc_dev_ptr[NOALLOC_MAX_DEVICES] = {};

// Writes the descriptor and clears what must start at zero: the
// accumulators, the look-back words and the outcome.  Without the magic
// word the twiddle table is not there (the array was re-created by a device
// reset): the product is forced to SSMUL_CUDA_ERROR, so its digits are
// zero-filled and the host builds the table again.
__global__ void k_noalloc_init(ProdDesc d, unsigned char* base) {
    if (threadIdx.x == 0) *reinterpret_cast<ProdDesc*>(base + NA_OFF_DESC) = d;
    unsigned int* st = reinterpret_cast<unsigned int*>(base + NA_OFF_ST);
    for (size_t i = threadIdx.x; i < sizeof(ProdState) / sizeof(unsigned int); i += blockDim.x)
        st[i] = 0u;
    uint32_t* fl = reinterpret_cast<uint32_t*>(base + NA_OFF_FLAGS);
    for (size_t i = threadIdx.x; i < NOALLOC_TILES; i += blockDim.x) fl[i] = 0u;
    unsigned char* res = base + NA_OFF_RES;
    for (size_t i = threadIdx.x; i < sizeof(ssmul_result); i += blockDim.x) res[i] = 0;
    __syncthreads();
    if (threadIdx.x == 0 &&
        *reinterpret_cast<const unsigned long long*>(base + NA_OFF_MAGIC) != NOALLOC_MAGIC)
        reinterpret_cast<ProdState*>(base + NA_OFF_ST)->forced = SSMUL_CUDA_ERROR;
}

__global__ void k_noalloc_mark(unsigned char* base) {
    *reinterpret_cast<unsigned long long*>(base + NA_OFF_MAGIC) = NOALLOC_MAGIC;
}

// Once per device, with that device current (and again after a device
// reset, which may move the array): find the array's device address, build
// the twiddle table in it, mark it built and allow the kernel's shared
// memory size.  Returns the address, or nullptr with *err set.  rebuild:
// the last call found the table missing.
unsigned char* noalloc_setup(int dev, cudaStream_t stream, bool rebuild, ssmul_status* err) {
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    void* ptr = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
    if (e != cudaSuccess || ptr == nullptr) {
        *err = cuda_status(e == cudaSuccess ? cudaErrorInvalidSymbol : e);
        return nullptr;
    }
    if (!rebuild && g_noalloc_dev_ptr[dev] == ptr) return g_noalloc_dev_ptr[dev];
    g_noalloc_dev_ptr[dev] = nullptr;
    unsigned char* base = static_cast<unsigned char*>(ptr);
    e = cudaFuncSetAttribute(k_small<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             int(NOALLOC_N * sizeof(CI<double>)));
    if (e == cudaSuccess) {
        k_twiddle_gen<<<int((NOALLOC_TAB + 255) / 256), 256, 0, stream>>>(
            reinterpret_cast<TwMid*>(base + NA_OFF_T64),
            reinterpret_cast<TwEntry<float>*>(base + NA_OFF_T32), NOALLOC_LOG_N, 1);
        k_noalloc_mark<<<1, 1, 0, stream>>>(base);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
    if (e != cudaSuccess) {
        *err = cuda_status(e);
        return nullptr;
    }
    g_noalloc_dev_ptr[dev] = base;
    return base;
}

// One product on the array at `base`; waits for it and reads its outcome.
ssmul_status noalloc_run(unsigned char* base, const uint8_t* d_a, size_t na, const uint8_t* d_b,
                         size_t nb, uint8_t* d_z, cudaStream_t stream, ssmul_result* out) {
    ProdDesc d{};
    d.a = d_a;
    d.b = d_b;
    d.z = d_z;
    d.na = uint32_t(na);
    d.nb = uint32_t(nb);
    d.log_n = log_n_for(na, nb);
    d.coeff = reinterpret_cast<int64_t*>(base + NA_OFF_COEFF);
    d.flags = reinterpret_cast<uint32_t*>(base + NA_OFF_FLAGS);
    d.st = reinterpret_cast<ProdState*>(base + NA_OFF_ST);
    d.res = reinterpret_cast<ssmul_result*>(base + NA_OFF_RES);
    const ProdDesc* slot = reinterpret_cast<const ProdDesc*>(base + NA_OFF_DESC);
    const TwTable tw{reinterpret_cast<const TwMid*>(base + NA_OFF_T64),
                     reinterpret_cast<const TwEntry<float>*>(base + NA_OFF_T32), NOALLOC_LOG_N};
    const int n = 1 << d.log_n;

    k_noalloc_init<<<1, 64, 0, stream>>>(d, base);
    k_small<double><<<1, threads_for(n), n * sizeof(CI<double>), stream>>>(slot, tw, nullptr);
    k_carry<<<unsigned(carry_tiles(na + nb)), CARRY_THREADS, 0, stream>>>(slot);
    k_finalize<<<1, 256, 0, stream>>>(slot);
    SS_TRY(cudaGetLastError());
    SS_TRY(cudaMemcpyAsync(out, base + NA_OFF_RES, sizeof(*out), cudaMemcpyDeviceToHost, stream));
    SS_TRY(cudaStreamSynchronize(stream));
    return SSMUL_OK;
}

}  // namespace

extern "C" ssmul_status ssmul_mul_noalloc(const uint8_t* d_a, size_t na, const uint8_t* d_b,
                                          size_t nb, uint8_t* d_z, ssmul_result* h_res,
                                          void* cuda_stream) {
    if (!d_a || !d_b || !d_z || na == 0 || nb == 0) return SSMUL_INVALID_ARG;
    if (na + nb > SSMUL_NOALLOC_MAX_DIGITS) return SSMUL_TOO_LARGE;
    int dev = -1;
    SS_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= NOALLOC_MAX_DEVICES) return SSMUL_CUDA_ERROR;
    cudaStream_t stream = static_cast<cudaStream_t>(cuda_stream);
    for (int attempt = 0;; ++attempt) {
        ssmul_status err = SSMUL_OK;
        unsigned char* base = noalloc_setup(dev, stream, attempt > 0, &err);
        if (!base) return err;
        ssmul_result r{};
        err = noalloc_run(base, d_a, na, d_b, nb, d_z, stream, &r);
        if (err != SSMUL_OK) return err;
        // the table was missing (see k_noalloc_init): build it, run once more
        if (r.status == SSMUL_CUDA_ERROR && attempt == 0) continue;
        if (h_res) *h_res = r;
        return ssmul_status(r.status);
    }
}
