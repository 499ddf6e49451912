// Internal declarations shared by the host runtime and the kernels.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <utility>
#include <vector>

#include "../../include/smf.h"

namespace smf {

// Largest basis the kernels handle (primes of at most 26 bits, up to ~6600
// bits of result bound).
constexpr int kMaxPrimes = 256;
// Largest result width (32-bit limbs of M) handled by the CRT kernel.
constexpr int kMaxMLimbs = kMaxPrimes + 1;

// Device-resident constants of a basis (Section 3.1: the basis carries its
// inverses and reduction constants, computed once when it is built).  All pointers index device memory owned by the basis.
struct BasisDev {
    int L;
    int m_limbs;              // 32-bit limbs of M = prod p_i
    const uint32_t* p;        // [L] primes, descending
    const uint64_t* mu;       // [L] floor((2^64 - 1) / p_i), Barrett reduction
    const uint32_t* pow32;    // [L] 2^32 mod p_i
    const double* inv_p;      // [L] 1/p_i rounded to fp64 (Section 3.1 fast reduction)
    // Garner: for j < i, w[i*L + j] = p_j mod p_i with its Shoup companion
    // floor(w * 2^32 / p_i); inv[i] = (p_0 ... p_{i-1})^-1 mod p_i likewise.
    const uint32_t* gw;
    const uint32_t* gws;
    const uint32_t* ginv;
    const uint32_t* ginvs;
    const uint32_t* m_words; // [m_limbs] limbs of M
};

// Host copies of the Garner constants (the CRT kernel takes them by value).
struct CrtHost {
    int L = 0, m_limbs = 0;
    const uint32_t* p = nullptr;      // [L]
    const uint32_t* gw = nullptr;     // [L*L], W_k mod p_i at i*L + k
    const uint32_t* gws = nullptr;    // [L*L] Shoup companions
    const uint32_t* ginv = nullptr;   // [L]
    const uint32_t* ginvs = nullptr;  // [L]
    const uint32_t* m = nullptr;      // [m_limbs] limbs of M
    // Lagrange form with H = (M-1)/2 and M_i = M / p_i
    const uint32_t* hmod = nullptr;   // [L] H mod p_i
    const uint32_t* c = nullptr;      // [L] M_i^-1 mod p_i
    const uint32_t* cs = nullptr;     // [L] Shoup companions of c
    const uint32_t* mi = nullptr;     // [L][m_limbs] limbs of M_i
    const uint32_t* h = nullptr;      // [m_limbs] limbs of H
};

}  // namespace smf

struct smf_basis {
    smf_ctx* ctx;
    int device;
    std::vector<uint32_t> primes;
    std::vector<uint32_t> m_limbs;  // host copy of M
    int m_bits;                     // bit length of M
    void* dev_blob;                 // one allocation holding all tables
    smf::BasisDev dev;
    // host copies of the CRT tables
    std::vector<uint32_t> gw, gws, ginv, ginvs, hmod, c, cs, mi, h;
    smf::CrtHost crt;
};

struct smf_prof_rec {
    int kind;
    cudaEvent_t start, stop;
};

// default thresholds of the eliminations by panels (smf_set_elim_panels)
constexpr int64_t kElimPanelMinN = 2560;       // determinants
constexpr int64_t kElimLocalPanelMinN = 1536;  // local Smith forms

struct smf_ctx {
    int device;
    smf_form form;
    size_t budget;
    int num_sms;
    std::string err;
    void* ws;          // context-owned workspace (lazily grown)
    size_t ws_bytes;
    int* d_status;     // device status word (bounded-wait timeouts)
    int inject;        // failure injection flags for the next limb launch (tests)
    cudaStream_t aux;  // side stream: the A reduction overlaps the B reduction
    cudaEvent_t ev_fork, ev_join;
    // host-operand pipeline: copy-in and copy-out streams and their events
    cudaStream_t h2d, d2h;
    cudaEvent_t pev[12];
    // grouped products: pinned staging of the launch descriptors, and the event
    // after which the last copy out of it has finished
    void* gdesc_host;
    size_t gdesc_cap;
    cudaEvent_t gdesc_ev;
    bool prof;
    std::vector<smf_prof_rec> prof_recs;
    std::vector<cudaEvent_t> event_pool;
    // bases cached by rns_matmul: (bound_bits, p_max) -> basis
    std::vector<std::pair<std::pair<int, uint32_t>, smf_basis*>> basis_cache;
    // 1: single products whose residue product can take the CRT in its
    // epilogue run as one fused kernel (smf_set_fused_crt)
    int fused_crt = 0;
    // eliminations over Z/(m) of matrices with at least this many columns run
    // by panels of 16 columns (smf_set_elim_panels): determinants, and local
    // Smith forms, whose column loop keeps every column live and so gains from
    // panels at smaller sizes (measured: n = 1009 9 % slower by panels, n = 2003
    // 9 % faster)
    int64_t elim_panel_min_n = kElimPanelMinN;
    int64_t elim_local_panel_min_n = kElimLocalPanelMinN;
    // grouped-product plans: the autotuner's measured choice per product class
    // (key: basis size, A's digit count and the log2 sizes; value: 1 = three digits)
    std::vector<std::pair<uint64_t, int>> tune_cache;
    // pinned host staging of the Smith-form driver's digit sums, kept across calls
    // (allocating and freeing pinned memory per call would synchronise the device)
    void* pinned[2] = {nullptr, nullptr};
    size_t pinned_cap[2] = {0, 0};
};

namespace smf {

// Programmatic dependent launch.  A kernel launched by launch_pdl may start
// while the kernel before it on the stream still runs: it calls pdl_wait()
// before it touches anything (griddepcontrol.wait returns once the previous
// grid has completed and its writes are visible), then pdl_trigger() so that
// the kernel after it may start early in turn.  In a normal launch both are
// no-ops.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

template <typename... KArgs, typename... Args>
cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                       Args&&... args) {
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}


// Kernel timing (smf_profile_enable): a scope brackets the launches issued in
// it with two events from the context's pool, recorded on its stream.
inline cudaEvent_t take_event(smf_ctx* c) {
    if (!c->event_pool.empty()) {
        cudaEvent_t e = c->event_pool.back();
        c->event_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

struct ProfScope {
    smf_ctx* c;
    int kind;
    cudaStream_t s;
    cudaEvent_t start = nullptr;
    ProfScope(smf_ctx* c_, int kind_, cudaStream_t s_) : c(c_), kind(kind_), s(s_) {
        if (c->prof) {
            start = take_event(c);
            cudaEventRecord(start, s);
        }
    }
    ~ProfScope() {
        if (start) {
            cudaEvent_t stop = take_event(c);
            cudaEventRecord(stop, s);
            c->prof_recs.push_back({kind, start, stop});
        }
    }
};

// Stream-ordered device scratch (cudaMallocAsync / cudaFreeAsync on the stream
// the work runs on): no device-wide synchronisation when it is freed, so calls
// on different streams keep overlapping.
struct StreamBuf {
    void* p = nullptr;
    cudaStream_t s = nullptr;
    StreamBuf() = default;
    StreamBuf(const StreamBuf&) = delete;
    StreamBuf& operator=(const StreamBuf&) = delete;
    cudaError_t alloc(size_t bytes, cudaStream_t st) {
        release();
        s = st;
        return cudaMallocAsync(&p, bytes ? bytes : 1, st);
    }
    void release() {
        if (p) cudaFreeAsync(p, s);
        p = nullptr;
    }
    ~StreamBuf() { release(); }
};

// Pinned host staging slot `slot` (0 or 1) of the context, at least `bytes`
// (grown when needed, freed with the context); nullptr on failure.
inline void* ctx_pinned(smf_ctx* c, int slot, size_t bytes) {
    if (c->pinned_cap[slot] < bytes) {
        if (c->pinned[slot]) cudaFreeHost(c->pinned[slot]);
        c->pinned[slot] = nullptr;
        c->pinned_cap[slot] = 0;
        if (cudaMallocHost(&c->pinned[slot], bytes) != cudaSuccess) {
            cudaGetLastError();
            c->pinned[slot] = nullptr;
            return nullptr;
        }
        c->pinned_cap[slot] = bytes;
    }
    return c->pinned[slot];
}

// A basis cached in the context (created on first use, destroyed with the context).
smf_basis* ctx_basis(smf_ctx* ctx, int bound_bits, uint32_t p_max, int* status);

// Device status word bits.
constexpr int kStatusTimeout = 1;
constexpr int kStatusInexact = 2;  // p-adic lifting: a residual was not divisible by p
constexpr int kStatusSingular = 4; // inverse mod p: a column without a pivot (p divides det A)
constexpr int kStatusBound = 8;    // an operand entry lies outside its declared bound (smf_bigmat.bits)

// ---------------------------------------------------------------- launches

// Generic reduction of a big-integer matrix to per-prime outputs.
enum class ReduceOut {
    kCanonical = 0,   // int32 [L][rows][cols] in [0, p)
    kCentered = 1,    // int32 [L][rows][cols] in [-(p-1)/2, (p-1)/2]
    kDigits = 2,      // bf16 digit planes [L][t][rows][ld_out]
    kDigitsT = 3,     // bf16 digit planes, transposed and digit-major: [t][L][cols][ld_out]
};

struct ReduceArgs {
    const uint64_t* X;
    int64_t rows, cols, ld;
    int W;
    void* out;
    int64_t ld_out;   // digit planes: leading dimension (elements)
    int t;            // digit planes: digits per residue
    int identity;     // 1: skip reduction, the value itself is centred (|x| small)
    int bits;         // declared bound |x| <= 2^bits: an entry beyond it sets kStatusBound (0: not checked)
    int* status;      // set by launch_reduce
};

cudaError_t launch_reduce(const BasisDev& b, const ReduceArgs& a, ReduceOut kind, int* d_status,
                          cudaStream_t s);

// Work lists of the grouped launches.  The work units of item i are
// [base_i, base_(i+1)) of one launch (bases ascending, base_0 = 0); a block
// walks units in steps of the grid and finds each unit's item by bisection.
struct ReduceItem {       // one operand of a grouped digit split or transposed reduce
    const uint64_t* X;
    int64_t rows, cols, ld;
    void* out;
    int64_t ld_out;
    int W, t;
    int bits;             // declared bound of the entries (checked; >= 64 W - 1: not checked)
    int rb;               // transposed reduce: rows per unit (set by reduce_t_units)
    int64_t base;
    // digit split: floor(e / cols) = (umulhi(e, div_m) + e) >> div_s for e < 2^32
    // (division by an invariant integer, Granlund and Montgomery; set by split_units)
    uint32_t div_m;
    int div_s;
};
struct CrtItem {          // one output of a grouped CRT
    const int32_t* R;     // [L][rows][cols]
    int64_t rows, cols;
    uint64_t* X;
    int64_t ld;
    int W;
    int64_t base;
};
#ifdef __CUDACC__
// (hi:lo) += a * b as one carry chain: the low word with carry out, the high
// word with carry in (the 64-bit sum must not overflow).  Two instructions per
// product, where a 64-bit accumulation written in C takes more.
__device__ __forceinline__ void mac64(uint32_t& lo, uint32_t& hi, uint32_t a, uint32_t b) {
    asm("mad.lo.cc.u32 %0, %2, %3, %0;\n\tmadc.hi.u32 %1, %2, %3, %1;" : "+r"(lo), "+r"(hi) : "r"(a), "r"(b));
}
template <class Item>
__device__ __forceinline__ const Item* find_item(const Item* items, int n, int64_t u) {
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (items[mid].base <= u) lo = mid;
        else hi = mid - 1;
    }
    return items + lo;
}
#endif
// Work units of one item: transposed reduce of B (rb rows by 1024 / rb
// columns, rb fitted to the row count and returned), digit split of a
// shared-digit A (2048 entries), CRT (128 entries).
int64_t reduce_t_units(int64_t rows, int64_t cols, int* rb);
bool reduce_t_groupable(const BasisDev& b, const ReduceArgs& a);  // W in {1, 2, 4, 8}, aligned, one prime group
int64_t split_units(int64_t rows, int64_t cols, uint32_t* div_m, int* div_s);
int64_t crt_units(int64_t rows, int64_t cols);
// One persistent launch each (grid: the SMs times the blocks resident per SM).
// Transposed reduce: every item has W words.  Split: items are centred values
// (identity), planes [t][rows][ld_out].
cudaError_t launch_reduce_t_grouped(const BasisDev& b, int W, const ReduceItem* items, int n, int64_t units,
                                    int num_sms, int* status, cudaStream_t s);
cudaError_t launch_split_grouped(const ReduceItem* items, int n, int64_t units, int num_sms, int* status,
                                 cudaStream_t s);

// int32 residues (any representative in (-p, p)) -> bf16 balanced digit
// planes, either [L][t][rows][ld_out] or transposed and digit-major
// [t][L][cols][ld_out].
cudaError_t launch_residue_digits(const BasisDev& b, const int32_t* R, int64_t prime_stride,
                                  int Lcount, int64_t rows, int64_t cols, void* out,
                                  int64_t ld_out, int t, bool transpose, cudaStream_t s);

// FP64 residue GEMM (Section 3.1: exact double-precision products).
struct Fp64GemmArgs {
    const int32_t* A;
    int64_t a_prime_stride;
    const int32_t* B;
    int32_t* C;
    int64_t M, N, K;
    int kblk;          // products accumulated between reductions
};
cudaError_t launch_gemm_fp64(const BasisDev& b, const Fp64GemmArgs& a, cudaStream_t s);
// Measured FP64 FMA throughput of the device (TFLOP/s; 0 on failure).  Synchronous.
double fp64_fma_peak_tflops(int num_sms, cudaStream_t s);

// INT8-limb residue GEMM on tcgen05 (bf16-held digits, fp32 TMEM accumulation).
struct LimbGemmArgs {
    const void* Adig;        // bf16 [planesA][M][lda]
    int64_t lda;
    int a_shared;            // 1: planes [TA][M][lda] shared by all primes
    const void* Bdig;        // bf16 [TB][L][N][ldb] (digit-major: each digit plane spans all primes)
    int64_t ldb;
    int32_t* C;              // [L][M][N]
    int64_t M, N, K;
    int TA, TB;
    int* d_status;
    int inject;              // SMF_INJECT_* flags (tests of the bounded waits)
    uint64_t amax, bmax;     // bounds on |A| and |B| entries: their digit bounds set the fold block
    // split-K (3x3 digits, few tiles): `split` launches of `kchunk` K steps each
    // write canonical partial residues to part [split][L][M][N], summed mod p into C
    int32_t* part;
    int split, kchunk;
    int keep_parts;          // 1: leave the partials for the caller's own kernel to sum (C is not written)
    int pdl;                 // 1: launch as a programmatic dependent of the kernel before it (launch_pdl)
    int pf;                  // grouped launch: K steps of L2 prefetch ahead of the loads (0: none)
    int bn;                  // kernels for fewer than 3x3 digits: tile width 48 (0) or 64 (1x3 and 2x3 digits)
};
// Split-K of a 3x3-digit product with too few tiles for the SMs: the number of
// K splits (1 = none) and the K steps of each (every split non-empty).
void limb_split(int L, int64_t M, int64_t N, int64_t K, bool a_shared, int TA, int TB, int num_sms, int* split,
                int* kchunk);
// Relative time of a limb product (waves x (K steps per unit + fill) x digit
// pairs x tile width), for choosing between digit counts of an operand.
double limb_cost(int L, int64_t M, int64_t N, int64_t K, bool a_shared, int TA, int TB, int num_sms);
// Tile width of the kernels for fewer than 3x3 digits: 64 (MMA N = 192, one
// tile for 64 columns) where its waves x width come out below 48's, else 48
// (num_sms = 0: 48).
int limb_narrow_bn(int L, int64_t M, int64_t N, int64_t K, bool a_shared, int TA, int TB, int num_sms);
// One launch over the tiles of several products (Adig, Bdig, C, shapes and A's
// digit count per product, one basis); desc_dev holds limb_group_desc_bytes(count).
size_t limb_group_desc_bytes(int count);
bool limb_group_supported(const LimbGemmArgs& a);  // TA in 1..3, TB = 3
struct LimbGroup {
    int count;      // non-empty products (descriptors written)
    int first;      // index of the first of them in the argument array
    int64_t tiles;  // tiles over all of them
    int kblk;       // the smallest fold block among them
};
// Host half: the descriptors of the non-empty products into `host`
// (limb_group_desc_bytes(count) bytes).  Device half: one persistent launch
// over those descriptors once they have been copied to `desc_dev`.
// tile_order: 0 longest K first, 1 most MMAs per tile (K times A's digits) first.
cudaError_t limb_group_encode(const BasisDev& b, const LimbGemmArgs* probs, int count, void* host, int tile_order,
                              LimbGroup* out);
cudaError_t limb_group_launch(smf_ctx* ctx, const BasisDev& b, const LimbGemmArgs* probs, const LimbGroup& g,
                              const void* desc_dev, cudaStream_t s);
// The same launch for products whose A has one digit, in the kernel whose
// ring holds five K steps of one-digit operands (40 KB each) instead of the
// 3x3-digit kernel's three 72 KB slots.
cudaError_t limb_group_launch_one_digit(smf_ctx* ctx, const BasisDev& b, const LimbGemmArgs* probs,
                                       const LimbGroup& g, const void* desc_dev, cudaStream_t s);
cudaError_t launch_gemm_limb(smf_ctx* ctx, const BasisDev& b, const LimbGemmArgs& a,
                             cudaStream_t s);
// The 3x3-digit residue product with the CRT in its epilogue: X (M x N, W
// words, leading dimension ld) = the integers of the residues it computes
// into a.C.  Fusable: 3x3 digits, no K split, at most 24 primes below 2^24,
// tiles within one prime (a shared A needs N a multiple of 64).  count:
// limb_crt_units(M, N) ints of scratch (zeroed by the launch on s).
bool limb_crt_fusable(const CrtHost& h, const LimbGemmArgs& a);
int64_t limb_crt_units(int64_t M, int64_t N);
cudaError_t launch_gemm_limb_crt(smf_ctx* ctx, const BasisDev& b, const CrtHost& h, const LimbGemmArgs& a,
                                 int* count, uint64_t* X, int64_t ld, int W, cudaStream_t s);

// CRT reconstruction: Lagrange form with an fp32 correction, exact mixed-radix (Garner) fallback.
cudaError_t launch_crt(const CrtHost& h, const int32_t* R, int64_t rows, int64_t cols,
                       uint64_t* X, int64_t ld, int W, cudaStream_t s);

cudaError_t launch_crt_grouped(const CrtHost& h, const CrtItem* items, int n, int64_t units, int num_sms,
                               cudaStream_t s);

// Conversion between RNS bases: residues [from.L][count] canonical -> [LQ][count]
// canonical modulo the target primes q (< 2^26), for the symmetric
// representatives of the source basis.  At most 48 primes on either side.
cudaError_t launch_convert(const CrtHost& from, const uint32_t* q, int LQ, const int32_t* R, int32_t* out,
                           int64_t count, int num_sms, cudaStream_t s);

// p-adic lifting: X_i (int32 canonical) -> int64 words; R = (R - AX) / p, exact.
cudaError_t launch_widen(const int32_t* x, int64_t count, int64_t* out, cudaStream_t s);
// A^-1 mod p by Gauss-Jordan over GF(p) (inverse.cu): res = A mod p (int32
// [n][n], canonical); M (n x 2n uint32), col (n) and flag (one int) are
// scratch; C gets A^-1 mod p ([n][n]) unless kStatusSingular is raised.
cudaError_t launch_inverse_mod_p(const int32_t* res, int64_t n, uint32_t p, uint32_t* M, uint32_t* col, int* flag,
                                 int32_t* C, int* status, int num_sms, cudaStream_t s);
// The blocked form (inverse.cu): [res | I] into M (n x 2n); one panel of bw
// columns from c0 reduced on the scratch T = [P | S] (n x 2bw, P filled from
// M, S zero) with its row swaps applied to M's columns [lo, hi); and the
// update of M's columns [c1, c1 + R) from C = S Mp (n x R, canonical).
cudaError_t launch_gj_init(const int32_t* res, int64_t n, uint32_t* M, cudaStream_t s);
cudaError_t launch_panel_factor(uint32_t* T, int64_t n, int bw, int64_t c0, uint32_t* M, int64_t ldM, int64_t lo,
                                int64_t hi, uint32_t p, uint32_t* col, int* flag, int* status, int num_sms,
                                cudaStream_t s);
cudaError_t launch_panel_update(uint32_t* M, int64_t ldM, int64_t n, int64_t c0, int64_t c1, int64_t R,
                                const int32_t* C, uint32_t p, cudaStream_t s);
// Column sums of the p-adic digits weighted by W (invariant.cu):
// out[s][j] = sum_i W[i][j] X[s][i][j] for X [steps][n][m], W [n][m].
cudaError_t launch_lift_combine(const int32_t* X, int64_t steps, int64_t n, int64_t m, const uint32_t* W,
                                uint64_t* out, cudaStream_t s);
// The limb form's step kernels (lift.cu): the product basis of A X_i, at most
// four primes (descending) with inv[j] = (q_0 ... q_(j-1))^-1 mod q_j.
constexpr int kLiftMaxPrimes = 4;
struct LiftBasis {
    int L;
    uint32_t q[kLiftMaxPrimes];
    uint32_t inv[kLiftMaxPrimes];
};
// part: [split][n][m] canonical partials of C R_i mod p -> X (n x m, [0, p)) and
// the centred residues of X modulo q as t-digit planes [t][L][m][ldd].
cudaError_t launch_lift_x(const int32_t* part, int split, int64_t n, int64_t m, uint32_t p, int32_t* X,
                          const LiftBasis& q, void* xdig, int64_t ldd, int t, cudaStream_t s);
// part: [split][L][n][m] canonical partials of A X_i mod q_j -> R = (R - A X_i) / p
// (flags kStatusInexact on a remainder); rdig, when not null, gets the t-digit
// planes [t][m][ldd] of R mod p (centred).
cudaError_t launch_lift_step(const int32_t* part, int split, int64_t n, int64_t m, const LiftBasis& q, int64_t* R,
                             int64_t ldR, uint32_t p, void* rdig, int64_t ldd, int t, int* status, cudaStream_t s);
cudaError_t launch_lift_update(int64_t* R, int64_t ldR, const int64_t* AX, int64_t rows, int64_t cols, uint32_t p,
                               int* status, cudaStream_t s);

// Bytes of device workspace for the digit planes of each form.
inline int64_t round_up(int64_t x, int64_t m) { return (x + m - 1) / m * m; }

// Digits in balanced base 2^8 needed for |x| <= h.  The lower t-1 digits lie
// in [-128, 127]; the top digit is the remaining quotient, |top| <= 128.
// t digits therefore cover |x| <= 128 * 256^(t-1) + 127 * (256^(t-1) - 1) / 255.
inline int digits_for(uint64_t h) {
    uint64_t lower = 0, scale = 1;  // 127 * (256^(t-1) - 1) / 255, 256^(t-1)
    int t = 1;
    while (128 * scale + lower < h) {
        lower += 127 * scale;
        scale *= 256;
        t++;
    }
    return t;
}

}  // namespace smf
