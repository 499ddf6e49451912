// Largest invariant factor s_n of a nonsingular integer matrix (the paper's
// Phase 1, Section 2: a Monte Carlo method that gives the initial modulus of
// the massager iterations).  Host driver over this library's calls:
//  1. a prime p below 2^24 (below 2^(60 - bits(A) - log2 n) for wide entries)
//     with A invertible mod p: A^-1 mod p by Gauss-Jordan on the device
//     (smf_inverse_mod_p); on p | det A the next prime below;
//  2. m random right-hand sides B (n x m, |b| <= 2^10) and p-adic lifting of
//     A^-1 B (smf_padic_lift), at most to k digits, p^k > 2 N D, where D bounds
//     det A and N the numerators below (Hadamard's bound on rows); it stops
//     earlier once every column's fraction has settled (below);
//  3. per column j, the weighted digit sums c_s,j = sum_i w_ij X_s,ij on the
//     device, so that z_j = sum_s c_s,j p^s = w_j . A^-1 b_j (mod p^k) for
//     random weights w_ij in [1, 2^16);
//  4. rational reconstruction of each z_j = a_j / d_j on the host (extended
//     Euclid), and s = lcm_j d_j.
// Every d_j divides s_n (s_n A^-1 is integral), so s divides s_n.  For a
// prime q | s_n, column j misses q's full power only if b_j falls in a
// sublattice of index q (probability at most 1/q + 2^-10 over the box of b)
// or the weights w_j cancel it (at most 1/q + 2^-16); for q = 2 that is about
// 3/4 per column, so all m columns miss it with probability about (3/4)^m.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <thread>

#include "smith_internal.h"

namespace smf {
namespace {

constexpr int kCombineThreads = 256;

__global__ void __launch_bounds__(kCombineThreads) lift_combine_kernel(const int32_t* __restrict__ X, int64_t n,
                                                                       int64_t m, const uint32_t* __restrict__ W,
                                                                       uint64_t* __restrict__ out) {
    extern __shared__ unsigned long long acc[];
    const int64_t s = blockIdx.x;
    for (int64_t j = threadIdx.x; j < m; j += kCombineThreads) acc[j] = 0;
    __syncthreads();
    const int32_t* xs = X + s * n * m;
    for (int64_t e = threadIdx.x; e < n * m; e += kCombineThreads)
        atomicAdd(&acc[e % m], (unsigned long long)W[e] * (uint32_t)xs[e]);
    __syncthreads();
    for (int64_t j = threadIdx.x; j < m; j += kCombineThreads) out[s * m + j] = acc[j];
}

// Pairing digit sums for the Smith-form driver's projection (Phase 2):
// out[s][a][j] = sum_i Q[i][a] X[s][i][j] for j < c (the first c of the m
// lifted columns) and a < CP functionals.  Thread (g, j) of a block (one
// block per digit) sums rows i = g mod G for all CP functionals in
// registers; the G partial sums meet in shared memory.  Every term is below
// 2^40 (Q < 2^16, X < 2^24) and n < 2^14, so the sums stay below 2^54.
template <int CP>
__global__ void __launch_bounds__(kCombineThreads) lift_pair_kernel(const int32_t* __restrict__ X, int64_t n,
                                                                    int64_t m, int c, const uint32_t* __restrict__ Qt,
                                                                    uint64_t* __restrict__ out) {
    extern __shared__ unsigned long long part[];  // [G][CP][c]
    const int G = kCombineThreads / c;
    const int g = threadIdx.x / c, j = threadIdx.x % c;
    const int64_t s = blockIdx.x;
    unsigned long long acc[CP];
#pragma unroll
    for (int a = 0; a < CP; a++) acc[a] = 0;
    if (g < G) {
        const int32_t* xs = X + s * n * m;
        for (int64_t i = g; i < n; i += G) {
            const unsigned long long x = (uint32_t)xs[i * m + j];
            const uint32_t* q = Qt + i * CP;
#pragma unroll
            for (int a = 0; a < CP; a++) acc[a] += x * q[a];
        }
#pragma unroll
        for (int a = 0; a < CP; a++) part[((size_t)g * CP + a) * c + j] = acc[a];
    }
    __syncthreads();
    for (int e = threadIdx.x; e < CP * c; e += kCombineThreads) {
        unsigned long long t = 0;
        for (int h = 0; h < G; h++) t += part[(size_t)h * CP * c + e];
        out[s * CP * c + e] = t;
    }
}

// splitmix64 (Steele, Lea and Flood, 2014): the driver's own random stream
struct SplitMix64 {
    uint64_t x;
    uint64_t next() {
        uint64_t z = (x += 0x9e3779b97f4a7c15ull);
        z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
        z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
        return z ^ (z >> 31);
    }
    uint64_t below(uint64_t bound) {  // uniform in [0, bound) by rejection
        const uint64_t lim = UINT64_MAX - UINT64_MAX % bound;
        uint64_t v;
        do v = next();
        while (v >= lim);
        return v % bound;
    }
};

int fail_with(smf_ctx* ctx, int code, const char* msg) {
    ctx->err = msg;
    return code;
}

constexpr int kRhsBits = 10;     // |b| <= 2^10
constexpr int kWeightBits = 16;  // w in [1, 2^16)
constexpr int kMaxTries = 8;     // primes tried before A is declared singular
constexpr int64_t kChunk = 64;   // lifting steps per call
constexpr int64_t kFirstCheckpoint = 128;  // digits before the first early reconstruction
constexpr int64_t kMarginBits = 64;        // bits of p^k' left unused by the early bounds
constexpr int64_t kAheadMinN = 3000;       // above this n, two chunks run during a checkpoint

int64_t clog2(int64_t k) {
    int64_t b = 0;
    while (((int64_t)1 << b) < k) b++;
    return b;
}

}  // namespace

cudaError_t launch_lift_combine(const int32_t* X, int64_t steps, int64_t n, int64_t m, const uint32_t* W,
                                uint64_t* out, cudaStream_t s) {
    if (steps == 0 || m == 0) return cudaSuccess;
    lift_combine_kernel<<<(unsigned)steps, kCombineThreads, sizeof(unsigned long long) * m, s>>>(X, n, m, W, out);
    return cudaGetLastError();
}

cudaError_t launch_lift_pair(const int32_t* X, int64_t steps, int64_t n, int64_t m, int c, int cp, const uint32_t* Qt,
                             uint64_t* out, cudaStream_t s) {
    if (steps == 0 || c == 0) return cudaSuccess;
    if (c > 32 || kCombineThreads % c || (cp != 16 && cp != 32)) return cudaErrorInvalidValue;
    const size_t smem = sizeof(unsigned long long) * (kCombineThreads / c) * cp * c;
    if (cp == 16) {
        cudaFuncSetAttribute(lift_pair_kernel<16>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        lift_pair_kernel<16><<<(unsigned)steps, kCombineThreads, smem, s>>>(X, n, m, c, Qt, out);
    } else {
        cudaFuncSetAttribute(lift_pair_kernel<32>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        lift_pair_kernel<32><<<(unsigned)steps, kCombineThreads, smem, s>>>(X, n, m, c, Qt, out);
    }
    return cudaGetLastError();
}

}  // namespace smf

using namespace smf;

int smf::lif_run(smf_ctx* ctx, const smf_bigmat* A, const LifOptions& o, LifResult* res, cudaStream_t s) {
    const int32_t m = o.m;
    const uint64_t seed = o.seed;
    const int cp = o.pair_rows, cq = o.pair_cols;
    if (!A || m < 1 || m > 1024)
        return fail_with(ctx, SMF_E_INVALID, "largest_invariant_factor: bad argument");
    if (cp && ((cp != 16 && cp != 32) || cq < 1 || cq > m || cq > 32 || 256 % cq))
        return fail_with(ctx, SMF_E_INVALID, "largest_invariant_factor: bad pairing shape");
    if (A->rows != A->cols || A->rows < 1 || A->words != 1 || A->ld < A->cols || !A->data || A->bits < 0)
        return fail_with(ctx, SMF_E_INVALID, "largest_invariant_factor: A must be n x n (n >= 1), single words");
    using clk = std::chrono::steady_clock;
    const auto t0 = clk::now();
    int dev0 = 0;
    cudaGetDevice(&dev0);
    cudaSetDevice(ctx->device);
    struct Restore {
        int d;
        ~Restore() { cudaSetDevice(d); }
    } restore{dev0};
    const int64_t n = A->rows;
    if (n >= (1 << 14))
        return fail_with(ctx, SMF_E_UNSUPPORTED, "largest_invariant_factor: n must stay below 16384 (digit sums)");
    const int abits = A->bits > 0 ? A->bits : 63;
    // 1. A on the host (the bounds) and contiguous on the device (the solves)
    std::vector<int64_t> Ah((size_t)n * n);
    // in order on s (A may have just been written there), then waited for
    if (cudaMemcpy2DAsync(Ah.data(), 8 * n, A->data, 8 * A->ld, 8 * n, n,
                          A->on_device ? cudaMemcpyDeviceToHost : cudaMemcpyHostToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) {
        cudaGetLastError();
        return fail_with(ctx, SMF_E_CUDA, "largest_invariant_factor: copy of A failed");
    }
    // Hadamard: |det A| <= prod_i ||a_i|| = 2^hd; a numerator of A^-1 b is a
    // determinant with one column replaced by b: at most prod_i (||a_i||^2 + b_i^2)^(1/2) = 2^hn
    double hd = 0, hn = 0;
    const double b2 = std::ldexp(1.0, 2 * kRhsBits);
    for (int64_t i = 0; i < n; i++) {
        double r2 = 0;
        for (int64_t j = 0; j < n; j++) r2 += (double)Ah[i * n + j] * (double)Ah[i * n + j];
        if (r2 == 0) return fail_with(ctx, SMF_E_SINGULAR, "largest_invariant_factor: A has a zero row");
        hd += 0.5 * std::log2(r2);
        hn += 0.5 * std::log2(r2 + b2);
    }
    // |w . adj(A) b| <= n 2^16 2^hn; one bit of margin each for rounding
    const int64_t db = (int64_t)std::ceil(hd) + 1;
    const int64_t nb = (int64_t)std::ceil(hn) + clog2(n) + kWeightBits + 1;
    // scratch in stream order on s (no device-wide synchronisation when freed)
    StreamBuf Ad, Cd, inv_ws, Rd, Wd, Xd, cd, lift_ws, Qd, pd;
    if (Ad.alloc(8 * (size_t)n * n, s) != cudaSuccess || Cd.alloc(4 * (size_t)n * n, s) != cudaSuccess) {
        cudaGetLastError();
        return fail_with(ctx, SMF_E_NOMEM, "largest_invariant_factor: device allocation failed");
    }
    if (cudaMemcpyAsync(Ad.p, Ah.data(), 8 * (size_t)n * n, cudaMemcpyHostToDevice, s) != cudaSuccess)
        return fail_with(ctx, SMF_E_CUDA, "largest_invariant_factor: copy of A failed");
    smf_bigmat Am{n, n, n, 1, abits, Ad.p, 1, 0};
    size_t inv_bytes = 0;
    smf_inverse_mod_p_workspace(ctx, n, &inv_bytes);
    if (inv_ws.alloc(inv_bytes, s) != cudaSuccess) {
        cudaGetLastError();
        return fail_with(ctx, SMF_E_NOMEM, "largest_invariant_factor: device allocation failed");
    }
    // 2. the prime (one-prime bases cached in the context)
    smf_basis* pb = nullptr;
    // the lifting prime: below 2^24, smaller for wide entries so that the
    // residuals (|R| <= 2 n |A| p) keep fitting 64-bit words
    const int64_t pb_cap = std::min<int64_t>(24, 62 - abits - clog2(n) - 2);
    if (pb_cap < 5)
        return fail_with(ctx, SMF_E_BOUND, "largest_invariant_factor: entries too wide for 64-bit residuals");
    uint32_t p = 0, p_max = 1u << pb_cap;
    int st = SMF_OK;
    for (int attempt = 0; attempt < kMaxTries; attempt++) {
        if (!(pb = ctx_basis(ctx, 1, p_max, &st))) return st;
        const uint32_t* primes = nullptr;
        int32_t L = 0;
        smf_basis_info(pb, &L, &primes);
        p = primes[0];
        if ((st = smf_inverse_mod_p(ctx, pb, &Am, (int32_t*)Cd.p, inv_ws.p, inv_bytes, s))) return st;
        st = smf_status_sync(ctx, s);
        if (st == SMF_OK) break;
        if (st != SMF_E_SINGULAR) return st;
        p_max = p;
    }
    if (st == SMF_E_SINGULAR)
        return fail_with(ctx, SMF_E_SINGULAR, "largest_invariant_factor: det A vanishes modulo 8 primes (singular)");
    const auto t1 = clk::now();
    int pbits = 0;
    while ((1ull << pbits) <= p) pbits++;
    if (abits + pbits + clog2(n) + 2 > 62)
        return fail_with(ctx, SMF_E_BOUND, "largest_invariant_factor: n |A| p too large for 64-bit residuals");
    // 3. lifting to k digits, p^k > 2^(nb + db + 1)
    // the projection's values s P (s <= 2^db, numerators below 2^nb) are read
    // with 65 bits to spare: its cap leaves room for them
    const int64_t cap_bits = nb + db + 1 + (cp ? db + 70 : 0);
    const int64_t k = (int64_t)std::ceil((double)cap_bits / std::log2((double)p)) + 1;
    SplitMix64 rng{seed};
    std::vector<int64_t> Bh((size_t)n * m);
    for (auto& b : Bh) b = (int64_t)rng.below((2ull << kRhsBits) + 1) - (1ll << kRhsBits);
    std::vector<uint32_t> Wh((size_t)n * m);
    for (auto& w : Wh) w = 1 + (uint32_t)rng.below((1u << kWeightBits) - 1);
    std::vector<uint32_t> Qh((size_t)n * cp);  // [i][a]: the functionals of the pairing
    for (auto& w : Qh) w = 1 + (uint32_t)rng.below((1u << kWeightBits) - 1);
    const int64_t chunk = std::min<int64_t>(kChunk, k);
    if (Rd.alloc(8 * (size_t)n * m, s) != cudaSuccess || Wd.alloc(4 * (size_t)n * m, s) != cudaSuccess ||
        Xd.alloc(4 * (size_t)chunk * n * m, s) != cudaSuccess || cd.alloc(8 * (size_t)chunk * m, s) != cudaSuccess ||
        (cp && (Qd.alloc(4 * (size_t)n * cp, s) != cudaSuccess ||
                pd.alloc(8 * (size_t)chunk * cp * cq, s) != cudaSuccess))) {
        cudaGetLastError();
        return fail_with(ctx, SMF_E_NOMEM, "largest_invariant_factor: device allocation failed");
    }
    if (cp && cudaMemcpyAsync(Qd.p, Qh.data(), 4 * (size_t)n * cp, cudaMemcpyHostToDevice, s) != cudaSuccess)
        return fail_with(ctx, SMF_E_CUDA, "largest_invariant_factor: copy of the functionals failed");
    if (cudaMemcpyAsync(Rd.p, Bh.data(), 8 * (size_t)n * m, cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaMemcpyAsync(Wd.p, Wh.data(), 4 * (size_t)n * m, cudaMemcpyHostToDevice, s) != cudaSuccess)
        return fail_with(ctx, SMF_E_CUDA, "largest_invariant_factor: copy of B failed");
    // |R_i| <= max(|B|, 2 n |A| p)
    const int rbits = (int)std::max<int64_t>(kRhsBits, abits + pbits + clog2(n) + 1);
    smf_bigmat Rm{n, m, m, 1, rbits, Rd.p, 1, 0};
    size_t lift_bytes = 0;
    if ((st = smf_padic_lift_workspace(ctx, pb, &Am, &Rm, &lift_bytes))) return st;
    if (lift_bytes && lift_ws.alloc(lift_bytes, s) != cudaSuccess) {
        cudaGetLastError();
        return fail_with(ctx, SMF_E_NOMEM, "largest_invariant_factor: device allocation failed");
    }
    // Lifting in chunks, with checkpoints geometric in the number of digits.
    // At a checkpoint of k' digits the unsettled columns are reconstructed with
    // balanced bounds that leave kMarginBits of p^k' unused (a fraction that
    // small arises by chance with probability about 2^-64), and a column
    // settles when the same denominator comes back at the next checkpoint one
    // chunk later.  The Hadamard precision k caps the lifting; there the
    // remaining columns are reconstructed with the proven bounds.
    struct {
        void* p;
    } cbuf{ctx_pinned(ctx, 0, 8 * (size_t)k * m)}, pbuf{cp ? ctx_pinned(ctx, 1, 8 * (size_t)k * cp * cq) : nullptr};
    if (!cbuf.p || (cp && !pbuf.p))
        return fail_with(ctx, SMF_E_NOMEM, "largest_invariant_factor: pinned host allocation failed");
    const uint64_t* c = (const uint64_t*)cbuf.p;
    std::vector<Nat> den(m), cand(m);
    std::vector<int> settled(m, 0), has_cand(m, 0), failed(m, 0);
    const int nt = (int)std::max<unsigned>(1, std::min<unsigned>(std::thread::hardware_concurrency(), m));
    const double lp = std::log2((double)p);
    double recon_s = 0;
    auto reconstruct = [&](int64_t kk, int64_t nbb, int64_t dbb, bool proven) {
        const auto r0 = clk::now();
        const Nat Pk = pow_small(p, kk);
        const std::vector<Nat> pw = horner_powers(p, kk);  // Horner by halves, shared by the columns
        // the columns' fractions have about the same size: before any column has
        // a candidate, a checkpoint tries the first unsettled column alone
        int64_t probe = -1, skip = -1;
        if (!proven && std::none_of(has_cand.begin(), has_cand.end(), [](int v) { return v != 0; }))
            probe = std::find(settled.begin(), settled.end(), 0) - settled.begin();
        // threads only for wide values (a thread costs tens of microseconds)
        const int nw = (double)kk * lp < 2048.0 ? 1 : nt;
        // A known denominator D < 2^dbb (the column's candidate, else the reference:
        // a denominator already found at this precision or settled) is tried first:
        // if D z mod P^k is within 2^nbb of 0, then (P^k > 2^(nbb + dbb + 1)) y / D
        // is z's fraction, whose denominator divides D, found by one product and
        // one Barrett reduction instead of an extended Euclid.
        const Nat* ref = nullptr;
        for (int64_t j = 0; j < m && !ref; j++) ref = settled[j] ? &den[j] : has_cand[j] ? &cand[j] : nullptr;
        Barrett br;
        bool have_br = false;
        auto divides = [&](const Nat& z, const Nat& D) {
            if (D.bits() > dbb) return false;
            const Nat y = barrett_mod(br, mul(D, barrett_mod(br, z)));
            return y.bits() <= nbb || sub(br.m, y).bits() <= nbb;
        };
        auto work = [&](int t) {
            for (int64_t j = t; j < m; j += nw) {
                if (settled[j] || (probe >= 0 && j != probe) || j == skip) continue;
                const Nat z = horner_split(c + j, kk, (size_t)m, p, 30 + pbits, pw);  // sums below n 2^16 p
                const Nat* D = has_cand[j] ? &cand[j] : ref;
                if (have_br && D && divides(z, *D)) {
                    if (proven || has_cand[j]) {  // the fraction persists (or the bounds are proven)
                        den[j] = *D;
                        settled[j] = 1;
                    } else {
                        cand[j] = *D;
                        has_cand[j] = 1;
                    }
                    continue;
                }
                Int a;
                Nat d;
                const bool found = rational_reconstruct(z, Pk, nbb, dbb, &a, &d);
                if (proven) {
                    failed[j] = !found;
                    den[j] = std::move(d);
                    settled[j] = 1;
                } else if (found && has_cand[j] && cmp(cand[j], d) == 0) {
                    den[j] = std::move(d);
                    settled[j] = 1;
                } else {
                    has_cand[j] = found;
                    cand[j] = std::move(d);
                }
            }
        };
        if (probe >= 0 && probe < m) {
            work((int)(probe % nw));  // the slot that holds the probe column
            if (!has_cand[probe]) {
                recon_s += std::chrono::duration<double>(clk::now() - r0).count();
                return;
            }
            skip = probe;  // found: the other columns at the same precision
            ref = &cand[probe];
            probe = -1;
        }
        Nat ref_copy;  // the threads may replace the candidate it came from
        if (ref) {
            ref_copy = *ref;
            ref = &ref_copy;
        }
        if (ref || std::any_of(has_cand.begin(), has_cand.end(), [](int v) { return v != 0; })) {
            br = barrett_of(Pk);
            have_br = true;
        }
        std::vector<std::thread> pool;
        for (int t = 1; t < nw; t++) pool.emplace_back(work, t);
        work(0);
        for (auto& th : pool) th.join();
        recon_s += std::chrono::duration<double>(clk::now() - r0).count();
    };
    auto enqueue = [&](int64_t done, int64_t steps) -> int {
        int rc = smf_padic_lift(ctx, pb, &Am, (const int32_t*)Cd.p, &Rm, (int32_t)steps, (int32_t*)Xd.p, &Rm,
                                lift_ws.p, lift_bytes, s);
        if (rc) return rc;
        if (launch_lift_combine((const int32_t*)Xd.p, steps, n, m, (const uint32_t*)Wd.p, (uint64_t*)cd.p, s) !=
                cudaSuccess ||
            cudaMemcpyAsync((uint64_t*)cbuf.p + done * m, cd.p, 8 * (size_t)steps * m, cudaMemcpyDeviceToHost, s) !=
                cudaSuccess ||
            (cp && (launch_lift_pair((const int32_t*)Xd.p, steps, n, m, cq, cp, (const uint32_t*)Qd.p,
                                     (uint64_t*)pd.p, s) != cudaSuccess ||
                    cudaMemcpyAsync((uint64_t*)pbuf.p + done * cp * cq, pd.p, 8 * (size_t)steps * cp * cq,
                                    cudaMemcpyDeviceToHost, s) != cudaSuccess))) {
            cudaGetLastError();
            return fail_with(ctx, SMF_E_CUDA, "largest_invariant_factor: launch failed");
        }
        return SMF_OK;
    };
    int64_t done = 0, checkpoint = std::min<int64_t>(k, kFirstCheckpoint);
    bool all = false;
    while (done < k && !all) {
        const int64_t steps = std::min<int64_t>(chunk, k - done);
        if ((st = enqueue(done, steps))) return st;
        done += steps;
        if (o.proven || done < checkpoint || done >= k) continue;
        if ((st = smf_status_sync(ctx, s))) return st;
        // the next chunks run on the device while the host reconstructs: for a
        // large n a checkpoint outlasts one chunk (measured: two chunks ahead took
        // n = 5003 from 0.79 to 0.70 s, and n = 1009 from 0.035 to 0.042 s through
        // the steps lifted after the fractions settled)
        const int lookahead = n > kAheadMinN ? 2 : 1;
        int64_t ahead = 0;
        for (int a = 0; a < lookahead && done + ahead < k; a++) {
            const int64_t more = std::min<int64_t>(chunk, k - done - ahead);
            if ((st = enqueue(done + ahead, more))) return st;
            ahead += more;
        }
        const int64_t budget = (int64_t)std::floor((double)done * lp) - 2 - kMarginBits;
        if (budget > 2) reconstruct(done, std::min(nb, budget / 2), std::min(db, budget / 2), false);
        done += ahead;
        all = std::all_of(settled.begin(), settled.end(), [](int v) { return v != 0; });
        const bool pending = std::any_of(has_cand.begin(), has_cand.end(), [](int v) { return v != 0; });
        checkpoint = pending ? done : std::max<int64_t>(done + chunk, (int64_t)std::ceil((double)done * 1.25));
    }
    if (all && cp && done < k) {  // one chunk more for the projection's margin
        const int64_t more = std::min<int64_t>(chunk, k - done);
        if ((st = enqueue(done, more))) return st;
        done += more;
    }
    if ((st = smf_status_sync(ctx, s))) return st;
    if (!all) reconstruct(k, nb, db, true);  // the cap: proven bounds
    const auto t2 = clk::now();
    Nat sn(1);
    for (int64_t j = 0; j < m; j++) {
        if (failed[j]) return fail_with(ctx, SMF_E_INVALID, "largest_invariant_factor: rational reconstruction failed");
        Nat q;
        divmod(den[j], gcd(sn, den[j]), &q, nullptr);
        sn = mul(sn, q);
    }
    const auto t3 = clk::now();
    res->seconds[0] = std::chrono::duration<double>(t1 - t0).count();
    res->seconds[1] = std::chrono::duration<double>(t2 - t1).count() - recon_s;
    res->seconds[2] = std::chrono::duration<double>(t3 - t2).count() + recon_s;
    res->seconds[3] = std::chrono::duration<double>(t3 - t0).count();
    res->s = std::move(sn);
    res->p = p;
    res->digits = done;
    res->cap_digits = k;
    if (cp) res->pair.assign((const uint64_t*)pbuf.p, (const uint64_t*)pbuf.p + (size_t)done * cp * cq);
    return SMF_OK;
}

extern "C" int smf_largest_invariant_factor(smf_ctx* ctx, const smf_bigmat* A, int32_t m, uint64_t seed,
                                            uint32_t* s_limbs, int32_t s_cap, int32_t* s_len, double seconds[4],
                                            void* stream) {
    if (!ctx) return SMF_E_INVALID;
    if (!A || !s_len || m < 1 || m > 1024 || s_cap < 0 || (s_cap > 0 && !s_limbs))
        return fail_with(ctx, SMF_E_INVALID, "largest_invariant_factor: bad argument");
    LifOptions o;
    o.m = m;
    o.seed = seed;
    LifResult r;
    const int st = lif_run(ctx, A, o, &r, (cudaStream_t)stream);
    if (st != SMF_OK) return st;
    *s_len = (int32_t)r.s.d.size();
    if (seconds)
        for (int i = 0; i < 4; i++) seconds[i] = r.seconds[i];
    if ((int64_t)r.s.d.size() > s_cap) return fail_with(ctx, SMF_E_NOMEM, "largest_invariant_factor: s_cap too small");
    for (size_t i = 0; i < r.s.d.size(); i++) s_limbs[i] = r.s.d[i];
    return SMF_OK;
}

// Rational reconstruction on the host (the driver's last step), exposed for
// tests: u and P as little-endian 32-bit limbs; a / b with a = b u (mod P),
// |a| < 2^nb, 0 < b < 2^db, in lowest terms.  num/den receive the limbs of |a|
// and b (capacity `cap` limbs each), *num_neg the sign of a.  Returns
// SMF_E_INVALID when no such fraction is found, SMF_E_NOMEM when cap is short.
extern "C" int smf_rational_reconstruct(const uint32_t* u, int32_t ulen, const uint32_t* P, int32_t plen, int64_t nb,
                                        int64_t db, uint32_t* num, int32_t* num_len, int32_t* num_neg, uint32_t* den,
                                        int32_t* den_len, int32_t cap) {
    if ((ulen > 0 && !u) || plen <= 0 || !P || !num || !num_len || !num_neg || !den || !den_len || cap < 0 ||
        ulen < 0 || nb < 0 || db < 0)
        return SMF_E_INVALID;
    Nat un, Pn;
    un.d.assign(u, u + ulen);
    un.trim();
    Pn.d.assign(P, P + plen);
    Pn.trim();
    if (Pn.zero()) return SMF_E_INVALID;
    Int a;
    Nat b;
    if (!rational_reconstruct(un, Pn, nb, db, &a, &b)) return SMF_E_INVALID;
    if ((int64_t)a.m.d.size() > cap || (int64_t)b.d.size() > cap) return SMF_E_NOMEM;
    for (size_t i = 0; i < a.m.d.size(); i++) num[i] = a.m.d[i];
    for (size_t i = 0; i < b.d.size(); i++) den[i] = b.d[i];
    *num_len = (int32_t)a.m.d.size();
    *den_len = (int32_t)b.d.size();
    *num_neg = a.neg ? 1 : 0;
    return SMF_OK;
}
