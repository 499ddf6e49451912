// The Smith form of a nonsingular integer matrix A (n x n): the unique
// diag(s_1, ..., s_n), s_i > 0, s_i | s_(i+1), with U A V = S for unimodular
// U, V (Section 1).  Host driver in the shape of the paper's three phases
// (Section 2), over this library's device calls:
//
// Phase 1 (Monte Carlo): s = s_n, the largest invariant factor, by p-adic
//   lifting of A^-1 B for m random columns B and rational reconstruction
//   (lif_run).  The same lifting keeps the digits of a projection of A^-1:
//   P = Q A^-1 J for 32 random functionals Q (rows of weights in [1, 2^16))
//   and 32 of the random columns J.
// Phase 2: s P is integral (s A^-1 is), and Rem(s P, s) is the projection the
//   paper reduces modulo s.  Its Smith form over Z/(s) - pivots that are units
//   after dividing out the content, so that the working modulus shrinks with
//   every invariant factor found - gives the largest invariant factors of A
//   (for a w x w corner of the projection the w - 8 largest, except with
//   probability about 2^-8 per prime).  The corner starts at 16 x 16 and grows
//   (up to 32, without lifting again) while it shows more factors above 2^62
//   than it holds reliably.  Those above 2^62 are kept; the first
//   one below, s', bounds all the others, and the last iteration works modulo
//   that word-size s' at once: the Smith form of A over Z/(s') is
//   diag(gcd(s_i, s')), taken prime power by prime power by elimination on the
//   device (local_smith_device).
// Phase 3: every value so found divides the true invariant factor in its
//   place, so the product of the candidate equals |det A| only if the
//   candidate is the Smith form.  The check compares det A mod q (elimination
//   over GF(q) on the device) with +- prod s_i mod q for four random primes
//   q in (2^30, 2^31) that do not divide prod s_i, with one sign for all; on a
//   mismatch the algorithm restarts from Phase 1 with fresh random choices.
//   (The paper's Phase 3 certifies unimodularity deterministically; here a
//   wrong candidate passes only if each q divides det A / prod s_i -+ 1, with
//   probability below 2^-40 for |det A| < 2^(2^20).)
#include <algorithm>
#include <chrono>
#include <cmath>
#include <thread>

#include "numtheory.h"
#include "pairing_smith.h"
#include "smith_internal.h"

namespace smf {
namespace {

using clk = std::chrono::steady_clock;

int fail_smith(smf_ctx* ctx, int code, const std::string& msg) {
    ctx->err = msg;
    return code;
}

double since(clk::time_point t) { return std::chrono::duration<double>(clk::now() - t).count(); }

// splitmix64 (Steele, Lea and Flood, 2014)
struct Rng {
    uint64_t x;
    uint64_t next() {
        uint64_t z = (x += 0x9e3779b97f4a7c15ull);
        z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
        z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
        return z ^ (z >> 31);
    }
};


// Rem(s P, s) for the leading w x w corner of the pairing digit sums (cp x cp
// per digit): z = sum_t sums[t] p^t = P (mod p^k); y = s z mod p^k, balanced;
// accepted when |y| s 2^65 < p^k (then y is the integer s P[a][j] unless
// s P[a][j] is not integral, which leaves a small y with probability about
// 2^-65).  Entries already in Y (have[e]) are kept.  False when an entry is
// not accepted.
bool pairing_mod_s(const LifResult& r, int cp, int w, std::vector<Nat>* Y, std::vector<char>* have) {
    const int64_t k = r.digits;
    const Nat P = pow_small(r.p, k);
    Nat half;
    divmod(P, Nat(2), &half, nullptr);
    const int64_t pbits = P.bits();
    const int64_t sbits = r.s.bits();
    const int count = cp * cp;
    if ((int)Y->size() != count) {
        Y->assign(count, Nat());
        have->assign(count, 0);
    }
    std::vector<int> todo;
    for (int a = 0; a < w; a++)
        for (int j = 0; j < w; j++)
            if (!(*have)[a * cp + j]) todo.push_back(a * cp + j);
    std::vector<char> ok(todo.size(), 0);
    // shared by the entries: the powers of p for Horner by halves, and Barrett's
    // reciprocal of p^k (two products per reduction instead of a long division)
    const std::vector<Nat> pw = horner_powers(r.p, k);
    const Barrett bP = barrett_of(P);
    // threads only for wide values (a thread costs tens of microseconds)
    const int nt = r.s.d.size() < 64 ? 1
                                     : (int)std::max<unsigned>(1, std::min<unsigned>(std::thread::hardware_concurrency(),
                                                                                     std::max<size_t>(1, todo.size())));
    auto work = [&](int t) {
        for (size_t u = t; u < todo.size(); u += nt) {
            const int e = todo[u];
            // digit sums below 2^(16 + bits(p) + 14)
            int pb = 0;
            while ((1ull << pb) <= r.p) pb++;
            const Nat z = barrett_mod(bP, horner_split(r.pair.data() + e, k, (size_t)count, r.p, 30 + pb, pw));
            Nat y = barrett_mod(bP, mul(r.s, z));  // s < p^k: the product stays below p^(2k)
            bool neg = false;
            if (cmp(y, half) > 0) {
                y = sub(P, y);
                neg = true;
            }
            if (y.bits() + sbits + 65 >= pbits) continue;
            Nat rem;
            divmod(y, r.s, nullptr, &rem);
            (*Y)[e] = (neg && !rem.zero()) ? sub(r.s, rem) : rem;
            ok[u] = 1;
        }
    };
    std::vector<std::thread> pool;
    for (int t = 1; t < nt; t++) pool.emplace_back(work, t);
    work(0);
    for (auto& th : pool) th.join();
    for (size_t u = 0; u < todo.size(); u++)
        if (ok[u]) (*have)[todo[u]] = 1;
    return std::all_of(ok.begin(), ok.end(), [](char v) { return v != 0; });
}

// The leading w x w corner of the cp x cp pairing values.
std::vector<Nat> corner(const std::vector<Nat>& Y, int cp, int w) {
    std::vector<Nat> out((size_t)w * w);
    for (int a = 0; a < w; a++)
        for (int j = 0; j < w; j++) out[(size_t)a * w + j] = Y[(size_t)a * cp + j];
    return out;
}

Nat nat_pow(uint64_t q, int e) {
    Nat r(1);
    for (int i = 0; i < e; i++) r = mul(r, Nat(q));
    return r;
}


constexpr int kAttempts = 4;       // Phase 1-3 runs before SMF_E_RETRY_EXHAUSTED
constexpr int kSafety = 8;         // projection columns beyond the invariant factors it must show
constexpr int kPairFirst = 16;     // the projection's first corner
constexpr int kPairMax = 32;       // the digits kept on the device: a 32 x 32 projection
constexpr int kDetPrimes = 4;      // Phase 3 primes
constexpr int64_t kSmallBits = 62; // the last iteration's modulus s' stays below 2^62

}  // namespace
}  // namespace smf

using namespace smf;

namespace {
// A on the device for the eliminations: the caller's buffer, or a copy of a host one.
struct DeviceA {
    StreamBuf copy;
    const int64_t* p = nullptr;
    int64_t ld = 0;
    bool load(const smf_bigmat* A, cudaStream_t s) {
        const int64_t n = A->rows;
        if (A->on_device || n == 0) {
            p = (const int64_t*)A->data;
            ld = A->ld;
            return true;
        }
        if (copy.alloc(8 * (size_t)n * n, s) != cudaSuccess ||
            cudaMemcpy2DAsync(copy.p, 8 * n, A->data, 8 * A->ld, 8 * n, n, cudaMemcpyHostToDevice, s) != cudaSuccess) {
            cudaGetLastError();
            return false;
        }
        p = (const int64_t*)copy.p;
        ld = n;
        return true;
    }
};

bool square_single_words(const smf_bigmat* A) {
    return A && A->rows == A->cols && A->rows >= 0 && A->words == 1 && A->ld >= A->cols && (A->rows == 0 || A->data);
}
}  // namespace

extern "C" int smf_det_mod(smf_ctx* ctx, const smf_bigmat* A, const uint64_t* q, int32_t count, uint64_t* det,
                           void* stream) {
    if (!ctx) return SMF_E_INVALID;
    if (!square_single_words(A) || !q || !det || count < 1 || count > 64)
        return fail_smith(ctx, SMF_E_INVALID, "det_mod: A must be square with single-word entries; 1 to 64 primes");
    for (int32_t i = 0; i < count; i++)
        if (!is_prime64(q[i]) || q[i] >= (1ull << 62))
            return fail_smith(ctx, SMF_E_INVALID, "det_mod: every q must be a prime below 2^62");
    int dev0 = 0;
    cudaGetDevice(&dev0);
    cudaSetDevice(ctx->device);
    DeviceA Ad;
    int st = Ad.load(A, (cudaStream_t)stream) ? det_mod_device(ctx, Ad.p, Ad.ld, A->rows, q, count, det, (cudaStream_t)stream)
                        : fail_smith(ctx, SMF_E_NOMEM, "det_mod: copy of A failed");
    cudaSetDevice(dev0);
    return st;
}

extern "C" int smf_smith_local(smf_ctx* ctx, const smf_bigmat* A, const uint64_t* q, const int32_t* e,
                               int32_t count, int64_t* counts, void* stream) {
    if (!ctx) return SMF_E_INVALID;
    if (!square_single_words(A) || !q || !e || !counts || count < 1 || count > 16)
        return fail_smith(ctx, SMF_E_INVALID, "smith_local: A must be square with single-word entries; 1 to 16 primes");
    for (int32_t i = 0; i < count; i++) {
        if (!is_prime64(q[i])) return fail_smith(ctx, SMF_E_INVALID, "smith_local: every q must be prime");
        for (int32_t j = 0; j < i; j++)
            if (q[j] == q[i]) return fail_smith(ctx, SMF_E_INVALID, "smith_local: the primes must differ");
    }
    int dev0 = 0;
    cudaGetDevice(&dev0);
    cudaSetDevice(ctx->device);
    DeviceA Ad;
    std::vector<std::vector<int64_t>> cnt;
    std::vector<int> ev(e, e + count);
    int st = Ad.load(A, (cudaStream_t)stream) ? local_smith_device(ctx, Ad.p, Ad.ld, A->rows, q, ev.data(), count, &cnt, (cudaStream_t)stream)
                        : fail_smith(ctx, SMF_E_NOMEM, "smith_local: copy of A failed");
    cudaSetDevice(dev0);
    if (st == SMF_OK) {
        int64_t off = 0;
        for (int32_t i = 0; i < count; i++)
            for (int t = 0; t <= e[i]; t++) counts[off++] = cnt[i][t];
    }
    return st;
}

extern "C" int smf_smith_form(smf_ctx* ctx, const smf_bigmat* A, uint64_t seed, uint32_t* limbs, int64_t cap,
                              int64_t* offsets, double seconds[4], int32_t* attempts, void* stream) {
    if (!ctx) return SMF_E_INVALID;
    if (!A || !offsets || cap < 0 || (cap > 0 && !limbs))
        return fail_smith(ctx, SMF_E_INVALID, "smith_form: bad argument");
    if (A->rows != A->cols || A->rows < 1 || A->words != 1 || A->ld < A->cols || !A->data || A->bits < 0)
        return fail_smith(ctx, SMF_E_INVALID, "smith_form: A must be n x n (n >= 1), single words");
    const auto t_start = clk::now();
    int dev0 = 0;
    cudaGetDevice(&dev0);
    cudaSetDevice(ctx->device);
    struct Restore {
        int d;
        ~Restore() { cudaSetDevice(d); }
    } restore{dev0};
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t n = A->rows;
    // A contiguous on the device (the eliminations), in stream order on s
    StreamBuf Ad;
    if (Ad.alloc(8 * (size_t)n * n, s) != cudaSuccess) {
        cudaGetLastError();
        return fail_smith(ctx, SMF_E_NOMEM, "smith_form: device allocation failed");
    }
    if (cudaMemcpy2DAsync(Ad.p, 8 * n, A->data, 8 * A->ld, 8 * n, n,
                          A->on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s) != cudaSuccess) {
        cudaGetLastError();
        return fail_smith(ctx, SMF_E_CUDA, "smith_form: copy of A failed");
    }
    smf_bigmat Am{n, n, n, 1, A->bits, Ad.p, 1, 0};
    const int64_t* Adev = (const int64_t*)Ad.p;
    double t1 = 0, t2 = 0, t3 = 0;
    int inject = ctx->inject;
    ctx->inject &= ~(SMF_INJECT_WRONG_SMITH | SMF_INJECT_WRONG_SMITH_ALWAYS);
    std::vector<Nat> result;  // descending
    std::string why = "Phase 3 rejected every attempt";
    int attempt = 0;
    for (; attempt < kAttempts; attempt++) {
        Rng rng{seed + 0x9e3779b97f4a7c15ull * (uint64_t)attempt};
        // ---- Phase 1, with the digits of a kPairMax x kPairMax projection
        auto ta = clk::now();
        LifOptions o;
        o.m = 32;
        o.seed = rng.next();
        o.pair_rows = kPairMax;
        o.pair_cols = kPairMax;
        LifResult r;
        int st = lif_run(ctx, &Am, o, &r, s);
        if (st != SMF_OK) return st;
        t1 += since(ta);
        // ---- Phase 2: Rem(s P, s) on a w x w corner of the projection, its Smith form over
        // Z/(s); the corner grows (up to kPairMax) while it shows too many factors above 2^62
        ta = clk::now();
        std::vector<Nat> Y, inv;
        std::vector<char> have;
        bool complete = false, fine = true;
        int w = kPairFirst, rtop = 0;
        for (;;) {
            if (!pairing_mod_s(r, kPairMax, w, &Y, &have)) {
                if (o.proven) {  // s was not a multiple of s_n: a new attempt
                    why = "Phase 2: the projection times s is not integral in any attempt (s below s_n)";
                    fine = false;
                    break;
                }
                // precision short of what some entry needs: lift to Hadamard's precision
                t2 += since(ta);
                ta = clk::now();
                o.proven = true;
                if ((st = lif_run(ctx, &Am, o, &r, s)) != SMF_OK) return st;
                t1 += since(ta);
                ta = clk::now();
                Y.clear();
                continue;
            }
            if (!pairing_smith(corner(Y, kPairMax, w), w, w, r.s, &inv, &complete)) {
                why = "Phase 2: no unit pivot in the projection's Smith form in any attempt";
                fine = false;
                break;
            }
            rtop = 0;  // invariant factors above 2^62, taken from the projection
            while (rtop < (int)inv.size() && inv[rtop].bits() > kSmallBits) rtop++;
            if (rtop < w - kSafety || (complete && rtop == (int)inv.size())) break;
            if (w == kPairMax) {
                t2 += since(ta);
                return fail_smith(ctx, SMF_E_UNSUPPORTED,
                                  "smith_form: more than 24 invariant factors above 2^62 (the projection's limit)");
            }
            w = std::min(kPairMax, rtop + 1 + kSafety);  // wide enough for one more than found
        }
        if (!fine) {
            t2 += since(ta);
            continue;
        }
        uint64_t sp = 1;  // s' = the largest invariant factor below 2^62 (1: none)
        if (rtop < (int)inv.size()) {
            const Nat& v = inv[rtop];
            sp = v.d.size() > 1 ? ((uint64_t)v.d[1] << 32) | v.d[0] : v.d[0];
        }
        // the last iteration: Smith form of A over Z/(s'), prime power by prime power
        std::vector<Nat> small(n, Nat(1));  // gcd(s_i, s'), i-th largest first
        if (sp > 1) {
            std::vector<uint64_t> f;
            factor64(sp, &f);
            std::sort(f.begin(), f.end());
            std::vector<uint64_t> qs;
            std::vector<int> es;
            for (size_t i = 0; i < f.size();) {
                qs.push_back(f[i]);
                es.push_back(0);
                while (i < f.size() && f[i] == qs.back()) {
                    es.back()++;
                    i++;
                }
            }
            // all prime powers of s' in one joint column loop, then the leftover block per prime
            std::vector<std::vector<int64_t>> counts;
            if ((st = local_smith_device(ctx, Adev, n, n, qs.data(), es.data(), (int)qs.size(), &counts, s)) !=
                SMF_OK)
                return st;
            for (size_t l = 0; l < qs.size(); l++)
                for (int64_t j = 0; j < n; j++) {
                    int v = 0;
                    for (int t = 1; t <= es[l]; t++)
                        if (counts[l][t] > j) v = t;
                    if (v) small[j] = mul(small[j], nat_pow(qs[l], v));
                }
        }
        // the r largest factors over Z/(s') are s' (multiples of s'): the projection's values replace them
        std::vector<Nat> cand(n);
        bool consistent = true;
        for (int64_t j = 0; j < n; j++) {
            if (j < rtop) {
                consistent &= cmp(small[j], Nat(sp)) == 0;
                cand[j] = inv[j];
            } else {
                cand[j] = small[j];
            }
        }
        if (inject & (SMF_INJECT_WRONG_SMITH | SMF_INJECT_WRONG_SMITH_ALWAYS)) {
            cand[0] = mul(cand[0], Nat(2));  // a wrong candidate for Phase 3 to reject
            inject &= ~SMF_INJECT_WRONG_SMITH;
        }
        t2 += since(ta);
        if (!consistent) {
            why = "Phase 2: the last iteration disagrees with the projection in every attempt";
            continue;
        }
        why = "Phase 3 rejected every attempt";
        // ---- Phase 3: prod s_i = +-det A modulo random primes
        ta = clk::now();
        uint64_t qs[kDetPrimes], prods[kDetPrimes], dets[kDetPrimes];
        for (int t = 0; t < kDetPrimes;) {
            uint64_t q = (1ull << 30) + (rng.next() >> 34);
            while (!is_prime64(q)) q++;
            uint64_t prod = 1;
            for (const Nat& v : cand) prod = mulmod64(prod, nat_rem32(v, (uint32_t)q), q);
            if (prod == 0 || std::find(qs, qs + t, q) != qs + t) continue;  // q divides the product: another
            qs[t] = q;
            prods[t++] = prod;
        }
        // the four determinants in one column loop
        if ((st = det_mod_device(ctx, Adev, n, n, qs, kDetPrimes, dets, s)) != SMF_OK) return st;
        int sign = 0;
        bool pass = true;
        for (int t = 0; t < kDetPrimes; t++) {
            const uint64_t q = qs[t], d = dets[t], prod = prods[t];
            const int sg = d == prod ? 1 : d == (q - prod) % q ? -1 : 0;
            if (sg == 0 || (sign && sg != sign)) pass = false;
            sign = sg;
        }
        t3 += since(ta);
        if (pass) {
            result = std::move(cand);
            break;
        }
    }
    if (attempts) *attempts = std::min(attempt + 1, kAttempts);
    if (seconds) {
        seconds[0] = t1;
        seconds[1] = t2;
        seconds[2] = t3;
        seconds[3] = since(t_start);
    }
    if (result.empty()) return fail_smith(ctx, SMF_E_RETRY_EXHAUSTED, "smith_form: " + why);
    // ascending order, s_1 | s_2 | ... | s_n
    int64_t off = 0;
    for (int64_t i = 0; i < n; i++) {
        offsets[i] = off;
        off += (int64_t)result[n - 1 - i].d.size();
    }
    offsets[n] = off;
    if (off > cap) return fail_smith(ctx, SMF_E_NOMEM, "smith_form: cap too small for the invariant factors");
    for (int64_t i = 0; i < n; i++) {
        const Nat& v = result[n - 1 - i];
        std::copy(v.d.begin(), v.d.end(), limbs + offsets[i]);
    }
    return SMF_OK;
}
