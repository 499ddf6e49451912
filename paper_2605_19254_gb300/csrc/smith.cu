// The Smith form of a nonsingular integer matrix A (n x n): the unique
// diag(s_1, ..., s_n), s_i > 0, s_i | s_(i+1), with U A V = S for unimodular
// U, V (Section 1).  Host driver in the shape of the paper's three phases
// (Section 2), over this library's device calls:
//
// Phase 1 (Monte Carlo): s = s_n, the largest invariant factor, by p-adic
//   lifting of A^-1 B for m random columns B and rational reconstruction
//   (lif_run).  The same lifting keeps the digits of a projection of A^-1:
//   P = Q A^-1 J for c' random functionals Q (rows of weights in [1, 2^16))
//   and c of the random columns J.
// Phase 2: s P is integral (s A^-1 is), and Rem(s P, s) is the projection the
//   paper reduces modulo s.  Its Smith form over Z/(s) - pivots that are units
//   after dividing out the content, so that the working modulus shrinks with
//   every invariant factor found - gives the largest invariant factors of A
//   (for a projection of c >= r + 8 random columns the r largest, except with
//   probability about 2^-8 per prime).  Those above 2^62 are kept; the first
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

uint64_t mulmod64(uint64_t a, uint64_t b, uint64_t m) { return (uint64_t)((unsigned __int128)a * b % m); }

uint64_t powmod64(uint64_t a, uint64_t e, uint64_t m) {
    uint64_t r = 1 % m;
    a %= m;
    while (e) {
        if (e & 1) r = mulmod64(r, a, m);
        a = mulmod64(a, a, m);
        e >>= 1;
    }
    return r;
}

// Miller-Rabin with the first twelve prime bases: deterministic below 3.3e24
bool is_prime64(uint64_t n) {
    if (n < 2) return false;
    static const uint64_t bases[] = {2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37};
    for (uint64_t b : bases)
        if (n % b == 0) return n == b;
    uint64_t d = n - 1;
    int r = 0;
    while (!(d & 1)) {
        d >>= 1;
        r++;
    }
    for (uint64_t b : bases) {
        uint64_t x = powmod64(b, d, n);
        if (x == 1 || x == n - 1) continue;
        bool comp = true;
        for (int i = 1; i < r && comp; i++) {
            x = mulmod64(x, x, n);
            if (x == n - 1) comp = false;
        }
        if (comp) return false;
    }
    return true;
}

uint64_t gcd64(uint64_t a, uint64_t b) {
    while (b) {
        const uint64_t t = a % b;
        a = b;
        b = t;
    }
    return a;
}

// a non-trivial factor of a composite n by Pollard's rho (Brent's cycle search)
uint64_t rho_factor(uint64_t n, uint64_t c) {
    if (!(n & 1)) return 2;
    uint64_t y = 2, x = 2, g = 1, q = 1, ys = 2;
    const uint64_t mstep = 128;
    for (uint64_t r = 1; g == 1; r <<= 1) {
        x = y;
        for (uint64_t i = 0; i < r; i++) y = (mulmod64(y, y, n) + c) % n;
        for (uint64_t k = 0; k < r && g == 1; k += mstep) {
            ys = y;
            for (uint64_t i = 0; i < std::min(mstep, r - k); i++) {
                y = (mulmod64(y, y, n) + c) % n;
                q = mulmod64(q, x > y ? x - y : y - x, n);
            }
            g = gcd64(q, n);
        }
    }
    if (g == n) {
        do {
            ys = (mulmod64(ys, ys, n) + c) % n;
            g = gcd64(x > ys ? x - ys : ys - x, n);
        } while (g == 1);
    }
    return g;
}

void factor64(uint64_t n, std::vector<uint64_t>* out) {
    if (n < 2) return;
    for (uint64_t p = 2; p < 1000 && p * p <= n; p++)
        while (n % p == 0) {
            out->push_back(p);
            n /= p;
        }
    if (n < 2) return;
    if (is_prime64(n)) {
        out->push_back(n);
        return;
    }
    uint64_t d = n;
    for (uint64_t c = 1; d == n; c++) d = rho_factor(n, c);
    factor64(d, out);
    factor64(n / d, out);
}

// Rem(s P, s) for the pairing digit sums: z = sum_t sums[t] p^t = P (mod p^k);
// y = s z mod p^k, balanced; accepted when |y| s 2^65 < p^k (then y is the
// integer s P[a][j] unless s P[a][j] is not integral, which leaves a small y
// with probability about 2^-65).  False when an entry is not accepted.
bool pairing_mod_s(const LifResult& r, int cp, int cq, std::vector<Nat>* Y, double* secs) {
    const auto t0 = clk::now();
    const int64_t k = r.digits;
    const Nat P = pow_small(r.p, k);
    const int64_t pbits = P.bits();
    const int64_t sbits = r.s.bits();
    const int count = cp * cq;
    Y->assign(count, Nat());
    std::vector<char> ok(count, 0);
    const int nt = (int)std::max<unsigned>(1, std::min<unsigned>(std::thread::hardware_concurrency(), count));
    auto work = [&](int t) {
        for (int e = t; e < count; e += nt) {
            Nat z;
            for (int64_t i = k; i-- > 0;) mul_add_small(z, r.p, r.pair[(size_t)i * count + e]);
            Nat y;
            divmod(mul(r.s, z), P, nullptr, &y);
            bool neg = false;
            Nat half;
            divmod(P, Nat(2), &half, nullptr);
            if (cmp(y, half) > 0) {
                y = sub(P, y);
                neg = true;
            }
            if (y.bits() + sbits + 65 >= pbits) continue;
            Nat rem;
            divmod(y, r.s, nullptr, &rem);
            (*Y)[e] = (neg && !rem.zero()) ? sub(r.s, rem) : rem;
            ok[e] = 1;
        }
    };
    std::vector<std::thread> pool;
    for (int t = 1; t < nt; t++) pool.emplace_back(work, t);
    work(0);
    for (auto& th : pool) th.join();
    *secs += since(t0);
    return std::all_of(ok.begin(), ok.end(), [](char v) { return v != 0; });
}

// Smith form of the c' x c matrix Y over Z/(s): at each step the content g
// (gcd of the modulus and the entries) is divided out, which shrinks the
// modulus to s / (product of the contents so far); then a unit entry is the
// pivot and its row and column are eliminated.  The invariant factor of A
// that a pivot stands for is the modulus at that step.  `complete`: the
// entries left vanished (every further invariant factor of the projection is
// 1).  False when no unit pivot turns up, also after random row combinations.
bool pairing_smith(std::vector<Nat> Y, int rows, int cols, const Nat& s, uint64_t seed, std::vector<Nat>* inv,
                   bool* complete) {
    Nat mod = s;
    std::vector<int> R(rows), C(cols);
    for (int i = 0; i < rows; i++) R[i] = i;
    for (int j = 0; j < cols; j++) C[j] = j;
    Rng rng{seed ^ 0x5bd1e995u};
    const int nt = (int)std::max<unsigned>(1, std::min<unsigned>(std::thread::hardware_concurrency(), 64));
    auto par_rows = [&](const std::vector<int>& rs, auto&& fn) {
        const int nr = (int)rs.size();
        const int w = std::min(nt, std::max(1, nr));
        std::vector<std::thread> pool;
        for (int t = 1; t < w; t++)
            pool.emplace_back([&, t] {
                for (int i = t; i < nr; i += w) fn(rs[i]);
            });
        for (int i = 0; i < nr; i += w) fn(rs[i]);
        for (auto& th : pool) th.join();
    };
    inv->clear();
    *complete = false;
    while (!R.empty() && !C.empty()) {
        // content
        Nat g = mod;
        for (int a : R) {
            for (int j : C) {
                const Nat& e = Y[(size_t)a * cols + j];
                if (e.zero()) continue;
                g = gcd(g, e);
                if (is_one(g)) break;
            }
            if (is_one(g)) break;
        }
        if (cmp(g, mod) == 0) {
            *complete = true;
            return true;
        }
        if (!is_one(g)) {
            bool exact = true;
            par_rows(R, [&](int a) {
                for (int j : C) {
                    Nat& e = Y[(size_t)a * cols + j];
                    Nat q, rem;
                    divmod(e, g, &q, &rem);
                    if (!rem.zero()) exact = false;
                    e = std::move(q);
                }
            });
            if (!exact) return false;
            Nat q;
            divmod(mod, g, &q, nullptr);
            mod = std::move(q);
        }
        // a unit pivot, if need be after adding random multiples of the other rows to one
        int pa = -1, pj = -1;
        for (int attempt = 0; attempt < 8 && pa < 0; attempt++) {
            for (int a : R) {
                for (int j : C) {
                    const Nat& e = Y[(size_t)a * cols + j];
                    if (!e.zero() && is_one(gcd(mod, e))) {
                        pa = a;
                        pj = j;
                        break;
                    }
                }
                if (pa >= 0) break;
            }
            if (pa >= 0 || R.size() < 2) break;
            const int a0 = R[0];
            for (size_t u = 1; u < R.size(); u++) {
                const Nat cfac((rng.next() >> 48) + 1);
                for (int j : C) {
                    Nat& e = Y[(size_t)a0 * cols + j];
                    Nat t;
                    divmod(add(e, mul(cfac, Y[(size_t)R[u] * cols + j])), mod, nullptr, &t);
                    e = std::move(t);
                }
            }
        }
        if (pa < 0) return false;
        inv->push_back(mod);
        Nat pinv;
        if (!inv_mod(Y[(size_t)pa * cols + pj], mod, &pinv)) return false;
        std::vector<int> others;
        for (int a : R)
            if (a != pa) others.push_back(a);
        par_rows(others, [&](int a) {
            Nat& ea = Y[(size_t)a * cols + pj];
            if (ea.zero()) return;
            const Nat f = mul_mod(ea, pinv, mod);
            for (int j : C) {
                if (j == pj) continue;
                Nat& e = Y[(size_t)a * cols + j];
                e = sub_mod(e, mul_mod(f, Y[(size_t)pa * cols + j], mod), mod);
            }
            ea = Nat();
        });
        R.erase(std::find(R.begin(), R.end(), pa));
        C.erase(std::find(C.begin(), C.end(), pj));
    }
    return true;
}

Nat nat_pow(uint64_t q, int e) {
    Nat r(1);
    for (int i = 0; i < e; i++) r = mul(r, Nat(q));
    return r;
}

uint32_t nat_mod32(const Nat& a, uint32_t q) {
    uint64_t r = 0;
    for (size_t i = a.d.size(); i-- > 0;) r = ((r << 32) | a.d[i]) % q;
    return (uint32_t)r;
}

constexpr int kAttempts = 4;       // Phase 1-3 runs before SMF_E_RETRY_EXHAUSTED
constexpr int kSafety = 8;         // projection columns beyond the invariant factors it must show
constexpr int kDetPrimes = 4;      // Phase 3 primes
constexpr int64_t kSmallBits = 62; // the last iteration's modulus s' stays below 2^62

}  // namespace
}  // namespace smf

using namespace smf;

extern "C" int smf_det_mod(smf_ctx* ctx, const smf_bigmat* A, uint64_t q, uint64_t* det, void* stream) {
    if (!ctx) return SMF_E_INVALID;
    if (!A || !det || A->rows != A->cols || A->rows < 0 || A->words != 1 || A->ld < A->cols ||
        (A->rows > 0 && !A->data))
        return fail_smith(ctx, SMF_E_INVALID, "det_mod: A must be square with single-word entries");
    if (!is_prime64(q) || q >= (1ull << 62)) return fail_smith(ctx, SMF_E_INVALID, "det_mod: q must be a prime below 2^62");
    int dev0 = 0;
    cudaGetDevice(&dev0);
    cudaSetDevice(ctx->device);
    const int64_t n = A->rows;
    cudaStream_t s = (cudaStream_t)stream;
    int st = SMF_OK;
    void* Ad = nullptr;
    if (n > 0 && !A->on_device) {
        if (cudaMalloc(&Ad, 8 * (size_t)n * n) != cudaSuccess ||
            cudaMemcpy2D(Ad, 8 * n, A->data, 8 * A->ld, 8 * n, n, cudaMemcpyHostToDevice) != cudaSuccess) {
            cudaGetLastError();
            if (Ad) cudaFree(Ad);
            cudaSetDevice(dev0);
            return fail_smith(ctx, SMF_E_NOMEM, "det_mod: copy of A failed");
        }
        st = det_mod_device(ctx, (const int64_t*)Ad, n, n, q, det, s);
        cudaFree(Ad);
    } else {
        st = det_mod_device(ctx, (const int64_t*)A->data, A->ld, n, q, det, s);
    }
    cudaSetDevice(dev0);
    return st;
}

extern "C" int smf_smith_local(smf_ctx* ctx, const smf_bigmat* A, uint64_t q, int32_t e, int64_t* counts,
                               void* stream) {
    if (!ctx) return SMF_E_INVALID;
    if (!A || !counts || A->rows != A->cols || A->rows < 0 || A->words != 1 || A->ld < A->cols ||
        (A->rows > 0 && !A->data))
        return fail_smith(ctx, SMF_E_INVALID, "smith_local: A must be square with single-word entries");
    if (!is_prime64(q)) return fail_smith(ctx, SMF_E_INVALID, "smith_local: q must be prime");
    int dev0 = 0;
    cudaGetDevice(&dev0);
    cudaSetDevice(ctx->device);
    const int64_t n = A->rows;
    cudaStream_t s = (cudaStream_t)stream;
    int st;
    void* Ad = nullptr;
    if (n > 0 && !A->on_device) {
        if (cudaMalloc(&Ad, 8 * (size_t)n * n) != cudaSuccess ||
            cudaMemcpy2D(Ad, 8 * n, A->data, 8 * A->ld, 8 * n, n, cudaMemcpyHostToDevice) != cudaSuccess) {
            cudaGetLastError();
            if (Ad) cudaFree(Ad);
            cudaSetDevice(dev0);
            return fail_smith(ctx, SMF_E_NOMEM, "smith_local: copy of A failed");
        }
        st = local_smith_device(ctx, (const int64_t*)Ad, n, n, q, e, counts, s);
        cudaFree(Ad);
    } else {
        st = local_smith_device(ctx, (const int64_t*)A->data, A->ld, n, q, e, counts, s);
    }
    cudaSetDevice(dev0);
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
    // A contiguous on the device (the eliminations) and on the host
    struct Buf {
        void* p = nullptr;
        ~Buf() {
            if (p) cudaFree(p);
        }
    } Ad;
    if (cudaMalloc(&Ad.p, 8 * (size_t)n * n) != cudaSuccess) {
        cudaGetLastError();
        return fail_smith(ctx, SMF_E_NOMEM, "smith_form: device allocation failed");
    }
    if (cudaMemcpy2D(Ad.p, 8 * n, A->data, 8 * A->ld, 8 * n, n,
                     A->on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice) != cudaSuccess) {
        cudaGetLastError();
        return fail_smith(ctx, SMF_E_CUDA, "smith_form: copy of A failed");
    }
    smf_bigmat Am{n, n, n, 1, A->bits, Ad.p, 1, 0};
    const int64_t* Adev = (const int64_t*)Ad.p;
    double t1 = 0, t2 = 0, t3 = 0;
    int inject = ctx->inject;
    ctx->inject &= ~(SMF_INJECT_WRONG_SMITH | SMF_INJECT_WRONG_SMITH_ALWAYS);
    int cp = 16;
    std::vector<Nat> result;  // descending
    std::string why = "Phase 3 rejected every attempt";
    int attempt = 0;
    for (; attempt < kAttempts; attempt++) {
        Rng rng{seed + 0x9e3779b97f4a7c15ull * (uint64_t)attempt};
        // ---- Phase 1 (and the projection's digits)
        auto ta = clk::now();
        LifOptions o;
        o.m = 32;
        o.seed = rng.next();
        o.pair_rows = cp;
        o.pair_cols = cp;
        LifResult r;
        int st = lif_run(ctx, &Am, o, &r, s);
        if (st != SMF_OK) return st;
        t1 += since(ta);
        // ---- Phase 2: Rem(s P, s), its Smith form over Z/(s)
        ta = clk::now();
        std::vector<Nat> Y;
        double pt = 0;
        if (!pairing_mod_s(r, cp, cp, &Y, &pt)) {
            // precision short of what some entry needs: lift to Hadamard's precision
            t2 += since(ta);
            ta = clk::now();
            o.proven = true;
            if ((st = lif_run(ctx, &Am, o, &r, s)) != SMF_OK) return st;
            t1 += since(ta);
            ta = clk::now();
            if (!pairing_mod_s(r, cp, cp, &Y, &pt)) {
                t2 += since(ta);
                why = "Phase 2: the projection times s is not integral in any attempt (s below s_n)";
                continue;  // s was not a multiple of s_n: a new attempt
            }
        }
        std::vector<Nat> inv;
        bool complete = false;
        if (!pairing_smith(Y, cp, cp, r.s, rng.next(), &inv, &complete)) {
            t2 += since(ta);
            why = "Phase 2: no unit pivot in the projection's Smith form in any attempt";
            continue;
        }
        const int reliable = cp - kSafety;
        int rtop = 0;  // invariant factors above 2^62, taken from the projection
        while (rtop < (int)inv.size() && inv[rtop].bits() > kSmallBits) rtop++;
        if (rtop >= reliable && !(complete && rtop == (int)inv.size())) {
            t2 += since(ta);
            if (cp < 32) {  // more large invariant factors than the projection shows reliably: a wider one
                cp = 32;
                attempt--;
                continue;
            }
            return fail_smith(ctx, SMF_E_UNSUPPORTED,
                              "smith_form: more than 25 invariant factors above 2^62 (the projection's limit)");
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
            for (size_t i = 0; i < f.size();) {
                const uint64_t q = f[i];
                int e = 0;
                while (i < f.size() && f[i] == q) {
                    e++;
                    i++;
                }
                std::vector<int64_t> counts(e + 1);
                if ((st = local_smith_device(ctx, Adev, n, n, q, e, counts.data(), s)) != SMF_OK) return st;
                for (int64_t j = 0; j < n; j++) {
                    int v = 0;
                    for (int t = 1; t <= e; t++)
                        if (counts[t] > j) v = t;
                    if (v) small[j] = mul(small[j], nat_pow(q, v));
                }
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
        int sign = 0;
        bool pass = true;
        for (int t = 0; t < kDetPrimes && pass;) {
            uint64_t q = (1ull << 30) + (rng.next() >> 34);
            while (!is_prime64(q)) q++;
            uint64_t prod = 1;
            for (const Nat& v : cand) prod = mulmod64(prod, nat_mod32(v, (uint32_t)q), q);
            if (prod == 0) continue;  // q divides the candidate's product: another prime
            uint64_t d = 0;
            if ((st = det_mod_device(ctx, Adev, n, n, q, &d, s)) != SMF_OK) return st;
            const int sg = d == prod ? 1 : d == (q - prod) % q ? -1 : 0;
            if (sg == 0 || (sign && sg != sign)) pass = false;
            sign = sg;
            t++;
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
