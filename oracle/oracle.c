/*
 * Oracle for the RNS exact integer matrix product (test infrastructure).
 *
 * A plain, slow, obviously correct CPU restatement of what the hot path
 * computes: reduction of big integers modulo word-size primes, the residue
 * products, CRT reconstruction, and the exact product itself.  Only the test
 * suite, the smoke check and the CPU-baseline leg of the benchmark may load
 * this library; the product path never calls it, and it shares no code with
 * the CUDA path.
 *
 * Paper: "A C implementation of the Smith massager algorithm", Section 3.1
 * (RNS arithmetic).  Each function below names the passage it follows.
 *
 * Big integers here are sign-magnitude arrays of base-2^32 limbs, least
 * significant limb first.  The interchange format with the caller is the
 * library-wide one: W little-endian 64-bit words per entry holding the two's
 * complement value.
 *
 * Parity status: every function is pinned by the CPU test suite against
 * Python integers, closed forms or brute force (see tests/test_oracle_*.py).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_OK 0
#define ORC_E_OVERFLOW 1
#define ORC_E_INVALID 2
#define ORC_E_NOMEM 3

/* ------------------------------------------------------------------------ */
/* Magnitude arithmetic on base-2^32 limb arrays.                           */
/* ------------------------------------------------------------------------ */

/* number of significant limbs */
static int mag_len(const uint32_t* a, int n) {
    while (n > 0 && a[n - 1] == 0) n--;
    return n;
}

/* compare |a| and |b|: -1, 0, 1 */
static int mag_cmp(const uint32_t* a, int na, const uint32_t* b, int nb) {
    na = mag_len(a, na);
    nb = mag_len(b, nb);
    if (na != nb) return na < nb ? -1 : 1;
    for (int i = na - 1; i >= 0; i--)
        if (a[i] != b[i]) return a[i] < b[i] ? -1 : 1;
    return 0;
}

/* r = a + b, r has room for max(na, nb) + 1 limbs; returns limbs written */
static int mag_add(const uint32_t* a, int na, const uint32_t* b, int nb, uint32_t* r) {
    int n = na > nb ? na : nb;
    uint64_t carry = 0;
    for (int i = 0; i < n; i++) {
        uint64_t s = carry;
        if (i < na) s += a[i];
        if (i < nb) s += b[i];
        r[i] = (uint32_t)s;
        carry = s >> 32;
    }
    r[n] = (uint32_t)carry;
    return n + 1;
}

/* r = a - b with |a| >= |b|; r has room for na limbs */
static void mag_sub(const uint32_t* a, int na, const uint32_t* b, int nb, uint32_t* r) {
    int64_t borrow = 0;
    for (int i = 0; i < na; i++) {
        int64_t d = (int64_t)a[i] - borrow - (i < nb ? (int64_t)b[i] : 0);
        borrow = 0;
        if (d < 0) { d += ((int64_t)1 << 32); borrow = 1; }
        r[i] = (uint32_t)d;
    }
}

/* r = a * b (schoolbook), r has room for na + nb limbs */
static void mag_mul(const uint32_t* a, int na, const uint32_t* b, int nb, uint32_t* r) {
    memset(r, 0, sizeof(uint32_t) * (size_t)(na + nb));
    for (int i = 0; i < na; i++) {
        uint64_t carry = 0;
        for (int j = 0; j < nb; j++) {
            uint64_t t = (uint64_t)a[i] * b[j] + r[i + j] + carry;
            r[i + j] = (uint32_t)t;
            carry = t >> 32;
        }
        r[i + nb] = (uint32_t)carry;
    }
}

/* a = a * m + c in place (a has room for n + 1 limbs); returns new length */
static int mag_mul_small_add(uint32_t* a, int n, uint32_t m, uint32_t c) {
    uint64_t carry = c;
    for (int i = 0; i < n; i++) {
        uint64_t t = (uint64_t)a[i] * m + carry;
        a[i] = (uint32_t)t;
        carry = t >> 32;
    }
    a[n] = (uint32_t)carry;
    return n + 1;
}

/* remainder of |a| modulo a 32-bit modulus, by long division from the top */
static uint32_t mag_mod_small(const uint32_t* a, int n, uint32_t p) {
    uint64_t r = 0;
    for (int i = n - 1; i >= 0; i--) r = ((r << 32) | a[i]) % p;
    return (uint32_t)r;
}

/* q = a / d exactly (remainder discarded), q has room for n limbs */
static void mag_div_small(const uint32_t* a, int n, uint32_t d, uint32_t* q) {
    uint64_t r = 0;
    for (int i = n - 1; i >= 0; i--) {
        uint64_t cur = (r << 32) | a[i];
        q[i] = (uint32_t)(cur / d);
        r = cur % d;
    }
}

/* ------------------------------------------------------------------------ */
/* Two's complement words <-> sign-magnitude limbs.                         */
/* ------------------------------------------------------------------------ */

/* Reads W words; writes |x| into mag[0 .. 2W) and returns 1 if x < 0. */
static int tc_to_sm(const uint64_t* w, int W, uint32_t* mag) {
    int neg = (int)(w[W - 1] >> 63);
    uint64_t carry = 1;
    for (int j = 0; j < W; j++) {
        uint64_t v = w[j];
        if (neg) {
            v = ~v + carry;
            carry = (carry && v == 0) ? 1 : 0;
        }
        mag[2 * j] = (uint32_t)v;
        mag[2 * j + 1] = (uint32_t)(v >> 32);
    }
    return neg;
}

/* Writes sign*|mag| as W two's complement words; ORC_E_OVERFLOW if it does
 * not fit in [-2^(64W-1), 2^(64W-1)). */
static int sm_to_tc(int neg, const uint32_t* mag, int n, uint64_t* w, int W) {
    n = mag_len(mag, n);
    if (n == 0) neg = 0;
    if (n > 2 * W) return ORC_E_OVERFLOW;
    /* limit = 2^(64W-1) as limbs: top limb 0x80000000 */
    uint32_t top = n == 2 * W ? mag[2 * W - 1] : 0;
    if (top > 0x80000000u) return ORC_E_OVERFLOW;
    if (top == 0x80000000u) {
        int rest_zero = 1;
        for (int i = 0; i < 2 * W - 1; i++)
            if (mag[i]) rest_zero = 0;
        if (!neg || !rest_zero) return ORC_E_OVERFLOW;
    }
    uint64_t carry = 1;
    for (int j = 0; j < W; j++) {
        uint64_t lo = 2 * j < n ? mag[2 * j] : 0;
        uint64_t hi = 2 * j + 1 < n ? mag[2 * j + 1] : 0;
        uint64_t v = lo | (hi << 32);
        if (neg) {
            v = ~v + carry;
            carry = (carry && v == 0) ? 1 : 0;
        }
        w[j] = v;
    }
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Primes of the RNS basis (Section 3.1: a run of consecutive primes just  */
/* under the bound).                                                        */
/* ------------------------------------------------------------------------ */

/* primality by trial division */
int orc_is_prime(uint64_t n) {
    if (n < 2) return 0;
    if (n % 2 == 0) return n == 2;
    for (uint64_t d = 3; d * d <= n; d += 2)
        if (n % d == 0) return 0;
    return 1;
}

/* The `count` largest primes strictly below `bound`, in descending order.
 * Returns the number found. */
int orc_primes_below(uint64_t bound, int count, uint32_t* out) {
    int found = 0;
    for (uint64_t c = bound; c > 2 && found < count;) {
        c--;
        if (orc_is_prime(c)) out[found++] = (uint32_t)c;
    }
    return found;
}

/* Section 3.1, exact double-precision accumulation: the largest p with
 * n (p-1)^2 + (p-1) < 2^53 - 1.  Found by scanning down from a float
 * estimate plus margin, testing the inequality in exact integers. */
uint64_t orc_fp64_prime_cap(uint64_t n) {
    const unsigned __int128 lim = ((unsigned __int128)1 << 53) - 1;
    uint64_t p = 2;
    /* grow by doubling, then bisect on the exact predicate */
    uint64_t lo = 1, hi = 2;
    for (;;) {
        unsigned __int128 t = (unsigned __int128)n * (hi - 1) * (hi - 1) + (hi - 1);
        if (t >= lim) break;
        lo = hi;
        hi *= 2;
    }
    /* predicate true at lo, false at hi */
    while (hi - lo > 1) {
        uint64_t mid = lo + (hi - lo) / 2;
        unsigned __int128 t = (unsigned __int128)n * (mid - 1) * (mid - 1) + (mid - 1);
        if (t < lim) lo = mid; else hi = mid;
    }
    p = lo;
    return p;
}

/* Number of primes (descending below `bound`) whose product M exceeds
 * 2^(bits+1), so that every x with |x| <= 2^bits has a unique symmetric
 * representative in (-M/2, M/2].  Writes the primes to `out` (room for
 * `cap`).  Returns the count, or -1 if `cap` is too small. */
int orc_basis(uint64_t bound, int bits, int cap, uint32_t* out) {
    int nl = (bits + 2) / 32 + 4;
    uint32_t* m = (uint32_t*)calloc((size_t)nl + (size_t)cap + 2, sizeof(uint32_t));
    if (!m) return -1;
    m[0] = 1;
    int n = 1, L = 0;
    uint64_t c = bound;
    for (;;) {
        /* bit length of M */
        int len = mag_len(m, n);
        int bl = 32 * (len - 1);
        for (uint32_t t = m[len - 1]; t; t >>= 1) bl++;
        if (bl >= bits + 2) break; /* M >= 2^(bits+1), odd, hence > */
        if (L == cap) { free(m); return -1; }
        uint32_t p = 0;
        while (c > 2) {
            c--;
            if (orc_is_prime(c)) { p = (uint32_t)c; break; }
        }
        if (!p) { free(m); return -1; }
        out[L++] = p;
        n = mag_mul_small_add(m, n, p, 0);
    }
    free(m);
    return L;
}

/* ------------------------------------------------------------------------ */
/* Reduction (Section 3.1: an integer matrix is reduced modulo each prime,  */
/* giving one residue matrix per prime).                                    */
/* ------------------------------------------------------------------------ */

/* residues[i][r][c] = X[r][c] mod primes[i] in [0, p_i).
 * X: rows x cols entries, leading dimension ld entries, W words each. */
int orc_reduce(const uint64_t* X, int64_t rows, int64_t cols, int64_t ld, int W,
               const uint32_t* primes, int L, int32_t* residues) {
    if (W < 1 || rows < 0 || cols < 0 || ld < cols || L < 0) return ORC_E_INVALID;
    uint32_t* mag = (uint32_t*)malloc(sizeof(uint32_t) * 2 * (size_t)W);
    if (!mag) return ORC_E_NOMEM;
    for (int64_t r = 0; r < rows; r++)
        for (int64_t c = 0; c < cols; c++) {
            int neg = tc_to_sm(X + (size_t)(r * ld + c) * W, W, mag);
            for (int i = 0; i < L; i++) {
                uint32_t p = primes[i];
                uint32_t m = mag_mod_small(mag, 2 * W, p);
                if (neg && m) m = p - m;
                residues[((size_t)i * rows + r) * cols + c] = (int32_t)m;
            }
        }
    free(mag);
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* The exact product over Z (the result the RNS route must reproduce).      */
/* ------------------------------------------------------------------------ */

/* C = A * B exactly.  A: M x K (lda entries, Wa words), B: K x N (ldb, Wb),
 * C: M x N (ldc, Wc).  Schoolbook: each C entry is the signed sum of the K
 * products.  ORC_E_OVERFLOW if some entry does not fit in Wc words (the
 * other entries are still written). */
int orc_matmul(const uint64_t* A, int64_t M, int64_t K, int64_t lda, int Wa,
               const uint64_t* B, int64_t N, int64_t ldb, int Wb,
               uint64_t* C, int64_t ldc, int Wc) {
    if (Wa < 1 || Wb < 1 || Wc < 1 || M < 0 || N < 0 || K < 0) return ORC_E_INVALID;
    int status = ORC_OK;
    const int na = 2 * Wa, nb = 2 * Wb;
    /* accumulator: product limbs + room for K-fold growth */
    const int nacc = na + nb + 4;
    /* B magnitudes and signs, converted once */
    uint32_t* bmag = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)nb * (size_t)(K * N + 1));
    int* bneg = (int*)malloc(sizeof(int) * (size_t)(K * N + 1));
    if (!bmag || !bneg) { free(bmag); free(bneg); return ORC_E_NOMEM; }
    for (int64_t k = 0; k < K; k++)
        for (int64_t n = 0; n < N; n++)
            bneg[k * N + n] = tc_to_sm(B + (size_t)(k * ldb + n) * Wb, Wb, bmag + (size_t)(k * N + n) * nb);

#pragma omp parallel
    {
        uint32_t* amag = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)na * (size_t)(K + 1));
        int* aneg = (int*)malloc(sizeof(int) * (size_t)(K + 1));
        uint32_t* prod = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)(na + nb));
        uint32_t* acc = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)nacc);
        uint32_t* tmp = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)(nacc + 1));
        int local_status = ORC_OK;
#pragma omp for schedule(dynamic, 1)
        for (int64_t m = 0; m < M; m++) {
            for (int64_t k = 0; k < K; k++)
                aneg[k] = tc_to_sm(A + (size_t)(m * lda + k) * Wa, Wa, amag + (size_t)k * na);
            for (int64_t n = 0; n < N; n++) {
                int acc_neg = 0;
                memset(acc, 0, sizeof(uint32_t) * (size_t)nacc);
                for (int64_t k = 0; k < K; k++) {
                    const uint32_t* a = amag + (size_t)k * na;
                    const uint32_t* b = bmag + (size_t)(k * N + n) * nb;
                    int la = mag_len(a, na), lb = mag_len(b, nb);
                    if (la == 0 || lb == 0) continue;
                    mag_mul(a, la, b, lb, prod);
                    int lp = la + lb;
                    int pneg = aneg[k] ^ bneg[k * N + n];
                    /* acc := acc + (pneg ? -prod : prod) in sign-magnitude */
                    if (pneg == acc_neg) {
                        mag_add(acc, nacc - 1, prod, lp, tmp);
                        memcpy(acc, tmp, sizeof(uint32_t) * (size_t)nacc);
                    } else if (mag_cmp(acc, nacc, prod, lp) >= 0) {
                        mag_sub(acc, nacc, prod, lp, acc);
                    } else {
                        memset(tmp, 0, sizeof(uint32_t) * (size_t)nacc);
                        memcpy(tmp, prod, sizeof(uint32_t) * (size_t)lp);
                        mag_sub(tmp, nacc, acc, nacc, acc);
                        acc_neg = pneg;
                    }
                }
                int rc = sm_to_tc(acc_neg, acc, nacc, C + (size_t)(m * ldc + n) * Wc, Wc);
                if (rc != ORC_OK) local_status = rc;
            }
        }
#pragma omp critical
        {
            if (local_status != ORC_OK) status = local_status;
        }
        free(amag); free(aneg); free(prod); free(acc); free(tmp);
    }
    free(bmag);
    free(bneg);
    return status;
}

/* ------------------------------------------------------------------------ */
/* Residue products (Section 3.1: one independent product per prime, each   */
/* reduced modulo its prime).                                               */
/* ------------------------------------------------------------------------ */

/* C_i = (A_i B_i) mod p_i in [0, p_i) for each of L primes.  Entries of the
 * residue operands are any int32 representatives.  A_i starts at
 * A + i * a_prime_stride (a stride of 0 shares one A across all primes).
 * The dot products are accumulated exactly in 128-bit integers. */
int orc_residue_gemm(const int32_t* A, int64_t a_prime_stride, const int32_t* B,
                     int64_t M, int64_t N, int64_t K, const uint32_t* primes, int L,
                     int32_t* C) {
    if (M < 0 || N < 0 || K < 0 || L < 0) return ORC_E_INVALID;
    for (int i = 0; i < L; i++) {
        const int32_t* Ai = A + (size_t)i * (size_t)a_prime_stride;
        const int32_t* Bi = B + (size_t)i * (size_t)(K * N);
        int32_t* Ci = C + (size_t)i * (size_t)(M * N);
        const __int128 p = primes[i];
#pragma omp parallel for schedule(static)
        for (int64_t m = 0; m < M; m++)
            for (int64_t n = 0; n < N; n++) {
                __int128 s = 0;
                for (int64_t k = 0; k < K; k++) s += (__int128)Ai[m * K + k] * Bi[k * N + n];
                __int128 r = s % p;
                if (r < 0) r += p;
                Ci[m * N + n] = (int32_t)r;
            }
    }
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* CRT reconstruction (Section 3.1: the exact product comes back from its  */
/* residues by CRT).  Lagrange form:                                        */
/*   x = sum_i r_i * (M/p_i) * ((M/p_i)^-1 mod p_i)  (mod M),               */
/* then the symmetric representative in (-M/2, M/2].                        */
/* ------------------------------------------------------------------------ */

static uint32_t mulmod32(uint32_t a, uint32_t b, uint32_t p) {
    return (uint32_t)(((uint64_t)a * b) % p);
}

static uint32_t powmod32(uint32_t a, uint32_t e, uint32_t p) {
    uint32_t r = 1 % p;
    a %= p;
    while (e) {
        if (e & 1) r = mulmod32(r, a, p);
        a = mulmod32(a, a, p);
        e >>= 1;
    }
    return r;
}

/* residues: [L][count] canonical; out: count entries of W words each. */
int orc_crt(const int32_t* residues, int64_t count, const uint32_t* primes, int L,
            uint64_t* out, int W) {
    if (L < 1 || W < 1 || count < 0) return ORC_E_INVALID;
    for (int i = 0; i < L; i++)
        if (!orc_is_prime(primes[i])) return ORC_E_INVALID;
    for (int i = 0; i < L; i++)
        for (int j = 0; j < i; j++)
            if (primes[i] == primes[j]) return ORC_E_INVALID;
    const int n = L + 2; /* limbs of M and of partial sums */
    uint32_t* Mm = (uint32_t*)calloc((size_t)n + 1, sizeof(uint32_t));
    uint32_t* Mi = (uint32_t*)calloc((size_t)L * (size_t)(n + 1), sizeof(uint32_t));
    uint32_t* yi = (uint32_t*)calloc((size_t)L, sizeof(uint32_t));
    uint32_t* half = (uint32_t*)calloc((size_t)n + 1, sizeof(uint32_t));
    if (!Mm || !Mi || !yi || !half) { free(Mm); free(Mi); free(yi); free(half); return ORC_E_NOMEM; }
    Mm[0] = 1;
    int nm = 1;
    for (int i = 0; i < L; i++) nm = mag_mul_small_add(Mm, nm, primes[i], 0);
    for (int i = 0; i < L; i++) {
        uint32_t* mi = Mi + (size_t)i * (n + 1);
        mag_div_small(Mm, n, primes[i], mi); /* M / p_i, exact */
        uint32_t c = mag_mod_small(mi, n, primes[i]);
        yi[i] = powmod32(c, primes[i] - 2, primes[i]); /* Fermat inverse */
    }
    /* (M - 1) / 2 for the symmetric range; M is odd */
    mag_div_small(Mm, n, 2, half);
    int status = ORC_OK;
#pragma omp parallel
    {
        uint32_t* x = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)(n + 2));
        uint32_t* t = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)(n + 2));
        uint32_t* u = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)(n + 2));
        int local = ORC_OK;
#pragma omp for schedule(static)
        for (int64_t e = 0; e < count; e++) {
            memset(x, 0, sizeof(uint32_t) * (size_t)(n + 2));
            for (int i = 0; i < L; i++) {
                uint32_t r = (uint32_t)residues[(size_t)i * count + e];
                if (r >= primes[i]) { local = ORC_E_INVALID; r %= primes[i]; }
                uint32_t coef = mulmod32(r, yi[i], primes[i]);
                /* t = M_i * coef  (< M) */
                memcpy(t, Mi + (size_t)i * (n + 1), sizeof(uint32_t) * (size_t)n);
                t[n] = 0;
                mag_mul_small_add(t, n, coef, 0);
                /* x += t; if x >= M: x -= M */
                mag_add(x, n + 1, t, n + 1, u);
                memcpy(x, u, sizeof(uint32_t) * (size_t)(n + 2));
                if (mag_cmp(x, n + 2, Mm, n) >= 0) mag_sub(x, n + 2, Mm, n, x);
            }
            /* symmetric representative: x > (M-1)/2  ->  x - M (negative) */
            int neg = 0;
            if (mag_cmp(x, n + 2, half, n) > 0) {
                memset(t, 0, sizeof(uint32_t) * (size_t)(n + 2));
                memcpy(t, Mm, sizeof(uint32_t) * (size_t)n);
                mag_sub(t, n + 2, x, n + 2, x); /* |x - M| = M - x */
                neg = 1;
            }
            int rc = sm_to_tc(neg, x, n + 2, out + (size_t)e * W, W);
            if (rc != ORC_OK) local = rc;
        }
#pragma omp critical
        {
            if (local != ORC_OK) status = local;
        }
        free(x); free(t); free(u);
    }
    free(Mm); free(Mi); free(yi); free(half);
    return status;
}

/* ------------------------------------------------------------------------ */
/* Balanced base-2^8 digits of a signed residue: r = sum_u d_u 2^(8u), the
 * lower t-1 digits in [-128, 127] and the top digit the remaining quotient,
 * which must satisfy |d_top| <= 128 (so every digit product is at most 2^14
 * in magnitude).  The lower digits are fixed by r mod 256^(t-1), so the
 * representation is unique. */

/* digits: [t][count]; returns ORC_E_OVERFLOW if t digits do not suffice */
int orc_balanced_digits(const int64_t* r, int64_t count, int t, int32_t* digits) {
    int status = ORC_OK;
    for (int64_t e = 0; e < count; e++) {
        int64_t v = r[e];
        for (int u = 0; u < t - 1; u++) {
            int64_t d = ((v % 256) + 256) % 256; /* 0..255 */
            if (d >= 128) d -= 256;              /* -128..127 */
            digits[(size_t)u * count + e] = (int32_t)d;
            v = (v - d) / 256;
        }
        if (v > 128 || v < -128) status = ORC_E_OVERFLOW;
        digits[(size_t)(t - 1) * count + e] = (int32_t)v;
    }
    return status;
}

/* ------------------------------------------------------------------------ */
/* det A mod q: the check of a Smith form at sizes where no exact Smith form  */
/* of the oracle finishes.  Section 2: the invariant factors of a nonsingular */
/* A multiply to |det A|, so prod s_i = +-det A modulo every prime q.         */
/* ------------------------------------------------------------------------ */

static uint64_t mulmod64(uint64_t a, uint64_t b, uint64_t q) {
    return (uint64_t)((unsigned __int128)a * b % q);
}

static uint64_t powmod64(uint64_t a, uint64_t e, uint64_t q) {
    uint64_t r = 1 % q;
    while (e) {
        if (e & 1) r = mulmod64(r, a, q);
        a = mulmod64(a, a, q);
        e >>= 1;
    }
    return r;
}

/* Gaussian elimination over GF(q) for a prime q < 2^63 on the n x n int64
 * matrix A (row-major, leading dimension lda): at step k the first row at or
 * below k with a nonzero entry in column k is swapped up (the determinant
 * changes sign), and every row below it subtracts the multiple of it that
 * clears column k.  det = sign * product of the pivots.  The rows of one step
 * are independent (OpenMP).  *det gets det A mod q in [0, q). */
int orc_det_mod(const int64_t* A, int64_t n, int64_t lda, uint64_t q, uint64_t* det) {
    if (n < 0 || lda < n || q < 2 || !det) return ORC_E_INVALID;
    uint64_t* M = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)(n > 0 ? n * n : 1));
    if (!M) return ORC_E_NOMEM;
    for (int64_t i = 0; i < n; i++)
        for (int64_t j = 0; j < n; j++) {
            const int64_t a = A[i * lda + j];
            const uint64_t m = (uint64_t)(a < 0 ? -(a + 1) : a) % q; /* |a| - 1 for negatives: no overflow */
            M[i * n + j] = a < 0 ? (q - (m + 1) % q) % q : m;
        }
    uint64_t d = 1 % q;
    for (int64_t k = 0; k < n && d; k++) {
        int64_t piv = -1;
        for (int64_t i = k; i < n; i++)
            if (M[i * n + k]) {
                piv = i;
                break;
            }
        if (piv < 0) {
            d = 0;
            break;
        }
        if (piv != k) {
            for (int64_t j = 0; j < n; j++) {
                const uint64_t t = M[k * n + j];
                M[k * n + j] = M[piv * n + j];
                M[piv * n + j] = t;
            }
            d = (q - d) % q;
        }
        const uint64_t p = M[k * n + k];
        d = mulmod64(d, p, q);
        const uint64_t inv = powmod64(p, q - 2, q); /* Fermat: q is prime */
#pragma omp parallel for schedule(static)
        for (int64_t i = k + 1; i < n; i++) {
            const uint64_t f = mulmod64(M[i * n + k], inv, q);
            if (!f) continue;
            for (int64_t j = k; j < n; j++) {
                const uint64_t t = mulmod64(f, M[k * n + j], q);
                const uint64_t x = M[i * n + j];
                M[i * n + j] = x >= t ? x - t : x + (q - t);
            }
        }
    }
    free(M);
    *det = d;
    return ORC_OK;
}
