// Arbitrary-precision integers for the host side of the Smith-form driver:
// naturals as little-endian base-2^32 limbs without leading zero limbs (zero
// has no limbs), signed values as sign and magnitude.  Schoolbook products,
// long division by Knuth's Algorithm D (TAOCP vol. 2, 4.3.1), Euclid's gcd,
// and rational reconstruction by the extended Euclidean algorithm (Wang's
// method: the first remainder below the numerator bound, with its cofactor),
// sped up by Lehmer's single-precision quotient runs.
#pragma once

#include <stdint.h>

#include <algorithm>
#include <utility>
#include <vector>

namespace smf {

struct Nat {
    std::vector<uint32_t> d;
    Nat() = default;
    explicit Nat(uint64_t v) {
        while (v) {
            d.push_back((uint32_t)v);
            v >>= 32;
        }
    }
    bool zero() const { return d.empty(); }
    void trim() {
        while (!d.empty() && d.back() == 0) d.pop_back();
    }
    int64_t bits() const {
        if (d.empty()) return 0;
        uint32_t t = d.back();
        int b = 0;
        while (t) {
            b++;
            t >>= 1;
        }
        return 32 * (int64_t)(d.size() - 1) + b;
    }
};

inline int cmp(const Nat& a, const Nat& b) {
    if (a.d.size() != b.d.size()) return a.d.size() < b.d.size() ? -1 : 1;
    for (size_t i = a.d.size(); i-- > 0;)
        if (a.d[i] != b.d[i]) return a.d[i] < b.d[i] ? -1 : 1;
    return 0;
}

inline Nat add(const Nat& a, const Nat& b) {
    const Nat& x = a.d.size() >= b.d.size() ? a : b;
    const Nat& y = a.d.size() >= b.d.size() ? b : a;
    Nat r;
    r.d.resize(x.d.size() + 1);
    uint64_t c = 0;
    for (size_t i = 0; i < x.d.size(); i++) {
        c += (uint64_t)x.d[i] + (i < y.d.size() ? y.d[i] : 0u);
        r.d[i] = (uint32_t)c;
        c >>= 32;
    }
    r.d[x.d.size()] = (uint32_t)c;
    r.trim();
    return r;
}

// a - b for a >= b
inline Nat sub(const Nat& a, const Nat& b) {
    Nat r;
    r.d.resize(a.d.size());
    uint32_t borrow = 0;
    for (size_t i = 0; i < a.d.size(); i++) {
        const uint64_t t = (uint64_t)a.d[i] - (i < b.d.size() ? b.d[i] : 0u) - borrow;
        r.d[i] = (uint32_t)t;
        borrow = (uint32_t)(t >> 63);  // the subtraction wrapped
    }
    r.trim();
    return r;
}

// a = a * m + c
inline void mul_add_small(Nat& a, uint32_t m, uint64_t c) {
    for (size_t i = 0; i < a.d.size(); i++) {
        const uint64_t t = (uint64_t)a.d[i] * m + (c & 0xffffffffu);
        a.d[i] = (uint32_t)t;
        c = (c >> 32) + (t >> 32);
    }
    while (c) {
        a.d.push_back((uint32_t)c);
        c >>= 32;
    }
    a.trim();
}

namespace nat_detail {
// r[0 .. na+nb) += a * b, schoolbook (r long enough, a carry never leaves it)
inline void mul_school(uint32_t* r, const uint32_t* a, size_t na, const uint32_t* b, size_t nb) {
    for (size_t i = 0; i < na; i++) {
        const uint64_t ai = a[i];
        uint64_t c = 0;
        for (size_t j = 0; j < nb; j++) {
            const uint64_t t = ai * b[j] + r[i + j] + c;  // <= 2^64 - 1
            r[i + j] = (uint32_t)t;
            c = t >> 32;
        }
        for (size_t k = i + nb; c; k++) {
            const uint64_t t = (uint64_t)r[k] + c;
            r[k] = (uint32_t)t;
            c = t >> 32;
        }
    }
}
// r[0 .. n) += x[0 .. nx) (nx <= n); the carry out of r[n - 1] is returned
inline uint32_t add_into(uint32_t* r, size_t n, const uint32_t* x, size_t nx) {
    uint64_t c = 0;
    size_t i = 0;
    for (; i < nx; i++) {
        c += (uint64_t)r[i] + x[i];
        r[i] = (uint32_t)c;
        c >>= 32;
    }
    for (; c && i < n; i++) {
        c += r[i];
        r[i] = (uint32_t)c;
        c >>= 32;
    }
    return (uint32_t)c;
}
// r[0 .. n) -= x[0 .. nx) (the result is known to be non-negative)
inline void sub_from(uint32_t* r, size_t n, const uint32_t* x, size_t nx) {
    int64_t b = 0;
    size_t i = 0;
    for (; i < nx; i++) {
        const int64_t t = (int64_t)r[i] - x[i] - b;
        r[i] = (uint32_t)t;
        b = t < 0;
    }
    for (; b && i < n; i++) {
        const int64_t t = (int64_t)r[i] - b;
        r[i] = (uint32_t)t;
        b = t < 0;
    }
}
constexpr size_t kKaratsuba = 32;  // limbs below which the schoolbook product is faster
// r[0 .. na+nb) = a * b by Karatsuba's method (r zero on entry): with a = a1 B^h + a0,
// b = b1 B^h + b0, a b = a1 b1 B^2h + ((a0 + a1)(b0 + b1) - a0 b0 - a1 b1) B^h + a0 b0.
// An operand much shorter than the other is taken against the longer one in pieces of
// its length, each product added in with its carry carried through.
inline void mul_kara(uint32_t* r, const uint32_t* a, size_t na, const uint32_t* b, size_t nb) {
    if (na < nb) {
        std::swap(a, b);
        std::swap(na, nb);
    }
    if (nb < kKaratsuba) {
        mul_school(r, a, na, b, nb);
        return;
    }
    if (na >= 2 * nb) {  // pieces of the longer operand, each about nb limbs
        std::vector<uint32_t> t(2 * nb);
        for (size_t off = 0; off < na; off += nb) {
            const size_t np = std::min(nb, na - off);
            std::fill(t.begin(), t.end(), 0u);
            mul_kara(t.data(), a + off, np, b, nb);
            add_into(r + off, na + nb - off, t.data(), np + nb);
        }
        return;
    }
    const size_t h = (na + 1) / 2;  // nb >= h since na < 2 nb
    const uint32_t *a0 = a, *a1 = a + h, *b0 = b, *b1 = b + h;
    const size_t na1 = na - h, nb1 = nb - h;
    std::vector<uint32_t> z0(2 * h, 0), z2(na1 + nb1, 0), sa(h + 1, 0), sb(h + 1, 0), z1(2 * h + 2, 0);
    mul_kara(z0.data(), a0, h, b0, h);
    mul_kara(z2.data(), a1, na1, b1, nb1);
    std::copy(a0, a0 + h, sa.begin());
    sa[h] = add_into(sa.data(), h, a1, na1);
    std::copy(b0, b0 + h, sb.begin());
    sb[h] = add_into(sb.data(), h, b1, nb1);
    mul_kara(z1.data(), sa.data(), h + 1, sb.data(), h + 1);
    sub_from(z1.data(), z1.size(), z0.data(), z0.size());
    sub_from(z1.data(), z1.size(), z2.data(), z2.size());
    size_t n1 = z1.size();
    while (n1 > 0 && z1[n1 - 1] == 0) n1--;
    const size_t nr = na + nb;
    add_into(r, nr, z0.data(), z0.size());
    add_into(r + h, nr - h, z1.data(), n1);
    add_into(r + 2 * h, nr - 2 * h, z2.data(), z2.size());
}
}  // namespace nat_detail

inline Nat mul(const Nat& a, const Nat& b) {
    Nat r;
    if (a.zero() || b.zero()) return r;
    r.d.assign(a.d.size() + b.d.size(), 0);
    nat_detail::mul_kara(r.d.data(), a.d.data(), a.d.size(), b.d.data(), b.d.size());
    r.trim();
    return r;
}

namespace nat_detail {
inline int clz32(uint32_t x) {
    int n = 0;
    while (!(x & 0x80000000u)) {
        x <<= 1;
        n++;
    }
    return n;
}
// x << s limb by limb (0 <= s < 32), with `extra` zero limbs appended first
inline std::vector<uint32_t> shl(const std::vector<uint32_t>& x, int s, size_t extra) {
    std::vector<uint32_t> r(x.size() + extra, 0);
    uint32_t carry = 0;
    for (size_t i = 0; i < x.size(); i++) {
        r[i] = s ? (x[i] << s) | carry : x[i];
        carry = s ? x[i] >> (32 - s) : 0;
    }
    if (extra) r[x.size()] = carry;
    return r;
}
}  // namespace nat_detail

// q = a / b and r = a mod b (b non-zero); either output may be null.
inline void divmod(const Nat& a, const Nat& b, Nat* q, Nat* r) {
    if (cmp(a, b) < 0) {
        if (q) *q = Nat();
        if (r) *r = a;
        return;
    }
    if (b.d.size() == 1) {
        const uint64_t v = b.d[0];
        Nat qq;
        qq.d.resize(a.d.size());
        uint64_t rem = 0;
        for (size_t i = a.d.size(); i-- > 0;) {
            const uint64_t cur = (rem << 32) | a.d[i];
            qq.d[i] = (uint32_t)(cur / v);
            rem = cur % v;
        }
        qq.trim();
        if (q) *q = std::move(qq);
        if (r) *r = Nat(rem);
        return;
    }
    // normalise so that the divisor's top limb has its high bit set
    const int s = nat_detail::clz32(b.d.back());
    std::vector<uint32_t> u = nat_detail::shl(a.d, s, 1);
    const std::vector<uint32_t> v = nat_detail::shl(b.d, s, 0);
    const size_t n = v.size(), m = u.size() - n;
    Nat qq;
    qq.d.assign(m, 0);
    const uint64_t B = 1ull << 32;
    for (size_t j = m; j-- > 0;) {
        // estimate the quotient limb from the top two limbs, then correct it
        const uint64_t num = ((uint64_t)u[j + n] << 32) | u[j + n - 1];
        uint64_t qhat = num / v[n - 1], rhat = num % v[n - 1];
        while (qhat >= B || qhat * v[n - 2] > ((rhat << 32) | u[j + n - 2])) {
            qhat--;
            rhat += v[n - 1];
            if (rhat >= B) break;
        }
        // u[j .. j+n] -= qhat * v
        uint64_t carry = 0;
        uint32_t borrow = 0;
        for (size_t i = 0; i < n; i++) {
            const uint64_t p = qhat * v[i] + carry;
            carry = p >> 32;
            const uint64_t t = (uint64_t)u[i + j] - (uint32_t)p - borrow;
            u[i + j] = (uint32_t)t;
            borrow = (uint32_t)(t >> 63);
        }
        const uint64_t t = (uint64_t)u[j + n] - carry - borrow;
        u[j + n] = (uint32_t)t;
        if (t >> 63) {  // qhat was one too large: add v back
            qhat--;
            uint64_t c = 0;
            for (size_t i = 0; i < n; i++) {
                c += (uint64_t)u[i + j] + v[i];
                u[i + j] = (uint32_t)c;
                c >>= 32;
            }
            u[j + n] += (uint32_t)c;
        }
        qq.d[j] = (uint32_t)qhat;
    }
    qq.trim();
    if (q) *q = std::move(qq);
    if (r) {
        Nat rr;
        rr.d.resize(n);
        for (size_t i = 0; i < n; i++)
            rr.d[i] = s ? (u[i] >> s) | (i + 1 < n + 1 ? (uint32_t)((uint64_t)u[i + 1] << (32 - s)) : 0u) : u[i];
        rr.trim();
        *r = std::move(rr);
    }
}

// sum_(t < k) c[t * stride] p^t by Horner's rule, taking g digits per pass
// over the limbs: g is the largest count with p^g < 2^32 whose grouped addend
// sum_(i < g) c_i p^i still fits 64 bits, given c_t < 2^cbits (for a 24-bit p
// one digit per pass; for an 8-bit p, digit sums below 2^38, four).
inline Nat horner(const uint64_t* c, int64_t k, size_t stride, uint32_t p, int cbits) {
    int pb = 0;
    while ((1ull << pb) <= p) pb++;
    int g = 1;
    uint64_t pg = p;  // p^g
    while (pg * p < (1ull << 32) && cbits + 1 + pb * g < 64) {
        pg *= p;
        g++;
    }
    Nat z;
    int64_t t = k;
    const int64_t top = k % g ? k % g : g;  // the top group may be short
    for (int64_t len = top; t > 0; len = g) {
        uint64_t add = 0, mult = 1;
        for (int64_t i = t - 1; i >= t - len; i--) add = add * p + c[(size_t)i * stride];
        for (int64_t i = 0; i < len; i++) mult *= p;
        mul_add_small(z, (uint32_t)mult, add);
        t -= len;
    }
    return z;
}

// The same z = sum_(t < k) c[t stride] p^t by halves: z = z_lo + p^h z_hi with
// h = kBlock 2^j the largest below the length, down to blocks of kBlock digits
// (horner).  pw[j] = p^(kBlock 2^j), from horner_powers(p, k).  With
// Karatsuba products this costs a few products of the final size instead of
// k products by a word that grow to it.
constexpr int64_t kHornerBlock = 128;
inline std::vector<Nat> horner_powers(uint32_t p, int64_t k) {
    std::vector<Nat> pw;
    Nat b(1);
    for (int64_t i = 0; i < kHornerBlock; i++) mul_add_small(b, p, 0);
    pw.push_back(b);
    while (kHornerBlock * ((int64_t)1 << pw.size()) < k) pw.push_back(mul(pw.back(), pw.back()));
    return pw;
}
inline Nat horner_split(const uint64_t* c, int64_t k, size_t stride, uint32_t p, int cbits,
                        const std::vector<Nat>& pw) {
    if (k <= kHornerBlock) return horner(c, k, stride, p, cbits);
    size_t j = 0;
    while (j + 1 < pw.size() && kHornerBlock * ((int64_t)2 << j) < k) j++;
    const int64_t h = kHornerBlock * ((int64_t)1 << j);
    Nat lo = horner_split(c, h, stride, p, cbits, pw);
    const Nat hi = horner_split(c + (size_t)h * stride, k - h, stride, p, cbits, pw);
    return add(lo, mul(hi, pw[j]));
}

// p^k by binary powering, top bit of k first: about log2 k squarings by the
// Karatsuba product, the last of the final size, in place of k products by a
// word that grow to it (at k = 9800 digits of a 24-bit p, 45 -> 5 ms on an x86
// host)
inline Nat pow_small(uint32_t p, int64_t k) {
    Nat r(1);
    if (k <= 0) return r;
    int top = 62;
    while (!((k >> top) & 1)) top--;
    for (int b = top; b >= 0; b--) {
        if (b != top) r = mul(r, r);
        if ((k >> b) & 1) mul_add_small(r, p, 0);
    }
    return r;
}

struct Int {
    bool neg = false;
    Nat m;
};

inline Int add(const Int& a, const Int& b) {
    if (a.neg == b.neg) return Int{a.neg && !(a.m.zero() && b.m.zero()), add(a.m, b.m)};
    const int c = cmp(a.m, b.m);
    if (c == 0) return Int{};
    return c > 0 ? Int{a.neg, sub(a.m, b.m)} : Int{b.neg, sub(b.m, a.m)};
}

// bits s .. s+63 of n (zeros above its top), s >= 0
inline uint64_t bits_at(const Nat& n, int64_t s) {
    const size_t w = (size_t)(s / 32);
    const int b = (int)(s % 32);
    auto limb = [&](size_t k) -> uint64_t { return k < n.d.size() ? n.d[k] : 0u; };
    const uint64_t lo = limb(w) | (limb(w + 1) << 32);
    return b ? (lo >> b) | (limb(w + 2) << (64 - b)) : lo;
}

// (x, y) <- (A x + B y, C x + D y) in one pass over the limbs, for
// single-word signed coefficients (|A|, |B|, |C|, |D| < 2^31): each result is
// accumulated with a signed 128-bit carry in two's complement over two limbs
// more than the inputs, then turned back into sign and magnitude.
inline void lin2(Int& x, Int& y, int64_t A, int64_t B, int64_t C, int64_t D) {
    const int64_t a = x.neg ? -A : A, b = y.neg ? -B : B, c = x.neg ? -C : C, d = y.neg ? -D : D;
    const size_t n = std::max(x.m.d.size(), y.m.d.size()) + 2;
    std::vector<uint32_t> r0(n), r1(n);
    __int128 k0 = 0, k1 = 0;
    for (size_t i = 0; i < n; i++) {
        const int64_t xi = i < x.m.d.size() ? x.m.d[i] : 0, yi = i < y.m.d.size() ? y.m.d[i] : 0;
        k0 += (__int128)a * xi + (__int128)b * yi;
        k1 += (__int128)c * xi + (__int128)d * yi;
        r0[i] = (uint32_t)(uint64_t)k0;
        r1[i] = (uint32_t)(uint64_t)k1;
        k0 >>= 32;  // arithmetic: the carry keeps the sign
        k1 >>= 32;
    }
    auto finish = [](std::vector<uint32_t>& r, bool negative, Int& out) {
        if (negative) {  // two's complement -> magnitude
            uint64_t carry = 1;
            for (auto& w : r) {
                const uint64_t t = (uint64_t)(uint32_t)~w + carry;
                w = (uint32_t)t;
                carry = t >> 32;
            }
        }
        out.m.d = std::move(r);
        out.m.trim();
        out.neg = negative && !out.m.zero();
    };
    finish(r0, k0 < 0, x);
    finish(r1, k1 < 0, y);
}

// Lehmer's acceleration of Euclid's algorithm (Knuth, TAOCP vol. 2, 4.5.2,
// Algorithm L): run the quotients of the leading 31 bits of (u, v), u >= v,
// while the two bounding quotients agree (then they are the true ones), and
// return their 2 x 2 cofactor matrix: the remainders advance as
// (u, v) <- (A u + B v, C u + D v).  B = 0 when no step is certain.
inline void lehmer_round(const Nat& u, const Nat& v, int64_t* A, int64_t* B, int64_t* C, int64_t* D) {
    const int64_t sh = u.bits() - 31;
    int64_t x = (int64_t)(bits_at(u, sh) & 0x7fffffffu), y = (int64_t)(bits_at(v, sh) & 0x7fffffffu);
    int64_t a = 1, b = 0, c = 0, d = 1;
    while (y + c > 0 && y + d > 0) {
        const int64_t q = (x + a) / (y + c);
        if (q != (x + b) / (y + d) || x + b < 0 || x + a < 0) break;
        int64_t t = a - q * c;
        a = c;
        c = t;
        t = b - q * d;
        b = d;
        d = t;
        t = x - q * y;
        x = y;
        y = t;
    }
    *A = a;
    *B = b;
    *C = c;
    *D = d;
}

inline Nat gcd(Nat a, Nat b) {
    if (cmp(a, b) < 0) std::swap(a, b);
    while (b.bits() > 64) {
        int64_t A, B, C, D;
        lehmer_round(a, b, &A, &B, &C, &D);
        if (B == 0) {
            Nat r;
            divmod(a, b, nullptr, &r);
            a = std::move(b);
            b = std::move(r);
            continue;
        }
        Int x{false, std::move(a)}, y{false, std::move(b)};
        lin2(x, y, A, B, C, D);  // Euclidean remainders: non-negative
        a = std::move(x.m);
        b = std::move(y.m);
    }
    while (!b.zero()) {
        Nat r;
        divmod(a, b, nullptr, &r);
        a = std::move(b);
        b = std::move(r);
    }
    return a;
}

// The fraction a / b (b > 0, gcd 1) with a = b u (mod P), |a| < 2^nb and
// b < 2^db, by the extended Euclidean algorithm on (P, u): the first
// remainder below 2^nb and its cofactor.  Unique when P > 2^(nb + db + 1).
// False when there is no such fraction: the stopping row's cofactor is not
// below 2^db, or it shares a factor with the row's remainder.
inline bool rational_reconstruct(const Nat& u, const Nat& P, int64_t nb, int64_t db, Int* a, Nat* b) {
    Nat r0 = P, r1;
    divmod(u, P, nullptr, &r1);
    Int t0, t1{false, Nat(1)};
    // Lehmer rounds advance the remainders and the cofactors t together; while
    // r1 keeps more than 96 bits above 2^nb a round cannot pass the stopping row
    while (r1.bits() > nb + 96) {
        int64_t A, B, C, D;
        lehmer_round(r0, r1, &A, &B, &C, &D);
        if (B == 0) {  // no step certain from the leading bits: one full division
            Nat q, rem;
            divmod(r0, r1, &q, &rem);
            r0 = std::move(r1);
            r1 = std::move(rem);
            Int t2 = add(t0, Int{!t1.neg, mul(q, t1.m)});
            if (t2.m.zero()) t2.neg = false;
            t0 = std::move(t1);
            t1 = std::move(t2);
            continue;
        }
        Int x{false, std::move(r0)}, y{false, std::move(r1)};
        lin2(x, y, A, B, C, D);  // remainders of the Euclidean sequence: non-negative
        r0 = std::move(x.m);
        r1 = std::move(y.m);
        lin2(t0, t1, A, B, C, D);
    }
    while (r1.bits() > nb) {
        Nat q, rem;
        divmod(r0, r1, &q, &rem);
        r0 = std::move(r1);
        r1 = std::move(rem);
        Int t2 = add(t0, Int{!t1.neg, mul(q, t1.m)});
        if (t2.m.zero()) t2.neg = false;
        t0 = std::move(t1);
        t1 = std::move(t2);
    }
    if (t1.m.zero() || t1.m.bits() > db) return false;
    // a fraction within the bounds exists only if this row's remainder and
    // cofactor are coprime, and then it is that row (Wang); a common factor
    // means there is none (dividing it out would break a = b u mod P)
    const Nat g = gcd(r1, t1.m);
    if (!(g.d.size() == 1 && g.d[0] == 1)) return false;
    a->neg = t1.neg && !r1.zero();
    a->m = std::move(r1);
    *b = std::move(t1.m);
    return true;
}


// a^-1 mod m (m > 1) by the extended Euclidean algorithm on (m, a mod m) with
// Lehmer's rounds: the remainders r_i keep r_i = t_i a (mod m); at the end
// r = gcd(a, m), and a is invertible exactly when it is 1.  False otherwise.
inline bool inv_mod(const Nat& a, const Nat& m, Nat* inv) {
    Nat r0 = m, r1;
    divmod(a, m, nullptr, &r1);
    Int t0, t1{false, Nat(1)};
    while (!r1.zero()) {
        int64_t A = 1, B = 0, C = 0, D = 1;
        if (r1.bits() > 64) lehmer_round(r0, r1, &A, &B, &C, &D);
        if (B == 0) {
            Nat q, rem;
            divmod(r0, r1, &q, &rem);
            r0 = std::move(r1);
            r1 = std::move(rem);
            Int t2 = add(t0, Int{!t1.neg, mul(q, t1.m)});
            if (t2.m.zero()) t2.neg = false;
            t0 = std::move(t1);
            t1 = std::move(t2);
            continue;
        }
        Int x{false, std::move(r0)}, y{false, std::move(r1)};
        lin2(x, y, A, B, C, D);
        r0 = std::move(x.m);
        r1 = std::move(y.m);
        lin2(t0, t1, A, B, C, D);
    }
    if (!(r0.d.size() == 1 && r0.d[0] == 1)) return false;
    Nat t;
    divmod(t0.m, m, nullptr, &t);
    *inv = (t0.neg && !t.zero()) ? sub(m, t) : t;
    return true;
}

// Extended Euclid: g = gcd(a, b) = x a + y b (x, y signed).
inline void xgcd(const Nat& a, const Nat& b, Nat* g, Int* x, Int* y) {
    Nat r0 = a, r1 = b;
    Int x0{false, Nat(1)}, x1, y0, y1{false, Nat(1)};
    while (!r1.zero()) {
        Nat q, rem;
        divmod(r0, r1, &q, &rem);
        r0 = std::move(r1);
        r1 = std::move(rem);
        Int x2 = add(x0, Int{!x1.neg, mul(q, x1.m)});
        Int y2 = add(y0, Int{!y1.neg, mul(q, y1.m)});
        if (x2.m.zero()) x2.neg = false;
        if (y2.m.zero()) y2.neg = false;
        x0 = std::move(x1);
        x1 = std::move(x2);
        y0 = std::move(y1);
        y1 = std::move(y2);
    }
    *g = std::move(r0);
    *x = std::move(x0);
    *y = std::move(y0);
}

// a signed value modulo m, in [0, m)
inline Nat mod_of(const Int& v, const Nat& m) {
    Nat r;
    divmod(v.m, m, nullptr, &r);
    return (v.neg && !r.zero()) ? sub(m, r) : r;
}

inline Nat mul_mod(const Nat& a, const Nat& b, const Nat& m) {
    Nat r;
    divmod(mul(a, b), m, nullptr, &r);
    return r;
}

// (a - b) mod m for a, b in [0, m)
inline Nat sub_mod(const Nat& a, const Nat& b, const Nat& m) { return cmp(a, b) >= 0 ? sub(a, b) : sub(add(a, m), b); }

inline bool is_one(const Nat& a) { return a.d.size() == 1 && a.d[0] == 1; }

// Barrett reduction modulo a fixed m of n limbs (Menezes, van Oorschot and
// Vanstone, Handbook of Applied Cryptography, Algorithm 14.42): with
// mu = floor(B^(2n) / m), B = 2^32, an x < B^(2n) has q = floor(floor(x / B^(n-1))
// mu / B^(n+1)) within 2 of floor(x / m), so x mod m = x - q m less at most two
// m.  One division to set up, then two products per reduction.
struct Barrett {
    Nat m, mu;
    size_t n = 0;
};

namespace nat_detail {
// x B^s and floor(x / B^s)
inline Nat shl_limbs(const Nat& x, size_t s) {
    Nat r;
    if (x.zero()) return r;
    r.d.assign(s, 0u);
    r.d.insert(r.d.end(), x.d.begin(), x.d.end());
    return r;
}
inline Nat shr_limbs(const Nat& x, size_t s, bool* rest = nullptr) {
    Nat r;
    if (rest) *rest = std::any_of(x.d.begin(), x.d.begin() + std::min(s, x.d.size()), [](uint32_t v) { return v != 0; });
    if (x.d.size() > s) r.d.assign(x.d.begin() + s, x.d.end());
    return r;
}
}  // namespace nat_detail

// floor(B^(2n) / m) for m of n limbs (Barrett's mu).  Up to kRecipSchool limbs
// by long division.  Above it, from y = floor(B^(2h) / m_t) for the top
// h = floor(n/2) + 3 limbs m_t of m (the same function): x0 = y B^(n-h) has a
// relative error below B^(2-h), one Newton step for the reciprocal,
// x1 = x0 + x0 (B^(2n) - m x0) / B^(2n), squares it (below B^(-n)), and an
// exact comparison of m x1 with B^(2n) settles the last units.  The result is
// exact whatever the approximation's error: a correction of more than a few
// units falls back to long division.  Cost: a few Karatsuba products of the
// size of m instead of a quadratic division (7350 limbs: 58 -> 24 ms on an x86
// host).
constexpr size_t kRecipSchool = 48;
inline Nat recip_floor(const Nat& m) {
    using namespace nat_detail;
    const size_t n = m.d.size();
    Nat X;  // B^(2n)
    X.d.assign(2 * n + 1, 0u);
    X.d[2 * n] = 1;
    auto by_division = [&] {
        Nat q;
        divmod(X, m, &q, nullptr);
        return q;
    };
    if (n <= kRecipSchool) return by_division();
    const size_t h = n / 2 + 3;  // < n here
    Nat mt;
    mt.d.assign(m.d.begin() + (n - h), m.d.end());
    const Nat y = recip_floor(mt);
    const Nat x0 = shl_limbs(y, n - h);
    const Nat t0 = shl_limbs(mul(m, y), n - h);  // m x0
    Nat x1, t;  // t = m x1, from m x0 and the Newton correction d (a product of half the size)
    bool rest = false;
    if (cmp(t0, X) <= 0) {  // x0 below: add d = floor(x0 (B^(2n) - m x0) / B^(2n))
        const Nat d = shr_limbs(mul(y, sub(X, t0)), n + h);
        x1 = add(x0, d);
        t = add(t0, mul(m, d));
    } else {  // above: subtract the ceiling of x0 (m x0 - B^(2n)) / B^(2n)
        Nat d = shr_limbs(mul(y, sub(t0, X)), n + h, &rest);
        if (rest) d = add(d, Nat(1));
        if (cmp(d, x0) > 0) return by_division();
        x1 = sub(x0, d);
        t = sub(t0, mul(m, d));
    }
    for (int it = 0; it < 8; it++) {
        if (cmp(t, X) > 0) {
            if (x1.zero()) break;
            x1 = sub(x1, Nat(1));
            t = sub(t, m);
            continue;
        }
        if (cmp(sub(X, t), m) >= 0) {
            x1 = add(x1, Nat(1));
            t = add(t, m);
            continue;
        }
        return x1;  // m x1 <= B^(2n) < m (x1 + 1)
    }
    return by_division();
}

inline Barrett barrett_of(const Nat& m) {
    Barrett b;
    b.m = m;
    b.n = m.d.size();
    b.mu = recip_floor(m);
    return b;
}

inline Nat barrett_mod(const Barrett& b, const Nat& x) {  // x < B^(2n)
    Nat q1, q3;
    if (x.d.size() > b.n - 1) q1.d.assign(x.d.begin() + (b.n - 1), x.d.end());
    const Nat q2 = mul(q1, b.mu);
    if (q2.d.size() > b.n + 1) q3.d.assign(q2.d.begin() + (b.n + 1), q2.d.end());
    Nat r = sub(x, mul(q3, b.m));
    while (cmp(r, b.m) >= 0) r = sub(r, b.m);
    return r;
}

}  // namespace smf
