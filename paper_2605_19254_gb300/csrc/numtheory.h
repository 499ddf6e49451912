// Word-size number theory on the host for the Smith-form driver (Section 2):
// Phase 2's last iteration factors the word-size modulus s' into prime powers,
// Phase 3 draws random primes, and the entry points check that their moduli
// are prime.  Header-only so that the CPU tests can check it against exact
// arithmetic.
#pragma once

#include <stdint.h>

#include <algorithm>
#include <vector>

namespace smf {

inline uint64_t mulmod64(uint64_t a, uint64_t b, uint64_t m) { return (uint64_t)((unsigned __int128)a * b % m); }

inline uint64_t powmod64(uint64_t a, uint64_t e, uint64_t m) {
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
inline bool is_prime64(uint64_t n) {
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

inline uint64_t gcd64(uint64_t a, uint64_t b) {
    while (b) {
        const uint64_t t = a % b;
        a = b;
        b = t;
    }
    return a;
}

// a non-trivial factor of a composite n by Pollard's rho (Brent's cycle search)
inline uint64_t rho_factor(uint64_t n, uint64_t c) {
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

inline void factor64(uint64_t n, std::vector<uint64_t>* out) {
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

}  // namespace smf
