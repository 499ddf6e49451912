// The Smith form over Z/(s) of the projection that Phase 2 of the Smith-form
// driver builds (Section 2: the modular Smith form of the projection gives
// the largest invariant factors of A), on the host with the library's big
// integers.  Header-only so that the CPU tests can check it against the
// closed form: over Z/(s) a matrix with integer invariant factors e_i has the
// invariant factors gcd(e_i, s).
#pragma once

#include <stdint.h>

#include <algorithm>
#include <thread>
#include <utility>
#include <vector>

#include "bignat.h"

namespace smf {

// a mod q for a word q
inline uint32_t nat_rem32(const Nat& a, uint32_t q) {
    uint64_t r = 0;
    for (size_t i = a.d.size(); i-- > 0;) r = ((r << 32) | a.d[i]) % q;
    return (uint32_t)r;
}

// The primes below 2^10.
inline const std::vector<uint32_t>& small_primes() {
    static const std::vector<uint32_t> ps = [] {
        std::vector<uint32_t> v;
        for (uint32_t q = 2; q < 1024; q++) {
            bool prime = true;
            for (uint32_t d = 2; d * d <= q && prime; d++) prime = q % d != 0;
            if (prime) v.push_back(q);
        }
        return v;
    }();
    return ps;
}

// Smith form of the c' x c matrix Y over Z/(s): at each step the content g
// (gcd of the modulus and the entries) is divided out, which shrinks the
// modulus to s / (product of the contents so far); then a unit entry is the
// pivot and its row and column are eliminated.  The invariant factor of A
// that a pivot stands for is the modulus at that step.  `complete`: the
// entries left vanished (every further invariant factor of the projection is
// 1).  False when no unit pivot turns up, also after merging the entries into
// one corner by Bezout steps (below).
inline bool pairing_smith(std::vector<Nat> Y, int rows, int cols, const Nat& s, std::vector<Nat>* inv, bool* complete) {
    Nat mod = s;
    std::vector<int> R(rows), C(cols);
    for (int i = 0; i < rows; i++) R[i] = i;
    for (int j = 0; j < cols; j++) C[j] = j;
    const int nt = (int)std::max<unsigned>(1, std::min<unsigned>(std::thread::hardware_concurrency(), 64));
    // threads only pay for themselves on wide numbers (a thread costs tens of
    // microseconds; a product of 64-limb numbers a few)
    auto threads_for = [&](int items) { return mod.d.size() < 64 ? 1 : std::min(nt, std::max(1, items)); };
    auto par_rows = [&](const std::vector<int>& rs, auto&& fn) {
        const int nr = (int)rs.size();
        const int w = threads_for(nr);
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
        // content: g = gcd(mod, first nonzero entry), then the other entries are
        // checked for divisibility by g in parallel (one division each instead of a
        // serial chain of gcds); an entry g does not divide lowers g and the check
        // runs again
        Nat g = mod;
        for (int a : R) {
            for (int j : C)
                if (!Y[(size_t)a * cols + j].zero()) {
                    g = gcd(g, Y[(size_t)a * cols + j]);
                    break;
                }
            if (cmp(g, mod) != 0) break;
        }
        while (!is_one(g)) {
            std::vector<Nat> misfit(rows);
            std::vector<char> bad(rows, 0);
            par_rows(R, [&](int a) {
                for (int j : C) {
                    const Nat& e = Y[(size_t)a * cols + j];
                    if (e.zero()) continue;
                    Nat rem;
                    divmod(e, g, nullptr, &rem);
                    if (!rem.zero()) {
                        misfit[a] = e;
                        bad[a] = 1;
                        return;
                    }
                }
            });
            const auto it = std::find(bad.begin(), bad.end(), 1);
            if (it == bad.end()) break;
            g = gcd(g, misfit[it - bad.begin()]);
        }
        if (cmp(g, mod) == 0) {
            *complete = true;
            return true;
        }
        if (!is_one(g)) {
            par_rows(R, [&](int a) {
                for (int j : C) {
                    Nat& e = Y[(size_t)a * cols + j];
                    Nat q;
                    divmod(e, g, &q, nullptr);
                    e = std::move(q);
                }
            });
            Nat q;
            divmod(mod, g, &q, nullptr);
            mod = std::move(q);
        }
        // a unit pivot; when no entry is one (a composite modulus can leave only
        // non-units, e.g. 2 and 3 modulo 6, although the content is 1) the entries
        // are merged into the corner (a0, j0) by unimodular 2 x 2 steps from
        // Bezout's identity - rows on column j0, then columns on row a0 - until
        // the corner holds the integer gcd of the block, coprime to the modulus
        int pa = -1, pj = -1;
        Nat pinv;
        bool have_inv = false;
        // the first entry (in order) that is a unit: an entry divisible by a small prime
        // factor of the modulus is passed over at the cost of word remainders; the others
        // are inverted modulo `mod`, a batch at a time in parallel, and the first that
        // inverts is the pivot (its inverse comes with it)
        auto find_unit = [&] {
            uint32_t prod[8];
            int nprod = 0;
            {
                uint64_t cur = 1;
                for (uint32_t q : small_primes()) {
                    if (nat_rem32(mod, q)) continue;
                    if (cur * q >= (1ull << 32)) {
                        if (nprod == 8) break;
                        prod[nprod++] = (uint32_t)cur;
                        cur = 1;
                    }
                    cur *= q;
                }
                if (cur > 1 && nprod < 8) prod[nprod++] = (uint32_t)cur;
            }
            auto passes = [&](const Nat& e) {
                if (e.zero()) return false;
                for (int t = 0; t < nprod; t++) {
                    uint32_t x = nat_rem32(e, prod[t]), y = prod[t];  // gcd(e mod P, P) = 1 iff no shared small prime
                    while (y) {
                        const uint32_t r = x % y;
                        x = y;
                        y = r;
                    }
                    if (x != 1) return false;
                }
                return true;
            };
            std::vector<std::pair<int, int>> cand;
            for (int a : R)
                for (int j : C)
                    if (passes(Y[(size_t)a * cols + j])) cand.push_back({a, j});
            const size_t batch = (size_t)threads_for((int)cand.size());
            for (size_t b0 = 0; b0 < cand.size() && pa < 0; b0 += batch) {
                const size_t nb = std::min(cand.size() - b0, batch);
                std::vector<Nat> iv(nb);
                std::vector<char> ok(nb, 0);
                std::vector<std::thread> pool;
                auto one = [&](size_t t) {
                    ok[t] = inv_mod(Y[(size_t)cand[b0 + t].first * cols + cand[b0 + t].second], mod, &iv[t]);
                };
                for (size_t t = 1; t < nb; t++) pool.emplace_back(one, t);
                one(0);
                for (auto& th : pool) th.join();
                for (size_t t = 0; t < nb; t++)
                    if (ok[t]) {
                        pa = cand[b0 + t].first;
                        pj = cand[b0 + t].second;
                        pinv = std::move(iv[t]);
                        have_inv = true;
                        break;
                    }
            }
        };
        // (u, v) <- (x u + y v, (-b/g) u + (a/g) v) on two lines of entries, mod `mod`
        auto bezout = [&](Nat* const* u, Nat* const* v, size_t len, const Nat& ea, const Nat& eb) {
            Nat g;
            Int x, y;
            xgcd(ea, eb, &g, &x, &y);
            Nat bq, aq;
            divmod(eb, g, &bq, nullptr);
            divmod(ea, g, &aq, nullptr);
            const Nat xm = mod_of(x, mod), ym = mod_of(y, mod), nb = mod_of(Int{!bq.zero(), bq}, mod);
            for (size_t t = 0; t < len; t++) {
                const Nat uu = *u[t], vv = *v[t];
                Nat r1, r2;
                divmod(add(mul(xm, uu), mul(ym, vv)), mod, nullptr, &r1);
                divmod(add(mul(nb, uu), mul(aq, vv)), mod, nullptr, &r2);
                *u[t] = std::move(r1);
                *v[t] = std::move(r2);
            }
        };
        find_unit();
        for (int round = 0; pa < 0 && round < 64; round++) {
            const int a0 = R[0], j0 = C[0];
            for (size_t u = 1; u < R.size(); u++) {  // rows: column j0's entries into (a0, j0)
                const int r = R[u];
                const Nat ea = Y[(size_t)a0 * cols + j0], eb = Y[(size_t)r * cols + j0];
                if (eb.zero()) continue;
                std::vector<Nat*> pu, pv;
                for (int j : C) {
                    pu.push_back(&Y[(size_t)a0 * cols + j]);
                    pv.push_back(&Y[(size_t)r * cols + j]);
                }
                bezout(pu.data(), pv.data(), pu.size(), ea, eb);
            }
            for (size_t u = 1; u < C.size(); u++) {  // columns: row a0's entries into (a0, j0)
                const int c = C[u];
                const Nat ea = Y[(size_t)a0 * cols + j0], eb = Y[(size_t)a0 * cols + c];
                if (eb.zero()) continue;
                std::vector<Nat*> pu, pv;
                for (int a : R) {
                    pu.push_back(&Y[(size_t)a * cols + j0]);
                    pv.push_back(&Y[(size_t)a * cols + c]);
                }
                bezout(pu.data(), pv.data(), pu.size(), ea, eb);
            }
            const Nat& corner_e = Y[(size_t)a0 * cols + j0];
            if (!corner_e.zero() && is_one(gcd(mod, corner_e))) {
                pa = a0;
                pj = j0;
                break;
            }
            // an entry the corner's gcd with the modulus does not divide: its row joins row a0
            const Nat gc = gcd(mod, corner_e);
            int add_row = -1;
            for (int a : R) {
                for (int j : C) {
                    Nat rem;
                    divmod(Y[(size_t)a * cols + j], gc, nullptr, &rem);
                    if (!rem.zero()) {
                        add_row = a;
                        break;
                    }
                }
                if (add_row >= 0) break;
            }
            if (add_row < 0 || add_row == a0) {
                find_unit();
                break;
            }
            for (int j : C) {
                Nat& e = Y[(size_t)a0 * cols + j];
                Nat t;
                divmod(add(e, Y[(size_t)add_row * cols + j]), mod, nullptr, &t);
                e = std::move(t);
            }
        }
        if (pa < 0) return false;
        inv->push_back(mod);
        if (!have_inv && !inv_mod(Y[(size_t)pa * cols + pj], mod, &pinv)) return false;
        std::vector<int> others;
        for (int a : R)
            if (a != pa) others.push_back(a);
        // products of entries below the modulus, reduced by Barrett's method
        const Barrett bm = barrett_of(mod);
        par_rows(others, [&](int a) {
            Nat& ea = Y[(size_t)a * cols + pj];
            if (ea.zero()) return;
            const Nat f = barrett_mod(bm, mul(ea, pinv));
            for (int j : C) {
                if (j == pj) continue;
                Nat& e = Y[(size_t)a * cols + j];
                e = sub_mod(e, barrett_mod(bm, mul(f, Y[(size_t)pa * cols + j])), mod);
            }
            ea = Nat();
        });
        R.erase(std::find(R.begin(), R.end(), pa));
        C.erase(std::find(C.begin(), C.end(), pj));
    }
    return true;
}

}  // namespace smf
