// Test harness for the host big-integer routines of the Smith-form driver
// (paper_2605_19254_gb300/csrc/bignat.h), the word-size modular arithmetic of
// its eliminations (csrc/modarith.h), its word-size number theory
// (csrc/numtheory.h) and Phase 2's Smith form over Z/(s) (csrc/pairing_smith.h):
// reads one operation per line from
// stdin, numbers in hexadecimal ("-" for a negative value), and writes the
// results on one line, so that tests/test_host_bignat.py can compare them with
// Python's integers.  Test infrastructure only; the library does not use it.
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>

#include <iostream>
#include <sstream>
#include <string>
#include <vector>

#include "bignat.h"
#include "modarith.h"
#include "numtheory.h"
#include "pairing_smith.h"

using smf::Int;
using smf::Nat;

static Nat parse_nat(const std::string& h) {
    Nat n;
    int64_t i = (int64_t)h.size();
    while (i > 0) {
        const int64_t j = i >= 8 ? i - 8 : 0;
        n.d.push_back((uint32_t)strtoul(h.substr(j, i - j).c_str(), nullptr, 16));
        i = j;
    }
    n.trim();
    return n;
}

static Int parse_int(const std::string& h) {
    Int v;
    if (!h.empty() && h[0] == '-') {
        v.m = parse_nat(h.substr(1));
        v.neg = !v.m.zero();
    } else {
        v.m = parse_nat(h);
    }
    return v;
}

static std::string hex(const Nat& n) {
    if (n.zero()) return "0";
    std::string s;
    char buf[16];
    snprintf(buf, sizeof buf, "%x", n.d.back());
    s += buf;
    for (size_t i = n.d.size() - 1; i-- > 0;) {
        snprintf(buf, sizeof buf, "%08x", n.d[i]);
        s += buf;
    }
    return s;
}

static std::string hex(const Int& v) { return (v.neg && !v.m.zero() ? "-" : "") + hex(v.m); }

int main() {
    std::string line;
    while (std::getline(std::cin, line)) {
        std::istringstream in(line);
        std::string op;
        if (!(in >> op)) continue;
        std::vector<std::string> a;
        for (std::string t; in >> t;) a.push_back(t);
        std::string out;
        if (op == "mul") {
            out = hex(smf::mul(parse_nat(a[0]), parse_nat(a[1])));
        } else if (op == "add") {
            out = hex(smf::add(parse_nat(a[0]), parse_nat(a[1])));
        } else if (op == "sub") {  // a >= b
            out = hex(smf::sub(parse_nat(a[0]), parse_nat(a[1])));
        } else if (op == "cmp") {
            out = std::to_string(smf::cmp(parse_nat(a[0]), parse_nat(a[1])));
        } else if (op == "iadd") {
            out = hex(smf::add(parse_int(a[0]), parse_int(a[1])));
        } else if (op == "divmod") {
            Nat q, r;
            smf::divmod(parse_nat(a[0]), parse_nat(a[1]), &q, &r);
            out = hex(q) + " " + hex(r);
        } else if (op == "gcd") {
            out = hex(smf::gcd(parse_nat(a[0]), parse_nat(a[1])));
        } else if (op == "xgcd") {
            Nat g;
            Int x, y;
            smf::xgcd(parse_nat(a[0]), parse_nat(a[1]), &g, &x, &y);
            out = hex(g) + " " + hex(x) + " " + hex(y);
        } else if (op == "inv") {
            Nat r;
            out = smf::inv_mod(parse_nat(a[0]), parse_nat(a[1]), &r) ? hex(r) : "none";
        } else if (op == "modof") {
            out = hex(smf::mod_of(parse_int(a[0]), parse_nat(a[1])));
        } else if (op == "mulmod") {
            out = hex(smf::mul_mod(parse_nat(a[0]), parse_nat(a[1]), parse_nat(a[2])));
        } else if (op == "submod") {
            out = hex(smf::sub_mod(parse_nat(a[0]), parse_nat(a[1]), parse_nat(a[2])));
        } else if (op == "barrett") {  // m x: x mod m, x < 2^(64 n) for m of n limbs
            const smf::Barrett b = smf::barrett_of(parse_nat(a[0]));
            out = hex(smf::barrett_mod(b, parse_nat(a[1])));
        } else if (op == "recip") {  // m: floor(2^(64 n) / m) for m of n limbs
            out = hex(smf::recip_floor(parse_nat(a[0])));
        } else if (op == "inv32") {  // a m (hexadecimal words): a^-1 mod m
            out = hex(Nat(smf::inv_mod32((uint32_t)strtoul(a[0].c_str(), nullptr, 16),
                                         (uint32_t)strtoul(a[1].c_str(), nullptr, 16))));
        } else if (op == "mulmod32") {  // a b m: a b mod m through floor((2^64 - 1) / m)
            const uint32_t m = (uint32_t)strtoul(a[2].c_str(), nullptr, 16);
            out = hex(Nat(smf::mulmod32_rcp((uint32_t)strtoul(a[0].c_str(), nullptr, 16),
                                            (uint32_t)strtoul(a[1].c_str(), nullptr, 16), m, UINT64_MAX / m)));
        } else if (op == "isprime") {  // n (hexadecimal)
            out = smf::is_prime64(strtoull(a[0].c_str(), nullptr, 16)) ? "1" : "0";
        } else if (op == "factor") {  // n: its prime factors with multiplicity, in any order
            std::vector<uint64_t> f;
            smf::factor64(strtoull(a[0].c_str(), nullptr, 16), &f);
            for (size_t i = 0; i < f.size(); i++) {
                char buf[24];
                snprintf(buf, sizeof buf, "%s%llx", i ? " " : "", (unsigned long long)f[i]);
                out += buf;
            }
            if (f.empty()) out = "-";
        } else if (op == "powmod") {  // a e m
            out = hex(Nat(smf::powmod64(strtoull(a[0].c_str(), nullptr, 16), strtoull(a[1].c_str(), nullptr, 16),
                                        strtoull(a[2].c_str(), nullptr, 16))));
        } else if (op == "psmith") {  // rows cols s y_00 y_01 ... (row-major, entries in [0, s))
            const int rows = (int)strtol(a[0].c_str(), nullptr, 16), cols = (int)strtol(a[1].c_str(), nullptr, 16);
            std::vector<Nat> Y;
            for (int e = 0; e < rows * cols; e++) Y.push_back(parse_nat(a[3 + e]));
            std::vector<Nat> inv;
            bool complete = false;
            if (!smf::pairing_smith(Y, rows, cols, parse_nat(a[2]), &inv, &complete)) {
                out = "fail";
            } else {
                out = complete ? "1" : "0";
                for (const Nat& v : inv) out += " " + hex(v);
            }
        } else if (op == "pow") {
            out = hex(smf::pow_small((uint32_t)strtoul(a[0].c_str(), nullptr, 16), strtoll(a[1].c_str(), nullptr, 16)));
        } else if (op == "horner" || op == "hsplit") {  // p cbits k c_0 .. c_(k-1)
            const uint32_t p = (uint32_t)strtoul(a[0].c_str(), nullptr, 16);
            const int cbits = (int)strtol(a[1].c_str(), nullptr, 16);
            const int64_t k = strtoll(a[2].c_str(), nullptr, 16);
            std::vector<uint64_t> c(k ? k : 1, 0);
            for (int64_t t = 0; t < k; t++) c[t] = strtoull(a[3 + t].c_str(), nullptr, 16);
            if (op == "horner") {
                out = hex(smf::horner(c.data(), k, 1, p, cbits));
            } else {
                const std::vector<Nat> pw = smf::horner_powers(p, k);
                out = hex(smf::horner_split(c.data(), k, 1, p, cbits, pw));
            }
        } else if (op == "rr") {  // u P nb db
            Int num;
            Nat den;
            const bool ok = smf::rational_reconstruct(parse_nat(a[0]), parse_nat(a[1]), strtoll(a[2].c_str(), nullptr, 16),
                                                      strtoll(a[3].c_str(), nullptr, 16), &num, &den);
            out = ok ? hex(num) + " " + hex(den) : "none";
        } else {
            out = "?";
        }
        std::cout << out << "\n";
    }
    return 0;
}
