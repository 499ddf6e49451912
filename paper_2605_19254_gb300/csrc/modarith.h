// Word-size modular arithmetic for moduli below 2^31, on the device and the
// host alike (the host build lets the CPU tests check these functions against
// exact integer arithmetic): the eliminations over Z/(m) of the Smith-form
// driver (Section 2's local Smith forms and determinants modulo primes) take a
// pivot's inverse once per column and a multiplier per row, and both sit on the
// column loop's critical path.
#pragma once

#include <stdint.h>

#ifdef __CUDACC__
#define SMF_HD __host__ __device__ __forceinline__
#else
#define SMF_HD inline
#endif

namespace smf {

// the high 64 bits of a b
SMF_HD uint64_t umulhi64(uint64_t a, uint64_t b) {
#ifdef __CUDA_ARCH__
    return __umul64hi(a, b);
#else
    return (uint64_t)(((unsigned __int128)a * b) >> 64);
#endif
}

// a^-1 mod m for 1 < m < 2^31 and a unit a (gcd(a, m) = 1), a < m: the
// extended Euclidean algorithm on (m, a) in 32-bit words; the remainders keep
// r_i = t_i a (mod m) with |t_i| <= m, so the cofactors fit 64-bit products of
// a 32-bit quotient by a cofactor without overflow.  (A 64-bit division, which
// the device emulates in software, made this chain several times longer.)
SMF_HD uint32_t inv_mod32(uint32_t a, uint32_t m) {
    uint32_t r0 = m, r1 = a;
    int64_t t0 = 0, t1 = 1;
    while (r1) {
        const uint32_t q = r0 / r1;
        const uint32_t r2 = r0 - q * r1;
        r0 = r1;
        r1 = r2;
        const int64_t t2 = t0 - (int64_t)q * t1;
        t0 = t1;
        t1 = t2;
    }
    return (uint32_t)(t0 < 0 ? t0 + (int64_t)m : t0);
}

// a b mod m for m < 2^31 and a, b < m, with rcp = floor((2^64 - 1) / m): for
// x = a b < 2^62, q = floor(x rcp / 2^64) is floor(x / m) or one less (the
// error of rcp is below one part in 2^64 / m, x / 2^64 < 1/4), so one
// conditional subtraction finishes.
SMF_HD uint32_t mulmod32_rcp(uint32_t a, uint32_t b, uint32_t m, uint64_t rcp) {
    const uint64_t x = (uint64_t)a * b;
    const uint64_t r = x - umulhi64(x, rcp) * m;
    return (uint32_t)(r >= m ? r - m : r);
}

}  // namespace smf
