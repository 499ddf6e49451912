// Device CRT reconstruction of one entry, shared by crt_reconstruct's kernels
// (crt.cu) and the residue product with the CRT fused into its epilogue
// (gemm_limb.cu).  Section 3.1: the exact product is recovered from its
// per-prime residues by CRT.
//
// Fast path (Lagrange form with a floating-point quotient).  With
// M_i = M / p_i, c_i = M_i^-1 mod p_i and H = (M-1)/2, the shifted value
// y = x + H (mod M), 0 <= y < M, satisfies
//   xi_i = ((r_i + H) mod p_i) * c_i mod p_i,
//   sum_i xi_i M_i = y + alpha M,   alpha = floor(sum_i xi_i / p_i),
// so x = sum_i xi_i M_i - alpha M - H.  The column sums of sum_i xi_i M_i over
// 32-bit limbs fit 64-bit registers (xi_i < 2^26, L <= 48).  alpha comes from
// an fp32 sum of xi_i * (1/p_i), whose error is below 2^-14; its fractional
// part is y / M, which lies near 1/2 for every |x| well inside (-M/2, M/2]
// (H shifts small results to the middle), so the floor is exact unless the
// fraction falls within 2^-12 of an integer.  Those entries take the exact
// Garner path below.
//
// Garner path (mixed radix).  With weights W_k = p_0 ... p_(k-1), x = sum_k v_k W_k,
//   v_i = (r_i - sum_(k<i) v_k W_k) * W_i^-1   (mod p_i),   0 <= v_i < p_i,
// produced column-wise (each finished digit is folded into the running sums
// of all later primes).  M is odd and (M-1)/2 = sum_k ((p_k - 1)/2) W_k, so
// x > (M-1)/2 iff the digit string exceeds ((p_k - 1)/2)_k lexicographically;
// those entries are returned as x - M.  x is rebuilt by Horner over 32-bit limbs.
//
// Every modular product is by a per-basis constant, reduced with Shoup's
// precomputed quotient (one high and two low multiplies, no division).
#ifndef SMF_CRT_DEV_H
#define SMF_CRT_DEV_H

#include "smf_internal.h"

namespace smf {
namespace {

// Residue loads: through the read-only path (inputs of a kernel that does not
// write them), or coherent at L2 (residues written earlier in the same launch
// by other blocks).
template <bool CG>
__device__ __forceinline__ uint32_t load_res(const int32_t* p) {
    if constexpr (CG) return (uint32_t)__ldcg(p);
    else return (uint32_t)__ldg(p);
}

// v * w (mod p) up to one multiple of p: a value in [0, 2p).
__device__ __forceinline__ uint32_t shoup_mul(uint32_t v, uint32_t w, uint32_t ws, uint32_t p) {
    const uint32_t q = __umulhi(v, ws);
    return v * w - q * p;
}

// Per-basis constants, passed by value so that they live in the kernel's
// parameter (constant) bank; with the loops fully unrolled every access is a
// compile-time offset.  gw/gws hold the strictly lower triangle (i, k), k < i,
// at index i(i-1)/2 + k.  The fast-path tables are used when FAST.
template <int LMAX, bool FAST, int PB>  // PB: bits of the largest prime (24 or 26)
struct CrtConst {
    static constexpr int MLMAX = (LMAX * PB + 31) / 32 + 1;
    uint32_t p[LMAX];
    uint32_t ginv[LMAX], ginvs[LMAX];
    uint32_t gw[LMAX * (LMAX - 1) / 2], gws[LMAX * (LMAX - 1) / 2];
    uint32_t m[MLMAX];
    // fast path
    uint32_t hmod[FAST ? LMAX : 1];                    // H mod p_i
    uint32_t c[FAST ? LMAX : 1], cs[FAST ? LMAX : 1];  // M_i^-1 mod p_i and its Shoup companion
    float invp[FAST ? LMAX : 1];                       // 1/p_i
    uint32_t mi[FAST ? LMAX * MLMAX : 1];              // limbs of M_i
    uint32_t h[FAST ? MLMAX : 1];                      // limbs of H
    int L, m_limbs;
};

template <int LMAX, bool FAST, int PB>
__device__ __forceinline__ void garner(const CrtConst<LMAX, FAST, PB>& q, const uint32_t (&r)[LMAX],
                                       uint32_t (&x)[CrtConst<LMAX, FAST, PB>::MLMAX], uint32_t& ext) {
    constexpr int MLMAX = CrtConst<LMAX, FAST, PB>::MLMAX;
    const int L = q.L;
    uint32_t t[LMAX];  // running sum_(k<i) v_k W_k mod p_i, kept in [0, 2 p_i)
    uint32_t v[LMAX];  // mixed-radix digits
#pragma unroll
    for (int i = 0; i < LMAX; i++) t[i] = 0;
#pragma unroll
    for (int k = 0; k < LMAX; k++) {
        if (k < L) {
            const uint32_t pk = q.p[k];
            uint32_t tk = t[k];
            if (tk >= pk) tk -= pk;
            const uint32_t d = r[k] >= tk ? r[k] - tk : r[k] + pk - tk;
            uint32_t vk = shoup_mul(d, q.ginv[k], q.ginvs[k], pk);
            if (vk >= pk) vk -= pk;
            v[k] = vk;
#pragma unroll
            for (int i = k + 1; i < LMAX; i++) {
                if (i < L) {
                    const int idx = i * (i - 1) / 2 + k;
                    const uint32_t pi = q.p[i];
                    const uint32_t sum = t[i] + shoup_mul(vk, q.gw[idx], q.gws[idx], pi);  // < 4 p_i
                    t[i] = sum >= 2 * pi ? sum - 2 * pi : sum;
                }
            }
        }
    }
    int cmp = 0;  // +1: x > (M-1)/2
#pragma unroll
    for (int k = LMAX - 1; k >= 0; k--) {
        if (k < L && cmp == 0) {
            const uint32_t hk = q.p[k] >> 1;
            if (v[k] != hk) cmp = v[k] > hk ? 1 : -1;
        }
    }
    // Horner; after digits k .. L-1 are in, x < 2^(26 (L-k)), so only the low limbs move
#pragma unroll
    for (int j = 0; j < MLMAX; j++) x[j] = 0;
#pragma unroll
    for (int k = LMAX - 1; k >= 0; k--) {
        if (k < L) {
            const uint32_t pk = k + 1 < L ? q.p[k] : 0;  // top digit: x = v_(L-1)
            uint32_t carry = v[k];
#pragma unroll
            for (int j = 0; j < MLMAX; j++) {
                if (j <= (26 * (LMAX - k) + 31) / 32) {
                    const uint64_t z = (uint64_t)x[j] * pk + carry;
                    x[j] = (uint32_t)z;
                    carry = (uint32_t)(z >> 32);
                }
            }
        }
    }
    ext = 0;
    if (cmp > 0) {  // x - M, negative
        uint32_t borrow = 0;
#pragma unroll
        for (int j = 0; j < MLMAX; j++) {
            const uint64_t d = (uint64_t)x[j] - q.m[j] - borrow;
            x[j] = (uint32_t)d;
            borrow = (uint32_t)(d >> 63);
        }
        ext = 0xFFFFFFFFu;
    }
}

// The same mixed-radix reconstruction with rolled loops (small code, local
// arrays): the fallback of the fast path, taken only by the rare entries whose
// quotient estimate is ambiguous.
template <int LMAX, bool FAST, int PB>
__device__ __noinline__ void garner_rolled(const CrtConst<LMAX, FAST, PB>& q, const uint32_t* r, uint32_t* x,
                                           uint32_t* ext_out) {
    constexpr int MLMAX = CrtConst<LMAX, FAST, PB>::MLMAX;
    const int L = q.L;
    uint32_t t[LMAX], v[LMAX];
#pragma unroll 1
    for (int i = 0; i < L; i++) t[i] = 0;
#pragma unroll 1
    for (int k = 0; k < L; k++) {
        const uint32_t pk = q.p[k];
        uint32_t tk = t[k];
        if (tk >= pk) tk -= pk;
        const uint32_t d = r[k] >= tk ? r[k] - tk : r[k] + pk - tk;
        uint32_t vk = shoup_mul(d, q.ginv[k], q.ginvs[k], pk);
        if (vk >= pk) vk -= pk;
        v[k] = vk;
#pragma unroll 1
        for (int i = k + 1; i < L; i++) {
            const int idx = i * (i - 1) / 2 + k;
            const uint32_t pi = q.p[i];
            const uint32_t sum = t[i] + shoup_mul(vk, q.gw[idx], q.gws[idx], pi);
            t[i] = sum >= 2 * pi ? sum - 2 * pi : sum;
        }
    }
    int cmp = 0;
#pragma unroll 1
    for (int k = L - 1; k >= 0 && cmp == 0; k--) {
        const uint32_t hk = q.p[k] >> 1;
        if (v[k] != hk) cmp = v[k] > hk ? 1 : -1;
    }
#pragma unroll 1
    for (int j = 0; j < MLMAX; j++) x[j] = 0;
#pragma unroll 1
    for (int k = L - 1; k >= 0; k--) {
        const uint32_t pk = k + 1 < L ? q.p[k] : 0;
        uint32_t carry = v[k];
#pragma unroll 1
        for (int j = 0; j < MLMAX; j++) {
            const uint64_t z = (uint64_t)x[j] * pk + carry;
            x[j] = (uint32_t)z;
            carry = (uint32_t)(z >> 32);
        }
    }
    uint32_t ext = 0;
    if (cmp > 0) {
        uint32_t borrow = 0;
#pragma unroll 1
        for (int j = 0; j < MLMAX; j++) {
            const uint64_t d = (uint64_t)x[j] - q.m[j] - borrow;
            x[j] = (uint32_t)d;
            borrow = (uint32_t)(d >> 63);
        }
        ext = 0xFFFFFFFFu;
    }
    *ext_out = ext;
}

// Fast path.  Returns false (x untouched) when alpha is not certain.
template <int LMAX, int PB, bool CG = false>
__device__ __forceinline__ bool lagrange(const CrtConst<LMAX, true, PB>& q, const int32_t* __restrict__ R,
                                         int64_t count, int64_t e, uint32_t (&x)[CrtConst<LMAX, true, PB>::MLMAX],
                                         uint32_t& ext) {
    constexpr int MLMAX = CrtConst<LMAX, true, PB>::MLMAX;
    const int L = q.L;
    uint64_t col[MLMAX];
#pragma unroll
    for (int j = 0; j < MLMAX; j++) col[j] = 0;
    float f = 0.f;
    // unrolled over the primes: every constant is a compile-time offset into
    // the parameter bank (no load instructions); the residues are loaded in
    // groups of eight ahead of use
    uint32_t rv[LMAX];
#pragma unroll
    for (int i = 0; i < LMAX; i++) rv[i] = i < L ? (uint32_t)load_res<CG>(R + (size_t)i * count + e) : 0u;
#pragma unroll
    for (int i = 0; i < LMAX; i++) {
        if (i < L) {
            const uint32_t pi = q.p[i];
            uint32_t a = rv[i] + q.hmod[i];
            if (a >= pi) a -= pi;
            uint32_t z = shoup_mul(a, q.c[i], q.cs[i], pi);
            if (z >= pi) z -= pi;
            f = fmaf((float)z, q.invp[i], f);
#pragma unroll
            for (int j = 0; j < MLMAX; j++) col[j] += (uint64_t)z * q.mi[i * MLMAX + j];
        }
    }
    const float fl = floorf(f);
    const float frac = f - fl;
    if (frac < 0x1p-12f || frac > 1.f - 0x1p-12f) return false;
    const uint32_t alpha = (uint32_t)fl;
    // y = sum_i xi_i M_i - alpha M limb by limb, then x = y - H
    uint64_t carry = 0;
    uint32_t borrow = 0, borrow2 = 0;
#pragma unroll
    for (int j = 0; j < MLMAX; j++) {
        const uint64_t s = col[j] + carry;
        carry = s >> 32;
        const uint64_t am = (uint64_t)alpha * q.m[j] + borrow;  // alpha M, limb j, plus borrow in
        const uint64_t d = (uint64_t)(uint32_t)s - (uint32_t)am;
        borrow = (uint32_t)(am >> 32) + (uint32_t)(d >> 63);
        const uint64_t d2 = (uint64_t)(uint32_t)d - q.h[j] - borrow2;
        borrow2 = (uint32_t)(d2 >> 63);
        x[j] = (uint32_t)d2;
    }
    ext = borrow2 ? 0xFFFFFFFFu : 0u;
    return true;
}

// Entry e of a [rows x cols] output whose residues are R[k * count + e].
template <int LMAX, bool FAST, int PB, bool CG = false>
__device__ __forceinline__ void crt_entry(const CrtConst<LMAX, FAST, PB>& q, const int32_t* __restrict__ R, int64_t count,
                                          int64_t cols, int64_t e, uint64_t* __restrict__ X, int64_t ld, int W) {
    constexpr int MLMAX = CrtConst<LMAX, FAST, PB>::MLMAX;
    const int L = q.L;
    uint32_t x[MLMAX];
    uint32_t ext;
    if constexpr (FAST) {
        if (!lagrange<LMAX, PB, CG>(q, R, count, e, x, ext)) {  // rare: exact mixed radix
            uint32_t rr[LMAX], xx[MLMAX];
#pragma unroll 1
            for (int k = 0; k < L; k++) rr[k] = (uint32_t)load_res<CG>(R + (size_t)k * count + e);
            garner_rolled<LMAX, FAST, PB>(q, rr, xx, &ext);
#pragma unroll
            for (int j = 0; j < MLMAX; j++) x[j] = xx[j];
        }
    } else {
        uint32_t r[LMAX];  // residues, loaded up front (coalesced across the warp)
#pragma unroll
        for (int k = 0; k < LMAX; k++) r[k] = k < L ? (uint32_t)load_res<CG>(R + (size_t)k * count + e) : 0;
        garner<LMAX, FAST, PB>(q, r, x, ext);
    }
    const int64_t row = e / cols, col = e % cols;
    uint64_t* out = X + (size_t)(row * ld + col) * W;
#pragma unroll
    for (int j = 0; j < MLMAX; j += 2) {
        if (j / 2 < W) {
            const uint32_t hi = j + 1 < MLMAX ? x[j + 1] : ext;
            out[j / 2] = (uint64_t)x[j] | ((uint64_t)hi << 32);
        }
    }
    const uint64_t ext64 = ((uint64_t)ext << 32) | ext;
    for (int w = (MLMAX + 1) / 2; w < W; w++) out[w] = ext64;
}


// The constants of a basis in the layout of CrtConst (host).
template <int LMAX, bool FAST, int PB>
void crt_const(const CrtHost& h, CrtConst<LMAX, FAST, PB>& q) {
    using Q = CrtConst<LMAX, FAST, PB>;
    q = Q{};
    const int L = h.L;
    for (int i = 0; i < L; i++) {
        q.p[i] = h.p[i];
        q.ginv[i] = h.ginv[i];
        q.ginvs[i] = h.ginvs[i];
        for (int k = 0; k < i; k++) {
            q.gw[i * (i - 1) / 2 + k] = h.gw[(size_t)i * L + k];
            q.gws[i * (i - 1) / 2 + k] = h.gws[(size_t)i * L + k];
        }
    }
    for (int j = 0; j < h.m_limbs && j < Q::MLMAX; j++) q.m[j] = h.m[j];
    if constexpr (FAST) {
        for (int i = 0; i < L; i++) {
            q.hmod[i] = h.hmod[i];
            q.c[i] = h.c[i];
            q.cs[i] = h.cs[i];
            q.invp[i] = 1.0f / (float)h.p[i];
            for (int j = 0; j < h.m_limbs && j < Q::MLMAX; j++)
                q.mi[i * Q::MLMAX + j] = h.mi[(size_t)i * h.m_limbs + j];
        }
        for (int j = 0; j < h.m_limbs && j < Q::MLMAX; j++) q.h[j] = h.h[j];
    }
    q.L = L;
    q.m_limbs = h.m_limbs;
}

}  // namespace
}  // namespace smf

#endif  // SMF_CRT_DEV_H
