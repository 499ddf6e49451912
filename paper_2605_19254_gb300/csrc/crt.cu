// crt_reconstruct: residues -> the signed integer (Section 3.1: the exact
// product is recovered from its per-prime residues by CRT), by Garner's
// mixed-radix method, one entry per thread.
//
// With weights W_k = p_0 ... p_(k-1), the unique x in [0, M) with
// x = r_i (mod p_i) is x = sum_k v_k W_k, where the mixed-radix digits are
//   v_i = (r_i - sum_(k<i) v_k W_k) * W_i^-1   (mod p_i),   0 <= v_i < p_i.
// The digits are produced column-wise: once v_k is known it is folded into
// the running sums t_i of every later prime, so the L(L-1)/2 modular products
// are independent of each other within a column.  Every product multiplies by
// a per-basis constant, so Shoup's precomputed quotient (one high multiply,
// one low multiply, no division) does the reduction.
//
// Sign: M is odd and (M-1)/2 = sum_k ((p_k - 1)/2) W_k, so x > (M-1)/2 iff the
// digit string (v_(L-1) ... v_0) exceeds ((p_(L-1)-1)/2 ... (p_0-1)/2)
// lexicographically; those entries are returned as x - M.
//
// x itself is rebuilt by Horner, x = (... (v_(L-1) p_(L-2) + v_(L-2)) ...) p_0 + v_0,
// over 32-bit limbs, and written as W two's complement words.
#include "smf_internal.h"

namespace smf {
namespace {

// t + v * w (mod p) up to a multiple of p: returns a value in [0, 2p).
__device__ __forceinline__ uint32_t shoup_mul(uint32_t v, uint32_t w, uint32_t ws, uint32_t p) {
    const uint32_t q = __umulhi(v, ws);
    return v * w - q * p;
}

// Per-basis constants, passed by value so that they live in the kernel's
// parameter (constant) bank; with the loops below fully unrolled every access
// is a compile-time offset.  gw/gws hold the strictly lower triangle
// (i, k), k < i, at index i(i-1)/2 + k.
template <int LMAX>
struct CrtConst {
    static constexpr int MLMAX = (LMAX * 26 + 31) / 32 + 1;
    uint32_t p[LMAX];
    uint32_t ginv[LMAX], ginvs[LMAX];
    uint32_t gw[LMAX * (LMAX - 1) / 2], gws[LMAX * (LMAX - 1) / 2];
    uint32_t m[MLMAX];
    int L, m_limbs;
};

template <int LMAX>
__global__ void __launch_bounds__(128)
crt_kernel(const __grid_constant__ CrtConst<LMAX> q, const int32_t* __restrict__ R, int64_t rows, int64_t cols,
           uint64_t* __restrict__ X, int64_t ld, int W) {
    constexpr int MLMAX = CrtConst<LMAX>::MLMAX;
    const int64_t count = rows * cols;
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= count) return;
    const int L = q.L;

    uint32_t r[LMAX];   // residues, loaded up front (coalesced across the warp)
#pragma unroll
    for (int k = 0; k < LMAX; k++) r[k] = k < L ? (uint32_t)__ldg(R + (size_t)k * count + e) : 0;

    uint32_t t[LMAX];   // running sum_(k<i) v_k W_k mod p_i, kept in [0, 2 p_i)
    uint32_t v[LMAX];   // mixed-radix digits
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
                    const uint32_t add = shoup_mul(vk, q.gw[idx], q.gws[idx], pi);
                    const uint32_t sum = t[i] + add;  // < 4 p_i
                    t[i] = sum >= 2 * pi ? sum - 2 * pi : sum;
                }
            }
        }
    }

    // sign test against the digits of (M-1)/2
    int cmp = 0;  // +1: x > (M-1)/2
#pragma unroll
    for (int k = LMAX - 1; k >= 0; k--) {
        if (k < L && cmp == 0) {
            const uint32_t hk = q.p[k] >> 1;
            if (v[k] != hk) cmp = v[k] > hk ? 1 : -1;
        }
    }

    // Horner over 32-bit limbs; after the digits k .. L-1 are in, x is below
    // p_k ... p_(L-1) < 2^(26 (L-k)), so only the low limbs can be non-zero.
    uint32_t x[MLMAX];
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
    uint32_t ext = 0;
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

template <int LMAX>
cudaError_t launch_crt_t(const CrtHost& h, const int32_t* R, int64_t rows, int64_t cols, uint64_t* X, int64_t ld,
                         int W, cudaStream_t s) {
    CrtConst<LMAX> q{};
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
    for (int j = 0; j < h.m_limbs && j < CrtConst<LMAX>::MLMAX; j++) q.m[j] = h.m[j];
    q.L = L;
    q.m_limbs = h.m_limbs;
    const int64_t count = rows * cols;
    const int threads = 128;
    crt_kernel<LMAX><<<(unsigned)((count + threads - 1) / threads), threads, 0, s>>>(q, R, rows, cols, X, ld, W);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_crt(const CrtHost& h, const int32_t* R, int64_t rows, int64_t cols, uint64_t* X, int64_t ld,
                       int W, cudaStream_t s) {
    if (rows == 0 || cols == 0) return cudaSuccess;
    if (h.L <= 8) return launch_crt_t<8>(h, R, rows, cols, X, ld, W, s);
    if (h.L <= 16) return launch_crt_t<16>(h, R, rows, cols, X, ld, W, s);
    if (h.L <= 24) return launch_crt_t<24>(h, R, rows, cols, X, ld, W, s);
    if (h.L <= 32) return launch_crt_t<32>(h, R, rows, cols, X, ld, W, s);
    if (h.L <= 48) return launch_crt_t<48>(h, R, rows, cols, X, ld, W, s);
    if (h.L <= 64) return launch_crt_t<64>(h, R, rows, cols, X, ld, W, s);
    return cudaErrorNotSupported;
}

}  // namespace smf
