// p-adic (Dixon) lifting: the elementwise steps between the products.
// With C = A^-1 mod p, each step computes X_i = C R_i mod p (a residue product)
// and A X_i (an exact product); these kernels widen X_i to the product's word
// layout and form R_(i+1) = (R_i - A X_i) / p, an exact division whose
// remainder is checked (a non-zero remainder means C is not A^-1 mod p).
//
// The limb form runs each step as two residue products and two kernels that
// stand between them and take the products' K-split partials as they are:
//   lift_x:    X_i = sum of the partials of C R_i mod p, stored, and X_i's
//              centred residues modulo the product basis q_0 .. q_(L-1), split
//              into the digit planes of A X_i's B operand;
//   lift_step: A X_i mod q_j summed over its partials, A X_i itself by Garner's
//              mixed radix (|A X_i| < Q/2, Q = q_0 ... q_(L-1) < 2^128),
//              R_(i+1) = (R_i - A X_i) / p in place, and the digit planes of
//              R_(i+1) mod p for the next step's C R_(i+1).
// The C and A digit planes are made once per call.
#include <cuda_bf16.h>

#include "smf_internal.h"

namespace smf {
namespace {

constexpr int kThreads = 256;

__global__ void __launch_bounds__(kThreads) widen_kernel(const int32_t* __restrict__ x, int64_t count,
                                                         int64_t* __restrict__ out) {
    const int64_t i = (int64_t)blockIdx.x * kThreads + threadIdx.x;
    if (i < count) out[i] = (int64_t)x[i];
}

__global__ void __launch_bounds__(kThreads) lift_update_kernel(int64_t* __restrict__ R, int64_t ldR,
                                                               const int64_t* __restrict__ AX, int64_t rows,
                                                               int64_t cols, int64_t p, int* status) {
    const int64_t e = (int64_t)blockIdx.x * kThreads + threadIdx.x;
    if (e >= rows * cols) return;
    const int64_t r = e / cols, c = e - r * cols;
    int64_t* rp = R + r * ldR + c;
    const int64_t t = *rp - AX[e];
    const int64_t q = t / p;
    if (q * p != t) atomicOr(status, kStatusInexact);
    *rp = q;
}

// Balanced base-2^8 digits of a centred value: t-1 digits in [-128, 127], then
// the remaining quotient (|v| <= 2^23 keeps it within +-128 for t = 3).  Digit u
// goes to d[u * plane].
__device__ __forceinline__ void put_digits(__nv_bfloat16* d, int64_t plane, int32_t v, int t) {
    for (int u = 0; u < t - 1; u++) {
        const int32_t lo = ((v + 128) & 255) - 128;
        d[u * plane] = __int2bfloat16_rn(lo);
        v = (v - lo) >> 8;  // exact: v - lo is a multiple of 256
    }
    d[(t - 1) * plane] = __int2bfloat16_rn(v);
}

// One thread per entry (k, c) of the n x m matrices, k fastest: the digit
// planes [t][L][m][ldd] are contiguous in k.
template <int LQ>
__global__ void __launch_bounds__(kThreads) lift_x_kernel(const int32_t* __restrict__ part, int split, int64_t n,
                                                          int64_t m, uint32_t p, int32_t* __restrict__ X, LiftBasis q,
                                                          __nv_bfloat16* __restrict__ xdig, int64_t ldd, int t) {
    const int64_t nm = n * m;
    const int64_t e = (int64_t)blockIdx.x * kThreads + threadIdx.x;
    if (e >= nm) return;
    const int64_t c = e / n, k = e - c * n, at = k * m + c;
    uint32_t x = 0;
    for (int sp = 0; sp < split; sp++) {
        x += (uint32_t)part[sp * nm + at];
        if (x >= p) x -= p;
    }
    X[at] = (int32_t)x;
    const int64_t plane = (int64_t)LQ * m * ldd;
#pragma unroll
    for (int j = 0; j < LQ; j++) {
        const uint32_t qj = q.q[j];
        int32_t r = (int32_t)(x % qj);
        if (r > (int32_t)(qj >> 1)) r -= (int32_t)qj;
        put_digits(xdig + (j * m + c) * ldd + k, plane, r, t);
    }
}

template <int LQ>
__global__ void __launch_bounds__(kThreads)
    lift_step_kernel(const int32_t* __restrict__ part, int split, int64_t n, int64_t m, LiftBasis q,
                     int64_t* __restrict__ R, int64_t ldR, int64_t p, __nv_bfloat16* __restrict__ rdig, int64_t ldd,
                     int t, int* status) {
    const int64_t nm = n * m;
    const int64_t e = (int64_t)blockIdx.x * kThreads + threadIdx.x;
    if (e >= nm) return;
    const int64_t c = e / n, k = e - c * n, at = k * m + c;
    // mixed-radix digits v_j of A X_i mod Q: with s_j = (v_0 + v_1 q_0 + ...
    // + v_(j-1) q_0...q_(j-2)) mod q_j, v_j = (r_j - s_j) (q_0...q_(j-1))^-1 mod q_j
    uint32_t v[LQ];
#pragma unroll
    for (int j = 0; j < LQ; j++) {
        const uint32_t qj = q.q[j];
        uint32_t r = 0;
        for (int sp = 0; sp < split; sp++) {
            r += (uint32_t)part[((int64_t)sp * LQ + j) * nm + at];
            if (r >= qj) r -= qj;
        }
        uint64_t sj = 0;
#pragma unroll
        for (int i = j - 1; i >= 0; i--) sj = (sj * q.q[i] + v[i]) % qj;
        v[j] = (uint32_t)((uint64_t)((r + qj - (uint32_t)sj) % qj) * q.inv[j] % qj);
    }
    unsigned __int128 x = 0, w = 1;
#pragma unroll
    for (int j = 0; j < LQ; j++) {
        x += (unsigned __int128)v[j] * w;
        w *= q.q[j];
    }
    // centred: Q is odd, values above (Q-1)/2 stand for x - Q
    const int64_t ax = x > (w >> 1) ? -(int64_t)(w - x) : (int64_t)x;
    int64_t* rp = R + k * ldR + c;
    const int64_t d = *rp - ax;
    const int64_t quo = d / p;
    if (quo * p != d) atomicOr(status, kStatusInexact);
    *rp = quo;
    if (rdig) {
        int64_t r = quo % p;
        if (r < 0) r += p;
        if (r > p / 2) r -= p;
        put_digits(rdig + c * ldd + k, m * ldd, (int32_t)r, t);
    }
}

}  // namespace

cudaError_t launch_lift_x(const int32_t* part, int split, int64_t n, int64_t m, uint32_t p, int32_t* X,
                          const LiftBasis& q, void* xdig, int64_t ldd, int t, cudaStream_t s) {
    const int64_t count = n * m;
    if (count == 0) return cudaSuccess;
    const unsigned grid = (unsigned)((count + kThreads - 1) / kThreads);
    __nv_bfloat16* xd = (__nv_bfloat16*)xdig;
    switch (q.L) {
    case 1: lift_x_kernel<1><<<grid, kThreads, 0, s>>>(part, split, n, m, p, X, q, xd, ldd, t); break;
    case 2: lift_x_kernel<2><<<grid, kThreads, 0, s>>>(part, split, n, m, p, X, q, xd, ldd, t); break;
    case 3: lift_x_kernel<3><<<grid, kThreads, 0, s>>>(part, split, n, m, p, X, q, xd, ldd, t); break;
    case 4: lift_x_kernel<4><<<grid, kThreads, 0, s>>>(part, split, n, m, p, X, q, xd, ldd, t); break;
    default: return cudaErrorNotSupported;
    }
    return cudaGetLastError();
}

cudaError_t launch_lift_step(const int32_t* part, int split, int64_t n, int64_t m, const LiftBasis& q, int64_t* R,
                             int64_t ldR, uint32_t p, void* rdig, int64_t ldd, int t, int* status, cudaStream_t s) {
    const int64_t count = n * m;
    if (count == 0) return cudaSuccess;
    const unsigned grid = (unsigned)((count + kThreads - 1) / kThreads);
    __nv_bfloat16* rd = (__nv_bfloat16*)rdig;
    const int64_t pp = (int64_t)p;
    switch (q.L) {
    case 1: lift_step_kernel<1><<<grid, kThreads, 0, s>>>(part, split, n, m, q, R, ldR, pp, rd, ldd, t, status); break;
    case 2: lift_step_kernel<2><<<grid, kThreads, 0, s>>>(part, split, n, m, q, R, ldR, pp, rd, ldd, t, status); break;
    case 3: lift_step_kernel<3><<<grid, kThreads, 0, s>>>(part, split, n, m, q, R, ldR, pp, rd, ldd, t, status); break;
    case 4: lift_step_kernel<4><<<grid, kThreads, 0, s>>>(part, split, n, m, q, R, ldR, pp, rd, ldd, t, status); break;
    default: return cudaErrorNotSupported;
    }
    return cudaGetLastError();
}

cudaError_t launch_widen(const int32_t* x, int64_t count, int64_t* out, cudaStream_t s) {
    if (count == 0) return cudaSuccess;
    widen_kernel<<<(unsigned)((count + kThreads - 1) / kThreads), kThreads, 0, s>>>(x, count, out);
    return cudaGetLastError();
}

cudaError_t launch_lift_update(int64_t* R, int64_t ldR, const int64_t* AX, int64_t rows, int64_t cols, uint32_t p,
                               int* status, cudaStream_t s) {
    const int64_t count = rows * cols;
    if (count == 0) return cudaSuccess;
    lift_update_kernel<<<(unsigned)((count + kThreads - 1) / kThreads), kThreads, 0, s>>>(R, ldR, AX, rows, cols,
                                                                                          (int64_t)p, status);
    return cudaGetLastError();
}

}  // namespace smf
