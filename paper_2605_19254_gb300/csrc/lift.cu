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

// The step kernels work on 32 x 32 tiles of the n x m matrices: entries are
// read and written along c (the matrices are row-major in k), and the digit
// planes [t][L][m][ldd], contiguous in k, are written along k after a
// transpose through shared memory.  Block: 32 x 32 threads, one entry each.
constexpr int kTile = 32;
constexpr int kTileRows = 32;

// Sum of `split` canonical partials (at most 16 below 2^26: the sum stays
// below 2^32) at stride `stride`, reduced mod q once.  The loads are
// independent of one another and unrolled, so they are all in flight at once.
__device__ __forceinline__ uint32_t sum_parts(const int32_t* __restrict__ part, int split, int64_t stride,
                                              uint32_t q) {
    uint32_t a0 = 0, a1 = 0, a2 = 0, a3 = 0;
    int sp = 0;
    for (; sp + 4 <= split; sp += 4) {
        a0 += (uint32_t)part[(sp + 0) * stride];
        a1 += (uint32_t)part[(sp + 1) * stride];
        a2 += (uint32_t)part[(sp + 2) * stride];
        a3 += (uint32_t)part[(sp + 3) * stride];
    }
    for (; sp < split; sp++) a0 += (uint32_t)part[sp * stride];
    return (a0 + a1 + a2 + a3) % q;
}

template <int LQ>
__global__ void __launch_bounds__(kTile * kTileRows)
    lift_x_kernel(const int32_t* __restrict__ part, int split, int64_t n, int64_t m, uint32_t p,
                  int32_t* __restrict__ X, LiftBasis q, __nv_bfloat16* __restrict__ xdig, int64_t ldd, int t) {
    __shared__ uint32_t tile[kTile][kTile + 1];
    pdl_wait();
    pdl_trigger();
    const int64_t nm = n * m;
    const int64_t k0 = (int64_t)blockIdx.x * kTile, c0 = (int64_t)blockIdx.y * kTile;
    const int tx = threadIdx.x, ty = threadIdx.y;
    // X_i = the K-split partials summed mod p, along c
    const int64_t c = c0 + tx;
#pragma unroll
    for (int r = ty; r < kTile; r += kTileRows) {
        const int64_t k = k0 + r;
        if (k < n && c < m) {
            const int64_t at = k * m + c;
            const uint32_t x = sum_parts(part + at, split, nm, p);
            X[at] = (int32_t)x;
            tile[r][tx] = x;
        }
    }
    __syncthreads();
    // its centred residues modulo q_j, as digit planes, along k
    const int64_t k = k0 + tx;
    if (k >= n) return;
    const int64_t plane = (int64_t)LQ * m * ldd;
#pragma unroll
    for (int r = ty; r < kTile; r += kTileRows) {
        const int64_t cc = c0 + r;
        if (cc >= m) break;
        const uint32_t x = tile[tx][r];
#pragma unroll
        for (int j = 0; j < LQ; j++) {
            const uint32_t qj = q.q[j];
            int32_t v = (int32_t)(x % qj);
            if (v > (int32_t)(qj >> 1)) v -= (int32_t)qj;
            put_digits(xdig + (j * m + cc) * ldd + k, plane, v, t);
        }
    }
}

template <int LQ>
__global__ void __launch_bounds__(kTile * kTileRows)
    lift_step_kernel(const int32_t* __restrict__ part, int split, int64_t n, int64_t m, LiftBasis q,
                     int64_t* __restrict__ R, int64_t ldR, int64_t p, __nv_bfloat16* __restrict__ rdig, int64_t ldd,
                     int t, int* status) {
    __shared__ int32_t tile[kTile][kTile + 1];
    pdl_wait();
    pdl_trigger();
    const int64_t nm = n * m;
    const int64_t k0 = (int64_t)blockIdx.x * kTile, c0 = (int64_t)blockIdx.y * kTile;
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int64_t c = c0 + tx;
#pragma unroll
    for (int rr = ty; rr < kTile; rr += kTileRows) {
        const int64_t k = k0 + rr;
        if (k >= n || c >= m) continue;
        const int64_t at = k * m + c;
        // mixed-radix digits v_j of A X_i mod Q: with s_j = (v_0 + v_1 q_0 + ...
        // + v_(j-1) q_0...q_(j-2)) mod q_j, v_j = (r_j - s_j) (q_0...q_(j-1))^-1 mod q_j
        uint32_t rj[LQ], v[LQ];
#pragma unroll
        for (int j = 0; j < LQ; j++) rj[j] = sum_parts(part + j * nm + at, split, LQ * nm, q.q[j]);
#pragma unroll
        for (int j = 0; j < LQ; j++) {
            const uint32_t qj = q.q[j], r = rj[j];
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
        int64_t res = quo % p;
        if (res < 0) res += p;
        if (res > p / 2) res -= p;
        tile[rr][tx] = (int32_t)res;
    }
    if (!rdig) return;  // uniform over the block
    __syncthreads();
    const int64_t k = k0 + tx;
    if (k >= n) return;
#pragma unroll
    for (int rr = ty; rr < kTile; rr += kTileRows) {
        const int64_t cc = c0 + rr;
        if (cc >= m) break;
        put_digits(rdig + cc * ldd + k, m * ldd, tile[tx][rr], t);
    }
}

}  // namespace

cudaError_t launch_lift_x(const int32_t* part, int split, int64_t n, int64_t m, uint32_t p, int32_t* X,
                          const LiftBasis& q, void* xdig, int64_t ldd, int t, cudaStream_t s) {
    if (n * m == 0) return cudaSuccess;
    const dim3 grid((unsigned)((n + kTile - 1) / kTile), (unsigned)((m + kTile - 1) / kTile));
    const dim3 block(kTile, kTileRows);
    __nv_bfloat16* xd = (__nv_bfloat16*)xdig;
    switch (q.L) {
    case 1: return launch_pdl(lift_x_kernel<1>, grid, block, 0, s, part, split, n, m, p, X, q, xd, ldd, t);
    case 2: return launch_pdl(lift_x_kernel<2>, grid, block, 0, s, part, split, n, m, p, X, q, xd, ldd, t);
    case 3: return launch_pdl(lift_x_kernel<3>, grid, block, 0, s, part, split, n, m, p, X, q, xd, ldd, t);
    case 4: return launch_pdl(lift_x_kernel<4>, grid, block, 0, s, part, split, n, m, p, X, q, xd, ldd, t);
    default: return cudaErrorNotSupported;
    }
    return cudaGetLastError();
}

cudaError_t launch_lift_step(const int32_t* part, int split, int64_t n, int64_t m, const LiftBasis& q, int64_t* R,
                             int64_t ldR, uint32_t p, void* rdig, int64_t ldd, int t, int* status, cudaStream_t s) {
    if (n * m == 0) return cudaSuccess;
    const dim3 grid((unsigned)((n + kTile - 1) / kTile), (unsigned)((m + kTile - 1) / kTile));
    const dim3 block(kTile, kTileRows);
    __nv_bfloat16* rd = (__nv_bfloat16*)rdig;
    const int64_t pp = (int64_t)p;
    switch (q.L) {
    case 1: return launch_pdl(lift_step_kernel<1>, grid, block, 0, s, part, split, n, m, q, R, ldR, pp, rd, ldd, t,
                               status);
    case 2: return launch_pdl(lift_step_kernel<2>, grid, block, 0, s, part, split, n, m, q, R, ldR, pp, rd, ldd, t,
                               status);
    case 3: return launch_pdl(lift_step_kernel<3>, grid, block, 0, s, part, split, n, m, q, R, ldR, pp, rd, ldd, t,
                               status);
    case 4: return launch_pdl(lift_step_kernel<4>, grid, block, 0, s, part, split, n, m, q, R, ldR, pp, rd, ldd, t,
                               status);
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
