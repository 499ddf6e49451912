// A^-1 mod p by Gauss-Jordan elimination over GF(p): the initialization of
// the p-adic lifting (Section 3 notes that it costs about as much as the
// lifting itself).
//
// The augmented n x 2n matrix [A mod p | I] is reduced column by column.
// Column k takes two launches:
//   gj_pivot: one block finds the first row r >= k whose entry in column k is
//             non-zero, swaps rows r and k, scales row k by that entry's
//             inverse (Fermat: a^(p-2)), and copies column k aside (f_i, with
//             f_k = 0);
//   gj_elim:  every row i != k subtracts f_i times row k, over the columns
//             j >= k (row k is zero left of column k).
// Afterwards the right half is A^-1 mod p.  A column without a pivot means
// p | det A: the pivot launch sets kStatusSingular and a device flag, and
// every later launch returns at once.
#include <algorithm>

#include "smf_internal.h"

namespace smf {
namespace {

constexpr int kPivotThreads = 1024;
constexpr int kElimThreads = 256;
constexpr int kMaxGridY = 65535;
constexpr int64_t kElimBlocksPerSM = 16;

// Barrett reduction of a product of two residues (p < 2^31): with
// mu = floor((2^64 - 1) / p) the estimate q falls short of the quotient by at
// most 2.
__device__ __forceinline__ uint32_t mulmod(uint32_t a, uint32_t b, uint32_t p, uint64_t mu) {
    const uint64_t x = (uint64_t)a * b;
    uint64_t r = x - __umul64hi(x, mu) * p;
    while (r >= p) r -= p;
    return (uint32_t)r;
}

__device__ uint32_t powmod(uint32_t a, uint32_t e, uint32_t p, uint64_t mu) {
    uint32_t r = 1 % p;
    while (e) {
        if (e & 1) r = mulmod(r, a, p, mu);
        a = mulmod(a, a, p, mu);
        e >>= 1;
    }
    return r;
}

__global__ void __launch_bounds__(kElimThreads) gj_init_kernel(const int32_t* __restrict__ res, int64_t n,
                                                               uint32_t* __restrict__ M) {
    const int64_t e = (int64_t)blockIdx.x * kElimThreads + threadIdx.x;
    if (e >= 2 * n * n) return;
    const int64_t i = e / (2 * n), j = e - i * 2 * n;
    M[e] = j < n ? (uint32_t)res[i * n + j] : (uint32_t)(j - n == i);
}

__global__ void __launch_bounds__(kPivotThreads) gj_pivot_kernel(uint32_t* __restrict__ M, int64_t n, int64_t k,
                                                                 uint32_t p, uint64_t mu, uint32_t* __restrict__ col,
                                                                 int* flag, int* status) {
    __shared__ unsigned long long s_piv;
    __shared__ uint32_t s_inv;
    pdl_wait();
    pdl_trigger();
    if (*flag) return;  // an earlier column had no pivot
    const int64_t ld = 2 * n;
    if (threadIdx.x == 0) s_piv = (unsigned long long)n;
    __syncthreads();
    for (int64_t r = k + threadIdx.x; r < n; r += kPivotThreads) {
        if (M[r * ld + k] != 0) {
            atomicMin(&s_piv, (unsigned long long)r);
            break;
        }
    }
    __syncthreads();
    const int64_t r = (int64_t)s_piv;
    if (r == n) {
        if (threadIdx.x == 0) {
            *flag = 1;
            atomicOr(status, kStatusSingular);
        }
        return;
    }
    if (r != k) {
        for (int64_t j = threadIdx.x; j < ld; j += kPivotThreads) {
            const uint32_t t = M[r * ld + j];
            M[r * ld + j] = M[k * ld + j];
            M[k * ld + j] = t;
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) s_inv = powmod(M[k * ld + k], p - 2, p, mu);
    __syncthreads();
    const uint32_t inv = s_inv;
    for (int64_t j = k + threadIdx.x; j < ld; j += kPivotThreads) M[k * ld + j] = mulmod(M[k * ld + j], inv, p, mu);
    for (int64_t i = threadIdx.x; i < n; i += kPivotThreads) col[i] = i == k ? 0u : M[i * ld + k];
}

__global__ void __launch_bounds__(kElimThreads) gj_elim_kernel(uint32_t* __restrict__ M, int64_t n, int64_t k,
                                                               uint32_t p, uint64_t mu,
                                                               const uint32_t* __restrict__ col, const int* flag) {
    pdl_wait();
    pdl_trigger();
    if (*flag) return;
    const int64_t ld = 2 * n;
    const int64_t j = k + (int64_t)blockIdx.x * kElimThreads + threadIdx.x;
    if (j >= ld) return;
    const uint32_t rk = M[k * ld + j];
    const int64_t gy = gridDim.y;
    int64_t i = blockIdx.y;
    // four rows at a time: their loads are issued before any store
    for (; i + 3 * gy < n; i += 4 * gy) {
        uint32_t f[4], v[4];
#pragma unroll
        for (int u = 0; u < 4; u++) {
            f[u] = col[i + u * gy];  // 0 for row k
            v[u] = M[(i + u * gy) * ld + j];
        }
#pragma unroll
        for (int u = 0; u < 4; u++) {
            if (f[u] == 0) continue;
            const uint32_t t = mulmod(f[u], rk, p, mu);
            M[(i + u * gy) * ld + j] = v[u] >= t ? v[u] - t : v[u] + p - t;
        }
    }
    for (; i < n; i += gy) {
        const uint32_t f = col[i];
        if (f == 0) continue;
        const uint32_t t = mulmod(f, rk, p, mu);
        uint32_t* e = M + i * ld + j;
        const uint32_t v = *e;
        *e = v >= t ? v - t : v + p - t;
    }
}

// ---- blocked form: panels of bw columns
//
// For panel columns [c0, c1) the scratch T = [P | S] (n x 2bw) holds a copy of
// the panel P and a block S that starts at zero.  Column k of the panel is
// reduced as above, restricted to T; the row swap is applied to M's columns
// [c1, 2n) as well, and S's entry (k, k - c0) gains 1 right after the swap,
// before the scaling.  By linearity S then ends as E S0, where E is the
// panel's elimination with all swaps done first and S0 the unit rows at the
// pivot positions c0 .. c1-1.  With Mp = M[c0:c1, c1:2n] after the swaps,
// the whole elimination of the remaining columns is
//   M[i, c1:] = (S Mp)_i                  for the pivot rows c0 <= i < c1,
//   M[i, c1:] = M[i, c1:] + (S Mp)_i     for every other row,
// one residue product with one prime (K = bw) and one elementwise pass.

__global__ void __launch_bounds__(kPivotThreads)
    panel_pivot_kernel(uint32_t* __restrict__ T, int64_t n, int bw, int64_t k, int j, uint32_t* __restrict__ M,
                       int64_t ldM, int64_t lo, int64_t hi, uint32_t p, uint64_t mu, uint32_t* __restrict__ col,
                       int* flag, int* status) {
    __shared__ unsigned long long s_piv;
    __shared__ uint32_t s_inv;
    pdl_wait();
    pdl_trigger();
    if (*flag) return;
    const int64_t ldT = 2 * (int64_t)bw;
    if (threadIdx.x == 0) s_piv = (unsigned long long)n;
    __syncthreads();
    for (int64_t r = k + threadIdx.x; r < n; r += kPivotThreads) {
        if (T[r * ldT + j] != 0) {
            atomicMin(&s_piv, (unsigned long long)r);
            break;
        }
    }
    __syncthreads();
    const int64_t r = (int64_t)s_piv;
    if (r == n) {
        if (threadIdx.x == 0) {
            *flag = 1;
            atomicOr(status, kStatusSingular);
        }
        return;
    }
    if (r != k) {
        for (int64_t c = threadIdx.x; c < ldT; c += kPivotThreads) {
            const uint32_t t = T[r * ldT + c];
            T[r * ldT + c] = T[k * ldT + c];
            T[k * ldT + c] = t;
        }
        for (int64_t c = lo + threadIdx.x; c < hi; c += kPivotThreads) {
            const uint32_t t = M[r * ldM + c];
            M[r * ldM + c] = M[k * ldM + c];
            M[k * ldM + c] = t;
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t* a = T + k * ldT + bw + j;  // S gains the unit of pivot row k
        *a = *a + 1 == p ? 0u : *a + 1;
        s_inv = powmod(T[k * ldT + j], p - 2, p, mu);
    }
    __syncthreads();
    const uint32_t inv = s_inv;
    for (int64_t c = j + threadIdx.x; c < ldT; c += kPivotThreads) T[k * ldT + c] = mulmod(T[k * ldT + c], inv, p, mu);
    for (int64_t i = threadIdx.x; i < n; i += kPivotThreads) col[i] = i == k ? 0u : T[i * ldT + j];
}

__global__ void __launch_bounds__(kElimThreads)
    panel_elim_kernel(uint32_t* __restrict__ T, int64_t n, int bw, int64_t k, int j, uint32_t p, uint64_t mu,
                      const uint32_t* __restrict__ col, const int* flag) {
    pdl_wait();
    pdl_trigger();
    if (*flag) return;
    const int64_t ldT = 2 * (int64_t)bw;
    const int64_t c = j + (int64_t)blockIdx.x * kElimThreads + threadIdx.x;
    if (c >= ldT) return;
    const uint32_t rk = T[k * ldT + c];
    if (rk == 0) return;
    for (int64_t i = blockIdx.y; i < n; i += gridDim.y) {
        const uint32_t f = col[i];
        if (f == 0) continue;
        const uint32_t t = mulmod(f, rk, p, mu);
        uint32_t* e = T + i * ldT + c;
        const uint32_t v = *e;
        *e = v >= t ? v - t : v + p - t;
    }
}

// M[i, c1 + jj] = C[i][jj] on the pivot rows, M + C mod p on the others
__global__ void __launch_bounds__(kElimThreads)
    panel_update_kernel(uint32_t* __restrict__ M, int64_t ldM, int64_t n, int64_t c0, int64_t c1, int64_t R,
                        const int32_t* __restrict__ C, uint32_t p) {
    const int64_t e = (int64_t)blockIdx.x * kElimThreads + threadIdx.x;
    if (e >= n * R) return;
    const int64_t i = e / R, jj = e - i * R;
    const uint32_t v = (uint32_t)C[e];
    uint32_t* m = M + i * ldM + c1 + jj;
    if (i >= c0 && i < c1) {
        *m = v;
    } else {
        const uint32_t w = *m + v;  // both below p < 2^31
        *m = w >= p ? w - p : w;
    }
}

}  // namespace

cudaError_t launch_panel_factor(uint32_t* T, int64_t n, int bw, int64_t c0, uint32_t* M, int64_t ldM, int64_t lo,
                                int64_t hi, uint32_t p, uint32_t* col, int* flag, int* status, int num_sms,
                                cudaStream_t s) {
    const uint64_t mu = UINT64_MAX / p;
    const int64_t blocks = kElimBlocksPerSM * (num_sms > 0 ? num_sms : 148);
    for (int j = 0; j < bw; j++) {
        const int64_t k = c0 + j;
        cudaError_t e = launch_pdl(panel_pivot_kernel, dim3(1), dim3(kPivotThreads), 0, s, T, n, bw, k, j, M, ldM, lo,
                                   hi, p, mu, col, flag, status);
        if (e != cudaSuccess) return e;
        const int64_t gx = (2 * (int64_t)bw - j + kElimThreads - 1) / kElimThreads;
        const int64_t gy = std::min<int64_t>(std::min<int64_t>(n, kMaxGridY), std::max<int64_t>(1, blocks / gx));
        e = launch_pdl(panel_elim_kernel, dim3((unsigned)gx, (unsigned)gy), dim3(kElimThreads), 0, s, T, n, bw, k, j, p,
                       mu, (const uint32_t*)col, (const int*)flag);
        if (e != cudaSuccess) return e;
    }
    return cudaGetLastError();
}

cudaError_t launch_panel_update(uint32_t* M, int64_t ldM, int64_t n, int64_t c0, int64_t c1, int64_t R,
                                const int32_t* C, uint32_t p, cudaStream_t s) {
    if (n * R == 0) return cudaSuccess;
    panel_update_kernel<<<(unsigned)((n * R + kElimThreads - 1) / kElimThreads), kElimThreads, 0, s>>>(M, ldM, n, c0,
                                                                                                        c1, R, C, p);
    return cudaGetLastError();
}

cudaError_t launch_gj_init(const int32_t* res, int64_t n, uint32_t* M, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    gj_init_kernel<<<(unsigned)((2 * n * n + kElimThreads - 1) / kElimThreads), kElimThreads, 0, s>>>(res, n, M);
    return cudaGetLastError();
}

cudaError_t launch_inverse_mod_p(const int32_t* res, int64_t n, uint32_t p, uint32_t* M, uint32_t* col, int* flag,
                                 int32_t* C, int* status, int num_sms, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    const uint64_t mu = UINT64_MAX / p;
    const int64_t blocks = kElimBlocksPerSM * (num_sms > 0 ? num_sms : 148);
    cudaError_t e = cudaMemsetAsync(flag, 0, sizeof(int), s);
    if (e != cudaSuccess) return e;
    gj_init_kernel<<<(unsigned)((2 * n * n + kElimThreads - 1) / kElimThreads), kElimThreads, 0, s>>>(res, n, M);
    for (int64_t k = 0; k < n; k++) {
        if ((e = launch_pdl(gj_pivot_kernel, dim3(1), dim3(kPivotThreads), 0, s, M, n, k, p, mu, col, flag, status)) !=
            cudaSuccess)
            return e;
        // about 16 blocks per SM in all, each over a strided set of rows
        const int64_t gx = (2 * n - k + kElimThreads - 1) / kElimThreads;
        const int64_t gy = std::min<int64_t>(std::min<int64_t>(n, kMaxGridY), std::max<int64_t>(1, blocks / gx));
        const dim3 grid((unsigned)gx, (unsigned)gy);
        if ((e = launch_pdl(gj_elim_kernel, grid, dim3(kElimThreads), 0, s, M, n, k, p, mu, (const uint32_t*)col,
                            (const int*)flag)) != cudaSuccess)
            return e;
    }
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    return cudaMemcpy2DAsync(C, sizeof(int32_t) * n, M + n, sizeof(uint32_t) * 2 * n, sizeof(int32_t) * n, n,
                             cudaMemcpyDeviceToDevice, s);
}

}  // namespace smf
