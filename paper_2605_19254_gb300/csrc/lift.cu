// p-adic (Dixon) lifting: the two elementwise steps between the products.
// With C = A^-1 mod p, each step computes X_i = C R_i mod p (a residue product)
// and A X_i (an exact product); these kernels widen X_i to the product's word
// layout and form R_(i+1) = (R_i - A X_i) / p, an exact division whose
// remainder is checked (a non-zero remainder means C is not A^-1 mod p).
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

}  // namespace

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
