// crt_reconstruct: residues -> the signed integer (Section 3.1: the exact
// product is recovered from its per-prime residues by CRT), one entry per
// thread, result in (-M/2, M/2] written as W two's complement words; and the
// conversion between RNS bases.  The per-entry reconstruction (Lagrange form
// with an fp32 quotient, exact mixed-radix fallback) is in crt_dev.h.
#include "crt_dev.h"

namespace smf {
namespace {

template <int LMAX, bool FAST, int PB>
__global__ void __launch_bounds__(128)
crt_kernel(const __grid_constant__ CrtConst<LMAX, FAST, PB> q, const int32_t* __restrict__ R, int64_t rows,
           int64_t cols, uint64_t* __restrict__ X, int64_t ld, int W) {
    const int64_t count = rows * cols;
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= count) return;
    crt_entry<LMAX, FAST, PB>(q, R, count, cols, e, X, ld, W);
}

// Several outputs of one basis in one launch: block u takes unit u, the 128
// consecutive entries u - base_i of item i (found by bisection).  One unit per
// block keeps the register count of crt_kernel; the search is a few loads from
// L1 against a block's tens of thousands of modular products.
template <int LMAX, bool FAST, int PB>
__global__ void __launch_bounds__(128)
crt_grouped_kernel(const __grid_constant__ CrtConst<LMAX, FAST, PB> q, const CrtItem* __restrict__ items, int n) {
    const CrtItem* it = find_item(items, n, (int64_t)blockIdx.x);
    const int64_t count = it->rows * it->cols;
    const int64_t e = ((int64_t)blockIdx.x - it->base) * 128 + threadIdx.x;
    if (e < count) crt_entry<LMAX, FAST, PB>(q, it->R, count, it->cols, e, it->X, it->ld, it->W);
}

// ---------------------------------------------------------------------------
// Conversion between RNS bases (Section 3.1: the Lagrange shortcut with a
// floating-point correction, no reconstruction).  With xi_i and alpha as in
// the fast path above, x + H = sum_i xi_i M_i - alpha M, so for a target prime q
//   x mod q = (sum_i xi_i (M_i mod q) - alpha (M mod q) - (H mod q)) mod q.
// Each term xi_i (M_i mod q) < 2^52 and at most 48 of them are summed in a
// 64-bit register, then one Barrett reduction.  When the fp32 estimate of
// alpha is too close to an integer to call, alpha is settled exactly: the
// true value is within one of floor(f), and it is the one that puts
// sum_i xi_i M_i - alpha M in [0, M), checked limb by limb.
template <int LMAX>
struct ConvConst {
    static constexpr int MLMAX = (LMAX * 26 + 31) / 32 + 1;
    uint32_t p[LMAX], hmod[LMAX], c[LMAX], cs[LMAX];
    float invp[LMAX];
    uint32_t mi[LMAX * MLMAX];     // limbs of M_i (exact alpha)
    uint32_t m[MLMAX];             // limbs of M
    uint32_t wt[LMAX * LMAX];      // M_i mod q_j at j * LMAX + i (zero for i >= L)
    // per target prime: {q, 2^32 mod q, its Shoup companion, floor(2^32 / q),
    // M mod q, H mod q, 0, 0}
    uint32_t qr[LMAX * 8];
    int L, LQ, m_limbs;
};
static_assert(sizeof(ConvConst<48>) <= 32000, "kernel parameter space");

template <int LMAX>
__device__ __noinline__ uint32_t exact_alpha(const ConvConst<LMAX>& v, const int32_t* __restrict__ R, int64_t count,
                                             int64_t e, uint32_t fl) {
    constexpr int MLMAX = ConvConst<LMAX>::MLMAX;
    const int L = v.L, ml = v.m_limbs;
    uint32_t xi[LMAX];  // recomputed here, so that the common path keeps its xi in registers
#pragma unroll 1
    for (int i = 0; i < L; i++) {
        const uint32_t pi = v.p[i];
        uint32_t a = (uint32_t)__ldg(R + (size_t)i * count + e) + v.hmod[i];
        if (a >= pi) a -= pi;
        uint32_t z = shoup_mul(a, v.c[i], v.cs[i], pi);
        if (z >= pi) z -= pi;
        xi[i] = z;
    }
    uint32_t d[MLMAX + 1];  // sum_i xi_i M_i - fl M, two's complement over ml + 1 limbs
    uint64_t carry = 0;
    uint32_t borrow = 0;
#pragma unroll 1
    for (int j = 0; j <= ml; j++) {
        uint64_t col = carry;
        if (j < ml) {
#pragma unroll 1
            for (int i = 0; i < L; i++) col += (uint64_t)xi[i] * v.mi[i * MLMAX + j];  // < 48 * 2^58 + 2^32
        }
        const uint32_t y = (uint32_t)col;
        carry = col >> 32;
        const uint64_t am = (uint64_t)fl * (j < ml ? v.m[j] : 0u) + borrow;
        const uint64_t diff = (uint64_t)y - (uint32_t)am;
        borrow = (uint32_t)(am >> 32) + (uint32_t)(diff >> 63);
        d[j] = (uint32_t)diff;
    }
    if (d[ml] >> 31) return fl - 1;  // below 0
    bool ge = d[ml] != 0;            // compare with M
    if (!ge) {
        ge = true;  // equal counts as >= M
#pragma unroll 1
        for (int j = ml - 1; j >= 0; j--) {
            if (d[j] != v.m[j]) {
                ge = d[j] > v.m[j];
                break;
            }
        }
    }
    return ge ? fl + 1 : fl;
}

template <int LMAX>
__global__ void __launch_bounds__(128)
convert_kernel(const __grid_constant__ ConvConst<LMAX> v, const int32_t* __restrict__ R, int32_t* __restrict__ out,
               int64_t count) {
    // The [j][i] table of M_i mod q_j and the per-target-prime records are
    // staged once per block in shared memory; the block then walks chunks of
    // 128 entries.  The loop over source primes is unrolled against 16-byte
    // shared loads, so xi stays in registers.
    __shared__ __align__(16) uint32_t ws[LMAX * LMAX];
    __shared__ __align__(16) uint32_t qs[LMAX * 8];
    const int L = v.L, LQ = v.LQ;
    for (int k = threadIdx.x; k < LQ * LMAX; k += blockDim.x) ws[k] = v.wt[k];
    for (int k = threadIdx.x; k < LQ * 8; k += blockDim.x) qs[k] = v.qr[k];
    __syncthreads();
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < count; e += (int64_t)gridDim.x * blockDim.x) {
        uint32_t rv[LMAX], xi[LMAX];
#pragma unroll
        for (int i = 0; i < LMAX; i++) rv[i] = i < L ? (uint32_t)__ldg(R + (size_t)i * count + e) : 0u;
        float f = 0.f;
#pragma unroll
        for (int i = 0; i < LMAX; i++) {
            xi[i] = 0;
            if (i < L) {
                const uint32_t pi = v.p[i];
                uint32_t a = rv[i] + v.hmod[i];
                if (a >= pi) a -= pi;
                uint32_t z = shoup_mul(a, v.c[i], v.cs[i], pi);
                if (z >= pi) z -= pi;
                xi[i] = z;
                f = fmaf((float)z, v.invp[i], f);
            }
        }
        const float fl = floorf(f);
        const float frac = f - fl;
        uint32_t alpha = (uint32_t)fl;
        if (frac < 0x1p-12f || frac > 1.f - 0x1p-12f) alpha = exact_alpha<LMAX>(v, R, count, e, alpha);
        int32_t* o = out + e;
#pragma unroll 1
        for (int j = 0; j < LQ; j++, o += count) {
            const uint4* wj = reinterpret_cast<const uint4*>(ws + j * LMAX);
            uint32_t l0 = 0, h0 = 0, l1 = 0, h1 = 0;  // two chains; xi_i = 0 and w = 0 beyond L
#pragma unroll
            for (int i4 = 0; i4 < LMAX / 4; i4++) {
                const uint4 w4 = wj[i4];
                mac64(l0, h0, xi[4 * i4], w4.x);
                mac64(l1, h1, xi[4 * i4 + 1], w4.y);
                mac64(l0, h0, xi[4 * i4 + 2], w4.z);
                mac64(l1, h1, xi[4 * i4 + 3], w4.w);
            }
            const uint4 c0 = *reinterpret_cast<const uint4*>(qs + 8 * j);
            const uint2 c1 = *reinterpret_cast<const uint2*>(qs + 8 * j + 4);
            const uint32_t qj = c0.x;
            // y - H = sum - alpha M - H; adding q 2^32 keeps it non-negative
            // (alpha (M mod q) + (H mod q) < 49 * 2^26 < 2^32) and below 2^59
            const uint64_t t = (((uint64_t)h0 << 32) | l0) + (((uint64_t)h1 << 32) | l1) + ((uint64_t)qj << 32) -
                               ((uint64_t)alpha * c1.x + c1.y);
            const uint32_t hi = (uint32_t)(t >> 32), lo = (uint32_t)t;
            const uint32_t t1 = hi * c0.y - __umulhi(hi, c0.z) * qj;  // [0, 2q)
            const uint32_t t2 = lo - __umulhi(lo, c0.w) * qj;         // [0, 2q)
            uint32_t r = t1 + t2;                                     // [0, 4q)
            if (r >= 2 * qj) r -= 2 * qj;
            if (r >= qj) r -= qj;
            *o = (int32_t)r;
        }
    }
}


template <int LMAX, bool FAST, int PB>
cudaError_t launch_crt_t(const CrtHost& h, const int32_t* R, int64_t rows, int64_t cols, uint64_t* X, int64_t ld,
                         int W, cudaStream_t s) {
    CrtConst<LMAX, FAST, PB> q;
    crt_const(h, q);
    const int64_t count = rows * cols;
    const int threads = 128;
    crt_kernel<LMAX, FAST, PB><<<(unsigned)((count + threads - 1) / threads), threads, 0, s>>>(q, R, rows, cols, X, ld,
                                                                                          W);
    return cudaGetLastError();
}

template <int LMAX, bool FAST, int PB>
cudaError_t launch_crt_grouped_t(const CrtHost& h, const CrtItem* items, int n, int64_t units, cudaStream_t s) {
    CrtConst<LMAX, FAST, PB> q;
    crt_const(h, q);
    crt_grouped_kernel<LMAX, FAST, PB><<<(unsigned)units, 128, 0, s>>>(q, items, n);
    return cudaGetLastError();
}

// a mod q of the integer with 32-bit limbs x[0 .. n) (q < 2^32)
uint32_t limbs_mod(const uint32_t* x, int n, uint32_t q) {
    uint64_t r = 0;
    for (int k = n - 1; k >= 0; k--) r = ((r << 32) | x[k]) % q;
    return (uint32_t)r;
}

template <int LMAX>
cudaError_t launch_convert_t(const CrtHost& h, const uint32_t* q, int LQ, const int32_t* R, int32_t* out,
                             int64_t count, int num_sms, cudaStream_t s) {
    using V = ConvConst<LMAX>;
    V v{};  // the parameter block, copied into the launch
    const int L = h.L;
    if (h.m_limbs > V::MLMAX) return cudaErrorInvalidValue;
    for (int i = 0; i < L; i++) {
        v.p[i] = h.p[i];
        v.hmod[i] = h.hmod[i];
        v.c[i] = h.c[i];
        v.cs[i] = h.cs[i];
        v.invp[i] = 1.0f / (float)h.p[i];
        for (int k = 0; k < h.m_limbs; k++) v.mi[i * V::MLMAX + k] = h.mi[(size_t)i * h.m_limbs + k];
    }
    for (int k = 0; k < h.m_limbs; k++) v.m[k] = h.m[k];
    for (int j = 0; j < LQ; j++) {
        const uint32_t qj = q[j];
        const uint32_t r32 = (uint32_t)((1ull << 32) % qj);
        uint32_t* rec = v.qr + 8 * j;
        rec[0] = qj;
        rec[1] = r32;
        rec[2] = (uint32_t)(((uint64_t)r32 << 32) / qj);
        rec[3] = (uint32_t)((1ull << 32) / qj);
        rec[4] = limbs_mod(h.m, h.m_limbs, qj);
        rec[5] = limbs_mod(h.h, h.m_limbs, qj);
        for (int i = 0; i < L; i++) v.wt[j * LMAX + i] = limbs_mod(h.mi + (size_t)i * h.m_limbs, h.m_limbs, qj);
    }
    v.L = L;
    v.LQ = LQ;
    v.m_limbs = h.m_limbs;
    // one block per 128 entries (measured faster than a persistent grid of
    // resident blocks walking the chunks: 0.164 against 0.183 ms for 1M entries)
    (void)num_sms;
    const int64_t chunks = (count + 127) / 128;
    if (chunks > 0x7FFFFFFF) return cudaErrorInvalidValue;
    convert_kernel<LMAX><<<(unsigned)chunks, 128, 0, s>>>(v, R, out, count);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_crt(const CrtHost& h, const int32_t* R, int64_t rows, int64_t cols, uint64_t* X, int64_t ld,
                       int W, cudaStream_t s) {
    if (rows == 0 || cols == 0) return cudaSuccess;
    const bool narrow = h.L > 0 && h.p[0] < (1u << 24);  // primes of at most 24 bits: fewer limbs of M
    if (h.L <= 8) return narrow ? launch_crt_t<8, true, 24>(h, R, rows, cols, X, ld, W, s) : launch_crt_t<8, true, 26>(h, R, rows, cols, X, ld, W, s);
    if (h.L <= 16) return narrow ? launch_crt_t<16, true, 24>(h, R, rows, cols, X, ld, W, s) : launch_crt_t<16, true, 26>(h, R, rows, cols, X, ld, W, s);
    if (h.L <= 24) return narrow ? launch_crt_t<24, true, 24>(h, R, rows, cols, X, ld, W, s) : launch_crt_t<24, true, 26>(h, R, rows, cols, X, ld, W, s);
    if (h.L <= 32) return narrow ? launch_crt_t<32, true, 24>(h, R, rows, cols, X, ld, W, s) : launch_crt_t<32, true, 26>(h, R, rows, cols, X, ld, W, s);
    if (h.L <= 48) return launch_crt_t<48, true, 26>(h, R, rows, cols, X, ld, W, s);
    if (h.L <= 64) return launch_crt_t<64, false, 26>(h, R, rows, cols, X, ld, W, s);
    return cudaErrorNotSupported;
}

int64_t crt_units(int64_t rows, int64_t cols) { return (rows * cols + 127) / 128; }

cudaError_t launch_crt_grouped(const CrtHost& h, const CrtItem* items, int n, int64_t units, int /*num_sms*/,
                               cudaStream_t s) {
    if (n == 0 || units == 0) return cudaSuccess;
    if (units > 0x7FFFFFFF) return cudaErrorInvalidValue;
    const bool narrow = h.L > 0 && h.p[0] < (1u << 24);
    if (h.L <= 8) return narrow ? launch_crt_grouped_t<8, true, 24>(h, items, n, units, s) : launch_crt_grouped_t<8, true, 26>(h, items, n, units, s);
    if (h.L <= 16) return narrow ? launch_crt_grouped_t<16, true, 24>(h, items, n, units, s) : launch_crt_grouped_t<16, true, 26>(h, items, n, units, s);
    if (h.L <= 24) return narrow ? launch_crt_grouped_t<24, true, 24>(h, items, n, units, s) : launch_crt_grouped_t<24, true, 26>(h, items, n, units, s);
    if (h.L <= 32) return narrow ? launch_crt_grouped_t<32, true, 24>(h, items, n, units, s) : launch_crt_grouped_t<32, true, 26>(h, items, n, units, s);
    if (h.L <= 48) return launch_crt_grouped_t<48, true, 26>(h, items, n, units, s);
    if (h.L <= 64) return launch_crt_grouped_t<64, false, 26>(h, items, n, units, s);
    return cudaErrorNotSupported;
}

cudaError_t launch_convert(const CrtHost& from, const uint32_t* q, int LQ, const int32_t* R, int32_t* out,
                           int64_t count, int num_sms, cudaStream_t s) {
    if (count == 0 || LQ == 0) return cudaSuccess;
    const int n = from.L > LQ ? from.L : LQ;
    if (n <= 8) return launch_convert_t<8>(from, q, LQ, R, out, count, num_sms, s);
    if (n <= 16) return launch_convert_t<16>(from, q, LQ, R, out, count, num_sms, s);
    if (n <= 24) return launch_convert_t<24>(from, q, LQ, R, out, count, num_sms, s);
    if (n <= 32) return launch_convert_t<32>(from, q, LQ, R, out, count, num_sms, s);
    if (n <= 48) return launch_convert_t<48>(from, q, LQ, R, out, count, num_sms, s);
    return cudaErrorNotSupported;
}

}  // namespace smf
