// rns_reduce: big-integer matrices -> residues modulo each prime of a basis
// (Section 3.1: the product starts by mapping each operand to one residue
// matrix per word-size prime), plus the balanced 8-bit digit split of the
// residues that feeds the tensor-core residue product.
//
// A two's complement entry of W words is x = sum_j v_j 2^(32 j) - s 2^(64 W)
// over its 2W unsigned 32-bit limbs v_j and sign bit s.  Hence
//   x mod p = (sum_j v_j c_j - s c_(2W)) mod p,   c_j = 2^(32 j) mod p,
// where every product v_j c_j < 2^58, so sixteen of them sum below 2^62 in a
// 64-bit register before one Barrett reduction.  The c_j of the primes in a
// launch's group are built once per block in shared memory.
#include <cuda_bf16.h>

#include "smf_internal.h"

namespace smf {
namespace {

constexpr int kThreads = 256;
constexpr int kTableWords = 4096;  // shared-memory table capacity (uint32)

__device__ __forceinline__ uint32_t barrett64(uint64_t x, uint32_t p, uint64_t mu) {
    // mu = floor((2^64-1)/p): the estimate q is at most 2 below floor(x/p)
    uint64_t q = __umul64hi(x, mu);
    uint64_t r = x - q * (uint64_t)p;
    if (r >= p) r -= p;
    if (r >= p) r -= p;
    return (uint32_t)r;
}

// bf16 bit pattern of an integer |d| <= 2^15: the fp32 value is formed exactly by
// the 1.5 * 2^23 offset trick (integer add, then one float subtract), and any
// integer with at most 8 significant bits converts to bf16 by truncation of
// the fp32 bits, exactly.  Callers pass |d| <= 256.
__device__ __forceinline__ uint16_t bf16_bits_small(int32_t d) {
    const float f = __int_as_float(0x4B400000 + d) - 12582912.0f;
    return (uint16_t)(__float_as_uint(f) >> 16);
}

// Balanced digits: lower digits in [-128, 127], top digit = remaining quotient.
// With a = r + 128: d0 = (a & 255) - 128 and the rest is a >> 8 (floor), so for
// two or three digits (|r| < 2^23) the split is in closed form.
__device__ __forceinline__ void store_digits(int64_t r, int t, __nv_bfloat16* dst, int64_t plane) {
    uint16_t* o = reinterpret_cast<uint16_t*>(dst);
    if (t == 3 || t == 2) {
        const int32_t a = (int32_t)r + 128;
        o[0] = bf16_bits_small((a & 255) - 128);
        if (t == 2) {
            o[plane] = bf16_bits_small(a >> 8);
        } else {
            const int32_t b = (a >> 8) + 128;
            o[plane] = bf16_bits_small((b & 255) - 128);
            o[2 * plane] = bf16_bits_small(b >> 8);
        }
        return;
    }
    for (int u = 0; u < t - 1; u++) {
        const int32_t d = (int32_t)(((r + 128) & 255) - 128);
        o[u * plane] = bf16_bits_small(d);
        r = (r - d) >> 8;
    }
    o[(t - 1) * plane] = bf16_bits_small((int32_t)r);  // |top| <= 128
}

// Declared-bound check: does the two's complement value of the 2W limbs v[]
// lie outside [-2^bits, 2^bits]?  Negative values fit when every bit from
// `bits` up is one; non-negative ones when every bit above `bits` is zero and,
// if bit `bits` is set, every bit below it is zero (x = 2^bits).
template <int WC>
__device__ __forceinline__ bool over_bits(const uint32_t (&v)[2 * WC], int W, int bits) {
    if (bits >= 64 * W - 1) return false;
    const int L = bits >> 5, sh = bits & 31;
    const bool neg = (v[2 * W - 1] >> 31) != 0;
    bool over = false, low_zero = true;
#pragma unroll
    for (int j = 0; j < 2 * WC; j++) {
        if (j >= 2 * W) break;
        if (j < L) {
            low_zero &= v[j] == 0;
        } else if (j == L) {
            const uint32_t hi = v[j] >> sh;
            if (neg) over |= hi != (0xFFFFFFFFu >> sh);
            else over |= hi > 1 || (hi == 1 && (!low_zero || (sh && (v[j] << (32 - sh)) != 0)));
        } else {
            over |= v[j] != (neg ? 0xFFFFFFFFu : 0u);
        }
    }
    return over;
}

// The same check for an entry that is its own centred value (the shared-digit
// path reads only the low word): |v| <= 2^bits, and the words above the low
// one (W > 1) are its sign extension.
__device__ __forceinline__ bool over_bits_low(int64_t v, int bits) {
    return bits < 63 && (v > (1ll << bits) || v < -(1ll << bits));
}

__device__ __forceinline__ void flag_bound(int* status) {
    if (status) atomicOr(status, kStatusBound);
}

// Residue of one entry whose 2W 32-bit limbs are v[] (two's complement sign s)
// modulo prime e of the block's group.
template <int WC>
__device__ __forceinline__ uint32_t entry_mod(const uint32_t (&v)[2 * WC], int W, uint32_t s, const uint32_t* ct,
                                              uint32_t p, uint64_t mu) {
    uint64_t acc = 0;
    uint32_t rr = 0;
#pragma unroll
    for (int j4 = 0; j4 < 2 * WC; j4 += 4) {
        if (j4 < 2 * W) {
            const uint4 c4 = *(const uint4*)(ct + j4);  // ct rows are 16-byte aligned
            const uint32_t cj[4] = {c4.x, c4.y, c4.z, c4.w};
#pragma unroll
            for (int q = 0; q < 4; q++) {
                const int j = j4 + q;
                if (j < 2 * W) {
                    acc += (uint64_t)v[j] * cj[q];
                    if ((j & 15) == 15) {  // 16 products: fold before 2^64
                        rr = barrett64(acc + rr, p, mu);
                        acc = 0;
                    }
                }
            }
        }
    }
    rr = barrett64(acc + rr, p, mu);
    if (s) {  // subtract 2^(64W) mod p
        const uint32_t cw = ct[2 * W];
        rr = rr >= cw ? rr - cw : rr + p - cw;
    }
    return rr;
}

// WC: compile-time word capacity (the entry's words are held in registers);
// W <= WC is the runtime word count.
template <ReduceOut KIND, int WC>
__global__ void __launch_bounds__(kThreads)
reduce_kernel(BasisDev b, ReduceArgs a, int group) {
    extern __shared__ uint32_t ctab[];  // [G][2W+1]
    const int i0 = blockIdx.z * group;
    const int G = min(group, b.L - i0);
    const int W = a.W;
    const int nw = (2 * W + 1 + 3) & ~3;  // row of one prime's constants, padded to 16 bytes
    if (!a.identity) {
        for (int e = threadIdx.x; e < G; e += blockDim.x) {
            const uint32_t p = b.p[i0 + e];
            const uint64_t mu = b.mu[i0 + e];
            const uint32_t r32 = b.pow32[i0 + e];
            uint32_t c = 1 % p;
            for (int j = 0; j < nw; j++) {
                ctab[e * nw + j] = j <= 2 * W ? c : 0u;
                c = barrett64((uint64_t)c * r32, p, mu);
            }
        }
        __syncthreads();
    }
    // Thread mapping: consecutive threads take consecutive output addresses.
    // Transposed digit planes are contiguous along rows, the others along cols.
    constexpr bool trans = KIND == ReduceOut::kDigitsT;
    const int64_t minor_n = trans ? a.rows : a.cols;
    const int64_t major_n = trans ? a.cols : a.rows;
    const int64_t minor = (int64_t)blockIdx.x * kThreads + threadIdx.x;
    if (minor >= minor_n) return;
    for (int64_t major = blockIdx.y; major < major_n; major += gridDim.y) {
        const int64_t r = trans ? minor : major;
        const int64_t c = trans ? major : minor;
        const uint64_t* x = a.X + (size_t)(r * a.ld + c) * W;
        // the entry's words, loaded once (16-byte loads when aligned)
        uint32_t v[2 * WC];
#pragma unroll
        for (int j = 0; j < WC; j++) {
            if (j < W) {
                uint64_t w;
                if ((W & 1) == 0 && (j & 1) == 0) {
                    const ulonglong2 q = __ldg((const ulonglong2*)(x + j));
                    w = q.x;
                    v[2 * j + 2] = (uint32_t)q.y;
                    v[2 * j + 3] = (uint32_t)(q.y >> 32);
                } else if ((W & 1) == 0) {
                    w = ((uint64_t)v[2 * j + 1] << 32) | v[2 * j];  // already loaded
                } else {
                    w = __ldg(x + j);
                }
                v[2 * j] = (uint32_t)w;
                v[2 * j + 1] = (uint32_t)(w >> 32);
            }
        }
        const uint32_t s = v[2 * W - 1] >> 31;
        if (a.status && blockIdx.z == 0) {
            bool over;
            if (a.identity) {
                const int64_t lo = (int64_t)(((uint64_t)v[1] << 32) | v[0]);
                over = over_bits_low(lo, a.bits);
                for (int j = 2; j < 2 * W; j++) over |= v[j] != (lo < 0 ? 0xFFFFFFFFu : 0u);
            } else {
                over = over_bits<WC>(v, W, a.bits);
            }
            if (over) flag_bound(a.status);
        }
        for (int e = 0; e < (a.identity ? 1 : G); e++) {
            const int i = i0 + e;
            int64_t val;  // centred residue, or the value itself (identity)
            uint32_t canon = 0;
            if (a.identity) {
                val = (int64_t)(((uint64_t)v[1] << 32) | v[0]);
            } else {
                const uint32_t p = b.p[i];
                canon = entry_mod<WC>(v, W, s, ctab + e * nw, p, b.mu[i]);
                val = (int64_t)canon > (int64_t)(p >> 1) ? (int64_t)canon - p : (int64_t)canon;
            }
            if constexpr (KIND == ReduceOut::kCanonical) {
                ((int32_t*)a.out)[((size_t)i * a.rows + r) * a.cols + c] = (int32_t)canon;
            } else if constexpr (KIND == ReduceOut::kCentered) {
                ((int32_t*)a.out)[((size_t)i * a.rows + r) * a.cols + c] = (int32_t)val;
            } else if constexpr (KIND == ReduceOut::kDigits) {  // [L][t][rows][ld_out]
                const int64_t plane = a.rows * a.ld_out;
                __nv_bfloat16* base = (__nv_bfloat16*)a.out + (size_t)i * a.t * plane;
                store_digits(val, a.t, base + r * a.ld_out + c, plane);
            } else {  // [t][L][cols][ld_out]
                const int64_t plane = a.cols * a.ld_out;
                __nv_bfloat16* base = (__nv_bfloat16*)a.out + (size_t)i * plane;
                store_digits(val, a.t, base + c * a.ld_out + r, plane * b.L);
            }
        }
    }
}

// rns_reduce of B straight into transposed, digit-major bf16 planes
// [t][L][cols][ld_out] (digit u of prime i at plane u * L + i).  A block takes
// 256 consecutive rows by NC columns; each thread reduces its row's NC
// entries (W words each, held in registers) modulo the block's group of
// primes, so the per-block table of 2^(32 j) mod p is amortised over NC
// entries.  With 2W <= 16 the limb products of one prime sum below 2^62 and a
// single Barrett reduction finishes each residue.
//
// Per prime: {p, 2^32 mod p, its Shoup companion, floor(2^32 / p)}, then
// c_j = 2^(32 j) mod p for j <= 2W, padded to 16-byte rows.
template <int W>
struct RtTable {
    static constexpr int NW = 4 + ((2 * W + 1 + 3) & ~3);
};

template <int W>
__device__ __forceinline__ void reduce_t_table(const BasisDev& b, uint32_t* ctab, int i0, int G) {
    constexpr int NW = RtTable<W>::NW;
    for (int e = threadIdx.x; e < G; e += blockDim.x) {
        const uint32_t p = b.p[i0 + e];
        const uint64_t mu = b.mu[i0 + e];
        const uint32_t r32 = b.pow32[i0 + e];
        uint32_t* row = ctab + e * NW;
        row[0] = p;
        row[1] = r32;
        row[2] = (uint32_t)(((uint64_t)r32 << 32) / p);
        row[3] = (uint32_t)((1ull << 32) / p);
        uint32_t c = 1 % p;
        for (int j = 0; j < NW - 4; j++) {
            row[4 + j] = j <= 2 * W ? c : 0u;
            c = barrett64((uint64_t)c * r32, p, mu);
        }
    }
}

// One thread of the transposed reduce: row r, columns [cb, cb + NC), primes
// i0 .. i0 + G - 1 (their table in ctab).
template <int W, int NC>
__device__ __forceinline__ void reduce_t_thread(const BasisDev& b, const uint32_t* ctab, int i0, int G,
                                                const uint64_t* __restrict__ X, int64_t rows, int64_t cols,
                                                int64_t ld, uint16_t* __restrict__ out, int64_t ld_out, int t,
                                                int64_t r, int64_t cb, int bits, int* status) {
    constexpr int NW = RtTable<W>::NW;
    if (r >= rows) return;
    const int64_t plane = cols * ld_out;
    const int64_t dstride = plane * b.L;  // between digit planes of one prime
    for (int cc = 0; cc < NC; cc++) {
        const int64_t c = cb + cc;
        if (c >= cols) break;
        const uint64_t* x = X + (size_t)(r * ld + c) * W;
        uint32_t v[2 * W];
#pragma unroll
        for (int j = 0; j < W; j += 2) {
            if (j + 1 < W) {
                const ulonglong2 q = __ldg((const ulonglong2*)(x + j));
                v[2 * j] = (uint32_t)q.x;
                v[2 * j + 1] = (uint32_t)(q.x >> 32);
                v[2 * j + 2] = (uint32_t)q.y;
                v[2 * j + 3] = (uint32_t)(q.y >> 32);
            } else {
                const uint64_t q = __ldg(x + j);
                v[2 * j] = (uint32_t)q;
                v[2 * j + 1] = (uint32_t)(q >> 32);
            }
        }
        const bool neg = (v[2 * W - 1] >> 31) != 0;
        if (status && i0 == 0 && over_bits<W>(v, W, bits)) flag_bound(status);
        uint16_t* o = out + (size_t)i0 * plane + c * ld_out + r;
        for (int e = 0; e < G; e++, o += plane) {
            const uint32_t* ct = ctab + e * NW;
            const uint4 hd = *(const uint4*)ct;
            const uint32_t p = hd.x;
            // sum_j v_j c_j < 16 * 2^56 < 2^62 (2W <= 16), as hi 2^32 + lo
            uint32_t lo = 0, hi = 0;
#pragma unroll
            for (int j4 = 0; j4 < 2 * W; j4 += 4) {
                const uint4 c4 = *(const uint4*)(ct + 4 + j4);
                const uint32_t cj[4] = {c4.x, c4.y, c4.z, c4.w};
#pragma unroll
                for (int q = 0; q < 4; q++)
                    if (j4 + q < 2 * W) mac64(lo, hi, v[j4 + q], cj[q]);
            }
            // hi (2^32 mod p) by Shoup, lo by its reciprocal quotient
            const uint32_t t1 = hi * hd.y - __umulhi(hi, hd.z) * p;  // [0, 2p)
            const uint32_t t2 = lo - __umulhi(lo, hd.w) * p;         // [0, 2p)
            uint32_t rr = t1 + t2;                                   // [0, 4p)
            if (rr >= 2 * p) rr -= 2 * p;
            if (rr >= p) rr -= p;
            if (neg) {  // subtract 2^(64W) mod p
                const uint32_t cw = ct[4 + 2 * W];
                rr = rr >= cw ? rr - cw : rr + p - cw;
            }
            int32_t val = rr > (p >> 1) ? (int32_t)rr - (int32_t)p : (int32_t)rr;
            if (t == 3) {  // balanced digits in closed form: a = v + 128, b = (a >> 8) + 128
                const int32_t a = val + 128;
                const int32_t b = (a >> 8) + 128;
                o[0] = bf16_bits_small((a & 255) - 128);
                o[dstride] = bf16_bits_small((b & 255) - 128);
                o[2 * dstride] = bf16_bits_small(b >> 8);
            } else {
                uint16_t* od = o;
                for (int u = 0; u < t - 1; u++, od += dstride) {
                    const int32_t d = ((val + 128) & 255) - 128;
                    *od = bf16_bits_small(d);
                    val = (val - d) >> 8;
                }
                *od = bf16_bits_small(val);
            }
        }
    }
}

template <int W, int NC>
__global__ void __launch_bounds__(kThreads)
reduce_digits_t_kernel(BasisDev b, const uint64_t* __restrict__ X, int64_t rows, int64_t cols, int64_t ld,
                       uint16_t* __restrict__ out, int64_t ld_out, int t, int group, int bits, int* status) {
    extern __shared__ uint32_t ctab[];  // [G][NW]
    const int i0 = blockIdx.z * group;
    const int G = min(group, b.L - i0);
    reduce_t_table<W>(b, ctab, i0, G);
    __syncthreads();
    reduce_t_thread<W, NC>(b, ctab, i0, G, X, rows, cols, ld, out, ld_out, t,
                           (int64_t)blockIdx.x * kThreads + threadIdx.x, (int64_t)blockIdx.y * NC, bits, status);
}

// The transposed reduce of several B operands (all of W words) in one
// persistent launch: the table of every prime is built once per block, then
// the block walks the items' units.  A unit is rb rows (rb = 32 .. 256, fitted
// to the item's row count so that short operands keep the threads busy) by
// (256 / rb) * NC columns; consecutive threads take consecutive rows.
template <int W, int NC>
__global__ void __launch_bounds__(kThreads, 4)  // 64 registers: four blocks per SM (measured 2 % faster than 74)
reduce_digits_t_grouped_kernel(BasisDev b, const ReduceItem* __restrict__ items, int n, int64_t units,
                               int* status) {
    extern __shared__ uint32_t ctab[];  // [L][NW]
    reduce_t_table<W>(b, ctab, 0, b.L);
    __syncthreads();
    for (int64_t u = blockIdx.x; u < units; u += gridDim.x) {
        const ReduceItem* it = find_item(items, n, u);
        const int rb = it->rb;
        const int64_t gx = (it->rows + rb - 1) / rb;
        const int64_t lu = u - it->base;
        const int64_t r = (lu % gx) * rb + threadIdx.x % rb;
        const int64_t cb = ((lu / gx) * (kThreads / rb) + threadIdx.x / rb) * NC;
        reduce_t_thread<W, NC>(b, ctab, 0, b.L, it->X, it->rows, it->cols, it->ld, (uint16_t*)it->out, it->ld_out,
                               it->t, r, cb, it->bits, status);
    }
}

// Digit split of a matrix whose int64 entries (low word of W) are their own
// centred residues (|x| <= (p_L - 1)/2): planes [t][rows][ld_out].  Eight
// consecutive entries per thread: 64 bytes in, 16 bytes out per plane.
__global__ void __launch_bounds__(kThreads)
split_digits8_kernel(const uint64_t* __restrict__ X, int64_t rows, int64_t cols, int64_t ld, int W,
                     __nv_bfloat16* __restrict__ out, int64_t ld_out, int t, int bits, int* status) {
    const int64_t groups = cols / 8;
    const int64_t g = (int64_t)blockIdx.x * kThreads + threadIdx.x;
    if (g >= groups) return;
    const int64_t plane = rows * ld_out;
    for (int64_t r = blockIdx.y; r < rows; r += gridDim.y) {
        const uint64_t* x = X + (size_t)(r * ld + g * 8) * W;
        int64_t v[8];
        if (W == 1) {
#pragma unroll
            for (int q = 0; q < 4; q++) {
                const ulonglong2 w = __ldg((const ulonglong2*)x + q);
                v[2 * q] = (int64_t)w.x;
                v[2 * q + 1] = (int64_t)w.y;
            }
        } else {
            bool ext = false;  // the upper words must be the low word's sign extension
#pragma unroll
            for (int q = 0; q < 8; q++) {
                v[q] = (int64_t)__ldg(x + (size_t)q * W);
                for (int j = 1; j < W; j++) ext |= __ldg(x + (size_t)q * W + j) != (v[q] < 0 ? ~0ull : 0ull);
            }
            if (ext) flag_bound(status);
        }
        {
            bool over = false;
#pragma unroll
            for (int q = 0; q < 8; q++) over |= over_bits_low(v[q], bits);
            if (over) flag_bound(status);
        }
        __nv_bfloat16* o = out + r * ld_out + g * 8;
        for (int u = 0; u < t; u++) {
            float f[8];
#pragma unroll
            for (int q = 0; q < 8; q++) {
                int32_t dq;
                if (u < t - 1) {
                    dq = (int32_t)(((v[q] + 128) & 255) - 128);
                    v[q] = (v[q] - dq) >> 8;
                } else {
                    dq = (int32_t)v[q];  // |top| <= 128
                }
                f[q] = __int_as_float(0x4B400000 + dq) - 12582912.0f;  // exact, |dq| <= 256
            }
            uint32_t w[4];
#pragma unroll
            for (int q = 0; q < 4; q++)
                w[q] = (__float_as_uint(f[2 * q]) >> 16) | (__float_as_uint(f[2 * q + 1]) & 0xFFFF0000u);
            *(uint4*)(o + u * plane) = make_uint4(w[0], w[1], w[2], w[3]);
        }
    }
}

// Digit split of several centred-value operands (shared-digit A: every entry
// is its own centred residue for all primes) in one persistent launch.  A unit
// is 2048 consecutive entries of one item in row-major order; consecutive
// threads take consecutive entries, so loads and plane stores coalesce along
// each row whatever the column count.
constexpr int kSplitPer = 8;  // entries per thread per unit
__global__ void __launch_bounds__(kThreads, 8)  // 32 registers: latency-bound, occupancy wins (measured)
split_digits_grouped_kernel(const ReduceItem* __restrict__ items, int n, int64_t units, int* status) {
    for (int64_t u = blockIdx.x; u < units; u += gridDim.x) {
        const ReduceItem* it = find_item(items, n, u);
        const int64_t cols = it->cols, count = it->rows * cols;
        const int64_t plane = it->rows * it->ld_out;
        __nv_bfloat16* out = (__nv_bfloat16*)it->out;
        const int64_t e0 = (u - it->base) * (kThreads * kSplitPer) + threadIdx.x;
#pragma unroll 4
        for (int q = 0; q < kSplitPer; q++) {
            const int64_t e = e0 + (int64_t)q * kThreads;
            if (e >= count) break;
            int64_t r, c;
            if (count <= 0xFFFFFFFFll) {  // quotient by the item's precomputed multiplier
                const uint32_t e32 = (uint32_t)e;
                r = (uint32_t)(((uint64_t)__umulhi(e32, it->div_m) + e32) >> it->div_s);
                c = e - r * cols;
            } else {
                r = e / cols;
                c = e - r * cols;
            }
            const uint64_t* x = it->X + (size_t)(r * it->ld + c) * it->W;
            const int64_t v = (int64_t)__ldg(x);
            bool over = over_bits_low(v, it->bits);
            for (int j = 1; j < it->W; j++) over |= __ldg(x + j) != (v < 0 ? ~0ull : 0ull);
            if (over) flag_bound(status);
            store_digits(v, it->t, out + r * it->ld_out + c, plane);
        }
    }
}

// int32 residues (any representative in (-p, p)) -> digit planes.
// Non-transposed: elementwise.  Transposed: 32 x 32 tiles through shared memory.
__global__ void __launch_bounds__(kThreads)
digits_kernel(BasisDev b, const int32_t* R, int64_t prime_stride, int64_t rows, int64_t cols,
              __nv_bfloat16* out, int64_t ld_out, int t, int shared_a) {
    const int i = blockIdx.z;
    const int32_t* Ri = R + (size_t)i * prime_stride;
    const int64_t plane = rows * ld_out;
    __nv_bfloat16* base = out + (size_t)i * t * plane;
    const uint32_t p = b.p[shared_a ? b.L - 1 : i];
    const int32_t h = (int32_t)(p >> 1);
    const int64_t c = (int64_t)blockIdx.x * kThreads + threadIdx.x;
    if (c >= cols) return;
    for (int64_t r = blockIdx.y; r < rows; r += gridDim.y) {
        int32_t v = Ri[r * cols + c];
        if (!shared_a) {
            if (v > h) v -= (int32_t)p;
            if (v < -h) v += (int32_t)p;
        }
        store_digits(v, t, base + r * ld_out + c, plane);
    }
}

__global__ void __launch_bounds__(256)
digits_t_kernel(BasisDev b, const int32_t* R, int64_t prime_stride, int64_t rows, int64_t cols,
                __nv_bfloat16* out, int64_t ld_out, int t) {
    // R_i is rows x cols; the planes are cols x ld_out (transposed), digit-major
    // across the primes: digit u of prime i at plane u * L + i.
    __shared__ int32_t tile[32][33];
    const int i = blockIdx.z;
    const int32_t* Ri = R + (size_t)i * prime_stride;
    const int64_t plane = cols * ld_out;
    __nv_bfloat16* base = out + (size_t)i * plane;
    const uint32_t p = b.p[i];
    const int32_t h = (int32_t)(p >> 1);
    const int64_t r0 = (int64_t)blockIdx.x * 32, c0 = (int64_t)blockIdx.y * 32;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    for (int k = ty; k < 32; k += 8) {
        const int64_t r = r0 + k, c = c0 + tx;
        int32_t v = 0;
        if (r < rows && c < cols) {
            v = Ri[r * cols + c];
            if (v > h) v -= (int32_t)p;
            if (v < -h) v += (int32_t)p;
        }
        tile[k][tx] = v;
    }
    __syncthreads();
    for (int k = ty; k < 32; k += 8) {
        const int64_t c = c0 + k, r = r0 + tx;
        if (c < cols && r < rows) store_digits(tile[tx][k], t, base + c * ld_out + r, plane * gridDim.z);
    }
}

}  // namespace

template <ReduceOut KIND>
cudaError_t launch_reduce_kind(const BasisDev& b, const ReduceArgs& a, dim3 grid, size_t smem, int group,
                               cudaStream_t s) {
    if (a.W <= 1) reduce_kernel<KIND, 1><<<grid, kThreads, smem, s>>>(b, a, group);
    else if (a.W <= 2) reduce_kernel<KIND, 2><<<grid, kThreads, smem, s>>>(b, a, group);
    else if (a.W <= 4) reduce_kernel<KIND, 4><<<grid, kThreads, smem, s>>>(b, a, group);
    else if (a.W <= 8) reduce_kernel<KIND, 8><<<grid, kThreads, smem, s>>>(b, a, group);
    else if (a.W <= 16) reduce_kernel<KIND, 16><<<grid, kThreads, smem, s>>>(b, a, group);
    else return cudaErrorNotSupported;
    return cudaGetLastError();
}

cudaError_t launch_reduce(const BasisDev& b, const ReduceArgs& a_in, ReduceOut kind, int* d_status,
                          cudaStream_t s) {
    if (a_in.rows == 0 || a_in.cols == 0) return cudaSuccess;
    // entries outside the declared bound set kStatusBound (bits <= 0: not checked)
    ReduceArgs a = a_in;
    if (a.bits <= 0) a.bits = 64 * a.W;
    a.status = a.bits < 64 * a.W - 1 ? d_status : nullptr;
    if (kind == ReduceOut::kDigits && a.identity && a.cols % 8 == 0 && a.ld % 2 == 0 && a.ld_out % 8 == 0 &&
        ((uintptr_t)a.X & 15) == 0 && ((uintptr_t)a.out & 15) == 0) {
        const int64_t groups = a.cols / 8;
        dim3 grid((unsigned)((groups + kThreads - 1) / kThreads), (unsigned)(a.rows < 65535 ? a.rows : 65535));
        split_digits8_kernel<<<grid, kThreads, 0, s>>>(a.X, a.rows, a.cols, a.ld, a.W, (__nv_bfloat16*)a.out,
                                                       a.ld_out, a.t, a.bits, a.status);
        return cudaGetLastError();
    }
    const int nw = (2 * a.W + 1 + 3) & ~3;
    int group = a.identity ? 1 : max(1, min(b.L, kTableWords / (nw + 4)));
    if (kind == ReduceOut::kDigitsT && !a.identity && (((uintptr_t)a.X & 15) == 0) &&
        (a.W == 1 || a.W == 2 || a.W == 4 || a.W == 8) && (a.W == 1 || a.ld % 2 == 0)) {
        constexpr int NC = 4;
        dim3 grid((unsigned)((a.rows + kThreads - 1) / kThreads), (unsigned)((a.cols + NC - 1) / NC),
                  (unsigned)((b.L + group - 1) / group));
        if (grid.y > 65535) goto generic;
        const size_t sm = sizeof(uint32_t) * (size_t)group * (nw + 4);
        uint16_t* o = (uint16_t*)a.out;
        switch (a.W) {
            case 1: reduce_digits_t_kernel<1, NC><<<grid, kThreads, sm, s>>>(b, a.X, a.rows, a.cols, a.ld, o, a.ld_out, a.t, group, a.bits, a.status); break;
            case 2: reduce_digits_t_kernel<2, NC><<<grid, kThreads, sm, s>>>(b, a.X, a.rows, a.cols, a.ld, o, a.ld_out, a.t, group, a.bits, a.status); break;
            case 4: reduce_digits_t_kernel<4, NC><<<grid, kThreads, sm, s>>>(b, a.X, a.rows, a.cols, a.ld, o, a.ld_out, a.t, group, a.bits, a.status); break;
            default: reduce_digits_t_kernel<8, NC><<<grid, kThreads, sm, s>>>(b, a.X, a.rows, a.cols, a.ld, o, a.ld_out, a.t, group, a.bits, a.status); break;
        }
        return cudaGetLastError();
    }
generic:
    const int groups = a.identity ? 1 : (b.L + group - 1) / group;
    const bool trans = kind == ReduceOut::kDigitsT;
    const int64_t minor_n = trans ? a.rows : a.cols;
    const int64_t major_n = trans ? a.cols : a.rows;
    dim3 grid((unsigned)((minor_n + kThreads - 1) / kThreads), (unsigned)(major_n < 65535 ? major_n : 65535),
              (unsigned)groups);
    size_t smem = a.identity ? 0 : sizeof(uint32_t) * (size_t)group * nw;
    switch (kind) {
        case ReduceOut::kCanonical: return launch_reduce_kind<ReduceOut::kCanonical>(b, a, grid, smem, group, s);
        case ReduceOut::kCentered: return launch_reduce_kind<ReduceOut::kCentered>(b, a, grid, smem, group, s);
        case ReduceOut::kDigits: return launch_reduce_kind<ReduceOut::kDigits>(b, a, grid, smem, group, s);
        case ReduceOut::kDigitsT: return launch_reduce_kind<ReduceOut::kDigitsT>(b, a, grid, smem, group, s);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_residue_digits(const BasisDev& b, const int32_t* R, int64_t prime_stride,
                                  int Lcount, int64_t rows, int64_t cols, void* out,
                                  int64_t ld_out, int t, bool transpose, cudaStream_t s) {
    if (rows == 0 || cols == 0 || Lcount == 0) return cudaSuccess;
    if (!transpose) {
        dim3 grid((unsigned)((cols + kThreads - 1) / kThreads), (unsigned)(rows < 65535 ? rows : 65535),
                  (unsigned)Lcount);
        digits_kernel<<<grid, kThreads, 0, s>>>(b, R, prime_stride, rows, cols, (__nv_bfloat16*)out,
                                                ld_out, t, prime_stride == 0 ? 1 : 0);
    } else {
        dim3 grid((unsigned)((rows + 31) / 32), (unsigned)((cols + 31) / 32), (unsigned)Lcount);
        digits_t_kernel<<<grid, 256, 0, s>>>(b, R, prime_stride, rows, cols, (__nv_bfloat16*)out,
                                             ld_out, t);
    }
    return cudaGetLastError();
}

namespace {
constexpr int kNC = 4;  // columns per block of the transposed reduce

// blocks of `kernel` resident per SM (at least one), computed once per kernel
template <class Kern>
int resident(Kern kernel, int threads, size_t smem) {
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kernel, threads, smem) != cudaSuccess) {
        cudaGetLastError();
        nb = 1;
    }
    return nb > 0 ? nb : 1;
}

int64_t persistent_grid(int64_t units, int num_sms, int per_sm) {
    const int64_t g = (int64_t)(num_sms > 0 ? num_sms : 148) * per_sm;
    return units < g ? units : g;
}

template <int W>
cudaError_t launch_rt_grouped_w(const BasisDev& b, const ReduceItem* items, int n, int64_t units, int num_sms,
                                int* status, cudaStream_t s) {
    const size_t sm = sizeof(uint32_t) * (size_t)b.L * RtTable<W>::NW;
    static int per_sm = 0;
    if (!per_sm) per_sm = resident(reduce_digits_t_grouped_kernel<W, kNC>, kThreads, sizeof(uint32_t) * 64 * RtTable<W>::NW);
    const int64_t grid = persistent_grid(units, num_sms, per_sm);
    reduce_digits_t_grouped_kernel<W, kNC><<<(unsigned)grid, kThreads, sm, s>>>(b, items, n, units, status);
    return cudaGetLastError();
}
}  // namespace

int64_t reduce_t_units(int64_t rows, int64_t cols, int* rb) {
    int h = 32;
    while (h < kThreads && h < rows) h *= 2;
    *rb = h;
    const int64_t cpu = (int64_t)(kThreads / h) * kNC;  // columns per unit
    return ((rows + h - 1) / h) * ((cols + cpu - 1) / cpu);
}

bool reduce_t_groupable(const BasisDev& b, const ReduceArgs& a) {
    const int nw = (2 * a.W + 1 + 3) & ~3;
    return !a.identity && ((uintptr_t)a.X & 15) == 0 && (a.W == 1 || a.W == 2 || a.W == 4 || a.W == 8) &&
           (a.W == 1 || a.ld % 2 == 0) && b.L <= 64 && b.L <= kTableWords / (nw + 4);
}

int64_t split_units(int64_t rows, int64_t cols, uint32_t* div_m, int* div_s) {
    // m = ceil(2^(32+s) / d) with 2^s >= d lies in (2^32, 2^33]; its low 32 bits
    // are kept and the 2^32 e term is added back in the kernel
    const uint64_t d = cols > 0 ? (uint64_t)cols : 1;
    int sh = 0;
    while (sh < 32 && (1ull << sh) < d) sh++;
    const unsigned __int128 num = (unsigned __int128)1 << (32 + sh);
    const unsigned __int128 m = (num + d - 1) / d;
    *div_m = (uint32_t)(m - ((unsigned __int128)1 << 32));
    *div_s = sh;
    return (rows * cols + kThreads * kSplitPer - 1) / (kThreads * kSplitPer);
}

cudaError_t launch_reduce_t_grouped(const BasisDev& b, int W, const ReduceItem* items, int n, int64_t units,
                                    int num_sms, int* status, cudaStream_t s) {
    if (n == 0 || units == 0) return cudaSuccess;
    switch (W) {
        case 1: return launch_rt_grouped_w<1>(b, items, n, units, num_sms, status, s);
        case 2: return launch_rt_grouped_w<2>(b, items, n, units, num_sms, status, s);
        case 4: return launch_rt_grouped_w<4>(b, items, n, units, num_sms, status, s);
        case 8: return launch_rt_grouped_w<8>(b, items, n, units, num_sms, status, s);
    }
    return cudaErrorNotSupported;
}

cudaError_t launch_split_grouped(const ReduceItem* items, int n, int64_t units, int num_sms, int* status,
                                 cudaStream_t s) {
    if (n == 0 || units == 0) return cudaSuccess;
    static int per_sm = 0;
    if (!per_sm) per_sm = resident(split_digits_grouped_kernel, kThreads, 0);
    const int64_t grid = persistent_grid(units, num_sms, per_sm);
    split_digits_grouped_kernel<<<(unsigned)grid, kThreads, 0, s>>>(items, n, units, status);
    return cudaGetLastError();
}

}  // namespace smf
