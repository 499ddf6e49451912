// Elimination over Z/(m) with unit pivots, on the device.  Two uses in the
// Smith-form driver (Section 2):
//  - the last iteration of Phase 2 works modulo a word-size s: the Smith form
//    of A over Z/(s) is the product over the prime powers q^e || s of the
//    local Smith forms over Z/(q^e), and each of those is found by
//    elimination with pivots that are units modulo q;
//  - Phase 3 checks prod s_i = +-det A modulo primes q: det A mod q by
//    Gaussian elimination over GF(q).
//
// Column k takes as pivot the first row not yet used whose entry in column k
// is a unit (not divisible by q).  Every other unused row i subtracts
// f_i = M[i][k] / M[p][k] times the pivot row (no row is moved, so the
// determinant is the sign of the permutation k -> pivot row times the product
// of the pivots).  A column without a unit is left for later ("deferred"):
// in the local form, once every column has been seen, the unused rows and the
// deferred columns hold a square block whose entries are all divisible by q;
// it is divided by q and reduced again modulo q^(e-1).  Its size at each
// level counts the invariant factors divisible by the next power of q.
//
// Products modulo m use Shoup's method: for a multiplier f fixed across a row,
// f' = floor(f 2^w / m) makes f y mod m = f y - floor(y f' / 2^w) m, at most
// one m too large (w = 32 for m < 2^31, 64 for m < 2^62).
//
// Determinants and lockstep local forms (two or more lanes) take one launch per
// column: the launch for column k eliminates
// it and, in the threads that update column k+1, copies that column's new values
// into a compact buffer and finds its first unused unit row (atomicMin).  The
// last of those blocks to finish (a counter, no waiting) takes that row as
// column k+1's pivot, marks it used and stores its inverse, so the next launch
// finds everything it needs; each block then forms the multipliers of its own
// rows from the compact column.  A local form in one lane keeps two launches
// per column (a one-block pivot step that writes every row's multiplier, then
// the update): there every column stays live and the per-block multipliers cost
// more than the pivot step saves (measured at n = 5003: 0.185 s against 0.227 s
// for one local form; four lockstep determinants 0.527 s against 0.418 s fused;
// four lockstep local forms 0.645 s against 0.604 s fused).
#include <algorithm>
#include <vector>

#include "modarith.h"
#include "smf_internal.h"

namespace smf {
namespace {

constexpr int kPivThreads = 256;
constexpr int kUpdThreads = 256;
// rows per update thread (the pivot row's entry is loaded once for them): eight
// for entries of up to 16 bytes, fewer for wider ones to stay in registers
template <typename T, int L>
__host__ __device__ constexpr int upd_rows() {
    return sizeof(T) * L <= 16 ? 8 : sizeof(T) * L <= 32 ? 4 : 2;
}

template <typename T>
struct ModOps;

template <>
struct ModOps<uint32_t> {
    __host__ __device__ static uint32_t shoup(uint32_t f, uint32_t m) {
        return (uint32_t)(((uint64_t)f << 32) / m);
    }
    __device__ static uint32_t mul(uint32_t y, uint32_t f, uint32_t fs, uint32_t m) {
        uint32_t r = f * y - __umulhi(y, fs) * m;
        return r >= m ? r - m : r;
    }
    __device__ static uint32_t mulmod(uint32_t a, uint32_t b, uint32_t m) {
        return (uint32_t)(((uint64_t)a * b) % m);
    }
    // shoup(f, m) from rcp = floor((2^64 - 1) / m): x = f 2^32 < 2^63, and
    // floor(x rcp / 2^64) is floor(x / m) or one less (x (2^64 / m - rcp) / 2^64 < 1/2)
    __device__ static uint32_t shoup_rcp(uint32_t f, uint32_t m, uint64_t rcp) {
        const uint64_t x = (uint64_t)f << 32;
        uint64_t q = __umul64hi(x, rcp);
        if (x - q * m >= m) q++;
        return (uint32_t)q;
    }
};

template <>
struct ModOps<uint64_t> {
    __host__ __device__ static uint64_t shoup(uint64_t f, uint64_t m) {
        return (uint64_t)(((unsigned __int128)f << 64) / m);
    }
    __device__ static uint64_t mul(uint64_t y, uint64_t f, uint64_t fs, uint64_t m) {
        uint64_t r = f * y - __umul64hi(y, fs) * m;
        return r >= m ? r - m : r;
    }
    __device__ static uint64_t mulmod(uint64_t a, uint64_t b, uint64_t m) {
        return (uint64_t)(((unsigned __int128)a * b) % m);
    }
};

// a^-1 mod m for a unit a (extended Euclid on signed 64-bit values, m < 2^62)
__device__ int64_t inv_mod(int64_t a, int64_t m) {
    int64_t r0 = m, r1 = a, t0 = 0, t1 = 1;
    while (r1) {
        const int64_t qq = r0 / r1;
        int64_t x = r0 - qq * r1;
        r0 = r1;
        r1 = x;
        x = t0 - qq * t1;
        t0 = t1;
        t1 = x;
    }
    return t0 < 0 ? t0 + m : t0;
}

// Up to L moduli m_l (units tested modulo the primes q_l | m_l) run in
// lockstep on one matrix whose entries hold L residues side by side: the
// pivot of a column is the first unused row that is a unit modulo every q_l,
// so one column loop serves all of them (Phase 3's primes; Phase 2's prime
// powers of s').
template <typename T, int L>
struct Lanes {
    int n;      // lanes in use (<= L)
    T m[L];
    T q[L];
    uint64_t rcp[L];  // floor((2^64 - 1) / m_l)
};

// A pivot's inverse and a multiplier's Shoup companion in lane l: 32-bit
// lanes (m < 2^31) by 32-bit Euclid and the lane's reciprocal of m, which keep
// 64-bit divisions (emulated on the device) off the column loop's critical
// path; 64-bit lanes as before.
template <typename T, int L>
__device__ __forceinline__ T inv_lane(T a, const Lanes<T, L>& md, int l) {
    if constexpr (sizeof(T) == 4) return inv_mod32(a, md.m[l]);
    else return (T)inv_mod((int64_t)a, (int64_t)md.m[l]);
}
template <typename T, int L>
__device__ __forceinline__ T shoup_lane(T f, const Lanes<T, L>& md, int l) {
    if constexpr (sizeof(T) == 4) return ModOps<uint32_t>::shoup_rcp(f, md.m[l], md.rcp[l]);
    else return ModOps<T>::shoup(f, md.m[l]);
}

// A (int64, row-major, lda) -> M[i][j][l] = A[i][j] mod m_l, canonical.
template <typename T, int L>
__global__ void elim_init_kernel(const int64_t* __restrict__ A, int64_t lda, int64_t n, T* __restrict__ M,
                                 Lanes<T, L> md) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n * n) return;
    const int64_t i = e / n, j = e - i * n;
    const int64_t a = A[i * lda + j];
#pragma unroll
    for (int l = 0; l < L; l++) {
        if (l >= md.n) break;
        const int64_t r = a % (int64_t)md.m[l];
        M[e * L + l] = (T)(r < 0 ? r + (int64_t)md.m[l] : r);
    }
}

template <typename T, int L>
__device__ __forceinline__ bool joint_unit(const T* __restrict__ x, const Lanes<T, L>& md) {
    bool u = true;
#pragma unroll
    for (int l = 0; l < L; l++)
        if (l < md.n) u &= x[l] % md.q[l] != 0;
    return u;
}

// One column's pivot: the first unused row that is a unit in every lane, then
// the multipliers of every other unused row (0 for used rows).
template <typename T, int L>
__global__ void __launch_bounds__(kPivThreads)
elim_pivot_kernel(T* __restrict__ M, int64_t n, int64_t k, Lanes<T, L> md, int field, int* __restrict__ used,
                  int64_t* __restrict__ pivrow, T* __restrict__ pivval, T* __restrict__ f, T* __restrict__ fs,
                  int* __restrict__ dead) {
    pdl_wait();
    __shared__ int64_t best;
    __shared__ T sinv[L], sinvs[L];
    if (threadIdx.x == 0) best = n;
    __syncthreads();
    const bool stop = *dead != 0;
    if (!stop) {
        // every row of the thread's stride is tested (independent loads), the first kept
        int64_t mine = n;
#pragma unroll 4
        for (int64_t i = threadIdx.x; i < n; i += kPivThreads)
            if (!used[i] && joint_unit<T, L>(M + (i * n + k) * L, md) && i < mine) mine = i;
        if (mine < n) atomicMin((unsigned long long*)&best, (unsigned long long)mine);
    }
    __syncthreads();
    const int64_t p = best;
    if (stop || p >= n) {
        if (threadIdx.x == 0) {
            pivrow[k] = -1;
            if (field) *dead = 1;  // the determinant: a column without a pivot means det = 0 (in some lane)
        }
        for (int64_t i = threadIdx.x; i < n * L; i += kPivThreads) f[i] = 0;
        pdl_trigger();
        return;
    }
    if (threadIdx.x < md.n) {
        const int l = threadIdx.x;
        const T pv = M[(p * n + k) * L + l];
        pivval[k * L + l] = pv;
        sinv[l] = inv_lane<T, L>(pv, md, l);
        sinvs[l] = shoup_lane<T, L>(sinv[l], md, l);
    }
    if (threadIdx.x == 0) {
        used[p] = 1;
        pivrow[k] = p;
    }
    __syncthreads();
    for (int64_t i = threadIdx.x; i < n; i += kPivThreads) {
        const bool live = !used[i];
#pragma unroll
        for (int l = 0; l < L; l++) {
            if (l >= md.n) break;
            T fi = 0;
            if (live) fi = ModOps<T>::mul(M[(i * n + k) * L + l], sinv[l], sinvs[l], md.m[l]);
            f[i * L + l] = fi;
            fs[i * L + l] = fi ? shoup_lane<T, L>(fi, md, l) : 0;
        }
    }
    pdl_trigger();
}

// The L residues of one entry, loaded and stored as one vector when they fill
// 8 or 16 bytes.
template <typename T, int L>
struct Entry {
    T v[L];
    __device__ __forceinline__ void load(const T* p) {
        if constexpr (sizeof(T) * L == 16) {
            const uint4 u = *reinterpret_cast<const uint4*>(p);
            memcpy(v, &u, 16);
        } else if constexpr (sizeof(T) * L == 8) {
            const uint2 u = *reinterpret_cast<const uint2*>(p);
            memcpy(v, &u, 8);
        } else {
#pragma unroll
            for (int l = 0; l < L; l++) v[l] = p[l];
        }
    }
    __device__ __forceinline__ void store(T* p) const {
        if constexpr (sizeof(T) * L == 16) {
            uint4 u;
            memcpy(&u, v, 16);
            *reinterpret_cast<uint4*>(p) = u;
        } else if constexpr (sizeof(T) * L == 8) {
            uint2 u;
            memcpy(&u, v, 8);
            *reinterpret_cast<uint2*>(p) = u;
        } else {
#pragma unroll
            for (int l = 0; l < L; l++) p[l] = v[l];
        }
    }
};

// Row i -= f_i * row p over the live columns (after k, or every column not yet
// a pivot column), every lane.  A thread takes one column and kUpdRows rows:
// it loads every row's multipliers and entries first, then updates them, so
// the loads of the rows overlap.
template <typename T, int L>
__global__ void __launch_bounds__(kUpdThreads)
elim_update_kernel(T* __restrict__ M, int64_t n, int64_t k, int64_t c0, Lanes<T, L> md,
                   const int64_t* __restrict__ pivrow, const T* __restrict__ f, const T* __restrict__ fs,
                   const int64_t* __restrict__ colpiv) {
    pdl_wait();
    const int64_t p = pivrow[k];
    const int64_t j = c0 + (int64_t)blockIdx.x * kUpdThreads + threadIdx.x;
    // colpiv (local form): columns that already have a pivot are never read again
    if (p >= 0 && j < n && j != k && !(colpiv && j < k && colpiv[j] >= 0)) {
        Entry<T, L> y;
        y.load(M + (p * n + j) * L);
        constexpr int kUpdRows = upd_rows<T, L>();
        const int64_t r0 = (int64_t)blockIdx.y * kUpdRows;
        T fi[kUpdRows][L];
        bool live[kUpdRows];
#pragma unroll
        for (int rr = 0; rr < kUpdRows; rr++) {
            const int64_t i = r0 + rr;
            live[rr] = false;
#pragma unroll
            for (int l = 0; l < L; l++) {
                fi[rr][l] = (i < n && l < md.n) ? f[i * L + l] : 0;
                live[rr] |= fi[rr][l] != 0;
            }
        }
        Entry<T, L> x[kUpdRows];
#pragma unroll
        for (int rr = 0; rr < kUpdRows; rr++)
            if (live[rr]) x[rr].load(M + ((r0 + rr) * n + j) * L);
#pragma unroll
        for (int rr = 0; rr < kUpdRows; rr++) {
            if (!live[rr]) continue;
            const int64_t i = r0 + rr;
#pragma unroll
            for (int l = 0; l < L; l++) {
                if (l >= md.n) break;
                const T t = ModOps<T>::mul(y.v[l], fi[rr][l], fs[i * L + l], md.m[l]);
                const T v = x[rr].v[l];
                x[rr].v[l] = v >= t ? v - t : v + (md.m[l] - t);
            }
            x[rr].store(M + (i * n + j) * L);
        }
    }
    pdl_trigger();
}

constexpr int kCountGroup = 32;  // blocks per first-level counter of the last-block count
constexpr int kStepRows = 8;  // rows per block of the column step (many blocks: the update is latency-bound)

// Column k: row i -= f_i * row p over the live columns (after k for a
// determinant; every column without a pivot yet for the local form), every
// lane, with f_i = M[i][k] / M[p][k] formed per block from the compact copy of
// column k; and column k+1's pivot search (see the top of this file).  A thread
// takes one column and kStepRows rows in groups of upd_rows, loading a group's
// entries before updating them.  k = -1 only searches column 0.
template <typename T, int L>
__global__ void __launch_bounds__(kUpdThreads)
elim_step_kernel(T* __restrict__ M, int64_t n, int64_t k, int64_t c0, Lanes<T, L> md, int field,
                 int* __restrict__ used, int64_t* __restrict__ pivrow, T* __restrict__ pivval, T* __restrict__ pinv,
                 T* __restrict__ pinvs, T* __restrict__ colbuf, unsigned* __restrict__ cand,
                 unsigned* __restrict__ counter, int* __restrict__ dead) {
    pdl_wait();
    constexpr int R = upd_rows<T, L>();
    static_assert(kStepRows % R == 0, "whole row groups");
    __shared__ T sf[kStepRows][L], sfs[kStepRows][L];
    __shared__ int s_last;
    const int64_t r0 = (int64_t)blockIdx.y * kStepRows;
    const bool stop = *dead != 0;  // a determinant that is already 0 in some lane
    const int64_t p = k >= 0 && !stop ? pivrow[k] : -1;
    const T* cur = colbuf + (size_t)(k & 1) * n * L;     // column k, copied by the launch before
    T* nxt = colbuf + (size_t)((k + 1) & 1) * n * L;     // column k+1, copied here
    if (p >= 0) {
        for (int t = threadIdx.x; t < kStepRows * L; t += kUpdThreads) {
            const int rr = t / L, l = t % L;
            const int64_t i = r0 + rr;
            T fi = 0;
            if (l < md.n && i < n && i != p && !used[i])
                fi = ModOps<T>::mul(cur[i * L + l], pinv[k * L + l], pinvs[k * L + l], md.m[l]);
            sf[rr][l] = fi;
            if constexpr (sizeof(T) == 4) sfs[rr][l] = fi ? ModOps<T>::shoup_rcp(fi, md.m[l], md.rcp[l]) : 0;
            else sfs[rr][l] = fi ? ModOps<T>::shoup(fi, md.m[l]) : 0;
        }
    }
    __syncthreads();
    const int64_t j = c0 + (int64_t)blockIdx.x * kUpdThreads + threadIdx.x;
    // local form: columns that already have a pivot are never read again
    const bool col_live = p >= 0 && j < n && j != k && !(!field && j < k && pivrow[j] >= 0);
    const bool search = !stop && k + 1 < n && j == k + 1;  // this thread copies column k+1 and searches it
    if (col_live || search) {
        Entry<T, L> y;
        if (col_live) y.load(M + (p * n + j) * L);
        unsigned best = 0xFFFFFFFFu;
        for (int g = 0; g < kStepRows; g += R) {
            bool live[R];
            Entry<T, L> x[R];
#pragma unroll
            for (int rr = 0; rr < R; rr++) {
                const int64_t i = r0 + g + rr;
                live[rr] = false;
                if (col_live && i < n) {
#pragma unroll
                    for (int l = 0; l < L; l++)
                        if (l < md.n) live[rr] |= sf[g + rr][l] != 0;
                }
            }
#pragma unroll
            for (int rr = 0; rr < R; rr++)
                if (live[rr] || (search && r0 + g + rr < n)) x[rr].load(M + ((r0 + g + rr) * n + j) * L);
#pragma unroll
            for (int rr = 0; rr < R; rr++) {
                const int64_t i = r0 + g + rr;
                if (live[rr]) {
#pragma unroll
                    for (int l = 0; l < L; l++) {
                        if (l >= md.n) break;
                        const T t = ModOps<T>::mul(y.v[l], sf[g + rr][l], sfs[g + rr][l], md.m[l]);
                        const T v = x[rr].v[l];
                        x[rr].v[l] = v >= t ? v - t : v + (md.m[l] - t);
                    }
                    x[rr].store(M + (i * n + j) * L);
                }
                if (search && i < n) {
                    x[rr].store(nxt + i * L);
                    if (i != p && !used[i] && joint_unit<T, L>(x[rr].v, md) && (unsigned)i < best) best = (unsigned)i;
                }
            }
        }
        // (the first unit row usually comes from an early block: skip the atomic when beaten)
        if (best != 0xFFFFFFFFu && best < *(volatile unsigned*)(cand + (k + 1))) atomicMin(cand + (k + 1), best);
    }
    // the last block over column k+1 settles its pivot; blocks are counted in groups
    // of kCountGroup (counter[1 + g]) and the groups in counter[0], so that no
    // address takes more than a few tens of atomics
    if (!stop && k + 1 < n && (k + 1 - c0) / kUpdThreads == (int64_t)blockIdx.x) {
        __threadfence();
        __syncthreads();
        if (threadIdx.x == 0) {
            const unsigned g = blockIdx.y / kCountGroup, ng = (gridDim.y + kCountGroup - 1) / kCountGroup;
            const unsigned in_g = min((unsigned)kCountGroup, gridDim.y - g * kCountGroup);
            s_last = 0;
            if (atomicAdd(counter + 1 + g, 1u) == in_g - 1) {
                counter[1 + g] = 0u;  // for the next launch
                __threadfence();
                s_last = atomicAdd(counter, 1u) == ng - 1;
            }
        }
        __syncthreads();
        if (s_last) {
            __threadfence();
            const unsigned q = atomicAdd(cand + (k + 1), 0u);
            if (q < (unsigned)n) {
                if (threadIdx.x < md.n) {
                    const int l = threadIdx.x;
                    const T pv = __ldcg(nxt + (size_t)q * L + l);
                    pivval[(k + 1) * L + l] = pv;
                    const T iv = inv_lane<T, L>(pv, md, l);
                    pinv[(k + 1) * L + l] = iv;
                    pinvs[(k + 1) * L + l] = shoup_lane<T, L>(iv, md, l);
                }
                if (threadIdx.x == 0) {
                    used[q] = 1;
                    pivrow[k + 1] = q;
                }
            } else if (threadIdx.x == 0) {
                pivrow[k + 1] = -1;
                if (field) *dead = 1;  // the determinant: a column without a pivot means det = 0 (in some lane)
            }
            if (threadIdx.x == 0) *counter = 0u;  // for the next launch
        }
    }
    pdl_trigger();
}

// out[a][b] = M[rows[a]][cols[b]][lane] / div (exact), a square block of size nb, one lane.
template <typename T, int L>
__global__ void elim_gather_kernel(const T* __restrict__ M, int64_t n, const int64_t* __restrict__ rows,
                                   const int64_t* __restrict__ cols, int64_t nb, int lane, T div,
                                   T* __restrict__ out) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= nb * nb) return;
    const int64_t a = e / nb, b = e - a * nb;
    out[e] = M[(rows[a] * n + cols[b]) * L + lane] / div;
}

// Scratch of an elimination of an n x n matrix with L lanes of type T.
// (stream-ordered: freeing them does not synchronise the device)
template <typename T, int L>
struct ElimBufs {
    StreamBuf M, used, pivrow, pivval, pinv, pinvs, colbuf, cand, counter, dead, f, fs;
    // the last-block count: one total and one per group of kCountGroup row blocks
    static size_t counters(int64_t n) {
        return 1 + (size_t)(((n + kStepRows - 1) / kStepRows + kCountGroup - 1) / kCountGroup);
    }
    cudaError_t alloc(int64_t n, cudaStream_t s) {
        cudaError_t e;
        const size_t nl = sizeof(T) * L * (size_t)n;
        if ((e = M.alloc(nl * (size_t)n, s)) || (e = used.alloc(sizeof(int) * (size_t)n, s)) ||
            (e = pivrow.alloc(sizeof(int64_t) * (size_t)n, s)) || (e = pivval.alloc(nl, s)) ||
            (e = pinv.alloc(nl, s)) || (e = pinvs.alloc(nl, s)) || (e = colbuf.alloc(2 * nl, s)) ||
            (e = cand.alloc(sizeof(unsigned) * (size_t)(n + 1), s)) ||
            (e = counter.alloc(sizeof(unsigned) * counters(n), s)) || (e = f.alloc(nl, s)) || (e = fs.alloc(nl, s)) ||
            (e = dead.alloc(sizeof(int), s)))
            return e;
        return cudaSuccess;
    }
};

// The column loop on the n x n matrix in `M`: each column's pivot row (-1 for a
// deferred column) and its values in every lane.  field: a determinant (only
// the columns after k are updated, a column without a pivot ends it); else the
// local form (every column but k stays current: deferred columns are kept).
template <typename T, int L>
cudaError_t elim_columns(ElimBufs<T, L>& b, T* M, int64_t n, const Lanes<T, L>& md, bool field,
                         std::vector<int64_t>* pivrow, std::vector<T>* pivval, cudaStream_t s) {
    cudaError_t e;
    if ((e = cudaMemsetAsync(b.used.p, 0, sizeof(int) * (size_t)n, s)) ||
        (e = cudaMemsetAsync(b.dead.p, 0, sizeof(int), s)) ||
        (e = cudaMemsetAsync(b.counter.p, 0, sizeof(unsigned) * ElimBufs<T, L>::counters(n), s)) ||
        (e = cudaMemsetAsync(b.cand.p, 0xFF, sizeof(unsigned) * (size_t)(n + 1), s)) ||
        (e = cudaMemsetAsync(b.pivrow.p, 0xFF, sizeof(int64_t) * (size_t)n, s)))
        return e;
    const bool fused = field || L > 1;
    for (int64_t k = 0; !fused && k < n; k++) {  // a one-lane local form: pivot step, then update
        e = launch_pdl(elim_pivot_kernel<T, L>, dim3(1), dim3(kPivThreads), 0, s, M, n, k, md, 0, (int*)b.used.p,
                       (int64_t*)b.pivrow.p, (T*)b.pivval.p, (T*)b.f.p, (T*)b.fs.p, (int*)b.dead.p);
        if (e) return e;
        constexpr int R = upd_rows<T, L>();
        const dim3 grid((unsigned)((n + kUpdThreads - 1) / kUpdThreads), (unsigned)((n + R - 1) / R));
        e = launch_pdl(elim_update_kernel<T, L>, grid, dim3(kUpdThreads), 0, s, M, n, k, (int64_t)0, md,
                       (const int64_t*)b.pivrow.p, (const T*)b.f.p, (const T*)b.fs.p, (const int64_t*)b.pivrow.p);
        if (e) return e;
    }
    // one launch per column (k = -1 only searches column 0)
    for (int64_t k = -1; fused && k < n; k++) {
        const int64_t c0 = field ? k + 1 : 0;
        if (c0 >= n) continue;
        const dim3 grid((unsigned)((n - c0 + kUpdThreads - 1) / kUpdThreads), (unsigned)((n + kStepRows - 1) / kStepRows));
        e = launch_pdl(elim_step_kernel<T, L>, grid, dim3(kUpdThreads), 0, s, M, n, k, c0, md, field ? 1 : 0,
                       (int*)b.used.p, (int64_t*)b.pivrow.p, (T*)b.pivval.p, (T*)b.pinv.p, (T*)b.pinvs.p,
                       (T*)b.colbuf.p, (unsigned*)b.cand.p, (unsigned*)b.counter.p, (int*)b.dead.p);
        if (e) return e;
    }
    pivrow->resize(n);
    pivval->resize((size_t)n * L);
    if ((e = cudaMemcpyAsync(pivrow->data(), b.pivrow.p, sizeof(int64_t) * n, cudaMemcpyDeviceToHost, s)) ||
        (e = cudaMemcpyAsync(pivval->data(), b.pivval.p, sizeof(T) * L * n, cudaMemcpyDeviceToHost, s)))
        return e;
    return cudaStreamSynchronize(s);
}

// ---------------------------------------------------------------------------
// Blocked elimination (32-bit lanes).  The column loop above reads and writes
// the whole trailing block once per column: about n^3/3 entry updates of
// 2 x 16 bytes for four lanes, which bounds it by memory.  Here panels of
// kPanel columns are eliminated first on the panel alone (per column: the
// pivot search, then every unused row's multiplier and the update of the
// panel's other live columns), the pivot rows' trailing parts are brought up
// to date within the panel (U), and the trailing columns take the panel's
// kPanel pivots in one pass: M[i][j] -= sum_t F[i][t] U[t][j].  The same
// pivots, the same multipliers and the same values as one column at a time;
// the trailing block is read and written once per panel.
//
// Two kinds (template flag LOC):
//  - a determinant (LOC = false): a column without a pivot ends the call (the
//    caller falls back to the column loop); the trailing columns are [c1, n);
//  - a local Smith form (LOC = true): a column without a unit pivot is
//    deferred and stays live, as in the column loop.  The deferred columns are
//    listed in increasing order (dcols[0 .. *ndef)); *ndef0 is their count
//    before the current panel.  The panel's own deferred columns are updated
//    within the panel by its later pivots; the trailing columns of the panel
//    are the earlier ones, dcols[0 .. *ndef0), followed by [c1, n).  A panel
//    position without a pivot contributes U = 0.
constexpr int kPanel = 16;
// Matrices below the context's thresholds (elim_panel_min_n, 2560, for
// determinants; elim_local_panel_min_n, 1536, for local forms; unless
// smf_set_elim_panels changes them) keep the column loop: its one launch per
// column against the panels' two per column plus two per panel (measured
// four-lane determinants: n = 2003 0.045 s by columns, 0.053 s blocked;
// n = 5003 0.416 against 0.205 s).

// trailing column x of a panel: an earlier deferred column, then [c1, n)
__device__ __forceinline__ int64_t trail_col(int64_t x, int64_t nd0, const int64_t* __restrict__ dcols, int64_t c1) {
    return x < nd0 ? dcols[x] : c1 + (x - nd0);
}

// The first unused row whose entry in column c is a unit in every lane
// (atomicMin of each block's smallest candidate).  A local form's first column
// of a panel also records the count of deferred columns before the panel.
template <int L, bool LOC>
__global__ void __launch_bounds__(256)
bd_search_kernel(const uint32_t* __restrict__ M, int64_t n, int64_t c, int64_t c0, Lanes<uint32_t, L> md,
                 const int* __restrict__ used, unsigned* __restrict__ cand, const int* __restrict__ dead,
                 const int* __restrict__ ndef, int* __restrict__ ndef0) {
    pdl_wait();
    pdl_trigger();
    if (*dead) return;
    if (LOC && c == c0 && blockIdx.x == 0 && threadIdx.x == 0) *ndef0 = *ndef;
    __shared__ unsigned wmin[8];
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    unsigned v = 0xFFFFFFFFu;
    if (i < n && !used[i] && joint_unit<uint32_t, L>(M + (i * n + c) * L, md)) v = (unsigned)i;
#pragma unroll
    for (int o = 16; o; o >>= 1) v = min(v, __shfl_xor_sync(0xffffffffu, v, o));
    if ((threadIdx.x & 31) == 0) wmin[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned b = wmin[0];
        for (int w = 1; w < (int)(blockDim.x >> 5); w++) b = min(b, wmin[w]);
        if (b != 0xFFFFFFFFu) atomicMin(cand + c, b);
    }
}

// Column c (panel [c0, c1)): its pivot p = cand[c], the pivot's inverse in
// every lane, each unused row's multiplier f = M[i][c] / M[p][c] with its
// Shoup companion (kept in F and Fs at panel position c - c0), and
// M[i][j] -= f M[p][j] for the panel's other live columns: j in (c, c1) and,
// in a local form, the panel's deferred columns before c.  No pivot: a
// determinant's call falls back to the column loop; a local form defers c.
template <int L, bool LOC>
__global__ void __launch_bounds__(256)
bd_panel_kernel(uint32_t* __restrict__ M, int64_t n, int64_t c, int64_t c0, int64_t c1, Lanes<uint32_t, L> md,
                int* __restrict__ used, const unsigned* __restrict__ cand, int64_t* __restrict__ pivrow,
                uint32_t* __restrict__ pivval, uint32_t* __restrict__ F, uint32_t* __restrict__ Fs,
                int* __restrict__ dead, int64_t* __restrict__ dcols, int* __restrict__ ndef) {
    pdl_wait();
    pdl_trigger();
    if (*dead) return;
    const unsigned pu = cand[c];
    if (pu >= (unsigned)n) {
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            if constexpr (LOC) {  // one writer: the list stays in column order
                const int d = *ndef;
                dcols[d] = c;
                *ndef = d + 1;
            } else {
                *dead = 1;
            }
        }
        return;
    }
    const int64_t p = pu;
    const uint32_t* prow = M + (p * n) * L;
    uint32_t inv[L];
#pragma unroll
    for (int l = 0; l < L; l++)
        inv[l] = l < md.n ? inv_mod32(prow[c * L + l], md.m[l]) : 0u;
    if (blockIdx.x == 0 && threadIdx.x == 0) {  // every other thread skips row p by its index
        pivrow[c] = p;
#pragma unroll
        for (int l = 0; l < L; l++) pivval[c * L + l] = prow[c * L + l];
        used[p] = 1;
    }
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n || i == p || used[i]) return;
    uint32_t* row = M + (i * n) * L;
    uint32_t f[L], fs[L];
#pragma unroll
    for (int l = 0; l < L; l++) {
        f[l] = fs[l] = 0;
        if (l < md.n) {
            f[l] = mulmod32_rcp(row[c * L + l], inv[l], md.m[l], md.rcp[l]);
            fs[l] = ModOps<uint32_t>::shoup_rcp(f[l], md.m[l], md.rcp[l]);
        }
        F[(i * kPanel + (c - c0)) * L + l] = f[l];
        Fs[(i * kPanel + (c - c0)) * L + l] = fs[l];
    }
    // (columns before c in the panel: only a local form's deferred ones, whose
    // pivrow was settled by an earlier launch, are still live)
    for (int64_t j = LOC ? c0 : c + 1; j < c1; j++) {
        if (LOC && j <= c && (j == c || pivrow[j] >= 0)) continue;
#pragma unroll
        for (int l = 0; l < L; l++) {
            if (l >= md.n) break;
            const uint32_t m = md.m[l];
            const uint32_t t = ModOps<uint32_t>::mul(prow[j * L + l], f[l], fs[l], m);
            const uint32_t a = row[j * L + l];
            row[j * L + l] = a >= t ? a - t : a + m - t;
        }
    }
}

// The panel's pivot rows on the trailing columns (a determinant: [c1, n); a
// local form: also the deferred columns before the panel): row p_t takes the
// panel's earlier pivots' eliminations, U_t = M[p_t] - sum_(t' < t) F[p_t][t'] U_t'
// (one thread per column, the panel's rows in registers), written back in
// place.  Threads beyond the count of trailing columns return.
template <int L, bool LOC>
__global__ void __launch_bounds__(128)
bd_urows_kernel(uint32_t* __restrict__ M, int64_t n, int64_t c0, int w, int64_t c1, Lanes<uint32_t, L> md,
                const int64_t* __restrict__ pivrow, const uint32_t* __restrict__ F, const uint32_t* __restrict__ Fs,
                const int* __restrict__ dead, const int64_t* __restrict__ dcols, const int* __restrict__ ndef0) {
    pdl_wait();
    pdl_trigger();
    if (*dead) return;
    const int64_t nd0 = LOC ? (int64_t)*ndef0 : 0;
    const int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= nd0 + (n - c1)) return;
    const int64_t j = trail_col(x, nd0, dcols, c1);
    uint32_t U[kPanel][L];
#pragma unroll
    for (int t = 0; t < kPanel; t++) {
        if (t >= w) break;
        const int64_t p = pivrow[c0 + t];
#pragma unroll
        for (int l = 0; l < L; l++) U[t][l] = 0;
        if (LOC && p < 0) continue;  // a deferred panel column: no elimination
        uint32_t* e = M + (p * n + j) * L;
#pragma unroll
        for (int l = 0; l < L; l++) {
            if (l >= md.n) continue;
            const uint32_t m = md.m[l];
            uint32_t u = e[l];
#pragma unroll
            for (int t2 = 0; t2 < kPanel; t2++) {
                if (t2 >= t) break;
                const size_t fi = ((size_t)p * kPanel + t2) * L + l;
                const uint32_t xx = ModOps<uint32_t>::mul(U[t2][l], F[fi], Fs[fi], m);
                u = u >= xx ? u - xx : u + m - xx;
            }
            U[t][l] = u;
            e[l] = u;
        }
    }
}

// The trailing block: every row still unused (after the panel) and every
// trailing column takes M[i][j] -= sum_t F[i][t] U_t[j].  A block covers 32
// rows by 64 trailing columns: the panel's U rows over its columns and its
// rows' multipliers in shared memory, eight entries per thread.
constexpr int kTrailRows = 32, kTrailCols = 64;
template <int L, bool LOC>
__global__ void __launch_bounds__(256)
bd_trail_kernel(uint32_t* __restrict__ M, int64_t n, int64_t c0, int w, int64_t c1, Lanes<uint32_t, L> md,
                const int* __restrict__ used, const int64_t* __restrict__ pivrow, const uint32_t* __restrict__ F,
                const uint32_t* __restrict__ Fs, const int* __restrict__ dead, const int64_t* __restrict__ dcols,
                const int* __restrict__ ndef0) {
    pdl_wait();
    pdl_trigger();
    if (*dead) return;
    const int64_t nd0 = LOC ? (int64_t)*ndef0 : 0;
    const int64_t ncols = nd0 + (n - c1);
    const int64_t x0 = (int64_t)blockIdx.x * kTrailCols;
    if (x0 >= ncols) return;  // (the grid bounds a local form's deferred count by c0)
    __shared__ uint32_t Us[kPanel][kTrailCols][L];
    __shared__ uint32_t Fsh[kTrailRows][kPanel][L], Fssh[kTrailRows][kPanel][L];
    __shared__ int live[kTrailRows];
    __shared__ int any;
    const int64_t r0 = (int64_t)blockIdx.y * kTrailRows;
    if (threadIdx.x == 0) any = 0;
    __syncthreads();
    if (threadIdx.x < kTrailRows) {
        const int64_t i = r0 + threadIdx.x;
        live[threadIdx.x] = i < n && !used[i];
        if (live[threadIdx.x]) any = 1;
    }
    __syncthreads();
    if (!any) return;  // every row of the tile is a pivot row already
    for (int x = threadIdx.x; x < kPanel * kTrailCols; x += blockDim.x) {
        const int t = x / kTrailCols, jj = x % kTrailCols;
        const int64_t xx = x0 + jj;
        const int64_t p = t < w ? pivrow[c0 + t] : -1;
        const bool ok = t < w && xx < ncols && p >= 0;
        const int64_t j = ok ? trail_col(xx, nd0, dcols, c1) : 0;
#pragma unroll
        for (int l = 0; l < L; l++) Us[t][jj][l] = ok ? M[(p * n + j) * L + l] : 0u;
    }
    for (int x = threadIdx.x; x < kTrailRows * kPanel; x += blockDim.x) {
        const int rr = x / kPanel, t = x % kPanel;
        const int64_t i = r0 + rr;
#pragma unroll
        for (int l = 0; l < L; l++) {
            const bool ok = t < w && live[rr];
            Fsh[rr][t][l] = ok ? F[((size_t)i * kPanel + t) * L + l] : 0u;
            Fssh[rr][t][l] = ok ? Fs[((size_t)i * kPanel + t) * L + l] : 0u;
        }
    }
    __syncthreads();
    const int jj = threadIdx.x % kTrailCols;
    const int64_t xx = x0 + jj;
    if (xx >= ncols) return;
    const int64_t j = trail_col(xx, nd0, dcols, c1);
    for (int rr = threadIdx.x / kTrailCols; rr < kTrailRows; rr += blockDim.x / kTrailCols) {
        if (!live[rr]) continue;
        uint32_t* e = M + ((r0 + rr) * n + j) * L;
        uint32_t v[L];
#pragma unroll
        for (int l = 0; l < L; l++) v[l] = e[l];
#pragma unroll
        for (int t = 0; t < kPanel; t++) {
            if (t >= w) break;
#pragma unroll
            for (int l = 0; l < L; l++) {
                if (l >= md.n) break;
                const uint32_t m = md.m[l];
                const uint32_t y = ModOps<uint32_t>::mul(Us[t][jj][l], Fsh[rr][t][l], Fssh[rr][t][l], m);
                v[l] = v[l] >= y ? v[l] - y : v[l] + m - y;
            }
        }
#pragma unroll
        for (int l = 0; l < L; l++) e[l] = v[l];
    }
}

// The blocked column loop on the n x n matrix in M (32-bit lanes): each
// column's pivot row (-1 for a local form's deferred column) and its values,
// as elim_columns gives them.  A determinant's *fallback: a column without a
// pivot that is a unit in every lane (the caller then takes the column loop
// above); a local form never falls back.
template <int L, bool LOC>
cudaError_t elim_blocked(ElimBufs<uint32_t, L>& b, uint32_t* M, int64_t n, const Lanes<uint32_t, L>& md,
                         std::vector<int64_t>* pivrow, std::vector<uint32_t>* pivval, bool* fallback, cudaStream_t s) {
    cudaError_t e;
    StreamBuf F, Fs, dl, nd;
    const size_t fb = sizeof(uint32_t) * (size_t)n * kPanel * L;
    if ((e = F.alloc(fb, s)) || (e = Fs.alloc(fb, s))) return e;
    if (LOC) {
        // a deferred panel position leaves F stale; zeros keep every read defined
        if ((e = dl.alloc(sizeof(int64_t) * (size_t)n, s)) || (e = nd.alloc(2 * sizeof(int), s)) ||
            (e = cudaMemsetAsync(nd.p, 0, 2 * sizeof(int), s)) || (e = cudaMemsetAsync(F.p, 0, fb, s)) ||
            (e = cudaMemsetAsync(Fs.p, 0, fb, s)))
            return e;
    }
    if ((e = cudaMemsetAsync(b.used.p, 0, sizeof(int) * (size_t)n, s)) ||
        (e = cudaMemsetAsync(b.dead.p, 0, sizeof(int), s)) ||
        (e = cudaMemsetAsync(b.cand.p, 0xFF, sizeof(unsigned) * (size_t)(n + 1), s)) ||
        (e = cudaMemsetAsync(b.pivrow.p, 0xFF, sizeof(int64_t) * (size_t)n, s)))
        return e;
    int* used = (int*)b.used.p;
    int* dead = (int*)b.dead.p;
    unsigned* cand = (unsigned*)b.cand.p;
    int64_t* pr = (int64_t*)b.pivrow.p;
    uint32_t* pv = (uint32_t*)b.pivval.p;
    int64_t* dcols = LOC ? (int64_t*)dl.p : nullptr;
    int* ndef = LOC ? (int*)nd.p : nullptr;  // [0]: deferred so far, [1]: before the current panel
    int* ndef0 = LOC ? (int*)nd.p + 1 : nullptr;
    const unsigned rblocks = (unsigned)((n + 255) / 256);
    for (int64_t c0 = 0; c0 < n; c0 += kPanel) {
        const int64_t c1 = std::min<int64_t>(n, c0 + kPanel);
        const int w = (int)(c1 - c0);
        for (int64_t c = c0; c < c1; c++) {
            if ((e = launch_pdl(bd_search_kernel<L, LOC>, dim3(rblocks), dim3(256), 0, s, (const uint32_t*)M, n, c, c0,
                                md, (const int*)used, cand, (const int*)dead, (const int*)ndef, ndef0)) ||
                (e = launch_pdl(bd_panel_kernel<L, LOC>, dim3(rblocks), dim3(256), 0, s, M, n, c, c0, c1, md, used,
                                (const unsigned*)cand, pr, pv, (uint32_t*)F.p, (uint32_t*)Fs.p, dead, dcols, ndef)))
                return e;
        }
        if (!LOC && c1 >= n) break;
        // trailing columns: at most c0 deferred ones (a local form) and [c1, n)
        const int64_t rest = (LOC ? c0 : 0) + (n - c1);
        if (rest == 0) continue;
        if ((e = launch_pdl(bd_urows_kernel<L, LOC>, dim3((unsigned)((rest + 127) / 128)), dim3(128), 0, s, M, n, c0,
                            w, c1, md, (const int64_t*)pr, (const uint32_t*)F.p, (const uint32_t*)Fs.p,
                            (const int*)dead, (const int64_t*)dcols, (const int*)ndef0)))
            return e;
        const dim3 grid((unsigned)((rest + kTrailCols - 1) / kTrailCols), (unsigned)((n + kTrailRows - 1) / kTrailRows));
        if ((e = launch_pdl(bd_trail_kernel<L, LOC>, grid, dim3(256), 0, s, M, n, c0, w, c1, md, (const int*)used,
                            (const int64_t*)pr, (const uint32_t*)F.p, (const uint32_t*)Fs.p, (const int*)dead,
                            (const int64_t*)dcols, (const int*)ndef0)))
            return e;
    }
    int dead_h = 0;
    pivrow->resize(n);
    pivval->resize((size_t)n * L);
    if ((e = cudaMemcpyAsync(&dead_h, dead, sizeof(int), cudaMemcpyDeviceToHost, s)) ||
        (e = cudaMemcpyAsync(pivrow->data(), pr, sizeof(int64_t) * n, cudaMemcpyDeviceToHost, s)) ||
        (e = cudaMemcpyAsync(pivval->data(), pv, sizeof(uint32_t) * L * n, cudaMemcpyDeviceToHost, s)) ||
        (e = cudaStreamSynchronize(s)))
        return e;
    *fallback = dead_h != 0;
    return cudaSuccess;
}

// The column loop of a local form (every column but k stays current), by
// panels when the entries are 32-bit and the matrix has at least
// ctx->elim_local_panel_min_n columns.
template <typename T, int L>
cudaError_t elim_local(smf_ctx* ctx, ElimBufs<T, L>& b, T* M, int64_t n, const Lanes<T, L>& md,
                       std::vector<int64_t>* pivrow, std::vector<T>* pivval, cudaStream_t s) {
    if constexpr (sizeof(T) == 4) {
        if (n >= ctx->elim_local_panel_min_n) {
            bool fallback = false;
            return elim_blocked<L, true>(b, M, n, md, pivrow, pivval, &fallback, s);
        }
    }
    return elim_columns<T, L>(b, M, n, md, false, pivrow, pivval, s);
}

uint64_t mulmod_host(uint64_t a, uint64_t b, uint64_t m) { return (uint64_t)((unsigned __int128)a * b % m); }

int elim_fail(smf_ctx* ctx, const char* what, cudaError_t e) {
    cudaGetLastError();
    ctx->err = std::string(what) + ": " + cudaGetErrorString(e);
    return e == cudaErrorMemoryAllocation ? SMF_E_NOMEM : SMF_E_CUDA;
}

// det A mod q_l for nq <= L primes in one column loop.  A column without a
// pivot that is nonzero modulo every prime sends the call back to one prime
// at a time (then such a column means det = 0 for that prime).
template <typename T, int L>
int det_lanes(smf_ctx* ctx, const int64_t* A, int64_t lda, int64_t n, const uint64_t* q, int nq, uint64_t* det,
              cudaStream_t s) {
    if (n == 0) {
        for (int l = 0; l < nq; l++) det[l] = 1 % q[l];
        return SMF_OK;
    }
    Lanes<T, L> md{};
    md.n = nq;
    for (int l = 0; l < nq; l++) {
        md.m[l] = md.q[l] = (T)q[l];
        md.rcp[l] = UINT64_MAX / (uint64_t)q[l];
    }
    ElimBufs<T, L> b;
    cudaError_t e = b.alloc(n, s);
    if (e) return elim_fail(ctx, "det_mod: device allocation", e);
    T* M = (T*)b.M.p;
    elim_init_kernel<T, L><<<(unsigned)((n * n + 255) / 256), 256, 0, s>>>(A, lda, n, M, md);
    std::vector<int64_t> pr;
    std::vector<T> pv;
    if ((e = cudaGetLastError())) return elim_fail(ctx, "det_mod", e);
    bool blocked = false;
    if constexpr (sizeof(T) == 4) {
        // 31-bit primes and a matrix of several panels: blocked elimination;
        // a column without a joint unit pivot goes back to the column loop
        if (n >= ctx->elim_panel_min_n) {
            bool fallback = false;
            if ((e = elim_blocked<L, false>(b, M, n, md, &pr, &pv, &fallback, s))) return elim_fail(ctx, "det_mod", e);
            blocked = !fallback;
            if (fallback) {  // the matrix again, for the column loop
                elim_init_kernel<T, L><<<(unsigned)((n * n + 255) / 256), 256, 0, s>>>(A, lda, n, M, md);
                if ((e = cudaGetLastError())) return elim_fail(ctx, "det_mod", e);
            }
        }
    }
    if (!blocked && (e = elim_columns<T, L>(b, M, n, md, true, &pr, &pv, s))) return elim_fail(ctx, "det_mod", e);
    if (std::any_of(pr.begin(), pr.end(), [](int64_t r) { return r < 0; })) {
        if (nq == 1) {
            det[0] = 0;
            return SMF_OK;
        }
        for (int l = 0; l < nq; l++) {
            const int st = det_lanes<T, L>(ctx, A, lda, n, q + l, 1, det + l, s);
            if (st) return st;
        }
        return SMF_OK;
    }
    // sign of the permutation k -> pr[k]: (-1)^(n - cycles)
    std::vector<char> seen(n, 0);
    int64_t cycles = 0;
    for (int64_t k = 0; k < n; k++) {
        if (seen[k]) continue;
        cycles++;
        for (int64_t j = k; !seen[j]; j = pr[j]) seen[j] = 1;
    }
    for (int l = 0; l < nq; l++) {
        uint64_t d = 1 % q[l];
        for (int64_t k = 0; k < n; k++) d = mulmod_host(d, (uint64_t)pv[k * L + l], q[l]);
        if (((n - cycles) & 1) && d) d = q[l] - d;
        det[l] = d;
    }
    return SMF_OK;
}

// The local Smith form at q over Z/(q^e) of the nb x nb matrix already in M
// (one lane, canonical modulo q^e): counts[t] += #(invariant factors divisible
// by q^t) for t = 1 .. e.
template <typename T>
int local_levels(smf_ctx* ctx, ElimBufs<T, 1>& b, StreamBuf& M2, int64_t nb, uint64_t q, int e, int64_t* counts,
                 cudaStream_t s) {
    uint64_t m = 1;
    for (int t = 0; t < e; t++) m *= q;
    T* M = (T*)b.M.p;
    T* Mn = (T*)M2.p;
    StreamBuf idx;
    cudaError_t ce = idx.alloc(sizeof(int64_t) * 2 * (size_t)std::max<int64_t>(nb, 1), s);
    if (ce) return elim_fail(ctx, "smith_local: device allocation", ce);
    int64_t size = nb;
    std::vector<int64_t> pr;
    std::vector<T> pv;
    // level t: the block left holds the invariant factors divisible by q^t, over Z/(q^(e-t))
    for (int t = 0; t < e && size > 0; t++) {
        Lanes<T, 1> md{};
        md.n = 1;
        md.m[0] = (T)m;
        md.q[0] = (T)q;
        md.rcp[0] = UINT64_MAX / m;
        if ((ce = elim_local<T, 1>(ctx, b, M, size, md, &pr, &pv, s))) return elim_fail(ctx, "smith_local", ce);
        std::vector<char> row_used(size, 0);
        std::vector<int64_t> id;  // unused rows, then deferred columns
        for (int64_t k = 0; k < size; k++)
            if (pr[k] >= 0) row_used[pr[k]] = 1;
        for (int64_t i = 0; i < size; i++)
            if (!row_used[i]) id.push_back(i);
        const int64_t k2 = (int64_t)id.size();
        for (int64_t k = 0; k < size; k++)
            if (pr[k] < 0) id.push_back(k);
        if ((int64_t)id.size() != 2 * k2) {
            ctx->err = "smith_local: unused rows and deferred columns differ in number";
            return SMF_E_INVALID;
        }
        counts[t + 1] += k2;  // invariant factors with q-valuation above t
        if (k2 == 0) break;
        m /= q;
        if (t + 1 == e) break;
        if ((ce = cudaMemcpyAsync(idx.p, id.data(), sizeof(int64_t) * 2 * k2, cudaMemcpyHostToDevice, s)))
            return elim_fail(ctx, "smith_local", ce);
        elim_gather_kernel<T, 1><<<(unsigned)((k2 * k2 + 255) / 256), 256, 0, s>>>(
            M, size, (const int64_t*)idx.p, (const int64_t*)idx.p + k2, k2, 0, (T)q, Mn);
        if ((ce = cudaGetLastError())) return elim_fail(ctx, "smith_local", ce);
        std::swap(M, Mn);
        size = k2;
    }
    return SMF_OK;
}

// The local Smith forms of A at the prime powers q_l^e_l (l < nq <= L) with one
// joint column loop over Z/(prod q_l^e_l) - pivots that are units modulo every
// q_l - and then, per prime, the levels of local_levels on the block of unused
// rows and deferred columns that is left.  counts[l][t], t = 0 .. e_l.
template <typename T, int L>
int local_lanes(smf_ctx* ctx, const int64_t* A, int64_t lda, int64_t n, const uint64_t* q, const int* e, int nq,
                std::vector<std::vector<int64_t>>* counts, cudaStream_t s) {
    counts->assign(nq, {});
    for (int l = 0; l < nq; l++) {
        (*counts)[l].assign(e[l] + 1, 0);
        (*counts)[l][0] = n;
    }
    if (n == 0) return SMF_OK;
    Lanes<T, L> md{};
    md.n = nq;
    for (int l = 0; l < nq; l++) {
        uint64_t m = 1;
        for (int t = 0; t < e[l]; t++) m *= q[l];
        md.m[l] = (T)m;
        md.q[l] = (T)q[l];
        md.rcp[l] = UINT64_MAX / m;
    }
    int64_t nb;
    std::vector<int64_t> id;
    StreamBuf joint, idx;
    {
        ElimBufs<T, L> b;
        cudaError_t ce = b.alloc(n, s);
        if (ce) return elim_fail(ctx, "smith_local: device allocation", ce);
        T* M = (T*)b.M.p;
        elim_init_kernel<T, L><<<(unsigned)((n * n + 255) / 256), 256, 0, s>>>(A, lda, n, M, md);
        std::vector<int64_t> pr;
        std::vector<T> pv;
        if ((ce = cudaGetLastError()) || (ce = elim_local<T, L>(ctx, b, M, n, md, &pr, &pv, s)))
            return elim_fail(ctx, "smith_local", ce);
        std::vector<char> row_used(n, 0);
        for (int64_t k = 0; k < n; k++)
            if (pr[k] >= 0) row_used[pr[k]] = 1;
        for (int64_t i = 0; i < n; i++)
            if (!row_used[i]) id.push_back(i);
        nb = (int64_t)id.size();
        for (int64_t k = 0; k < n; k++)
            if (pr[k] < 0) id.push_back(k);
        if ((int64_t)id.size() != 2 * nb) {
            ctx->err = "smith_local: unused rows and deferred columns differ in number";
            return SMF_E_INVALID;
        }
        if (nb == 0) return SMF_OK;  // every invariant factor is prime to every q_l
        // keep the joint matrix, free the rest of the scratch
        std::swap(joint.p, b.M.p);
        joint.s = s;
        if ((ce = idx.alloc(sizeof(int64_t) * 2 * nb, s)) ||
            (ce = cudaMemcpyAsync(idx.p, id.data(), sizeof(int64_t) * 2 * nb, cudaMemcpyHostToDevice, s)))
            return elim_fail(ctx, "smith_local", ce);
    }
    // each prime on the block that is left (the joint pivots are units for all of them)
    ElimBufs<T, 1> b1;
    StreamBuf M2;
    cudaError_t ce = b1.alloc(nb, s);
    if (!ce) ce = M2.alloc(sizeof(T) * (size_t)nb * nb, s);
    if (ce) return elim_fail(ctx, "smith_local: device allocation", ce);
    for (int l = 0; l < nq; l++) {
        elim_gather_kernel<T, L><<<(unsigned)((nb * nb + 255) / 256), 256, 0, s>>>(
            (const T*)joint.p, n, (const int64_t*)idx.p, (const int64_t*)idx.p + nb, nb, l, (T)1, (T*)b1.M.p);
        if ((ce = cudaGetLastError())) return elim_fail(ctx, "smith_local", ce);
        const int st = local_levels<T>(ctx, b1, M2, nb, q[l], e[l], (*counts)[l].data(), s);
        if (st) return st;
    }
    return SMF_OK;
}

template <typename T>
int det_dispatch(smf_ctx* ctx, const int64_t* A, int64_t lda, int64_t n, const uint64_t* q, int nq, uint64_t* det,
                 cudaStream_t s) {
    if (nq <= 1) return det_lanes<T, 1>(ctx, A, lda, n, q, nq, det, s);
    if (nq <= 2) return det_lanes<T, 2>(ctx, A, lda, n, q, nq, det, s);
    if (nq <= 4) return det_lanes<T, 4>(ctx, A, lda, n, q, nq, det, s);
    for (int i = 0; i < nq; i += 4) {  // groups of four
        const int st = det_lanes<T, 4>(ctx, A, lda, n, q + i, std::min(4, nq - i), det + i, s);
        if (st) return st;
    }
    return SMF_OK;
}

// Prime powers below 2^31 in lockstep groups of four 32-bit lanes (16-byte
// entries, one column loop per group), wider ones one at a time in 64-bit words.
// A joint loop of all eleven prime powers of the n = 5003 test in 64-bit lanes
// was slower than one at a time (4.35 s against 1.94 s): every update moved 88
// bytes per entry.
int local_dispatch(smf_ctx* ctx, const int64_t* A, int64_t lda, int64_t n, const uint64_t* q, const int* e, int nq,
                   const std::vector<char>& wide, std::vector<std::vector<int64_t>>* counts, cudaStream_t s) {
    counts->assign(nq, {});
    std::vector<int> narrow;
    for (int l = 0; l < nq; l++) {
        if (!wide[l]) {
            narrow.push_back(l);
            continue;
        }
        std::vector<std::vector<int64_t>> one;
        const int st = local_lanes<uint64_t, 1>(ctx, A, lda, n, q + l, e + l, 1, &one, s);
        if (st) return st;
        (*counts)[l] = std::move(one[0]);
    }
    for (size_t g = 0; g < narrow.size(); g += 4) {
        const int k = (int)std::min<size_t>(4, narrow.size() - g);
        std::vector<uint64_t> qg;
        std::vector<int> eg;
        for (int t = 0; t < k; t++) {
            qg.push_back(q[narrow[g + t]]);
            eg.push_back(e[narrow[g + t]]);
        }
        std::vector<std::vector<int64_t>> grp;
        const int st = k == 1   ? local_lanes<uint32_t, 1>(ctx, A, lda, n, qg.data(), eg.data(), 1, &grp, s)
                       : k == 2 ? local_lanes<uint32_t, 2>(ctx, A, lda, n, qg.data(), eg.data(), 2, &grp, s)
                                : local_lanes<uint32_t, 4>(ctx, A, lda, n, qg.data(), eg.data(), k, &grp, s);
        if (st) return st;
        for (int t = 0; t < k; t++) (*counts)[narrow[g + t]] = std::move(grp[t]);
    }
    return SMF_OK;
}

}  // namespace

int det_mod_device(smf_ctx* ctx, const int64_t* A, int64_t lda, int64_t n, const uint64_t* q, int nq, uint64_t* det,
                   cudaStream_t s) {
    bool wide = false;
    for (int l = 0; l < nq; l++) {
        if (q[l] < 2 || q[l] >= (1ull << 62)) {
            ctx->err = "det_mod: q must be a prime below 2^62";
            return SMF_E_INVALID;
        }
        wide |= q[l] >= (1ull << 31);
    }
    return wide ? det_dispatch<uint64_t>(ctx, A, lda, n, q, nq, det, s)
                : det_dispatch<uint32_t>(ctx, A, lda, n, q, nq, det, s);
}

int local_smith_device(smf_ctx* ctx, const int64_t* A, int64_t lda, int64_t n, const uint64_t* q, const int* e,
                       int nq, std::vector<std::vector<int64_t>>* counts, cudaStream_t s) {
    if (nq < 1 || nq > 16) {
        ctx->err = "smith_local: 1 to 16 prime powers";
        return SMF_E_INVALID;
    }
    std::vector<char> wide(nq, 0);
    for (int l = 0; l < nq; l++) {
        unsigned __int128 m = 1;
        for (int t = 0; t < e[l]; t++) m *= q[l];
        if (q[l] < 2 || e[l] < 1 || e[l] > 62 || m >= ((unsigned __int128)1 << 62)) {
            ctx->err = "smith_local: need primes q and q^e below 2^62";
            return SMF_E_INVALID;
        }
        wide[l] = m >= (1u << 31);
    }
    return local_dispatch(ctx, A, lda, n, q, e, nq, wide, counts, s);
}

}  // namespace smf
