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
#include <algorithm>
#include <vector>

#include "smf_internal.h"

namespace smf {
namespace {

constexpr int kPivThreads = 256;
constexpr int kUpdThreads = 256;
constexpr int kUpdRows = 16;  // rows per update block: the pivot row's entry is loaded once for them

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

// A (int64, row-major, lda) -> M = A mod m, canonical.
template <typename T>
__global__ void elim_init_kernel(const int64_t* __restrict__ A, int64_t lda, int64_t n, T* __restrict__ M,
                                 T m) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n * n) return;
    const int64_t i = e / n, j = e - i * n;
    const int64_t a = A[i * lda + j];
    const int64_t r = a % (int64_t)m;
    M[e] = (T)(r < 0 ? r + (int64_t)m : r);
}

// One column's pivot: the first unused row with a unit in column k, then the
// multipliers of every other unused row (0 for used rows and zero entries).
template <typename T>
__global__ void __launch_bounds__(kPivThreads)
elim_pivot_kernel(T* __restrict__ M, int64_t n, int64_t k, T m, T q, int field, int* __restrict__ used,
                  int64_t* __restrict__ pivrow, T* __restrict__ pivval, T* __restrict__ f, T* __restrict__ fs,
                  int* __restrict__ dead) {
    pdl_wait();
    __shared__ int64_t best;
    __shared__ T sinv, sinvs;
    if (threadIdx.x == 0) best = n;
    __syncthreads();
    const bool stop = *dead != 0;
    if (!stop) {
        int64_t mine = n;
        for (int64_t i = threadIdx.x; i < n; i += kPivThreads)
            if (!used[i] && M[i * n + k] % q != 0) {
                mine = i;
                break;
            }
        if (mine < n) atomicMin((unsigned long long*)&best, (unsigned long long)mine);
    }
    __syncthreads();
    const int64_t p = best;
    if (stop || p >= n) {
        if (threadIdx.x == 0) {
            pivrow[k] = -1;
            pivval[k] = 0;
            if (field) *dead = 1;  // the determinant: a column without a pivot means det = 0
        }
        for (int64_t i = threadIdx.x; i < n; i += kPivThreads) f[i] = 0;
        pdl_trigger();
        return;
    }
    if (threadIdx.x == 0) {
        const T pv = M[p * n + k];
        used[p] = 1;
        pivrow[k] = p;
        pivval[k] = pv;
        sinv = (T)inv_mod((int64_t)pv, (int64_t)m);
        sinvs = ModOps<T>::shoup(sinv, m);
    }
    __syncthreads();
    for (int64_t i = threadIdx.x; i < n; i += kPivThreads) {
        T fi = 0;
        if (!used[i]) fi = ModOps<T>::mul(M[i * n + k], sinv, sinvs, m);
        f[i] = fi;
        fs[i] = fi ? ModOps<T>::shoup(fi, m) : 0;
    }
    pdl_trigger();
}

// Row i -= f_i * row p over columns [c0, n) except k.
template <typename T>
__global__ void __launch_bounds__(kUpdThreads)
elim_update_kernel(T* __restrict__ M, int64_t n, int64_t k, int64_t c0, T m, const int64_t* __restrict__ pivrow,
                   const T* __restrict__ f, const T* __restrict__ fs) {
    pdl_wait();
    const int64_t p = pivrow[k];
    const int64_t j = c0 + (int64_t)blockIdx.x * kUpdThreads + threadIdx.x;
    if (p >= 0 && j < n && j != k) {
        const T y = M[p * n + j];
        const int64_t r0 = (int64_t)blockIdx.y * kUpdRows;
        const int64_t r1 = min(n, r0 + kUpdRows);
        for (int64_t i = r0; i < r1; i++) {
            const T fi = f[i];
            if (!fi) continue;
            const T t = ModOps<T>::mul(y, fi, fs[i], m);
            T x = M[i * n + j];
            M[i * n + j] = x >= t ? x - t : x + (m - t);
        }
    }
    pdl_trigger();
}

// out[a][b] = M[rows[a]][cols[b]] / q (exact), a square block of size nb.
template <typename T>
__global__ void elim_gather_kernel(const T* __restrict__ M, int64_t n, const int64_t* __restrict__ rows,
                                   const int64_t* __restrict__ cols, int64_t nb, T q, T* __restrict__ out) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= nb * nb) return;
    const int64_t a = e / nb, b = e - a * nb;
    out[e] = M[rows[a] * n + cols[b]] / q;
}

struct DevMem {
    void* p = nullptr;
    ~DevMem() {
        if (p) cudaFree(p);
    }
    cudaError_t alloc(size_t bytes) { return cudaMalloc(&p, bytes ? bytes : 1); }
};

// Scratch of one elimination of an n x n matrix.
template <typename T>
struct ElimBufs {
    DevMem M, M2, used, pivrow, pivval, f, fs, dead, idx;
    cudaError_t alloc(int64_t n) {
        cudaError_t e;
        if ((e = M.alloc(sizeof(T) * (size_t)n * n)) || (e = M2.alloc(sizeof(T) * (size_t)n * n)) ||
            (e = used.alloc(sizeof(int) * (size_t)n)) || (e = pivrow.alloc(sizeof(int64_t) * (size_t)n)) ||
            (e = pivval.alloc(sizeof(T) * (size_t)n)) || (e = f.alloc(sizeof(T) * (size_t)n)) ||
            (e = fs.alloc(sizeof(T) * (size_t)n)) || (e = dead.alloc(sizeof(int))) ||
            (e = idx.alloc(sizeof(int64_t) * 2 * (size_t)n)))
            return e;
        return cudaSuccess;
    }
};

// The column loop on the n x n matrix in `M`: pivots found for every column
// (row index, or -1 for a deferred column) and their values.  c0_all: update
// every column except k (the local form keeps deferred columns current); else
// only the columns after k (a field: nothing is deferred).
template <typename T>
cudaError_t elim_columns(ElimBufs<T>& b, T* M, int64_t n, T m, T q, bool c0_all, std::vector<int64_t>* pivrow,
                         std::vector<T>* pivval, cudaStream_t s) {
    cudaError_t e;
    if ((e = cudaMemsetAsync(b.used.p, 0, sizeof(int) * (size_t)n, s)) ||
        (e = cudaMemsetAsync(b.dead.p, 0, sizeof(int), s)))
        return e;
    for (int64_t k = 0; k < n; k++) {
        e = launch_pdl(elim_pivot_kernel<T>, dim3(1), dim3(kPivThreads), 0, s, M, n, k, m, q, c0_all ? 0 : 1,
                       (int*)b.used.p,
                       (int64_t*)b.pivrow.p, (T*)b.pivval.p, (T*)b.f.p, (T*)b.fs.p, (int*)b.dead.p);
        if (e) return e;
        const int64_t c0 = c0_all ? 0 : k + 1;
        if (c0 >= n) continue;
        const dim3 grid((unsigned)((n - c0 + kUpdThreads - 1) / kUpdThreads), (unsigned)((n + kUpdRows - 1) / kUpdRows));
        e = launch_pdl(elim_update_kernel<T>, grid, dim3(kUpdThreads), 0, s, M, n, k, c0, m,
                       (const int64_t*)b.pivrow.p, (const T*)b.f.p, (const T*)b.fs.p);
        if (e) return e;
    }
    pivrow->resize(n);
    pivval->resize(n);
    if ((e = cudaMemcpyAsync(pivrow->data(), b.pivrow.p, sizeof(int64_t) * n, cudaMemcpyDeviceToHost, s)) ||
        (e = cudaMemcpyAsync(pivval->data(), b.pivval.p, sizeof(T) * n, cudaMemcpyDeviceToHost, s)))
        return e;
    return cudaStreamSynchronize(s);
}

uint64_t mulmod_host(uint64_t a, uint64_t b, uint64_t m) { return (uint64_t)((unsigned __int128)a * b % m); }

template <typename T>
int det_mod_t(smf_ctx* ctx, const int64_t* A, int64_t lda, int64_t n, uint64_t q, uint64_t* det, cudaStream_t s) {
    if (n == 0) {
        *det = 1 % q;
        return SMF_OK;
    }
    ElimBufs<T> b;
    cudaError_t e = b.alloc(n);
    if (e) {
        cudaGetLastError();
        ctx->err = "det_mod: device allocation failed";
        return SMF_E_NOMEM;
    }
    T* M = (T*)b.M.p;
    elim_init_kernel<T><<<(unsigned)((n * n + 255) / 256), 256, 0, s>>>(A, lda, n, M, (T)q);
    std::vector<int64_t> pr;
    std::vector<T> pv;
    if ((e = cudaGetLastError()) || (e = elim_columns<T>(b, M, n, (T)q, (T)q, false, &pr, &pv, s))) {
        ctx->err = std::string("det_mod: ") + cudaGetErrorString(e);
        return SMF_E_CUDA;
    }
    uint64_t d = 1 % q;
    for (int64_t k = 0; k < n; k++) {
        if (pr[k] < 0) {
            *det = 0;
            return SMF_OK;
        }
        d = mulmod_host(d, (uint64_t)pv[k], q);
    }
    // sign of the permutation k -> pr[k]: (-1)^(n - cycles)
    std::vector<char> seen(n, 0);
    int64_t cycles = 0;
    for (int64_t k = 0; k < n; k++) {
        if (seen[k]) continue;
        cycles++;
        for (int64_t j = k; !seen[j]; j = pr[j]) seen[j] = 1;
    }
    if (((n - cycles) & 1) && d) d = q - d;
    *det = d;
    return SMF_OK;
}

template <typename T>
int local_smith_t(smf_ctx* ctx, const int64_t* A, int64_t lda, int64_t n, uint64_t q, int e, int64_t* counts,
                  cudaStream_t s) {
    counts[0] = n;
    for (int t = 1; t <= e; t++) counts[t] = 0;
    if (n == 0) return SMF_OK;
    ElimBufs<T> b;
    cudaError_t ce = b.alloc(n);
    if (ce) {
        cudaGetLastError();
        ctx->err = "smith_local: device allocation failed";
        return SMF_E_NOMEM;
    }
    uint64_t m = 1;
    for (int t = 0; t < e; t++) m *= q;
    T* M = (T*)b.M.p;
    T* M2 = (T*)b.M2.p;
    elim_init_kernel<T><<<(unsigned)((n * n + 255) / 256), 256, 0, s>>>(A, lda, n, M, (T)m);
    if ((ce = cudaGetLastError())) {
        ctx->err = std::string("smith_local: ") + cudaGetErrorString(ce);
        return SMF_E_CUDA;
    }
    int64_t size = n;
    std::vector<int64_t> pr;
    std::vector<T> pv;
    // level t: the block left holds the invariants divisible by q^t, over Z/(q^(e-t))
    for (int t = 0; t < e && size > 0; t++) {
        if ((ce = elim_columns<T>(b, M, size, (T)m, (T)q, true, &pr, &pv, s))) {
            ctx->err = std::string("smith_local: ") + cudaGetErrorString(ce);
            return SMF_E_CUDA;
        }
        std::vector<char> row_used(size, 0);
        std::vector<int64_t> idx;  // unused rows, then deferred columns
        for (int64_t k = 0; k < size; k++)
            if (pr[k] >= 0) row_used[pr[k]] = 1;
        for (int64_t i = 0; i < size; i++)
            if (!row_used[i]) idx.push_back(i);
        const int64_t nb = (int64_t)idx.size();
        for (int64_t k = 0; k < size; k++)
            if (pr[k] < 0) idx.push_back(k);
        if ((int64_t)idx.size() != 2 * nb) {
            ctx->err = "smith_local: unused rows and deferred columns differ in number";
            return SMF_E_INVALID;
        }
        counts[t + 1] = nb;  // invariants with q-valuation above t
        if (nb == 0) break;
        m /= q;
        if (t + 1 == e) break;
        if ((ce = cudaMemcpyAsync(b.idx.p, idx.data(), sizeof(int64_t) * 2 * nb, cudaMemcpyHostToDevice, s))) {
            ctx->err = std::string("smith_local: ") + cudaGetErrorString(ce);
            return SMF_E_CUDA;
        }
        elim_gather_kernel<T><<<(unsigned)((nb * nb + 255) / 256), 256, 0, s>>>(
            M, size, (const int64_t*)b.idx.p, (const int64_t*)b.idx.p + nb, nb, (T)q, M2);
        if ((ce = cudaGetLastError())) {
            ctx->err = std::string("smith_local: ") + cudaGetErrorString(ce);
            return SMF_E_CUDA;
        }
        std::swap(M, M2);
        size = nb;
    }
    return SMF_OK;
}

}  // namespace

int det_mod_device(smf_ctx* ctx, const int64_t* A, int64_t lda, int64_t n, uint64_t q, uint64_t* det,
                   cudaStream_t s) {
    if (q < 2 || q >= (1ull << 62)) {
        ctx->err = "det_mod: q must be a prime below 2^62";
        return SMF_E_INVALID;
    }
    return q < (1ull << 31) ? det_mod_t<uint32_t>(ctx, A, lda, n, q, det, s)
                            : det_mod_t<uint64_t>(ctx, A, lda, n, q, det, s);
}

int local_smith_device(smf_ctx* ctx, const int64_t* A, int64_t lda, int64_t n, uint64_t q, int e, int64_t* counts,
                       cudaStream_t s) {
    unsigned __int128 m = 1;
    for (int t = 0; t < e; t++) m *= q;
    if (q < 2 || e < 1 || e > 62 || m >= ((unsigned __int128)1 << 62)) {
        ctx->err = "smith_local: need a prime q and q^e below 2^62";
        return SMF_E_INVALID;
    }
    return m < (1u << 31) ? local_smith_t<uint32_t>(ctx, A, lda, n, q, e, counts, s)
                          : local_smith_t<uint64_t>(ctx, A, lda, n, q, e, counts, s);
}

}  // namespace smf
