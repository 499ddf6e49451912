// Host runtime behind the C ABI (include/smf.h): contexts, prime bases with
// their device-resident constants, workspace planning and the launch sequence
// of the RNS product (Section 3.1).
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cstdio>
#include <cstring>
#include <string>

#include "smf_internal.h"

using namespace smf;

namespace {

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        cudaGetDevice(&prev);
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard() {
        int cur = -1;
        cudaGetDevice(&cur);
        if (prev >= 0 && cur != prev) cudaSetDevice(prev);
    }
};

int fail(smf_ctx* c, int code, const std::string& msg) {
    if (c) c->err = msg;
    return code;
}

#define SMF_CU(ctx, call)                                                                  \
    do {                                                                                   \
        cudaError_t e_ = (call);                                                           \
        if (e_ != cudaSuccess)                                                             \
            return fail(ctx, SMF_E_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

// ------------------------------------------------------------ host number theory

bool is_prime_u32(uint32_t n) {
    if (n < 2) return false;
    if (n % 2 == 0) return n == 2;
    for (uint32_t d = 3; (uint64_t)d * d <= n; d += 2)
        if (n % d == 0) return false;
    return true;
}

uint32_t inv_mod(uint32_t a, uint32_t p) {  // extended Euclid, p prime, a != 0 mod p
    int64_t t = 0, nt = 1, r = p, nr = a % p;
    while (nr) {
        int64_t q = r / nr;
        int64_t x = t - q * nt;
        t = nt;
        nt = x;
        x = r - q * nr;
        r = nr;
        nr = x;
    }
    if (t < 0) t += p;
    return (uint32_t)t;
}

uint32_t shoup(uint32_t w, uint32_t p) { return (uint32_t)(((uint64_t)w << 32) / p); }

// Bit length of a limb vector.
int bitlen(const std::vector<uint32_t>& x) {
    for (int i = (int)x.size() - 1; i >= 0; i--)
        if (x[i]) return 32 * i + (32 - __builtin_clz(x[i]));
    return 0;
}

void mul_small(std::vector<uint32_t>& x, uint32_t m) {
    uint64_t carry = 0;
    for (auto& w : x) {
        uint64_t z = (uint64_t)w * m + carry;
        w = (uint32_t)z;
        carry = z >> 32;
    }
    if (carry) x.push_back((uint32_t)carry);
}

// ------------------------------------------------------------ profiling: take_event and ProfScope (smf_internal.h)

int64_t entry_bits(const smf_bigmat* X) { return X->bits > 0 ? X->bits : 64LL * X->words - 1; }

int check_bigmat(smf_ctx* c, const smf_bigmat* X, const char* name, bool need_device) {
    if (!X) return fail(c, SMF_E_INVALID, std::string(name) + ": null");
    if (X->rows < 0 || X->cols < 0 || X->ld < X->cols || X->words < 1 || X->bits < 0)
        return fail(c, SMF_E_INVALID, std::string(name) + ": bad shape");
    if (X->rows * X->cols > 0 && !X->data) return fail(c, SMF_E_INVALID, std::string(name) + ": null data");
    if (need_device && !X->on_device) return fail(c, SMF_E_INVALID, std::string(name) + ": must be on the device");
    if (X->on_device && ((uintptr_t)X->data & 15)) return fail(c, SMF_E_INVALID, std::string(name) + ": not 16-byte aligned");
    return SMF_OK;
}

// True for device (or managed) memory of any device; a null pointer is not.
bool device_ptr(const void* p) {
    if (!p) return false;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

int64_t ceil_log2(int64_t k) {
    int64_t b = 0;
    while (((int64_t)1 << b) < k) b++;
    return b;
}

uint32_t default_pmax(smf_form f) { return f == SMF_FORM_INT8LIMB ? (1u << 24) : (1u << 26); }

// Workspace layout of one residue product (offsets in bytes, 256-aligned).
struct GemmPlan {
    int TA = 0, TB = 0;
    int64_t lda = 0, ldb = 0;
    int split = 1, kchunk = 0;  // split-K of a product with few tiles
    int bn = 48;                // tile width of the kernels for fewer than 3x3 digits
    size_t a_off = 0, b_off = 0, part_off = 0, bytes = 0;
};

size_t align256(size_t x) { return (x + 255) / 256 * 256; }

// A copy of `height` rows of `width` bytes: one linear copy when both sides
// are contiguous, a pitched copy otherwise.
cudaError_t copy_rows(void* dst, size_t dpitch, const void* src, size_t spitch, size_t width, size_t height,
                      cudaMemcpyKind kind, cudaStream_t s) {
    if (dpitch == width && spitch == width) return cudaMemcpyAsync(dst, src, width * height, kind, s);
    return cudaMemcpy2DAsync(dst, dpitch, src, spitch, width, height, kind, s);
}

// num_sms > 0 lets a product with few tiles split K across the SMs (the
// partial residues get their own slot); 0 keeps one launch per tile.
GemmPlan plan_limb(int L, int64_t M, int64_t N, int64_t K, bool a_shared, uint64_t amax, uint64_t bmax,
                   int num_sms = 0) {
    GemmPlan g;
    g.TA = digits_for(amax);
    g.TB = digits_for(bmax);
    g.lda = round_up(std::max<int64_t>(K, 1), 8);
    g.ldb = g.lda;
    const size_t a_bytes = (size_t)g.TA * (a_shared ? 1 : L) * M * g.lda * 2;
    const size_t b_bytes = (size_t)g.TB * L * N * g.ldb * 2;
    g.a_off = 0;
    g.b_off = align256(a_bytes);
    g.bytes = g.b_off + align256(b_bytes);
    limb_split(L, M, N, K, a_shared, g.TA, g.TB, num_sms, &g.split, &g.kchunk);
    g.bn = limb_narrow_bn(L, M, N, K, a_shared, g.TA, g.TB, num_sms);
    if (g.split > 1) {
        g.part_off = g.bytes;
        g.bytes += align256((size_t)4 * g.split * L * M * N);
    }
    return g;
}

// Largest kblk with p + kblk * amax * bmax < 2^53 (exact fp64 accumulation).
int64_t fp64_kblk(uint32_t pmax, uint64_t amax, uint64_t bmax) {
    const unsigned __int128 prod = (unsigned __int128)amax * bmax;
    if (prod == 0) return 1 << 30;
    const unsigned __int128 room = ((unsigned __int128)1 << 53) - pmax - 1;
    const unsigned __int128 k = room / prod;
    return k > (1u << 30) ? (1 << 30) : (int64_t)k;
}

int basis_build(smf_ctx* ctx, int32_t bound_bits, uint32_t p_max, smf_basis** out) {
    if (bound_bits < 0 || bound_bits > 200000) return fail(ctx, SMF_E_INVALID, "basis: bound_bits out of range");
    if (p_max == 0) p_max = default_pmax(ctx->form);
    if (p_max > (1u << 26) || p_max < 3) return fail(ctx, SMF_E_INVALID, "basis: p_max must be in [3, 2^26]");
    auto* b = new smf_basis();
    b->ctx = ctx;
    b->device = ctx->device;
    b->dev_blob = nullptr;
    std::vector<uint32_t> M{1};
    uint32_t c = p_max;
    while (bitlen(M) < bound_bits + 2) {
        uint32_t p = 0;
        while (c > 3) {
            c--;
            if (is_prime_u32(c)) {
                p = c;
                break;
            }
        }
        if (!p || (int)b->primes.size() >= kMaxPrimes) {
            delete b;
            return fail(ctx, SMF_E_UNSUPPORTED, "basis: not enough primes below p_max for the bound");
        }
        b->primes.push_back(p);
        mul_small(M, p);
    }
    const int L = (int)b->primes.size();
    b->m_limbs = M;
    b->m_bits = bitlen(M);
    // host tables
    std::vector<uint32_t> p(b->primes), pow32(L), gw((size_t)L * L, 0), gws((size_t)L * L, 0), ginv(L), ginvs(L);
    std::vector<uint64_t> mu(L);
    std::vector<double> inv_p(L);
    for (int i = 0; i < L; i++) {
        mu[i] = UINT64_MAX / p[i];
        pow32[i] = (uint32_t)((1ull << 32) % p[i]);
        inv_p[i] = 1.0 / (double)p[i];
        // W_k mod p_i for k <= i, W_k = p_0 ... p_(k-1)
        uint32_t w = 1 % p[i];
        for (int k = 0; k < i; k++) {
            gw[(size_t)i * L + k] = w;
            gws[(size_t)i * L + k] = shoup(w, p[i]);
            w = (uint32_t)((uint64_t)w * (p[k] % p[i]) % p[i]);
        }
        ginv[i] = inv_mod(w, p[i]);
        ginvs[i] = shoup(ginv[i], p[i]);
    }
    // device blob
    const int ml = (int)M.size();
    size_t off = 0;
    auto slot = [&](size_t bytes) {
        size_t o = off;
        off = align256(off + bytes);
        return o;
    };
    const size_t o_p = slot(4 * L), o_mu = slot(8 * L), o_pow = slot(4 * L), o_inv = slot(8 * L);
    const size_t o_gw = slot(4 * (size_t)L * L), o_gws = slot(4 * (size_t)L * L), o_ginv = slot(4 * L),
                 o_ginvs = slot(4 * L), o_m = slot(4 * ml);
    std::vector<uint8_t> host(off, 0);
    memcpy(&host[o_p], p.data(), 4 * L);
    memcpy(&host[o_mu], mu.data(), 8 * L);
    memcpy(&host[o_pow], pow32.data(), 4 * L);
    memcpy(&host[o_inv], inv_p.data(), 8 * L);
    memcpy(&host[o_gw], gw.data(), 4 * (size_t)L * L);
    memcpy(&host[o_gws], gws.data(), 4 * (size_t)L * L);
    memcpy(&host[o_ginv], ginv.data(), 4 * L);
    memcpy(&host[o_ginvs], ginvs.data(), 4 * L);
    memcpy(&host[o_m], M.data(), 4 * ml);
    DeviceGuard g(ctx->device);
    cudaError_t e = cudaMalloc(&b->dev_blob, off);
    // A copy from pageable memory may return before its DMA lands, and kernels on
    // non-blocking streams are not ordered after the legacy stream: wait for it.
    if (e == cudaSuccess) e = cudaMemcpyAsync(b->dev_blob, host.data(), off, cudaMemcpyHostToDevice, cudaStreamLegacy);
    if (e == cudaSuccess) e = cudaStreamSynchronize(cudaStreamLegacy);
    if (e != cudaSuccess) {
        if (b->dev_blob) cudaFree(b->dev_blob);
        delete b;
        return fail(ctx, SMF_E_CUDA, std::string("basis tables: ") + cudaGetErrorString(e));
    }
    b->gw = gw;
    b->gws = gws;
    b->ginv = ginv;
    b->ginvs = ginvs;
    // Lagrange-form tables: H = (M-1)/2, M_i = M / p_i, c_i = M_i^-1 mod p_i
    {
        std::vector<uint32_t> H(ml, 0);
        for (int j = 0; j < ml; j++) H[j] = (M[j] >> 1) | (j + 1 < ml ? (M[j + 1] << 31) : 0u);  // M odd
        b->h = H;
        b->hmod.resize(L);
        b->c.resize(L);
        b->cs.resize(L);
        b->mi.assign((size_t)L * ml, 0);
        for (int i = 0; i < L; i++) {
            uint64_t rem = 0, hr = 0;
            for (int j = ml - 1; j >= 0; j--) {
                const uint64_t cur = (rem << 32) | M[j];
                b->mi[(size_t)i * ml + j] = (uint32_t)(cur / p[i]);
                rem = cur % p[i];
                hr = ((hr << 32) | H[j]) % p[i];
            }
            uint64_t mimod = 0;  // M_i mod p_i
            for (int j = ml - 1; j >= 0; j--) mimod = ((mimod << 32) | b->mi[(size_t)i * ml + j]) % p[i];
            b->hmod[i] = (uint32_t)hr;
            b->c[i] = inv_mod((uint32_t)mimod, p[i]);
            b->cs[i] = shoup(b->c[i], p[i]);
        }
    }
    b->crt.hmod = b->hmod.data();
    b->crt.c = b->c.data();
    b->crt.cs = b->cs.data();
    b->crt.mi = b->mi.data();
    b->crt.h = b->h.data();
    b->crt.L = L;
    b->crt.m_limbs = ml;
    b->crt.p = b->primes.data();
    b->crt.gw = b->gw.data();
    b->crt.gws = b->gws.data();
    b->crt.ginv = b->ginv.data();
    b->crt.ginvs = b->ginvs.data();
    b->crt.m = b->m_limbs.data();
    uint8_t* d = (uint8_t*)b->dev_blob;
    b->dev.L = L;
    b->dev.m_limbs = ml;
    b->dev.p = (const uint32_t*)(d + o_p);
    b->dev.mu = (const uint64_t*)(d + o_mu);
    b->dev.pow32 = (const uint32_t*)(d + o_pow);
    b->dev.inv_p = (const double*)(d + o_inv);
    b->dev.gw = (const uint32_t*)(d + o_gw);
    b->dev.gws = (const uint32_t*)(d + o_gws);
    b->dev.ginv = (const uint32_t*)(d + o_ginv);
    b->dev.ginvs = (const uint32_t*)(d + o_ginvs);
    b->dev.m_words = (const uint32_t*)(d + o_m);
    *out = b;
    return SMF_OK;
}

smf_basis* cached_basis(smf_ctx* ctx, int bound_bits, uint32_t p_max, int* status) {
    for (auto& kv : ctx->basis_cache)
        if (kv.first.first == bound_bits && kv.first.second == p_max) return kv.second;
    smf_basis* b = nullptr;
    *status = basis_build(ctx, bound_bits, p_max, &b);
    if (*status != SMF_OK) return nullptr;
    ctx->basis_cache.push_back({{bound_bits, p_max}, b});
    return b;
}

// Residue product on prepared operands (int32 residues).  amax/bmax bound
// the centred operands.  Used by smf_residue_gemm and smf_rns_matmul.
int run_residue_gemm_i32(smf_ctx* ctx, const smf_basis* b, const int32_t* A, int64_t a_stride, const int32_t* B,
                         int32_t* C, int64_t M, int64_t N, int64_t K, uint64_t amax, uint64_t bmax, void* ws,
                         size_t ws_bytes, cudaStream_t s) {
    const int L = (int)b->primes.size();
    const uint32_t p0 = b->primes[0];
    if (K == 0) {  // empty inner dimension: every residue is 0
        if (M * N > 0) SMF_CU(ctx, cudaMemsetAsync(C, 0, sizeof(int32_t) * (size_t)L * M * N, s));
        return SMF_OK;
    }
    if (ctx->form == SMF_FORM_FP64) {
        const int64_t kblk = fp64_kblk(p0, amax, bmax);
        if (kblk < 1) return fail(ctx, SMF_E_UNSUPPORTED, "fp64 form: operands too large for exact fp64 products");
        Fp64GemmArgs g{A, a_stride, B, C, M, N, K, (int)std::min<int64_t>(kblk, 1 << 30)};
        ProfScope ps(ctx, 2, s);
        SMF_CU(ctx, launch_gemm_fp64(b->dev, g, s));
        return SMF_OK;
    }
    const bool shared = a_stride == 0;
    GemmPlan g = plan_limb(L, M, N, K, shared, amax, bmax, ctx->num_sms);
    if ((unsigned __int128)K * amax * bmax >= ((unsigned __int128)1 << 62))
        return fail(ctx, SMF_E_UNSUPPORTED, "limb form: K * |a| * |b| must stay below 2^62");
    if (g.TA > 3 || g.TB > 3) return fail(ctx, SMF_E_UNSUPPORTED, "limb form: more than 3 digits per residue");
    if (!ws || ws_bytes < g.bytes) return fail(ctx, SMF_E_NOMEM, "residue_gemm: workspace too small");
    uint8_t* w = (uint8_t*)ws;
    {
        ProfScope ps(ctx, 1, s);
        SMF_CU(ctx, launch_residue_digits(b->dev, A, a_stride, shared ? 1 : L, M, K, w + g.a_off, g.lda, g.TA,
                                          false, s));
        SMF_CU(ctx, launch_residue_digits(b->dev, B, K * N, L, K, N, w + g.b_off, g.ldb, g.TB, true, s));
    }
    LimbGemmArgs la{w + g.a_off, g.lda, shared ? 1 : 0, w + g.b_off, g.ldb, C, M, N, K, g.TA, g.TB, ctx->d_status,
                    ctx->inject, amax, bmax, (int32_t*)(w + g.part_off), g.split, g.kchunk};
    la.bn = g.bn;
    ctx->inject = 0;
    ProfScope ps(ctx, 2, s);
    SMF_CU(ctx, launch_gemm_limb(ctx, b->dev, la, s));
    return SMF_OK;
}

}  // namespace

smf_basis* smf::ctx_basis(smf_ctx* ctx, int bound_bits, uint32_t p_max, int* status) {
    return cached_basis(ctx, bound_bits, p_max, status);
}


namespace {

struct MatmulPlan {
    int64_t M, N, K;
    int bound;
    uint32_t p_max;
    bool a_shared;
    uint64_t amax, bmax;
    // Row chunks of A (and C).  With A or C in host memory the product runs as
    // row chunks whose copies overlap the other chunks' kernels; otherwise one
    // chunk of all M rows.  Chunk c covers rows chunk_m0[c] .. chunk_m0[c+1]-1.
    int chunks;
    int64_t chunk_m0[5];
    int64_t chunk_rows;                      // rows of the largest chunk (sizes the buffers)
    // byte offsets into the workspace
    size_t a_stage[2], b_stage, c_stage[2];  // device copies of host operands (two per chunked operand)
    size_t a_op, b_op;                       // operand residues / digit planes (A: one chunk)
    size_t part_op = 0;                      // split-K partial residues (limb form, one chunk only)
    size_t r_off;                            // [L][chunk_rows][N] int32 residues of C
    size_t cnt_off = 0;                      // limb form: per-unit tile counters of the fused CRT
    size_t bytes;
    GemmPlan g;
};

// Row chunks of the host-operand pipeline.  The first chunk's copy-in and the
// last chunk's copy-out cannot overlap kernels, so those two are short (about
// M/12 rows); the middle chunks split the rest in two, so that their residue
// products fill whole waves of tiles.  Chunks are whole 128-row tiles; small
// products run as one chunk.
void plan_chunks(int64_t M, bool host_rows, MatmulPlan* P) {
    int n = 0;
    P->chunk_m0[n++] = 0;
    if (host_rows && M > 1024) {
        const int64_t edge = std::max<int64_t>(128, round_up((M + 11) / 12, 128));
        const int64_t mid = round_up((M - 2 * edge + 1) / 2, 128);
        for (int64_t m : {edge, edge + mid, M - edge})
            if (m > P->chunk_m0[n - 1] && m < M) P->chunk_m0[n++] = m;
    }
    P->chunk_m0[n] = M;
    P->chunks = n;
    P->chunk_rows = 1;
    for (int c = 0; c < n; c++) P->chunk_rows = std::max(P->chunk_rows, P->chunk_m0[c + 1] - P->chunk_m0[c]);
}

int plan_matmul(smf_ctx* ctx, const smf_bigmat* A, const smf_bigmat* B, const smf_bigmat* C, MatmulPlan* P,
                smf_basis** basis) {
    int st;
    if ((st = check_bigmat(ctx, A, "A", false)) || (st = check_bigmat(ctx, B, "B", false)) ||
        (st = check_bigmat(ctx, C, "C", false)))
        return st;
    if (A->cols != B->rows || C->rows != A->rows || C->cols != B->cols)
        return fail(ctx, SMF_E_INVALID, "rns_matmul: shapes do not chain");
    P->M = A->rows;
    P->N = B->cols;
    P->K = A->cols;
    const int64_t ab = entry_bits(A), bb = entry_bits(B);
    const int64_t bound = ab + bb + ceil_log2(std::max<int64_t>(P->K, 1));
    if (64LL * C->words < bound + 2) return fail(ctx, SMF_E_BOUND, "rns_matmul: C.words cannot hold K*|A|*|B|");
    if (bound > 100000) return fail(ctx, SMF_E_UNSUPPORTED, "rns_matmul: result bound too large");
    P->bound = (int)bound;
    P->p_max = default_pmax(ctx->form);
    smf_basis* b = cached_basis(ctx, P->bound, P->p_max, &st);
    if (!b) return st;
    *basis = b;
    const int L = (int)b->primes.size();
    if (L > 64) return fail(ctx, SMF_E_UNSUPPORTED, "rns_matmul: more than 64 primes");
    const uint64_t hL = b->primes.back() / 2, h0 = b->primes[0] / 2;
    // Shortcut: when |A| <= (p_L - 1)/2, A is its own centred residue for
    // every prime, so one copy serves all L residue products.
    P->a_shared = ab < 62 && (1ull << ab) <= hL && ab <= 30;
    P->amax = P->a_shared ? (1ull << ab) : h0;
    P->bmax = h0;
    size_t off = 0;
    auto slot = [&](size_t bytes) {
        size_t o = off;
        off = align256(off + bytes);
        return o;
    };
    const int64_t M = P->M, N = P->N, K = P->K;
    plan_chunks(M, !A->on_device || !C->on_device, P);
    const int nbuf = P->chunks > 1 ? 2 : 1;
    const int64_t Mc = std::min<int64_t>(M, P->chunk_rows);
    for (int i = 0; i < 2; i++) {
        P->a_stage[i] = A->on_device || i >= nbuf ? 0 : slot((size_t)Mc * A->cols * A->words * 8);
        P->c_stage[i] = C->on_device || i >= nbuf ? 0 : slot((size_t)Mc * C->cols * C->words * 8);
    }
    P->b_stage = B->on_device ? 0 : slot((size_t)B->rows * B->cols * B->words * 8);
    if (ctx->form == SMF_FORM_INT8LIMB) {
        P->g = plan_limb(L, Mc, N, K, P->a_shared, P->amax, P->bmax, P->chunks > 1 ? 0 : ctx->num_sms);
        if (P->g.TA > 3 || P->g.TB > 3) return fail(ctx, SMF_E_UNSUPPORTED, "limb form: more than 3 digits");
        if ((unsigned __int128)std::max<int64_t>(K, 1) * P->amax * P->bmax >= ((unsigned __int128)1 << 62))
            return fail(ctx, SMF_E_UNSUPPORTED, "limb form: K * |a| * |b| must stay below 2^62");
        const size_t base = slot(P->g.bytes);
        P->a_op = base + P->g.a_off;
        P->b_op = base + P->g.b_off;
        P->part_op = base + P->g.part_off;
    } else {
        P->a_op = slot((size_t)4 * (P->a_shared ? 1 : L) * Mc * K);
        P->b_op = slot((size_t)4 * L * K * N);
        if (fp64_kblk(b->primes[0], P->amax, P->bmax) < 1)
            return fail(ctx, SMF_E_UNSUPPORTED, "fp64 form: operands too large for exact fp64 products");
    }
    P->r_off = slot((size_t)4 * L * Mc * N);
    if (ctx->form == SMF_FORM_INT8LIMB) P->cnt_off = slot(sizeof(int) * (size_t)limb_crt_units(Mc, N));
    P->bytes = off;
    return SMF_OK;
}

// Events of the host-operand pipeline (indices into smf_ctx::pev).
enum { kEvFork = 0, kEvBIn = 1, kEvAIn = 2, kEvAFree = 4, kEvCReady = 6, kEvCFree = 8, kEvJoinIn = 10, kEvJoinOut = 11 };

// Product of row chunks with host operands (Section 3.1's product, one row
// block of A and C at a time).  B is copied in K-row chunks and each chunk is
// reduced as soon as it lands.  Per row chunk c: copy in A's rows (copy-in
// stream), reduce or split them, the residue product and the CRT (caller's
// stream), copy out C's rows (copy-out stream).  The staging buffers of A and
// C alternate between two slots, so chunk c's copies overlap the kernels of
// its neighbours; operand, residue and digit buffers are reused in stream order.
int run_pipelined(smf_ctx* ctx, const MatmulPlan& P, smf_basis* basis, const smf_bigmat* A, const smf_bigmat* B,
                  smf_bigmat* C, uint8_t* w, cudaStream_t s) {
    const int64_t M = P.M, N = P.N, K = P.K;
    const int L = (int)basis->primes.size();
    const bool limb = ctx->form == SMF_FORM_INT8LIMB;
    cudaEvent_t* ev = ctx->pev;
    cudaStream_t hin = ctx->h2d, hout = ctx->d2h;
    // the copy streams start after the work already queued on s (it may still use the workspace)
    SMF_CU(ctx, cudaEventRecord(ev[kEvFork], s));
    SMF_CU(ctx, cudaStreamWaitEvent(hin, ev[kEvFork], 0));
    SMF_CU(ctx, cudaStreamWaitEvent(hout, ev[kEvFork], 0));
    // B: the limb form's digit planes are K-contiguous, so a K-row chunk of B
    // reduces into an offset of them
    const int nbc = !B->on_device && limb ? (int)std::min<int64_t>(4, (K + 255) / 256) : 1;
    const int64_t kc_rows = (K + nbc - 1) / nbc;
    for (int j = 0; j < nbc && K > 0; j++) {
        const int64_t k0 = (int64_t)j * kc_rows, kc = std::min<int64_t>(kc_rows, K - k0);
        if (kc <= 0) break;
        const uint64_t* dB = (const uint64_t*)B->data + (size_t)k0 * B->ld * B->words;
        int64_t ldB = B->ld;
        if (!B->on_device) {
            uint64_t* st = (uint64_t*)(w + P.b_stage) + (size_t)k0 * N * B->words;
            {
                ProfScope ps(ctx, 4, hin);
                SMF_CU(ctx, copy_rows(st, (size_t)N * B->words * 8, dB, (size_t)B->ld * B->words * 8,
                                      (size_t)N * B->words * 8, (size_t)kc, cudaMemcpyHostToDevice, hin));
            }
            SMF_CU(ctx, cudaEventRecord(ev[kEvBIn], hin));
            SMF_CU(ctx, cudaStreamWaitEvent(s, ev[kEvBIn], 0));
            dB = st;
            ldB = N;
        }
        ProfScope ps(ctx, 0, s);
        if (limb) {
            ReduceArgs rb{dB, kc, N, ldB, B->words, w + P.b_op + 2 * (size_t)k0, P.g.ldb, P.g.TB, 0,
                          (int)entry_bits(B)};
            SMF_CU(ctx, launch_reduce(basis->dev, rb, ReduceOut::kDigitsT, ctx->d_status, s));
        } else {
            ReduceArgs rb{dB, K, N, ldB, B->words, w + P.b_op, 0, 0, 0, (int)entry_bits(B)};
            SMF_CU(ctx, launch_reduce(basis->dev, rb, ReduceOut::kCentered, ctx->d_status, s));
        }
    }
    int32_t* R = (int32_t*)(w + P.r_off);
    for (int c = 0; c < P.chunks; c++) {
        const int64_t m0 = P.chunk_m0[c];
        const int64_t mc = P.chunk_m0[c + 1] - m0;
        const int slot = c & 1;
        const uint64_t* dA = (const uint64_t*)A->data + (size_t)m0 * A->ld * A->words;
        int64_t ldA = A->ld;
        if (!A->on_device && K > 0) {
            // chunk c-2's reduction has read this slot
            if (c >= 2) SMF_CU(ctx, cudaStreamWaitEvent(hin, ev[kEvAFree + slot], 0));
            uint8_t* st = w + P.a_stage[slot];
            {
                ProfScope ps(ctx, 4, hin);
                SMF_CU(ctx, copy_rows(st, (size_t)K * A->words * 8, dA, (size_t)A->ld * A->words * 8,
                                      (size_t)K * A->words * 8, (size_t)mc, cudaMemcpyHostToDevice, hin));
            }
            SMF_CU(ctx, cudaEventRecord(ev[kEvAIn + slot], hin));
            SMF_CU(ctx, cudaStreamWaitEvent(s, ev[kEvAIn + slot], 0));
            dA = (const uint64_t*)st;
            ldA = K;
        }
        if (K > 0) {
            {
                ProfScope ps(ctx, 0, s);
                ReduceArgs ra{dA, mc, K, ldA, A->words, w + P.a_op, 0, 0, P.a_shared ? 1 : 0, (int)entry_bits(A)};
                if (limb) {
                    ra.ld_out = P.g.lda;
                    ra.t = P.g.TA;
                    SMF_CU(ctx, launch_reduce(basis->dev, ra, ReduceOut::kDigits, ctx->d_status, s));
                } else {
                    SMF_CU(ctx, launch_reduce(basis->dev, ra, ReduceOut::kCentered, ctx->d_status, s));
                }
            }
            if (!A->on_device) SMF_CU(ctx, cudaEventRecord(ev[kEvAFree + slot], s));
            ProfScope ps(ctx, 2, s);
            if (limb) {
                LimbGemmArgs la{w + P.a_op, P.g.lda, P.a_shared ? 1 : 0, w + P.b_op, P.g.ldb, R, mc, N, K,
                                P.g.TA, P.g.TB, ctx->d_status, ctx->inject, P.amax, P.bmax, nullptr, 1, 0};
                la.bn = P.g.bn;
                ctx->inject = 0;
                SMF_CU(ctx, launch_gemm_limb(ctx, basis->dev, la, s));
            } else {
                Fp64GemmArgs fa{(const int32_t*)(w + P.a_op), P.a_shared ? 0 : mc * K, (const int32_t*)(w + P.b_op),
                                R, mc, N, K, (int)fp64_kblk(basis->primes[0], P.amax, P.bmax)};
                SMF_CU(ctx, launch_gemm_fp64(basis->dev, fa, s));
            }
        } else {
            SMF_CU(ctx, cudaMemsetAsync(R, 0, sizeof(int32_t) * (size_t)L * mc * N, s));
        }
        uint64_t* X = (uint64_t*)C->data + (size_t)m0 * C->ld * C->words;
        int64_t ldX = C->ld;
        if (!C->on_device) {
            // chunk c-2's copy-out has read this slot
            if (c >= 2) SMF_CU(ctx, cudaStreamWaitEvent(s, ev[kEvCFree + slot], 0));
            X = (uint64_t*)(w + P.c_stage[slot]);
            ldX = N;
        }
        {
            ProfScope ps(ctx, 3, s);
            SMF_CU(ctx, launch_crt(basis->crt, R, mc, N, X, ldX, C->words, s));
        }
        if (!C->on_device) {
            SMF_CU(ctx, cudaEventRecord(ev[kEvCReady + slot], s));
            SMF_CU(ctx, cudaStreamWaitEvent(hout, ev[kEvCReady + slot], 0));
            {
                ProfScope ps(ctx, 4, hout);
                SMF_CU(ctx, copy_rows((uint64_t*)C->data + (size_t)m0 * C->ld * C->words,
                                      (size_t)C->ld * C->words * 8, X, (size_t)N * C->words * 8,
                                      (size_t)N * C->words * 8, (size_t)mc, cudaMemcpyDeviceToHost, hout));
            }
            SMF_CU(ctx, cudaEventRecord(ev[kEvCFree + slot], hout));
        }
    }
    // the caller's stream orders after every copy of this product
    SMF_CU(ctx, cudaEventRecord(ev[kEvJoinIn], hin));
    SMF_CU(ctx, cudaStreamWaitEvent(s, ev[kEvJoinIn], 0));
    SMF_CU(ctx, cudaEventRecord(ev[kEvJoinOut], hout));
    SMF_CU(ctx, cudaStreamWaitEvent(s, ev[kEvJoinOut], 0));
    return SMF_OK;
}

}  // namespace

// ======================================================================== ABI

extern "C" {

const char* smf_version(void) { return "smf-gb300 0.1 (sm_103a)"; }

int smf_create(smf_ctx** out, int device, smf_form form, size_t hbm_budget_bytes) {
    if (!out) return SMF_E_INVALID;
    *out = nullptr;
    if (form != SMF_FORM_FP64 && form != SMF_FORM_INT8LIMB) return SMF_E_INVALID;
    int n = 0;
    if (cudaGetDeviceCount(&n) != cudaSuccess || device < 0 || device >= n) return SMF_E_INVALID;
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, device) != cudaSuccess) return SMF_E_CUDA;
    if (!(prop.major == 10 && prop.minor == 3)) return SMF_E_UNSUPPORTED;
    auto* c = new smf_ctx();
    c->device = device;
    c->form = form;
    c->budget = hbm_budget_bytes;
    c->num_sms = prop.multiProcessorCount;
    c->ws = nullptr;
    c->ws_bytes = 0;
    c->prof = false;
    c->inject = 0;
    c->aux = c->h2d = c->d2h = nullptr;
    c->ev_fork = c->ev_join = nullptr;
    for (auto& e : c->pev) e = nullptr;
    c->d_status = nullptr;
    c->gdesc_host = nullptr;
    c->gdesc_cap = 0;
    c->gdesc_ev = nullptr;
    DeviceGuard g(device);
    bool ok = cudaMalloc(&c->d_status, 256) == cudaSuccess && cudaMemset(c->d_status, 0, 256) == cudaSuccess &&
              cudaStreamSynchronize(cudaStreamLegacy) == cudaSuccess &&  // cleared before any stream reads it
              cudaStreamCreateWithFlags(&c->aux, cudaStreamNonBlocking) == cudaSuccess &&
              cudaStreamCreateWithFlags(&c->h2d, cudaStreamNonBlocking) == cudaSuccess &&
              cudaStreamCreateWithFlags(&c->d2h, cudaStreamNonBlocking) == cudaSuccess &&
              cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming) == cudaSuccess &&
              cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming) == cudaSuccess;
    for (auto& e : c->pev) ok = ok && cudaEventCreateWithFlags(&e, cudaEventDisableTiming) == cudaSuccess;
    ok = ok && cudaEventCreateWithFlags(&c->gdesc_ev, cudaEventDisableTiming) == cudaSuccess;
    if (!ok) {
        for (cudaStream_t st : {c->aux, c->h2d, c->d2h})
            if (st) cudaStreamDestroy(st);
        for (cudaEvent_t e : {c->ev_fork, c->ev_join})
            if (e) cudaEventDestroy(e);
        for (auto e : c->pev)
            if (e) cudaEventDestroy(e);
        if (c->gdesc_ev) cudaEventDestroy(c->gdesc_ev);
        if (c->d_status) cudaFree(c->d_status);
        delete c;
        return SMF_E_CUDA;
    }
    *out = c;
    return SMF_OK;
}

int smf_destroy(smf_ctx* c) {
    if (!c) return SMF_OK;
    DeviceGuard g(c->device);
    cudaDeviceSynchronize();
    for (auto& kv : c->basis_cache) smf_basis_destroy(kv.second);
    for (auto& r : c->prof_recs) {
        cudaEventDestroy(r.start);
        cudaEventDestroy(r.stop);
    }
    for (auto e : c->event_pool) cudaEventDestroy(e);
    if (c->ws) cudaFree(c->ws);
    if (c->d_status) cudaFree(c->d_status);
    for (cudaStream_t st : {c->aux, c->h2d, c->d2h})
        if (st) cudaStreamDestroy(st);
    for (cudaEvent_t e : {c->ev_fork, c->ev_join})
        if (e) cudaEventDestroy(e);
    for (auto e : c->pev)
        if (e) cudaEventDestroy(e);
    if (c->gdesc_ev) cudaEventDestroy(c->gdesc_ev);
    if (c->gdesc_host) cudaFreeHost(c->gdesc_host);
    for (void* ph : c->pinned)
        if (ph) cudaFreeHost(ph);
    delete c;
    return SMF_OK;
}

const char* smf_last_error(const smf_ctx* c) { return c ? c->err.c_str() : "null context"; }

int smf_basis_create(smf_ctx* ctx, int32_t bound_bits, uint32_t p_max, smf_basis** out) {
    if (!ctx || !out) return SMF_E_INVALID;
    return basis_build(ctx, bound_bits, p_max, out);
}

int smf_basis_destroy(smf_basis* b) {
    if (!b) return SMF_OK;
    if (b->dev_blob) {
        DeviceGuard g(b->device);
        cudaFree(b->dev_blob);
    }
    delete b;
    return SMF_OK;
}

int smf_basis_info(const smf_basis* b, int32_t* L, const uint32_t** primes) {
    if (!b) return SMF_E_INVALID;
    if (L) *L = (int32_t)b->primes.size();
    if (primes) *primes = b->primes.data();
    return SMF_OK;
}

int smf_rns_reduce(smf_ctx* ctx, const smf_basis* b, const smf_bigmat* X, int32_t* residues, void* stream) {
    if (!ctx || !b) return SMF_E_INVALID;
    int st = check_bigmat(ctx, X, "X", true);
    if (st) return st;
    if (X->rows * X->cols > 0 && !residues) return fail(ctx, SMF_E_INVALID, "residues: null");
    DeviceGuard g(ctx->device);
    cudaStream_t s = (cudaStream_t)stream;
    ReduceArgs a{(const uint64_t*)X->data, X->rows, X->cols, X->ld, X->words, residues, 0, 0, 0};
    ProfScope ps(ctx, 0, s);
    SMF_CU(ctx, launch_reduce(b->dev, a, ReduceOut::kCanonical, ctx->d_status, s));
    return SMF_OK;
}

int smf_residue_gemm_workspace(smf_ctx* ctx, const smf_basis* b, int64_t M, int64_t N, int64_t K, int a_shared,
                               size_t* bytes) {
    if (!ctx || !b || !bytes || M < 0 || N < 0 || K < 0) return SMF_E_INVALID;
    if (ctx->form == SMF_FORM_FP64) {
        *bytes = 0;
        return SMF_OK;
    }
    const uint32_t h0 = b->primes[0] / 2, hL = b->primes.back() / 2;
    *bytes = plan_limb((int)b->primes.size(), M, N, K, a_shared != 0, a_shared ? hL : h0, h0, ctx->num_sms).bytes;
    return SMF_OK;
}

int smf_residue_gemm(smf_ctx* ctx, const smf_basis* b, const int32_t* A, int64_t a_prime_stride, const int32_t* B,
                     int32_t* C, int64_t M, int64_t N, int64_t K, void* workspace, size_t workspace_bytes,
                     void* stream) {
    if (!ctx || !b) return SMF_E_INVALID;
    if (M < 0 || N < 0 || K < 0 || a_prime_stride < 0) return fail(ctx, SMF_E_INVALID, "residue_gemm: bad sizes");
    if (a_prime_stride != 0 && a_prime_stride < M * K)
        return fail(ctx, SMF_E_INVALID, "residue_gemm: a_prime_stride overlaps");
    if (M * N > 0 && (!C || (K > 0 && (!A || !B)))) return fail(ctx, SMF_E_INVALID, "residue_gemm: null operand");
    DeviceGuard g(ctx->device);
    const uint32_t h0 = b->primes[0] / 2, hL = b->primes.back() / 2;
    return run_residue_gemm_i32(ctx, b, A, a_prime_stride, B, C, M, N, K, a_prime_stride == 0 ? hL : h0, h0,
                                workspace, workspace_bytes, (cudaStream_t)stream);
}

int smf_crt_reconstruct(smf_ctx* ctx, const smf_basis* b, const int32_t* residues, smf_bigmat* X, void* stream) {
    if (!ctx || !b) return SMF_E_INVALID;
    int st = check_bigmat(ctx, X, "X_out", true);
    if (st) return st;
    if (64LL * X->words < b->m_bits) return fail(ctx, SMF_E_BOUND, "crt: output words cannot hold (-M/2, M/2]");
    if (b->primes.size() > 64) return fail(ctx, SMF_E_UNSUPPORTED, "crt: more than 64 primes");
    if (X->rows * X->cols > 0 && !residues) return fail(ctx, SMF_E_INVALID, "residues: null");
    DeviceGuard g(ctx->device);
    cudaStream_t s = (cudaStream_t)stream;
    ProfScope ps(ctx, 3, s);
    SMF_CU(ctx, launch_crt(b->crt, residues, X->rows, X->cols, (uint64_t*)X->data, X->ld, X->words, s));
    return SMF_OK;
}


int smf_base_convert(smf_ctx* ctx, const smf_basis* from, const smf_basis* to, const int32_t* residues_in,
                     int32_t* residues_out, int64_t count, void* stream) {
    if (!ctx) return SMF_E_INVALID;
    if (!from || !to || count < 0) return fail(ctx, SMF_E_INVALID, "base_convert: null basis or negative count");
    if (from->primes.size() > 48 || to->primes.size() > 48)
        return fail(ctx, SMF_E_UNSUPPORTED, "base_convert: more than 48 primes in a basis");
    if (count == 0) return SMF_OK;
    DeviceGuard g(ctx->device);
    if (!device_ptr(residues_in) || !device_ptr(residues_out))
        return fail(ctx, SMF_E_INVALID, "base_convert: residues must be device memory");
    cudaStream_t s = (cudaStream_t)stream;
    ProfScope ps(ctx, 3, s);
    SMF_CU(ctx, launch_convert(from->crt, to->primes.data(), (int)to->primes.size(), residues_in, residues_out, count,
                               ctx->num_sms, s));
    return SMF_OK;
}

int smf_rns_matmul_workspace(smf_ctx* ctx, const smf_bigmat* A, const smf_bigmat* B, const smf_bigmat* C,
                             size_t* bytes) {
    if (!ctx || !bytes) return SMF_E_INVALID;
    MatmulPlan P;
    smf_basis* b = nullptr;
    int st = plan_matmul(ctx, A, B, C, &P, &b);
    if (st) return st;
    *bytes = P.bytes;
    return SMF_OK;
}

int smf_rns_matmul(smf_ctx* ctx, const smf_bigmat* A, const smf_bigmat* B, smf_bigmat* C, void* workspace,
                   size_t workspace_bytes, void* stream) {
    if (!ctx) return SMF_E_INVALID;
    DeviceGuard dg(ctx->device);
    MatmulPlan P;
    smf_basis* basis = nullptr;
    int st = plan_matmul(ctx, A, B, C, &P, &basis);
    if (st) return st;
    cudaStream_t s = (cudaStream_t)stream;
    if (!workspace) {
        if (ctx->budget && P.bytes > ctx->budget) return fail(ctx, SMF_E_NOMEM, "rns_matmul: workspace over budget");
        if (ctx->ws_bytes < P.bytes) {
            if (ctx->ws) {
                cudaStreamSynchronize(s);
                cudaFree(ctx->ws);
                ctx->ws = nullptr;
                ctx->ws_bytes = 0;
            }
            SMF_CU(ctx, cudaMalloc(&ctx->ws, P.bytes));
            ctx->ws_bytes = P.bytes;
        }
        workspace = ctx->ws;
        workspace_bytes = ctx->ws_bytes;
    }
    if (workspace_bytes < P.bytes) return fail(ctx, SMF_E_NOMEM, "rns_matmul: workspace too small");
    uint8_t* w = (uint8_t*)workspace;
    const int64_t M = P.M, N = P.N, K = P.K;
    const int L = (int)basis->primes.size();
    if (M == 0 || N == 0) return SMF_OK;
    if (P.chunks > 1) return run_pipelined(ctx, P, basis, A, B, C, w, s);
    // operands on the device
    const uint64_t* dA = (const uint64_t*)A->data;
    const uint64_t* dB = (const uint64_t*)B->data;
    int64_t ldA = A->ld, ldB = B->ld;
    {
        ProfScope ps(ctx, 4, s);
        if (!A->on_device && M * K > 0) {
            SMF_CU(ctx, copy_rows(w + P.a_stage[0], (size_t)K * A->words * 8, A->data,
                                          (size_t)A->ld * A->words * 8, (size_t)K * A->words * 8, (size_t)M,
                                          cudaMemcpyHostToDevice, s));
            dA = (const uint64_t*)(w + P.a_stage[0]);
            ldA = K;
        }
        if (!B->on_device && K * N > 0) {
            SMF_CU(ctx, copy_rows(w + P.b_stage, (size_t)N * B->words * 8, B->data,
                                          (size_t)B->ld * B->words * 8, (size_t)N * B->words * 8, (size_t)K,
                                          cudaMemcpyHostToDevice, s));
            dB = (const uint64_t*)(w + P.b_stage);
            ldB = N;
        }
    }
    int32_t* R = (int32_t*)(w + P.r_off);
    if (K > 0) {
        ProfScope ps(ctx, 0, s);
        ReduceArgs ra{dA, M, K, ldA, A->words, w + P.a_op, 0, 0, P.a_shared ? 1 : 0, (int)entry_bits(A)};
        ReduceArgs rb{dB, K, N, ldB, B->words, w + P.b_op, 0, 0, 0, (int)entry_bits(B)};
        if (ctx->form == SMF_FORM_INT8LIMB) {
            ra.ld_out = P.g.lda;
            ra.t = P.g.TA;
            rb.ld_out = P.g.ldb;
            rb.t = P.g.TB;
            // A's digit split (memory bound) runs on the side stream while B's
            // reduction (integer bound) runs here; the join orders both before the GEMM
            SMF_CU(ctx, cudaEventRecord(ctx->ev_fork, s));
            SMF_CU(ctx, cudaStreamWaitEvent(ctx->aux, ctx->ev_fork, 0));
            SMF_CU(ctx, launch_reduce(basis->dev, ra, ReduceOut::kDigits, ctx->d_status, ctx->aux));
            SMF_CU(ctx, launch_reduce(basis->dev, rb, ReduceOut::kDigitsT, ctx->d_status, s));
            SMF_CU(ctx, cudaEventRecord(ctx->ev_join, ctx->aux));
            SMF_CU(ctx, cudaStreamWaitEvent(s, ctx->ev_join, 0));
        } else {
            SMF_CU(ctx, launch_reduce(basis->dev, ra, ReduceOut::kCentered, ctx->d_status, s));
            SMF_CU(ctx, launch_reduce(basis->dev, rb, ReduceOut::kCentered, ctx->d_status, s));
        }
    }
    uint64_t* dC = C->on_device ? (uint64_t*)C->data : (uint64_t*)(w + P.c_stage[0]);
    const int64_t ldC = C->on_device ? C->ld : N;
    bool fused = false;  // the CRT ran in the residue product's epilogue
    if (K == 0) {
        SMF_CU(ctx, cudaMemsetAsync(R, 0, sizeof(int32_t) * (size_t)L * M * N, s));
    } else {
        ProfScope ps(ctx, 2, s);
        if (ctx->form == SMF_FORM_INT8LIMB) {
            LimbGemmArgs la{w + P.a_op, P.g.lda, P.a_shared ? 1 : 0, w + P.b_op, P.g.ldb, R, M, N, K,
                            P.g.TA, P.g.TB, ctx->d_status, ctx->inject, P.amax, P.bmax,
                            (int32_t*)(w + P.part_op), P.g.split, P.g.kchunk};
            la.bn = P.g.bn;
            ctx->inject = 0;
            fused = ctx->fused_crt && limb_crt_fusable(basis->crt, la);
            if (fused)
                SMF_CU(ctx, launch_gemm_limb_crt(ctx, basis->dev, basis->crt, la, (int*)(w + P.cnt_off), dC, ldC,
                                                 C->words, s));
            else
                SMF_CU(ctx, launch_gemm_limb(ctx, basis->dev, la, s));
        } else {
            Fp64GemmArgs fa{(const int32_t*)(w + P.a_op), P.a_shared ? 0 : M * K, (const int32_t*)(w + P.b_op), R,
                            M, N, K, (int)fp64_kblk(basis->primes[0], P.amax, P.bmax)};
            SMF_CU(ctx, launch_gemm_fp64(basis->dev, fa, s));
        }
    }
    if (!fused) {
        ProfScope ps(ctx, 3, s);
        SMF_CU(ctx, launch_crt(basis->crt, R, M, N, dC, ldC, C->words, s));
    }
    if (!C->on_device) {
        ProfScope ps(ctx, 4, s);
        SMF_CU(ctx, copy_rows(C->data, (size_t)C->ld * C->words * 8, dC, (size_t)N * C->words * 8,
                                      (size_t)N * C->words * 8, (size_t)M, cudaMemcpyDeviceToHost, s));
    }
    return SMF_OK;
}

}  // extern "C"

namespace {

// One product of a grouped call.
struct GroupItem {
    int64_t M, N, K;
    bool a_shared;
    uint64_t amax, bmax;
    GemmPlan g;
    size_t ops, r_off;  // digit planes of A then B; residues [L][M][N]
};

// Launch descriptors of a grouped call, staged together: the products' tile
// descriptors, the digit-split and transposed-reduce work lists, the CRT list.
struct GroupDescs {
    size_t gemm = 0, split = 0, bt = 0, crt = 0, bytes = 0;
    explicit GroupDescs(int count) {
        split = align256(limb_group_desc_bytes(count));
        bt = split + align256(sizeof(ReduceItem) * (size_t)count);
        crt = bt + align256(sizeof(ReduceItem) * (size_t)count);
        bytes = crt + align256(sizeof(CrtItem) * (size_t)count);
    }
};

struct GroupPlan {
    smf_basis* basis = nullptr;
    bool grouped = false;  // limb form, and every product within the grouped GEMM's digit counts
    std::vector<GroupItem> items;
    size_t desc_off = 0, bytes = 0;
};

// The context's pinned staging buffer, at least `bytes` long, once the copy
// out of it by the previous grouped call has finished.
void* stage_host(smf_ctx* ctx, size_t bytes, cudaError_t* err) {
    *err = cudaSuccess;
    if (ctx->gdesc_host && (*err = cudaEventSynchronize(ctx->gdesc_ev)) != cudaSuccess) return nullptr;
    if (ctx->gdesc_cap < bytes) {
        if (ctx->gdesc_host) cudaFreeHost(ctx->gdesc_host);
        ctx->gdesc_host = nullptr;
        ctx->gdesc_cap = 0;
        const size_t cap = bytes < 65536 ? 65536 : bytes;
        if ((*err = cudaHostAlloc(&ctx->gdesc_host, cap, cudaHostAllocDefault)) != cudaSuccess) return nullptr;
        ctx->gdesc_cap = cap;
    }
    return ctx->gdesc_host;
}

// pad (optional, one flag per product): a shared A whose entries need fewer
// than three digits still takes three (the autotuner's alternative to the
// one- or two-digit tile; the extra digits are zero).
int plan_grouped(smf_ctx* ctx, int count, const smf_bigmat* A, const smf_bigmat* B, const smf_bigmat* C,
                 GroupPlan* G, const uint8_t* pad = nullptr) {
    if (count < 0 || (count > 0 && (!A || !B || !C)))
        return fail(ctx, SMF_E_INVALID, "rns_matmul_grouped: bad count or null arrays");
    int64_t bound = 0;
    for (int i = 0; i < count; i++) {
        int st;
        if ((st = check_bigmat(ctx, &A[i], "A[i]", true)) || (st = check_bigmat(ctx, &B[i], "B[i]", true)) ||
            (st = check_bigmat(ctx, &C[i], "C[i]", true)))
            return st;
        if (A[i].cols != B[i].rows || C[i].rows != A[i].rows || C[i].cols != B[i].cols)
            return fail(ctx, SMF_E_INVALID, "rns_matmul_grouped: shapes of product " + std::to_string(i) +
                                                " do not chain");
        const int64_t b_i = entry_bits(&A[i]) + entry_bits(&B[i]) + ceil_log2(std::max<int64_t>(A[i].cols, 1));
        if (64LL * C[i].words < b_i + 2)
            return fail(ctx, SMF_E_BOUND, "rns_matmul_grouped: C[" + std::to_string(i) + "].words cannot hold K*|A|*|B|");
        bound = std::max(bound, b_i);
    }
    if (bound > 100000) return fail(ctx, SMF_E_UNSUPPORTED, "rns_matmul_grouped: result bound too large");
    int st = SMF_OK;
    G->basis = cached_basis(ctx, (int)bound, default_pmax(ctx->form), &st);
    if (!G->basis) return st;
    const int L = (int)G->basis->primes.size();
    const uint64_t hL = G->basis->primes.back() / 2, h0 = G->basis->primes[0] / 2;
    size_t off = 0;
    auto slot = [&](size_t bytes) {
        size_t o = off;
        off = align256(off + bytes);
        return o;
    };
    G->grouped = ctx->form == SMF_FORM_INT8LIMB && L <= 64;
    G->items.resize(count);
    size_t single = 0;  // workspace of the largest single product (the loop used otherwise)
    for (int i = 0; i < count; i++) {
        GroupItem& it = G->items[i];
        it.M = A[i].rows;
        it.N = B[i].cols;
        it.K = A[i].cols;
        const int64_t ab = entry_bits(&A[i]);
        it.a_shared = ab < 62 && (1ull << ab) <= hL && ab <= 30;
        it.amax = it.a_shared ? (1ull << ab) : h0;
        if (pad && pad[i] && it.a_shared) it.amax = std::max<uint64_t>(it.amax, 1ull << 16);
        it.bmax = h0;
        it.g = plan_limb(L, it.M, it.N, it.K, it.a_shared, it.amax, it.bmax);
        LimbGemmArgs probe{};
        probe.TA = it.g.TA;
        probe.TB = it.g.TB;
        if (!limb_group_supported(probe) ||
            (unsigned __int128)std::max<int64_t>(it.K, 1) * it.amax * it.bmax >= ((unsigned __int128)1 << 62))
            G->grouped = false;
        size_t b1 = 0;
        if ((st = smf_rns_matmul_workspace(ctx, &A[i], &B[i], &C[i], &b1))) return st;
        single = std::max(single, b1);
    }
    if (!G->grouped) {
        G->bytes = single;
        return SMF_OK;
    }
    for (auto& it : G->items) {
        it.ops = slot(it.g.bytes);
        it.r_off = slot((size_t)4 * L * it.M * it.N);
    }
    G->desc_off = slot(GroupDescs(count).bytes);
    G->bytes = off;
    return SMF_OK;
}

// p-adic lifting: workspace slots and the descriptors of the per-step buffers.
struct LiftPlan {
    int64_t n = 0, m = 0;
    uint32_t p = 0;
    size_t bytes = 0;
    // FP64 form: each step through the generic calls
    smf_bigmat X64{}, AX{};  // X_i as words, A X_i (single words); data set at run time
    size_t rp_off = 0, x64_off = 0, ax_off = 0, gemm_off = 0, gemm_bytes = 0, mm_off = 0, mm_bytes = 0;
    // limb form: C R_i mod p (plan g1, one prime) and A X_i modulo the product
    // basis Q (plan g2); their partials stay in c1 / c2 for the step kernels
    bool fused = false;
    smf_basis* Q = nullptr;
    LiftBasis lq{};
    GemmPlan g1, g2;
    bool a_shared = false;
    uint64_t amax2 = 0, bmax2 = 0;
    size_t g1_off = 0, g2_off = 0, c1_off = 0, c2_off = 0;
};

int plan_lift_limb(smf_ctx* ctx, const smf_bigmat* A, int pbits, LiftPlan* P) {
    const int64_t n = P->n, m = P->m;
    int st;
    // |A X_i| <= n |A| (p - 1): the product basis covers bits(A) + bits(p) + ceil(log2 n)
    const int64_t ab = entry_bits(A);
    smf_basis* Q = cached_basis(ctx, (int)(ab + pbits + ceil_log2(std::max<int64_t>(n, 1))), default_pmax(ctx->form), &st);
    if (!Q) return st;
    const int LQ = (int)Q->primes.size();
    if (LQ > kLiftMaxPrimes) return fail(ctx, SMF_E_UNSUPPORTED, "padic_lift: product basis over four primes");
    P->Q = Q;
    P->lq.L = LQ;
    for (int j = 0; j < LQ; j++) {
        P->lq.q[j] = Q->primes[j];
        P->lq.inv[j] = Q->ginv[j];
    }
    const uint64_t h = P->p / 2, hL = Q->primes.back() / 2, h0 = Q->primes[0] / 2;
    P->a_shared = ab < 62 && (1ull << ab) <= hL && ab <= 30;
    P->amax2 = P->a_shared ? (1ull << ab) : h0;
    P->bmax2 = h0;
    // a narrow A still takes three digits when the 3 x 3-digit kernel, which
    // splits K over idle SMs, is expected to finish first
    {
        const int ta = digits_for(P->amax2), tb = digits_for(P->bmax2);
        if (ta < 3 && tb == 3 &&
            limb_cost(LQ, n, m, n, P->a_shared, 3, 3, ctx->num_sms) <
                limb_cost(LQ, n, m, n, P->a_shared, ta, tb, ctx->num_sms))
            P->amax2 = std::max<uint64_t>(P->amax2, 1ull << 16);
    }
    P->g1 = plan_limb(1, n, m, n, false, h, h, ctx->num_sms);
    P->g2 = plan_limb(LQ, n, m, n, P->a_shared, P->amax2, P->bmax2, ctx->num_sms);
    for (const GemmPlan* g : {&P->g1, &P->g2})
        if (g->TA > 3 || g->TB > 3) return fail(ctx, SMF_E_UNSUPPORTED, "limb form: more than 3 digits per residue");
    if ((unsigned __int128)n * h * h >= ((unsigned __int128)1 << 62) ||
        (unsigned __int128)n * P->amax2 * P->bmax2 >= ((unsigned __int128)1 << 62))
        return fail(ctx, SMF_E_UNSUPPORTED, "limb form: K * |a| * |b| must stay below 2^62");
    size_t off = 0;
    auto slot = [&](size_t bytes) {
        const size_t o = off;
        off = align256(off + bytes);
        return o;
    };
    P->g1_off = slot(P->g1.bytes);
    P->g2_off = slot(P->g2.bytes);
    P->c1_off = P->g1.split > 1 ? P->g1_off + P->g1.part_off : slot((size_t)4 * n * m);
    P->c2_off = P->g2.split > 1 ? P->g2_off + P->g2.part_off : slot((size_t)4 * LQ * n * m);
    P->fused = true;
    P->bytes = off;
    return SMF_OK;
}

int plan_lift(smf_ctx* ctx, const smf_basis* pb, const smf_bigmat* A, const smf_bigmat* B, LiftPlan* P) {
    if (!pb || pb->primes.size() != 1) return fail(ctx, SMF_E_INVALID, "padic_lift: the basis must hold one prime");
    int st;
    if ((st = check_bigmat(ctx, A, "A", true)) || (st = check_bigmat(ctx, B, "B", true))) return st;
    if (A->rows != A->cols || B->rows != A->rows)
        return fail(ctx, SMF_E_INVALID, "padic_lift: A must be n x n and B n x m");
    if (A->words != 1 || B->words != 1) return fail(ctx, SMF_E_INVALID, "padic_lift: single-word A and B");
    const int64_t n = A->rows, m = B->cols;
    const uint32_t p = pb->primes[0];
    int pbits = 0;
    while ((1ull << pbits) <= p) pbits++;  // p < 2^pbits
    // |R_i| <= max(|B|, 2 n |A| p) and |A X_i| < n |A| p must stay below 2^62
    if (entry_bits(A) + pbits + ceil_log2(std::max<int64_t>(n, 1)) + 2 > 62 || entry_bits(B) > 61)
        return fail(ctx, SMF_E_BOUND, "padic_lift: n |A| p or |B| too large for 64-bit residuals");
    P->n = n;
    P->m = m;
    P->p = p;
    if (ctx->form == SMF_FORM_INT8LIMB) return plan_lift_limb(ctx, A, pbits, P);
    size_t off = 0;
    auto slot = [&](size_t bytes) {
        const size_t o = off;
        off = align256(off + bytes);
        return o;
    };
    P->rp_off = slot(4 * (size_t)n * m);
    P->x64_off = slot(8 * (size_t)n * m);
    P->ax_off = slot(8 * (size_t)n * m);
    size_t gb = 0;
    if ((st = smf_residue_gemm_workspace(ctx, pb, n, m, n, 0, &gb))) return st;
    P->gemm_off = slot(gb);
    P->gemm_bytes = gb;
    // the exact product's plan needs only shapes and bounds: a placeholder address
    P->X64 = smf_bigmat{n, m, m, 1, pbits, (void*)256, 1, 0};
    P->AX = smf_bigmat{n, m, m, 1, 0, (void*)256, 1, 0};
    size_t mb = 0;
    if ((st = smf_rns_matmul_workspace(ctx, A, &P->X64, &P->AX, &mb))) return st;
    P->mm_off = slot(mb);
    P->mm_bytes = mb;
    P->bytes = off;
    return SMF_OK;
}

// A^-1 mod p: workspace slots.  The blocked form (limb form, residues of at
// most three digits, n above kInvBlockedMin) adds the panel scratch, the
// panel's transform, the pivot rows, the product and its operand planes.
constexpr int64_t kInvPanel = 128;
constexpr int64_t kInvBlockedMin = 256;

struct InverseLayout {
    size_t res = 0, M = 0, col = 0, flag = 0, T = 0, S = 0, Mp = 0, C = 0, gemm = 0, gemm_bytes = 0, bytes = 0;
};

bool inverse_blocked(const smf_ctx* ctx, int64_t n, int digits) {
    return ctx->form == SMF_FORM_INT8LIMB && n > kInvBlockedMin && digits <= 3;
}

InverseLayout inverse_layout(const smf_ctx* ctx, int64_t n, bool blocked) {
    InverseLayout Lw;
    size_t off = 0;
    auto slot = [&](size_t bytes) {
        const size_t o = off;
        off = align256(off + bytes);
        return o;
    };
    Lw.res = slot((size_t)4 * n * n);
    Lw.M = slot((size_t)8 * n * n);
    Lw.col = slot((size_t)4 * n);
    Lw.flag = slot(4);
    if (blocked) {
        Lw.T = slot((size_t)8 * n * kInvPanel);
        Lw.S = slot((size_t)4 * n * kInvPanel);
        Lw.Mp = slot((size_t)8 * n * kInvPanel);
        Lw.C = slot((size_t)8 * n * n);
        // the largest product plan over the panels (three-digit residues)
        for (int64_t c0 = 0; c0 < n; c0 += kInvPanel) {
            const int64_t b = std::min<int64_t>(kInvPanel, n - c0);
            const GemmPlan g = plan_limb(1, n, 2 * n - c0 - b, b, false, 1u << 23, 1u << 23, ctx->num_sms);
            Lw.gemm_bytes = std::max(Lw.gemm_bytes, g.bytes);
        }
        Lw.gemm = slot(Lw.gemm_bytes);
    }
    Lw.bytes = off;
    return Lw;
}

// The launch lists of a grouped call, built on the host: its descriptors are
// written into a staging buffer that one copy moves to the workspace.
struct GroupBuild {
    struct BtClass {
        int W, first, n;
        int64_t units;
    };
    int nsplit = 0, ncrt = 0;
    int64_t usplit = 0, ucrt = 0;
    std::vector<BtClass> classes;                                  // transposed reduce of B, one launch per W
    std::vector<std::pair<ReduceArgs, ReduceOut>> one_by_one;      // operands outside the grouped reduces
    std::vector<std::pair<int32_t*, size_t>> zero_res;             // K = 0: residues are zero
    std::vector<LimbGemmArgs> args;      // residue products in the 3x3-digit kernel
    LimbGroup lg{};
    std::vector<LimbGemmArgs> args_one;  // one-digit A in the one-digit kernel (kVarOneDigit)
    LimbGroup lg_one{};                  // its descriptors come first in the list
};

// Order of the products' tiles in the grouped residue-product launch.
constexpr int kOrderK = 0;     // longest K first
constexpr int kOrderWork = 1;  // most MMA work per tile first (K times A's digit count)

// Launch variants of one product in a grouped plan (bits): its narrow shared A
// padded to three digits; the residue-product producer prefetching K steps
// into L2 ahead of its loads; a one-digit A's product in the kernel whose ring
// holds five one-digit K steps (a launch of its own before the 3x3-digit one).
constexpr uint8_t kVarPad = 1, kVarPrefetch = 2, kVarOneDigit = 4;
constexpr int kPrefetchSteps = 4;

// Fill `hs` (GroupDescs(count).bytes, host) with the descriptors of plan G
// over the workspace `w`, and `out` with what the launches need.  var
// (optional, per product): kVarPrefetch sets the producer's L2 prefetch.
int build_grouped(smf_ctx* ctx, const GroupPlan& G, int count, const smf_bigmat* A, const smf_bigmat* B,
                  const smf_bigmat* C, uint8_t* w, uint8_t* hs, int order, int inject, GroupBuild* out,
                  const uint8_t* var = nullptr) {
    const smf_basis* basis = G.basis;
    const int L = (int)basis->primes.size();
    const GroupDescs D(count);
    ReduceItem* split = (ReduceItem*)(hs + D.split);
    ReduceItem* bt = (ReduceItem*)(hs + D.bt);
    CrtItem* crt = (CrtItem*)(hs + D.crt);
    GroupBuild& b = *out;
    std::vector<ReduceItem> bt_w[4];  // by W = 1, 2, 4, 8
    b.args.reserve(count);
    for (int i = 0; i < count; i++) {
        const GroupItem& it = G.items[i];
        if (it.M == 0 || it.N == 0) continue;
        int32_t* R = (int32_t*)(w + it.r_off);
        crt[b.ncrt++] = CrtItem{R, it.M, it.N, (uint64_t*)C[i].data, C[i].ld, C[i].words, b.ucrt};
        b.ucrt += crt_units(it.M, it.N);
        if (it.K == 0) {
            b.zero_res.emplace_back(R, sizeof(int32_t) * (size_t)L * it.M * it.N);
            continue;
        }
        void* adig = w + it.ops + it.g.a_off;
        void* bdig = w + it.ops + it.g.b_off;
        const ReduceArgs ra{(const uint64_t*)A[i].data, it.M, it.K, A[i].ld, A[i].words, adig, it.g.lda, it.g.TA,
                            it.a_shared ? 1 : 0, (int)entry_bits(&A[i])};
        const ReduceArgs rb{(const uint64_t*)B[i].data, it.K, it.N, B[i].ld, B[i].words, bdig, it.g.ldb, it.g.TB, 0,
                            (int)entry_bits(&B[i])};
        if (it.a_shared) {
            ReduceItem& si = split[b.nsplit++];
            si = ReduceItem{ra.X, ra.rows, ra.cols, ra.ld, adig, ra.ld_out, ra.W, ra.t, ra.bits, 0, b.usplit, 0u, 0};
            b.usplit += split_units(it.M, it.K, &si.div_m, &si.div_s);
        } else {
            b.one_by_one.emplace_back(ra, ReduceOut::kDigits);
        }
        if (reduce_t_groupable(basis->dev, rb)) {
            const int cls = rb.W == 1 ? 0 : rb.W == 2 ? 1 : rb.W == 4 ? 2 : 3;
            bt_w[cls].push_back(
                ReduceItem{rb.X, rb.rows, rb.cols, rb.ld, bdig, rb.ld_out, rb.W, rb.t, rb.bits, 0, 0, 0u, 0});
        } else {
            b.one_by_one.emplace_back(rb, ReduceOut::kDigitsT);
        }
        const bool one = var && (var[i] & kVarOneDigit) && it.g.TA == 1 && it.g.TB == 3;
        std::vector<LimbGemmArgs>& list = one ? b.args_one : b.args;
        const bool first = b.args.empty() && b.args_one.empty();
        list.push_back(LimbGemmArgs{adig, it.g.lda, it.a_shared ? 1 : 0, bdig, it.g.ldb, R, it.M, it.N, it.K, it.g.TA,
                                    it.g.TB, ctx->d_status, first ? inject : 0, it.amax, it.bmax});
        if (var && (var[i] & kVarPrefetch)) list.back().pf = kPrefetchSteps;
    }
    int nbt = 0;
    for (int c = 0; c < 4; c++) {
        if (bt_w[c].empty()) continue;
        GroupBuild::BtClass k{1 << c, nbt, 0, 0};
        for (ReduceItem r : bt_w[c]) {
            r.base = k.units;
            k.units += reduce_t_units(r.rows, r.cols, &r.rb);
            bt[nbt++] = r;
            k.n++;
        }
        b.classes.push_back(k);
    }
    SMF_CU(ctx, limb_group_encode(basis->dev, b.args_one.data(), (int)b.args_one.size(), hs + D.gemm, order,
                                  &b.lg_one));
    SMF_CU(ctx, limb_group_encode(basis->dev, b.args.data(), (int)b.args.size(),
                                  hs + D.gemm + limb_group_desc_bytes(b.lg_one.count), order, &b.lg));
    return SMF_OK;
}

// The launches of a grouped call whose descriptors are at `dd` (device): the
// digit split and reduces, the residue products, the CRT.  Only kernel
// launches and memsets, so the sequence can be captured in a CUDA graph.
int enqueue_grouped(smf_ctx* ctx, const GroupPlan& G, const GroupBuild& b, uint8_t* dd, cudaStream_t s) {
    const smf_basis* basis = G.basis;
    const int sms = ctx->num_sms;
    const GroupDescs D((int)G.items.size());
    {
        ProfScope ps(ctx, 0, s);
        for (auto& z : b.zero_res) SMF_CU(ctx, cudaMemsetAsync(z.first, 0, z.second, s));
        SMF_CU(ctx, launch_split_grouped((const ReduceItem*)(dd + D.split), b.nsplit, b.usplit, sms, ctx->d_status, s));
        for (const GroupBuild::BtClass& k : b.classes)
            SMF_CU(ctx, launch_reduce_t_grouped(basis->dev, k.W, (const ReduceItem*)(dd + D.bt) + k.first, k.n,
                                                k.units, sms, ctx->d_status, s));
        for (auto& r : b.one_by_one) SMF_CU(ctx, launch_reduce(basis->dev, r.first, r.second, ctx->d_status, s));
    }
    if (b.lg.count > 0 || b.lg_one.count > 0) {
        ProfScope ps(ctx, 2, s);
        SMF_CU(ctx, limb_group_launch_one_digit(ctx, basis->dev, b.args_one.data(), b.lg_one, dd + D.gemm, s));
        SMF_CU(ctx, limb_group_launch(ctx, basis->dev, b.args.data(), b.lg,
                                      dd + D.gemm + limb_group_desc_bytes(b.lg_one.count), s));
    }
    {
        ProfScope ps(ctx, 3, s);
        SMF_CU(ctx, launch_crt_grouped(basis->crt, (const CrtItem*)(dd + D.crt), b.ncrt, b.ucrt, sms, s));
    }
    return SMF_OK;
}

}  // namespace

extern "C" {

int smf_rns_matmul_grouped_workspace(smf_ctx* ctx, int count, const smf_bigmat* A, const smf_bigmat* B,
                                     const smf_bigmat* C, size_t* bytes) {
    if (!ctx || !bytes) return SMF_E_INVALID;
    DeviceGuard dg(ctx->device);
    GroupPlan G;
    const int st = plan_grouped(ctx, count, A, B, C, &G);
    if (st) return st;
    *bytes = G.bytes;
    return SMF_OK;
}

int smf_rns_matmul_grouped(smf_ctx* ctx, int count, const smf_bigmat* A, const smf_bigmat* B, smf_bigmat* C,
                           void* workspace, size_t workspace_bytes, void* stream) {
    if (!ctx) return SMF_E_INVALID;
    DeviceGuard dg(ctx->device);
    GroupPlan G;
    int st = plan_grouped(ctx, count, A, B, C, &G);
    if (st) return st;
    cudaStream_t s = (cudaStream_t)stream;
    if (!workspace && G.bytes > 0) {
        if (ctx->budget && G.bytes > ctx->budget)
            return fail(ctx, SMF_E_NOMEM, "rns_matmul_grouped: workspace over budget");
        if (ctx->ws_bytes < G.bytes) {
            if (ctx->ws) {
                cudaStreamSynchronize(s);
                cudaFree(ctx->ws);
                ctx->ws = nullptr;
                ctx->ws_bytes = 0;
            }
            SMF_CU(ctx, cudaMalloc(&ctx->ws, G.bytes));
            ctx->ws_bytes = G.bytes;
        }
        workspace = ctx->ws;
        workspace_bytes = ctx->ws_bytes;
    }
    if (workspace_bytes < G.bytes) return fail(ctx, SMF_E_NOMEM, "rns_matmul_grouped: workspace too small");
    if (!G.grouped) {  // FP64 form (or a product outside the 3x3-digit kernel): one product at a time
        for (int i = 0; i < count; i++)
            if ((st = smf_rns_matmul(ctx, &A[i], &B[i], &C[i], workspace, workspace_bytes, stream))) return st;
        return SMF_OK;
    }
    const GroupDescs D(count);
    cudaError_t ce;
    uint8_t* hs = (uint8_t*)stage_host(ctx, D.bytes, &ce);
    if (!hs) SMF_CU(ctx, ce);
    GroupBuild gb;
    if ((st = build_grouped(ctx, G, count, A, B, C, (uint8_t*)workspace, hs, kOrderK, ctx->inject, &gb))) return st;
    // every descriptor in one copy; the staging buffer is rewritten only after it
    uint8_t* dd = (uint8_t*)workspace + G.desc_off;
    SMF_CU(ctx, cudaMemcpyAsync(dd, hs, D.bytes, cudaMemcpyHostToDevice, s));
    SMF_CU(ctx, cudaEventRecord(ctx->gdesc_ev, s));
    if (gb.lg.count > 0 || gb.lg_one.count > 0) ctx->inject = 0;
    return enqueue_grouped(ctx, G, gb, dd, s);
}

}  // extern "C"

// A grouped product prepared once and replayed (smf_group_plan_*).
struct smf_group_plan {
    smf_ctx* ctx = nullptr;
    int device = 0;
    int count = 0;
    std::vector<smf_bigmat> A, B, C;  // the operands (their buffers stay fixed)
    bool grouped = false;             // limb form through the grouped kernels; else one product per call
    void* ws = nullptr;               // plan-owned workspace
    size_t ws_bytes = 0;
    cudaGraphExec_t exec = nullptr;   // the captured launches (null: nothing to launch)
    int order = 0;
    std::vector<uint8_t> var;         // per product: kVarPad | kVarPrefetch
    int padded = 0, prefetched = 0, one_digit = 0, classes_tuned = 0, classes_cached = 0;
    double tune_ms = 0;
    std::string report;
};

namespace {

// Product class of the autotuner: basis size, A's natural digit count, a
// shared A, and the rounded-up log2 of K, M and N.
uint64_t tune_key(int L, const GroupItem& it) {
    return (uint64_t)L | ((uint64_t)it.g.TA << 8) | ((uint64_t)(it.a_shared ? 1 : 0) << 11) |
           ((uint64_t)ceil_log2(it.K) << 12) | ((uint64_t)ceil_log2(it.M) << 20) | ((uint64_t)ceil_log2(it.N) << 28);
}

std::vector<uint8_t> pad_bits(const std::vector<uint8_t>& var) {
    std::vector<uint8_t> p(var.size());
    for (size_t i = 0; i < var.size(); i++) p[i] = var[i] & kVarPad;
    return p;
}

const char* var_name(int v) {
    switch (v) {
        case 0: return "natural";
        case kVarPad: return "three digits";
        case kVarPrefetch: return "natural+prefetch";
        case kVarOneDigit: return "one-digit kernel";
        default: return "three digits+prefetch";
    }
}

// Median device time of `reps` grouped launches (after one untimed) over the
// products idx of (A, B, C) with launch variants var_all[i] and tile order
// `order`, run in the workspace ws.  The products' outputs are written.
int time_grouped(smf_ctx* ctx, const std::vector<int>& idx, const smf_bigmat* A, const smf_bigmat* B,
                 const smf_bigmat* C, const std::vector<uint8_t>& var_all, int order, void* ws, size_t ws_bytes,
                 cudaStream_t s, int reps, double* ms) {
    const int n = (int)idx.size();
    std::vector<smf_bigmat> a, b, c;
    std::vector<uint8_t> vr;
    for (int i : idx) {
        a.push_back(A[i]);
        b.push_back(B[i]);
        c.push_back(C[i]);
        vr.push_back(var_all[i]);
    }
    GroupPlan G;
    int st = plan_grouped(ctx, n, a.data(), b.data(), c.data(), &G, pad_bits(vr).data());
    if (st) return st;
    if (!G.grouped || G.bytes > ws_bytes) return fail(ctx, SMF_E_INVALID, "group plan: autotune workspace");
    std::vector<uint8_t> hs(GroupDescs(n).bytes);
    GroupBuild gb;
    if ((st = build_grouped(ctx, G, n, a.data(), b.data(), c.data(), (uint8_t*)ws, hs.data(), order, 0, &gb,
                            vr.data())))
        return st;
    uint8_t* dd = (uint8_t*)ws + G.desc_off;
    SMF_CU(ctx, cudaMemcpyAsync(dd, hs.data(), hs.size(), cudaMemcpyHostToDevice, s));
    SMF_CU(ctx, cudaStreamSynchronize(s));
    std::vector<cudaEvent_t> ev(2 * reps, nullptr);
    for (auto& e : ev) SMF_CU(ctx, cudaEventCreate(&e));
    std::vector<float> t(reps, 0.f);
    for (int r = -1; r < reps && !st; r++) {
        if (r >= 0) cudaEventRecord(ev[2 * r], s);
        st = enqueue_grouped(ctx, G, gb, dd, s);
        if (r >= 0) cudaEventRecord(ev[2 * r + 1], s);
    }
    cudaError_t ce = cudaStreamSynchronize(s);
    for (int r = 0; r < reps && ce == cudaSuccess && !st; r++) ce = cudaEventElapsedTime(&t[r], ev[2 * r], ev[2 * r + 1]);
    for (auto& e : ev) cudaEventDestroy(e);
    if (st) return st;
    SMF_CU(ctx, ce);
    std::sort(t.begin(), t.end());
    *ms = t[reps / 2];
    return SMF_OK;
}

// The autotuner of a grouped plan (flag SMF_PLAN_AUTOTUNE): per class of
// products, the class alone in each of its candidate variants (natural, with
// the producer's L2 prefetch, and for a shared A of one or two digits also
// padded to three digits), the fastest kept and remembered by the context for
// later plans; then, when digit counts differ in the batch, the whole batch in
// both tile orders.
int autotune_plan(smf_group_plan* P, cudaStream_t s) {
    smf_ctx* ctx = P->ctx;
    const int count = P->count;
    GroupPlan G0, Gpad;
    int st = plan_grouped(ctx, count, P->A.data(), P->B.data(), P->C.data(), &G0);
    if (st) return st;
    std::vector<uint8_t> ones(count, 1);
    if ((st = plan_grouped(ctx, count, P->A.data(), P->B.data(), P->C.data(), &Gpad, ones.data()))) return st;
    const int L = (int)G0.basis->primes.size();
    std::vector<std::pair<uint64_t, std::vector<int>>> classes;
    for (int i = 0; i < count; i++) {
        const GroupItem& it = G0.items[i];
        if (it.M == 0 || it.N == 0 || it.K == 0) continue;
        const uint64_t key = tune_key(L, it);
        auto c = std::find_if(classes.begin(), classes.end(), [&](const auto& x) { return x.first == key; });
        if (c == classes.end()) classes.push_back({key, {i}});
        else c->second.push_back(i);
    }
    const size_t tb = std::max(G0.bytes, Gpad.bytes);
    if (ctx->budget && tb > ctx->budget) return fail(ctx, SMF_E_NOMEM, "group plan: autotune workspace over budget");
    void* tws = nullptr;
    SMF_CU(ctx, cudaMalloc(&tws, tb));
    const auto t0 = std::chrono::steady_clock::now();
    char line[512];
    for (const auto& c : classes) {
        auto hit = std::find_if(ctx->tune_cache.begin(), ctx->tune_cache.end(),
                                [&](const auto& x) { return x.first == c.first; });
        const GroupItem& it = G0.items[c.second[0]];
        const int n0 = snprintf(line, sizeof line, "class ta=%d%s K<=2^%lld M<=2^%lld N<=2^%lld: %zu products", it.g.TA,
                                it.a_shared ? " shared" : "", (long long)ceil_log2(it.K), (long long)ceil_log2(it.M),
                                (long long)ceil_log2(it.N), c.second.size());
        int choice = 0;
        if (hit != ctx->tune_cache.end()) {
            choice = hit->second;
            P->classes_cached++;
            snprintf(line + n0, sizeof line - n0, ", cached -> %s\n", var_name(choice));
        } else {
            std::vector<int> cand{0, kVarPrefetch};
            if (it.a_shared && it.g.TA < 3) cand.push_back(kVarPad);
            if (it.g.TA == 1) cand.push_back(kVarOneDigit);
            std::vector<uint8_t> vr(count, 0);
            double best = 0;
            int n1 = n0;
            for (int v : cand) {
                for (int i : c.second) vr[i] = (uint8_t)v;
                double ms = 0;
                if ((st = time_grouped(ctx, c.second, P->A.data(), P->B.data(), P->C.data(), vr, kOrderK, tws, tb, s,
                                       3, &ms)))
                    break;
                n1 += snprintf(line + n1, sizeof line - n1, ", %s %.4f ms", var_name(v), ms);
                if (v == 0 || ms < best) {
                    best = ms;
                    choice = v;
                }
            }
            if (st) break;
            snprintf(line + n1, sizeof line - n1, " -> %s\n", var_name(choice));
            ctx->tune_cache.push_back({c.first, choice});
            P->classes_tuned++;
        }
        P->report += line;
        for (int i : c.second) P->var[i] = (uint8_t)choice;
    }
    // tile order, when the batch mixes digit counts
    bool mixed = false;
    int ta_first = 0;
    for (int i = 0; i < count && !st; i++) {
        const GroupItem& it = G0.items[i];
        if (it.M == 0 || it.N == 0 || it.K == 0) continue;
        const int ta = (P->var[i] & kVarPad) ? 3 : it.g.TA;
        if (!ta_first) ta_first = ta;
        mixed |= ta != ta_first;
    }
    if (mixed && !st) {
        std::vector<int> all(count);
        for (int i = 0; i < count; i++) all[i] = i;
        double ms[2] = {0, 0};
        for (int o = 0; o < 2 && !st; o++)
            st = time_grouped(ctx, all, P->A.data(), P->B.data(), P->C.data(), P->var, o, tws, tb, s, 3, &ms[o]);
        if (!st) {
            P->order = ms[1] < ms[0] ? kOrderWork : kOrderK;
            snprintf(line, sizeof line, "tile order: longest K first %.4f ms, most MMAs first %.4f ms -> %s\n", ms[0],
                     ms[1], P->order ? "most MMAs first" : "longest K first");
            P->report += line;
        }
    }
    cudaStreamSynchronize(s);
    cudaFree(tws);
    P->tune_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    return st;
}

void free_plan(smf_group_plan* P) {
    if (!P) return;
    if (P->exec) cudaGraphExecDestroy(P->exec);
    if (P->ws) cudaFree(P->ws);
    delete P;
}

}  // namespace

extern "C" {

int smf_group_plan_create(smf_ctx* ctx, int count, const smf_bigmat* A, const smf_bigmat* B, smf_bigmat* C,
                          int flags, smf_group_plan** out, void* stream) {
    if (!ctx || !out) return SMF_E_INVALID;
    *out = nullptr;
    DeviceGuard dg(ctx->device);
    cudaStream_t s = (cudaStream_t)stream;
    GroupPlan G;
    int st = plan_grouped(ctx, count, A, B, C, &G);
    if (st) return st;
    auto* P = new smf_group_plan();
    P->ctx = ctx;
    P->device = ctx->device;
    P->count = count;
    P->A.assign(A, A + count);
    P->B.assign(B, B + count);
    P->C.assign(C, C + count);
    P->grouped = G.grouped;
    const uint8_t fixed = (uint8_t)(((flags & SMF_PLAN_PAD_ALL) ? kVarPad : 0) |
                                    ((flags & SMF_PLAN_PREFETCH) ? kVarPrefetch : 0) |
                                    ((flags & SMF_PLAN_ONE_DIGIT) ? kVarOneDigit : 0));
    P->var.assign(count, fixed);
    P->order = (flags & SMF_PLAN_ORDER_WORK) ? kOrderWork : kOrderK;
    if (P->grouped && (flags & SMF_PLAN_AUTOTUNE) && count > 0) {
        std::fill(P->var.begin(), P->var.end(), 0);
        P->order = kOrderK;
        if ((st = autotune_plan(P, s))) {
            free_plan(P);
            return st;
        }
    }
    const GroupPlan G0 = G;  // natural digit counts
    if (P->grouped && (st = plan_grouped(ctx, count, A, B, C, &G, pad_bits(P->var).data()))) {
        free_plan(P);
        return st;
    }
    for (int i = 0; i < count && P->grouped; i++) {
        const GroupItem& it = G.items[i];
        const bool live = it.K > 0 && it.M > 0 && it.N > 0;
        P->padded += live && it.g.TA > G0.items[i].g.TA;
        P->prefetched += live && (P->var[i] & kVarPrefetch);
        P->one_digit += live && (P->var[i] & kVarOneDigit) && it.g.TA == 1;
    }
    if (ctx->budget && G.bytes > ctx->budget) {
        free_plan(P);
        return fail(ctx, SMF_E_NOMEM, "group plan: workspace over budget");
    }
    P->ws_bytes = G.bytes;
    if (G.bytes > 0) {
        const cudaError_t e = cudaMalloc(&P->ws, G.bytes);
        if (e != cudaSuccess) {
            cudaGetLastError();
            P->ws = nullptr;
            free_plan(P);
            return fail(ctx, SMF_E_NOMEM, std::string("group plan: workspace: ") + cudaGetErrorString(e));
        }
    }
    if (!P->grouped) {  // FP64 form, or a product outside the grouped kernels: one product per call
        *out = P;
        return SMF_OK;
    }
    std::vector<uint8_t> hs(GroupDescs(count).bytes);
    GroupBuild gb;
    if ((st = build_grouped(ctx, G, count, A, B, C, (uint8_t*)P->ws, hs.data(), P->order, 0, &gb, P->var.data()))) {
        free_plan(P);
        return st;
    }
    if (gb.zero_res.empty() && !gb.nsplit && gb.classes.empty() && gb.one_by_one.empty() && !gb.lg.count &&
        !gb.lg_one.count && !gb.ncrt) {  // every product empty: nothing to launch
        *out = P;
        return SMF_OK;
    }
    uint8_t* dd = (uint8_t*)P->ws + G.desc_off;
    cudaError_t ce = cudaMemcpyAsync(dd, hs.data(), hs.size(), cudaMemcpyHostToDevice, s);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(s);
    cudaStream_t cs = nullptr;
    if (ce == cudaSuccess) ce = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
    if (ce != cudaSuccess) {
        if (cs) cudaStreamDestroy(cs);
        free_plan(P);
        return fail(ctx, SMF_E_CUDA, std::string("group plan: ") + cudaGetErrorString(ce));
    }
    // the launches, captured once (profiling scopes off: a graph replays no events)
    const bool prof = ctx->prof;
    ctx->prof = false;
    cudaGraph_t graph = nullptr;
    ce = cudaStreamBeginCapture(cs, cudaStreamCaptureModeRelaxed);
    if (ce == cudaSuccess) {
        st = enqueue_grouped(ctx, G, gb, dd, cs);
        ce = cudaStreamEndCapture(cs, &graph);
    }
    ctx->prof = prof;
    if (ce == cudaSuccess && !st) ce = cudaGraphInstantiate(&P->exec, graph, 0);
    if (graph) cudaGraphDestroy(graph);
    cudaStreamDestroy(cs);
    if (st || ce != cudaSuccess) {
        free_plan(P);
        return st ? st : fail(ctx, SMF_E_CUDA, std::string("group plan: capture: ") + cudaGetErrorString(ce));
    }
    *out = P;
    return SMF_OK;
}

int smf_group_plan_launch(smf_group_plan* P, void* stream) {
    if (!P) return SMF_E_INVALID;
    smf_ctx* ctx = P->ctx;
    DeviceGuard dg(ctx->device);
    if (P->grouped) {
        if (P->exec) SMF_CU(ctx, cudaGraphLaunch(P->exec, (cudaStream_t)stream));
        return SMF_OK;
    }
    for (int i = 0; i < P->count; i++) {
        const int st = smf_rns_matmul(ctx, &P->A[i], &P->B[i], &P->C[i], P->ws, P->ws_bytes, stream);
        if (st) return st;
    }
    return SMF_OK;
}

int smf_group_plan_info(const smf_group_plan* P, int32_t* graph, int32_t* padded, int32_t* prefetched,
                        int32_t* one_digit, int32_t* tile_order, int32_t* classes_tuned, int32_t* classes_cached,
                        double* tune_ms, size_t* workspace_bytes) {
    if (!P) return SMF_E_INVALID;
    if (graph) *graph = P->grouped ? 1 : 0;
    if (padded) *padded = P->padded;
    if (prefetched) *prefetched = P->prefetched;
    if (one_digit) *one_digit = P->one_digit;
    if (tile_order) *tile_order = P->order;
    if (classes_tuned) *classes_tuned = P->classes_tuned;
    if (classes_cached) *classes_cached = P->classes_cached;
    if (tune_ms) *tune_ms = P->tune_ms;
    if (workspace_bytes) *workspace_bytes = P->ws_bytes;
    return SMF_OK;
}

int smf_group_plan_report(const smf_group_plan* P, char* buf, int64_t cap) {
    if (!P || !buf || cap <= 0) return SMF_E_INVALID;
    const size_t n = std::min<size_t>(P->report.size(), (size_t)cap - 1);
    memcpy(buf, P->report.data(), n);
    buf[n] = 0;
    return SMF_OK;
}

int smf_group_plan_destroy(smf_group_plan* P) {
    if (!P) return SMF_OK;
    DeviceGuard dg(P->device);  // the context may already be gone
    free_plan(P);
    return SMF_OK;
}

int smf_padic_lift_workspace(smf_ctx* ctx, const smf_basis* p_basis, const smf_bigmat* A, const smf_bigmat* B,
                             size_t* bytes) {
    if (!ctx || !bytes) return SMF_E_INVALID;
    DeviceGuard g(ctx->device);
    LiftPlan P;
    const int st = plan_lift(ctx, p_basis, A, B, &P);
    if (st) return st;
    *bytes = P.bytes;
    return SMF_OK;
}

int smf_padic_lift(smf_ctx* ctx, const smf_basis* p_basis, const smf_bigmat* A, const int32_t* A_inv_mod_p,
                   const smf_bigmat* B, int32_t steps, int32_t* X_digits, smf_bigmat* R, void* workspace,
                   size_t workspace_bytes, void* stream) {
    if (!ctx) return SMF_E_INVALID;
    DeviceGuard dg(ctx->device);
    LiftPlan P;
    int st = plan_lift(ctx, p_basis, A, B, &P);
    if (st) return st;
    if (steps < 0) return fail(ctx, SMF_E_INVALID, "padic_lift: negative step count");
    if ((st = check_bigmat(ctx, R, "R", true))) return st;
    if (R->rows != P.n || R->cols != P.m || R->words != 1)
        return fail(ctx, SMF_E_INVALID, "padic_lift: R must be n x m single-word entries");
    if (P.n * P.m == 0) return SMF_OK;
    if (!device_ptr(A_inv_mod_p) || (steps > 0 && !device_ptr(X_digits)))
        return fail(ctx, SMF_E_INVALID, "padic_lift: A_inv_mod_p and X_digits must be device memory");
    cudaStream_t s = (cudaStream_t)stream;
    if (!workspace && P.bytes > 0) {
        if (ctx->budget && P.bytes > ctx->budget) return fail(ctx, SMF_E_NOMEM, "padic_lift: workspace over budget");
        if (ctx->ws_bytes < P.bytes) {
            if (ctx->ws) {
                cudaStreamSynchronize(s);
                cudaFree(ctx->ws);
                ctx->ws = nullptr;
                ctx->ws_bytes = 0;
            }
            SMF_CU(ctx, cudaMalloc(&ctx->ws, P.bytes));
            ctx->ws_bytes = P.bytes;
        }
        workspace = ctx->ws;
        workspace_bytes = ctx->ws_bytes;
    }
    if (workspace_bytes < P.bytes) return fail(ctx, SMF_E_NOMEM, "padic_lift: workspace too small");
    uint8_t* w = (uint8_t*)workspace;
    int32_t* Rp = (int32_t*)(w + P.rp_off);
    int64_t* X64 = (int64_t*)(w + P.x64_off);
    int64_t* AX = (int64_t*)(w + P.ax_off);
    P.X64.data = X64;
    P.AX.data = AX;
    if (R->data != B->data)
        SMF_CU(ctx, copy_rows(R->data, (size_t)R->ld * 8, B->data, (size_t)B->ld * 8, (size_t)P.m * 8, (size_t)P.n,
                              cudaMemcpyDeviceToDevice, s));
    const uint64_t h = P.p / 2;
    if (P.fused) {
        uint8_t* w1 = w + P.g1_off;
        uint8_t* w2 = w + P.g2_off;
        void* cdig = w1 + P.g1.a_off;
        void* rdig = w1 + P.g1.b_off;
        void* adig = w2 + P.g2.a_off;
        void* xdig = w2 + P.g2.b_off;
        int32_t* c1 = (int32_t*)(w + P.c1_off);
        int32_t* c2 = (int32_t*)(w + P.c2_off);
        const int64_t n = P.n, m = P.m;
        if (steps > 0) {  // the operands' digit planes: C and A once, R_0 = B for the first step
            SMF_CU(ctx, launch_residue_digits(p_basis->dev, A_inv_mod_p, n * n, 1, n, n, cdig, P.g1.lda, P.g1.TA,
                                              false, s));
            const ReduceArgs ra{(const uint64_t*)A->data, n, n, A->ld, 1, adig, P.g2.lda, P.g2.TA,
                                P.a_shared ? 1 : 0, (int)entry_bits(A)};
            SMF_CU(ctx, launch_reduce(P.Q->dev, ra, ReduceOut::kDigits, ctx->d_status, s));
            const ReduceArgs rr{(const uint64_t*)R->data, n, m, R->ld, 1, rdig, P.g1.ldb, P.g1.TB, 0};
            SMF_CU(ctx, launch_reduce(p_basis->dev, rr, ReduceOut::kDigitsT, ctx->d_status, s));
        }
        for (int32_t i = 0; i < steps; i++) {
            int32_t* Xi = X_digits + (size_t)i * n * m;
            LimbGemmArgs l1{cdig, P.g1.lda, 0, rdig, P.g1.ldb, c1, n, m, n, P.g1.TA, P.g1.TB, ctx->d_status,
                            ctx->inject, h, h, c1, P.g1.split, P.g1.kchunk, 1, 1};
            l1.bn = P.g1.bn;
            ctx->inject = 0;
            SMF_CU(ctx, launch_gemm_limb(ctx, p_basis->dev, l1, s));
            SMF_CU(ctx, launch_lift_x(c1, P.g1.split, n, m, P.p, Xi, P.lq, xdig, P.g2.ldb, P.g2.TB, s));
            LimbGemmArgs l2{adig, P.g2.lda, P.a_shared ? 1 : 0, xdig, P.g2.ldb, c2, n, m, n, P.g2.TA,
                            P.g2.TB, ctx->d_status, 0, P.amax2, P.bmax2, c2, P.g2.split, P.g2.kchunk, 1, 1};
            l2.bn = P.g2.bn;
            SMF_CU(ctx, launch_gemm_limb(ctx, P.Q->dev, l2, s));
            SMF_CU(ctx, launch_lift_step(c2, P.g2.split, n, m, P.lq, (int64_t*)R->data, R->ld, P.p,
                                         i + 1 < steps ? rdig : nullptr, P.g1.ldb, P.g1.TB, ctx->d_status, s));
        }
        return SMF_OK;
    }
    for (int32_t i = 0; i < steps; i++) {
        // R_i mod p, X_i = C R_i mod p, A X_i exactly, R_(i+1) = (R_i - A X_i) / p
        const ReduceArgs ra{(const uint64_t*)R->data, P.n, P.m, R->ld, 1, Rp, 0, 0, 0};
        SMF_CU(ctx, launch_reduce(p_basis->dev, ra, ReduceOut::kCanonical, ctx->d_status, s));
        int32_t* Xi = X_digits + (size_t)i * P.n * P.m;
        if ((st = run_residue_gemm_i32(ctx, p_basis, A_inv_mod_p, P.n * P.n, Rp, Xi, P.n, P.m, P.n, h, h,
                                       w + P.gemm_off, P.gemm_bytes, s)))
            return st;
        SMF_CU(ctx, launch_widen(Xi, P.n * P.m, X64, s));
        if ((st = smf_rns_matmul(ctx, A, &P.X64, &P.AX, w + P.mm_off, P.mm_bytes, s))) return st;
        SMF_CU(ctx, launch_lift_update((int64_t*)R->data, R->ld, AX, P.n, P.m, P.p, ctx->d_status, s));
    }
    return SMF_OK;
}

int smf_inverse_mod_p_workspace(smf_ctx* ctx, int64_t n, size_t* bytes) {
    if (!ctx || !bytes || n < 0) return SMF_E_INVALID;
    *bytes = inverse_layout(ctx, n, inverse_blocked(ctx, n, 3)).bytes;
    return SMF_OK;
}

int smf_inverse_mod_p(smf_ctx* ctx, const smf_basis* p_basis, const smf_bigmat* A, int32_t* A_inv, void* workspace,
                      size_t workspace_bytes, void* stream) {
    if (!ctx) return SMF_E_INVALID;
    DeviceGuard dg(ctx->device);
    if (!p_basis || p_basis->primes.size() != 1)
        return fail(ctx, SMF_E_INVALID, "inverse_mod_p: the basis must hold one prime");
    int st;
    if ((st = check_bigmat(ctx, A, "A", true))) return st;
    if (A->rows != A->cols) return fail(ctx, SMF_E_INVALID, "inverse_mod_p: A must be square");
    const int64_t n = A->rows;
    if (n == 0) return SMF_OK;
    if (!device_ptr(A_inv)) return fail(ctx, SMF_E_INVALID, "inverse_mod_p: A_inv must be device memory");
    const uint32_t p = p_basis->primes[0];
    const bool blocked = inverse_blocked(ctx, n, digits_for(p / 2));
    const InverseLayout Lw = inverse_layout(ctx, n, blocked);
    cudaStream_t s = (cudaStream_t)stream;
    if (!workspace) {
        if (ctx->budget && Lw.bytes > ctx->budget) return fail(ctx, SMF_E_NOMEM, "inverse_mod_p: workspace over budget");
        if (ctx->ws_bytes < Lw.bytes) {
            if (ctx->ws) {
                cudaStreamSynchronize(s);
                cudaFree(ctx->ws);
                ctx->ws = nullptr;
                ctx->ws_bytes = 0;
            }
            SMF_CU(ctx, cudaMalloc(&ctx->ws, Lw.bytes));
            ctx->ws_bytes = Lw.bytes;
        }
        workspace = ctx->ws;
        workspace_bytes = ctx->ws_bytes;
    }
    if (workspace_bytes < Lw.bytes) return fail(ctx, SMF_E_NOMEM, "inverse_mod_p: workspace too small");
    uint8_t* w = (uint8_t*)workspace;
    int32_t* res = (int32_t*)(w + Lw.res);
    uint32_t* M = (uint32_t*)(w + Lw.M);
    uint32_t* col = (uint32_t*)(w + Lw.col);
    int* flag = (int*)(w + Lw.flag);
    const ReduceArgs ra{(const uint64_t*)A->data, n, n, A->ld, A->words, res, 0, 0, 0};
    SMF_CU(ctx, launch_reduce(p_basis->dev, ra, ReduceOut::kCanonical, ctx->d_status, s));
    if (!blocked) {
        SMF_CU(ctx, launch_inverse_mod_p(res, n, p, M, col, flag, A_inv, ctx->d_status, ctx->num_sms, s));
        return SMF_OK;
    }
    // panels of kInvPanel columns; the rest of the elimination of each panel is
    // one residue product with the panel's transform (inverse.cu)
    uint32_t* T = (uint32_t*)(w + Lw.T);
    int32_t* Sc = (int32_t*)(w + Lw.S);
    int32_t* Mp = (int32_t*)(w + Lw.Mp);
    int32_t* Cb = (int32_t*)(w + Lw.C);
    const int64_t ld = 2 * n;
    const uint64_t h = p / 2;
    SMF_CU(ctx, cudaMemsetAsync(flag, 0, sizeof(int), s));
    SMF_CU(ctx, launch_gj_init(res, n, M, s));
    for (int64_t c0 = 0; c0 < n; c0 += kInvPanel) {
        const int64_t b = std::min<int64_t>(kInvPanel, n - c0), c1 = c0 + b, R = ld - c1;
        SMF_CU(ctx, cudaMemcpy2DAsync(T, 8 * b, M + c0, 4 * ld, 4 * b, n, cudaMemcpyDeviceToDevice, s));
        SMF_CU(ctx, cudaMemset2DAsync(T + b, 8 * b, 0, 4 * b, n, s));
        SMF_CU(ctx, launch_panel_factor(T, n, (int)b, c0, M, ld, c1, ld, p, col, flag, ctx->d_status, ctx->num_sms, s));
        SMF_CU(ctx, cudaMemcpy2DAsync(Sc, 4 * b, T + b, 8 * b, 4 * b, n, cudaMemcpyDeviceToDevice, s));
        SMF_CU(ctx, cudaMemcpy2DAsync(Mp, 4 * R, M + c0 * ld + c1, 4 * ld, 4 * R, b, cudaMemcpyDeviceToDevice, s));
        if ((st = run_residue_gemm_i32(ctx, p_basis, Sc, n * b, Mp, Cb, n, R, b, h, h, w + Lw.gemm, Lw.gemm_bytes, s)))
            return st;
        SMF_CU(ctx, launch_panel_update(M, ld, n, c0, c1, R, Cb, p, s));
    }
    SMF_CU(ctx, cudaMemcpy2DAsync(A_inv, 4 * n, M + n, 4 * ld, 4 * n, n, cudaMemcpyDeviceToDevice, s));
    return SMF_OK;
}

int smf_set_fused_crt(smf_ctx* ctx, int enable) {
    if (!ctx) return SMF_E_INVALID;
    ctx->fused_crt = enable ? 1 : 0;
    return SMF_OK;
}

int smf_set_elim_panels(smf_ctx* ctx, int64_t min_n) {
    if (!ctx || min_n < 0) return SMF_E_INVALID;
    ctx->elim_panel_min_n = min_n ? min_n : kElimPanelMinN;
    ctx->elim_local_panel_min_n = min_n ? min_n : kElimLocalPanelMinN;
    return SMF_OK;
}

int smf_debug_inject(smf_ctx* ctx, int flags) {
    if (!ctx || (flags & ~(SMF_INJECT_STALL_LOADS | SMF_INJECT_WRONG_SMITH | SMF_INJECT_WRONG_SMITH_ALWAYS)))
        return SMF_E_INVALID;
    ctx->inject = flags;
    return SMF_OK;
}

int smf_profile_enable(smf_ctx* ctx, int enable) {
    if (!ctx) return SMF_E_INVALID;
    ctx->prof = enable != 0;
    return SMF_OK;
}

int smf_profile_read(smf_ctx* ctx, int32_t counts[SMF_PROF_KINDS], double ms[SMF_PROF_KINDS]) {
    if (!ctx) return SMF_E_INVALID;
    for (int k = 0; k < SMF_PROF_KINDS; k++) {
        if (counts) counts[k] = 0;
        if (ms) ms[k] = 0.0;
    }
    DeviceGuard g(ctx->device);
    for (auto& r : ctx->prof_recs) {
        float t = 0.f;
        SMF_CU(ctx, cudaEventSynchronize(r.stop));
        SMF_CU(ctx, cudaEventElapsedTime(&t, r.start, r.stop));
        if (counts) counts[r.kind]++;
        if (ms) ms[r.kind] += t;
        ctx->event_pool.push_back(r.start);
        ctx->event_pool.push_back(r.stop);
    }
    ctx->prof_recs.clear();
    return SMF_OK;
}

int smf_fp64_peak(smf_ctx* ctx, double* tflops, void* stream) {
    if (!ctx || !tflops) return SMF_E_INVALID;
    DeviceGuard g(ctx->device);
    *tflops = fp64_fma_peak_tflops(ctx->num_sms, (cudaStream_t)stream);
    return *tflops > 0 ? SMF_OK : fail(ctx, SMF_E_CUDA, "fp64_peak: the probe kernel failed");
}

int smf_status_sync(smf_ctx* ctx, void* stream) {
    if (!ctx) return SMF_E_INVALID;
    DeviceGuard g(ctx->device);
    SMF_CU(ctx, cudaStreamSynchronize((cudaStream_t)stream));
    int h = 0;
    SMF_CU(ctx, cudaMemcpy(&h, ctx->d_status, sizeof(int), cudaMemcpyDeviceToHost));
    if (h) {
        SMF_CU(ctx, cudaMemsetAsync(ctx->d_status, 0, sizeof(int), (cudaStream_t)stream));
        SMF_CU(ctx, cudaStreamSynchronize((cudaStream_t)stream));
        if (h & kStatusTimeout) return fail(ctx, SMF_E_TIMEOUT, "a bounded device wait gave up");
        if (h & kStatusInexact)
            return fail(ctx, SMF_E_INVALID, "padic_lift: a residual was not divisible by p (A_inv_mod_p is not A^-1 mod p)");
        if (h & kStatusSingular) return fail(ctx, SMF_E_SINGULAR, "inverse_mod_p: p divides det A");
        if (h & kStatusBound)
            return fail(ctx, SMF_E_BOUND, "an operand entry lies outside its declared bound (smf_bigmat.bits)");
    }
    return SMF_OK;
}

}  // extern "C"
