// residue_gemm, INT8-limb form, on the sm_103a tensor cores (tcgen05).
//
// Section 3.1 computes each residue product C_i = A_i B_i mod p_i as an exact
// floating-point GEMM.  Here each centred residue is split into balanced
// base-2^8 digits (lower digits in [-128, 127], top digit |d| <= 128):
//   a = sum_u a_u 2^(8u),  b = sum_v b_v 2^(8v),
//   a b = sum_(u,v) a_u b_v 2^(8(u+v)).
// The digits are exact in bf16, every digit product is at most 2^14 in
// magnitude, so an fp32 accumulator holding at most KBLK = 1024 of them stays
// an exact integer of magnitude <= 2^24.  The kernel therefore
//   - stages the TA digit planes of an A tile (128 rows) and the TB digit
//     planes of a B tile (BN rows) per 64-wide K step with TMA (128-byte
//     swizzle), all B planes stacked into one N = TB*BN operand;
//   - issues, per 16-wide K slice, TA tcgen05.mma (kind::f16, bf16 inputs,
//     fp32 accumulate), one per A digit, each into its own TMEM accumulator
//     of TB*BN columns (column block u*TB*BN + v*BN holds sum a_u b_v);
//   - every KBLK products, drains TMEM into exact int64 sums per output,
//     R += sum_(u,v) acc_uv * 2^(8(u+v)), then hands TMEM back to the MMA;
//   - reduces R modulo p_i once at the end and stores canonical residues.
// Warp roles: warp 0 issues TMA, warp 1 owns TMEM and issues MMA, warps 2..5
// drain TMEM (warp w reads TMEM lanes 32*(w%4) .. 32*(w%4)+31).
// Every wait is bounded (about two seconds of %globaltimer); on expiry the
// kernel records a timeout in the status word and unwinds.
#include <cuda.h>
#include <cuda_bf16.h>

#include <mutex>

#include "smf_internal.h"

namespace smf {
namespace {

constexpr int BM = 128;          // MMA M: rows of A per tile (= TMEM lanes)
constexpr int BK = 64;           // bf16 per 128-byte swizzled row
constexpr int KBLK_TILES = 16;   // 16 * 64 = 1024 products between drains
constexpr int kThreads = 192;    // 6 warps
constexpr uint64_t kWaitNs = 2000000000ull;

// exactness of the fp32 accumulator between drains: KBLK * 2^14 <= 2^24
static_assert(KBLK_TILES * BK * 128 * 128 <= (1 << 24), "fp32 accumulation would not be exact");

template <int TA, int TB, int BN>
struct Cfg {
    static constexpr int NMMA = TB * BN;
    static constexpr int TMEM_USED = TA * NMMA;
    static constexpr uint32_t TMEM_COLS = TMEM_USED <= 32 ? 32 : TMEM_USED <= 64 ? 64
                                        : TMEM_USED <= 128 ? 128 : TMEM_USED <= 256 ? 256 : 512;
    static constexpr int A_BYTES = BM * BK * 2;
    static constexpr int B_BYTES = BN * BK * 2;
    static constexpr int STAGE_BYTES = TA * A_BYTES + TB * B_BYTES;
    static constexpr int STAGES = (200 * 1024 / STAGE_BYTES) < 8 ? (200 * 1024 / STAGE_BYTES) : 8;
    static constexpr int SMEM = STAGES * STAGE_BYTES + 1024 /*align*/ + 256 /*barriers*/;
    static_assert(NMMA % 16 == 0 && NMMA >= 16 && NMMA <= 256, "invalid MMA N for M = 128");
    static_assert(TMEM_USED <= 512, "accumulators exceed TMEM");
    static_assert(BN % 16 == 0, "B tile rows must fill 1024-byte swizzle atoms; drain in x16");
    static_assert(STAGES >= 2, "pipeline needs two stages");
    // instruction descriptor: D fp32, A/B bf16, both K-major, N>>3, M>>4
    static constexpr uint32_t IDESC = (1u << 4) | (1u << 7) | (1u << 10) |
                                      ((uint32_t)(NMMA >> 3) << 17) | ((uint32_t)(BM >> 4) << 24);
};

struct EpiParams {
    int32_t* C;
    int64_t M, N, K;
    int L, n_tiles, a_shared;
    const uint32_t* p;
    const uint64_t* mu;
    int* status;
};

// ------------------------------------------------------------------ PTX helpers

__device__ __forceinline__ uint32_t smem_u32(const void* ptr) {
    return (uint32_t)__cvta_generic_to_shared(ptr);
}
__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count));
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}
// Bounded wait; false (and the timeout bit set) when it gives up.
__device__ __noinline__ bool mbar_wait(uint32_t bar, uint32_t parity, int* status) {
    if (mbar_try(bar, parity)) return true;
    const uint64_t t0 = global_ns();
    for (uint32_t it = 1;; it++) {
        if (mbar_try(bar, parity)) return true;
        if ((it & 255) == 0 && global_ns() - t0 > kWaitNs) {
            atomicOr(status, kStatusTimeout);
            return false;
        }
    }
}
__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap* map, uint32_t bar, int x, int y,
                                            int z) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(dst),
        "l"((uint64_t)map), "r"(x), "r"(y), "r"(z), "r"(bar)
        : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// UMMA shared-memory descriptor, K-major, 128-byte swizzle: 8-row atoms of
// 1024 bytes (stride byte offset), descriptor version 1, swizzle mode 2.
__device__ __forceinline__ uint64_t sdesc(uint32_t addr) {
    return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) |
           ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}
__device__ __forceinline__ void mma_bf16(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
        "l"(a), "l"(b), "r"(idesc), "r"(acc));
}
__device__ __forceinline__ void mma_commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&r)[16]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
}
__device__ __forceinline__ void tmem_ld_wait() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// ------------------------------------------------------------------ kernel

template <int TA, int TB, int BN>
__global__ void __launch_bounds__(kThreads, 1)
limb_gemm_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, EpiParams ep) {
    using C = Cfg<TA, TB, BN>;
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint64_t* bars = (uint64_t*)(smem + C::STAGES * C::STAGE_BYTES);
    // bars: full[STAGES], empty[STAGES], acc_full, acc_empty, done; then TMEM address
    const uint32_t full0 = smem_u32(bars), empty0 = smem_u32(bars + C::STAGES);
    const uint32_t acc_full = smem_u32(bars + 2 * C::STAGES), acc_empty = acc_full + 8, done = acc_full + 16;
    uint32_t* tmem_slot = (uint32_t*)(bars + 2 * C::STAGES + 3);

    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    const int mt = blockIdx.x;
    const int prime = blockIdx.y / ep.n_tiles, nt = blockIdx.y % ep.n_tiles;
    const int m0 = mt * BM, n0 = nt * BN;
    const int nk = (int)((ep.K + BK - 1) / BK);
    const int nkb = (nk + KBLK_TILES - 1) / KBLK_TILES;

    if (threadIdx.x == 0) {
        for (int s = 0; s < C::STAGES; s++) {
            mbar_init(full0 + 8 * s, 1);
            mbar_init(empty0 + 8 * s, 1);
        }
        mbar_init(acc_full, 1);
        mbar_init(acc_empty, 128);
        mbar_init(done, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(C::TMEM_COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp == 0 && lane == 0) {
        // ---------------- TMA producer
        const int planeA = ep.a_shared ? 0 : prime * TA;
        int issued = 0;
        for (int kt = 0; kt < nk; kt++) {
            const int s = kt % C::STAGES;
            const uint32_t ph = (kt / C::STAGES) & 1;
            if (!mbar_wait(empty0 + 8 * s, ph ^ 1, ep.status)) break;
            const uint32_t fb = full0 + 8 * s;
            mbar_expect_tx(fb, C::STAGE_BYTES);
            const uint32_t sa = smem_u32(smem + s * C::STAGE_BYTES);
            const uint32_t sb = sa + TA * C::A_BYTES;
#pragma unroll
            for (int u = 0; u < TA; u++) tma_load_3d(sa + u * C::A_BYTES, &tmA, fb, kt * BK, m0, planeA + u);
#pragma unroll
            for (int v = 0; v < TB; v++) tma_load_3d(sb + v * C::B_BYTES, &tmB, fb, kt * BK, n0, prime * TB + v);
            issued = kt + 1;
        }
        // let copies still in flight land before the block can exit
        for (int kt = max(0, issued - C::STAGES); kt < issued; kt++)
            mbar_wait(full0 + 8 * (kt % C::STAGES), (kt / C::STAGES) & 1, ep.status);
    } else if (warp == 1 && lane == 0) {
        // ---------------- MMA issuer
        bool ok = true;
        int issued = 0;
        for (int kt = 0; kt < nk && ok; kt++) {
            const int s = kt % C::STAGES;
            const uint32_t ph = (kt / C::STAGES) & 1;
            const int kb = kt / KBLK_TILES, kin = kt % KBLK_TILES;
            if (kin == 0 && kb > 0) ok = mbar_wait(acc_empty, (kb - 1) & 1, ep.status);
            if (ok) ok = mbar_wait(full0 + 8 * s, ph, ep.status);
            if (!ok) break;
            tc_fence_after();
            const uint32_t sa = smem_u32(smem + s * C::STAGE_BYTES);
            const uint32_t sb = sa + TA * C::A_BYTES;
#pragma unroll
            for (int k16 = 0; k16 < BK / 16; k16++) {
                const uint64_t bd = sdesc(sb + 32 * k16);
#pragma unroll
                for (int u = 0; u < TA; u++)
                    mma_bf16(tmem + u * C::NMMA, sdesc(sa + u * C::A_BYTES + 32 * k16), bd, C::IDESC,
                             (kin > 0 || k16 > 0) ? 1u : 0u);
            }
            mma_commit(empty0 + 8 * s);
            if (kin == KBLK_TILES - 1 || kt == nk - 1) mma_commit(acc_full);
            issued = kt + 1;
        }
        if (issued > 0) {  // all issued MMAs complete before TMEM can be freed
            mma_commit(done);
            mbar_wait(done, 0, ep.status);
        }
    } else if (warp >= 2) {
        // ---------------- epilogue: drain TMEM into exact int64 sums
        const int quad = warp % 4;
        const int row = quad * 32 + lane;
        const uint32_t tbase = tmem + ((uint32_t)(quad * 32) << 16);
        int64_t R[BN];
#pragma unroll
        for (int n = 0; n < BN; n++) R[n] = 0;
        bool ok = true;
        for (int kb = 0; kb < nkb && ok; kb++) {
            ok = mbar_wait(acc_full, kb & 1, ep.status);
            ok = __all_sync(0xffffffffu, ok);  // tcgen05.ld below is warp-collective
            if (!ok) break;
            tc_fence_after();
#pragma unroll 1
            for (int u = 0; u < TA; u++) {
#pragma unroll
                for (int v = 0; v < TB; v++) {
#pragma unroll
                    for (int c = 0; c < BN; c += 16) {
                        uint32_t r[16];
                        tmem_ld16(tbase + u * C::NMMA + v * BN + c, r);
                        tmem_ld_wait();
#pragma unroll
                        for (int j = 0; j < 16; j++) {
                            const int64_t x = (int64_t)__float2int_rn(__uint_as_float(r[j]));
                            R[c + j] += x * ((int64_t)1 << (8 * (u + v)));
                        }
                    }
                }
            }
            tc_fence_before();
            mbar_arrive(acc_empty);
        }
        // R = exact dot product of the centred residues; reduce mod p
        const int64_t m = (int64_t)m0 + row;
        if (ok && m < ep.M) {
            const uint32_t p = ep.p[prime];
            const uint64_t mu = ep.mu[prime];
            int32_t* out = ep.C + ((size_t)prime * ep.M + m) * ep.N + n0;
#pragma unroll
            for (int n = 0; n < BN; n++) {
                if (n0 + n < ep.N) {
                    const int64_t x = R[n];
                    const uint64_t ax = x < 0 ? (uint64_t)(-x) : (uint64_t)x;
                    const uint64_t q = __umul64hi(ax, mu);
                    uint64_t rr = ax - q * p;
                    if (rr >= p) rr -= p;
                    if (rr >= p) rr -= p;
                    if (x < 0 && rr) rr = p - rr;
                    out[n] = (int32_t)rr;
                }
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        __syncwarp();
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(C::TMEM_COLS));
    }
}

// ------------------------------------------------------------------ host side

using EncodeFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                              const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                              CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeFn get_encode() {
    static EncodeFn fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* ptr = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &ptr, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (EncodeFn)ptr;
    });
    return fn;
}

// 3-D bf16 tensor {K, rows, planes} with row stride ld elements, box {64, box_rows, 1}.
bool encode_planes(CUtensorMap* map, const void* base, int64_t K, int64_t rows, int64_t planes, int64_t ld,
                   int box_rows) {
    EncodeFn enc = get_encode();
    if (!enc) return false;
    cuuint64_t dims[3] = {(cuuint64_t)K, (cuuint64_t)rows, (cuuint64_t)planes};
    cuuint64_t strides[2] = {(cuuint64_t)(ld * 2), (cuuint64_t)(ld * 2 * rows)};
    cuuint32_t box[3] = {(cuuint32_t)BK, (cuuint32_t)box_rows, 1};
    cuuint32_t estr[3] = {1, 1, 1};
    CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<void*>(base), dims, strides, box, estr,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

template <int TA, int TB, int BN>
cudaError_t launch_cfg(const BasisDev& b, const LimbGemmArgs& a, cudaStream_t s) {
    using C = Cfg<TA, TB, BN>;
    static std::once_flag once;
    static cudaError_t attr_err = cudaSuccess;
    std::call_once(once, [] {
        attr_err = cudaFuncSetAttribute(limb_gemm_kernel<TA, TB, BN>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        C::SMEM);
    });
    if (attr_err != cudaSuccess) return attr_err;
    CUtensorMap tmA, tmB;
    const int64_t planesA = a.a_shared ? TA : (int64_t)TA * b.L;
    if (!encode_planes(&tmA, a.Adig, a.K, a.M, planesA, a.lda, BM)) return cudaErrorInvalidValue;
    if (!encode_planes(&tmB, a.Bdig, a.K, a.N, (int64_t)TB * b.L, a.ldb, BN)) return cudaErrorInvalidValue;
    EpiParams ep;
    ep.C = a.C;
    ep.M = a.M;
    ep.N = a.N;
    ep.K = a.K;
    ep.L = b.L;
    ep.n_tiles = (int)((a.N + BN - 1) / BN);
    ep.a_shared = a.a_shared;
    ep.p = b.p;
    ep.mu = b.mu;
    ep.status = a.d_status;
    const int m_tiles = (int)((a.M + BM - 1) / BM);
    if ((int64_t)ep.n_tiles * b.L > 65535) return cudaErrorInvalidConfiguration;
    dim3 grid((unsigned)m_tiles, (unsigned)(ep.n_tiles * b.L));
    limb_gemm_kernel<TA, TB, BN><<<grid, kThreads, C::SMEM, s>>>(tmA, tmB, ep);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_gemm_limb(smf_ctx*, const BasisDev& b, const LimbGemmArgs& a, cudaStream_t s) {
    if (a.M == 0 || a.N == 0) return cudaSuccess;
#define SMF_LIMB_CASE(ta, tb, bn) \
    if (a.TA == ta && a.TB == tb) return launch_cfg<ta, tb, bn>(b, a, s);
    SMF_LIMB_CASE(1, 1, 32)
    SMF_LIMB_CASE(2, 1, 32)
    SMF_LIMB_CASE(3, 1, 32)
    SMF_LIMB_CASE(1, 2, 32)
    SMF_LIMB_CASE(2, 2, 32)
    SMF_LIMB_CASE(3, 2, 32)
    SMF_LIMB_CASE(1, 3, 32)
    SMF_LIMB_CASE(2, 3, 32)
    SMF_LIMB_CASE(3, 3, 32)
#undef SMF_LIMB_CASE
    return cudaErrorNotSupported;
}

}  // namespace smf
