// residue_gemm, INT8-limb form, on the sm_103a tensor cores (tcgen05).
//
// Section 3.1 computes each residue product C_i = A_i B_i mod p_i as an exact
// floating-point GEMM.  Here each centred residue is split into balanced
// base-2^8 digits (lower digits in [-128, 127], top digit |d| <= 128):
//   a = sum_u a_u 2^(8u),  b = sum_v b_v 2^(8v),
//   a b = sum_s 2^(8s) D_s,   D_s = sum_(u+v=s) a_u b_v.
// Digits are exact in bf16 and every digit product is at most 2^14 in
// magnitude.  One fp32 TMEM accumulator per weight s (a "diagonal") collects
// the pairs (u, v) with u + v = s; it stays an exact integer of magnitude
// <= 2^24 for a fold block of KBLK products, KBLK * sum_(u+v=s) |a_u| |b_v|
// <= 2^24 (digit bounds from the operands' bounds: 128, except a top digit
// that covers less, e.g. 16 for |a| <= 2^20), after which it is drained into
// integer registers.
//
// Kernel structure of limb_gemm_kernel (one persistent CTA per SM, tiles of
// 128 rows of A by BN columns of B, where the columns of all primes' B form
// one space of L*N columns; BN = 48 keeps the MMA N = TB*48 large while two
// sets of diagonals still fit the 512 TMEM columns; three digits on each side
// take limb_gemm_wide_kernel further down, with BN = 64):
//  - warp 0 streams, per 64-wide K step, the TA digit planes of the A tile and
//    the TB digit planes of the B tile into shared memory with TMA (128-byte
//    swizzle); the B planes are stacked into one N = TB*BN operand;
//  - warp 1 owns TMEM and issues, per 16-wide K slice, one tcgen05.mma
//    (kind::f16, bf16 in, fp32 accumulate) per A digit u against the stacked
//    B planes; the MMA for u writes TMEM columns [u*BN, (u+TB)*BN), i.e. the
//    diagonals u .. u+TB-1, so the TA MMAs overlap on the shared diagonals;
//    every MMA accumulates (one instruction shape throughout): the drain warps
//    write zeros back into an accumulator set right after reading it;
//  - TMEM holds two accumulator sets of (TA+TB-1)*BN columns: while warps
//    2..9 (two per TMEM lane quadrant, half the columns each) drain one set
//    into exact int64 sums T += sum_s D_s 2^(8s), the MMAs fill the other;
//  - at the end of a tile the drain warps reduce T modulo p_i and store
//    canonical residues, while the MMAs already run on the next tile.
// Every wait is bounded (about two seconds of %globaltimer); on expiry the
// kernel records a timeout in the status word and unwinds.
#include <cuda.h>
#include <cuda_bf16.h>

#include <mutex>

#include <algorithm>

#include "crt_dev.h"
#include "smf_internal.h"
#include "tc_ptx.h"

namespace smf {
namespace {

constexpr int BM = 128;          // MMA M: rows of A per tile (= TMEM lanes)
constexpr int BK = 64;           // bf16 per 128-byte swizzled row
constexpr int kEpiWarps = 8;     // two drain warps per TMEM lane quadrant
constexpr int kThreads = 64 + 32 * kEpiWarps;
constexpr int kFoldKb = 64;      // the int64 sums are reduced mod p this often

template <int TA, int TB, int BN>
struct Cfg {
    static constexpr int NMMA = TB * BN;              // MMA N (stacked B planes)
    static constexpr int NDIAG = TA + TB - 1;         // accumulators per tile
    static constexpr int BUF = NDIAG * BN;            // TMEM columns of one set
    static constexpr int PAIRS = TA < TB ? TA : TB;   // most (u, v) pairs on one diagonal
    static constexpr int KBLK_TILES = 16 / PAIRS;     // fewest 64-wide K steps between drains (any digits)
    static constexpr uint32_t TMEM_COLS = 2 * BUF <= 32 ? 32 : 2 * BUF <= 64 ? 64
                                        : 2 * BUF <= 128 ? 128 : 2 * BUF <= 256 ? 256 : 512;
    static constexpr int CPE = BN * 4 / kEpiWarps;    // columns per drain warp per diagonal
    static constexpr int A_BYTES = BM * BK * 2;
    static constexpr int B_BYTES = BN * BK * 2;
    static constexpr int STAGE_BYTES = TA * A_BYTES + TB * B_BYTES;
    static constexpr int STAGES = (200 * 1024 / STAGE_BYTES) < 8 ? (200 * 1024 / STAGE_BYTES) : 8;
    static constexpr int SMEM = STAGES * STAGE_BYTES + 1024 /*align*/ + 256 /*barriers*/;
    // exactness: a diagonal holds at most KBLK * PAIRS products of |x| <= 2^14
    static_assert(KBLK_TILES * BK * PAIRS * 128 * 128 <= (1 << 24), "fp32 accumulation would not be exact");
    static_assert(NMMA % 16 == 0 && NMMA >= 16 && NMMA <= 256, "invalid MMA N for M = 128");
    static_assert(2 * BUF <= 512, "two accumulator sets must fit TMEM");
    static_assert(BN % 16 == 0 && CPE % 8 == 0, "B tile rows fill 1024-byte swizzle atoms; drains in x8");
    static_assert(STAGES >= 2, "pipeline needs two stages");
    // instruction descriptors: D fp32, A/B bf16, both K-major, N>>3, M>>4
    __host__ __device__ static constexpr uint32_t idesc(int n) {
        return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(BM >> 4) << 24);
    }
};

struct EpiParams {
    int32_t* C;
    int64_t M, N, K;
    int L, n_tiles, m_tiles, a_shared;
    int n_sub;      // per-prime tiling: column tiles per prime (0: tiles run over all L*N columns)
    int64_t tiles;
    int kblk;       // 64-wide K steps per fold block (every diagonal stays below 2^24)
    const uint32_t* p;
    const uint64_t* mu;
    int* status;
    int inject;     // SMF_INJECT_STALL_LOADS: the producer issues nothing (tests)
    // split-K (wide kernel, one product): tile t' covers tile t' % tiles over the
    // K steps [s kchunk, (s+1) kchunk), s = t' / tiles, writing to C + s part_stride
    int split, kchunk;
    int64_t part_stride;
};

// Tile t covers rows m0 .. m0+127 of A and the B columns c0 .. c0+BN-1 of the
// combined (prime, n) column space, c = prime * N + n, up to c_end.  With a
// shared A the tiles run straight over all L*N columns (a tile may span two
// primes); otherwise every tile stays within one prime, whose A it uses.
// Raster order: groups of kGroupM row tiles sweep all column tiles, so the
// A rows of a group stay in L2 while B streams once per group.
constexpr int kGroupRows = 2048;   // rows of A per raster group
__device__ __forceinline__ void tile_coords(const EpiParams& ep, int64_t t, int BN, int tile_m, int& m0, int64_t& c0,
                                            int64_t& c_end, int& prime_a) {
    const int group_m = kGroupRows / tile_m;
    const int64_t per_group = (int64_t)group_m * ep.n_tiles;
    const int64_t grp = t / per_group, local = t - grp * per_group;
    const int gm = min(group_m, ep.m_tiles - (int)grp * group_m);  // row tiles in this group
    const int64_t y = local / gm;
    m0 = (int)(grp * group_m + local % gm) * tile_m;
    if (ep.n_sub == 0) {
        c0 = y * BN;
        c_end = (int64_t)ep.L * ep.N;
        prime_a = 0;
    } else {
        prime_a = (int)(y / ep.n_sub);
        c0 = (int64_t)prime_a * ep.N + (y % ep.n_sub) * BN;
        c_end = (int64_t)(prime_a + 1) * ep.N;
    }
}

// x mod p in [0, p) for |x| < 2^63, by Barrett reduction with
// mu = floor((2^64-1)/p) and two corrections.
__device__ __forceinline__ int64_t mod_p(int64_t x, uint32_t p, uint64_t mu) {
    const uint64_t ax = x < 0 ? (uint64_t)(-x) : (uint64_t)x;
    const uint64_t q = __umul64hi(ax, mu);
    uint64_t rr = ax - q * p;
    if (rr >= p) rr -= p;
    if (rr >= p) rr -= p;
    if (x < 0 && rr) rr = p - rr;
    return (int64_t)rr;
}

// The nk K steps of a tile split into nkb = ceil(nk / kblk) fold blocks.  The
// double-buffered kernel makes them near-equal (block b has nk / nkb steps, one
// more for the first nk % nkb blocks): a short last block would leave the MMAs
// too little work to cover the drain of the block before it.
__device__ __forceinline__ int fold_blocks(int nk, int kblk) { return (nk + kblk - 1) / kblk; }
__device__ __forceinline__ int block_steps(int nk, int nkb, int b) { return nkb ? nk / nkb + (b < nk % nkb ? 1 : 0) : 0; }

// One product of a grouped launch: its tensor maps, shapes and output, and the
// first tile it owns in the launch's tile sequence.
struct GroupDesc {  // 128-byte aligned through its tensor maps
    CUtensorMap tmA, tmB;
    int32_t* C;
    int64_t M, N, K, tile_base;
    int m_tiles, n_tiles, n_sub, a_shared, ta;  // ta: A's digits (B always has 3)
    int kblk;                                   // K steps per fold block
    int pf;                                     // K steps ahead that the producer prefetches into L2 (0: none)
};
static_assert(alignof(GroupDesc) >= 64 && sizeof(GroupDesc) % 64 == 0, "descriptors stay 64-byte aligned in an array");
__device__ __forceinline__ int k_steps(int64_t K) { return (int)((K + BK - 1) / BK); }
// The product that owns tile t (tile_base ascending, gd[0].tile_base = 0).
__device__ __forceinline__ const GroupDesc* group_of(const GroupDesc* gd, int ng, int64_t t) {
    int lo = 0, hi = ng - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (gd[mid].tile_base <= t) lo = mid;
        else hi = mid - 1;
    }
    return gd + lo;
}
// Tiles of a CTA ascend, so each role finds its product by moving a cursor forward.
__device__ __forceinline__ int advance_group(const GroupDesc* gd, int ng, int cur, int64_t t) {
    while (cur + 1 < ng && gd[cur + 1].tile_base <= t) cur++;
    return cur;
}
__device__ __forceinline__ void set_group(EpiParams& e, const GroupDesc& g) {
    e.kblk = g.kblk;
    e.C = g.C;
    e.M = g.M;
    e.N = g.N;
    e.K = g.K;
    e.m_tiles = g.m_tiles;
    e.n_tiles = g.n_tiles;
    e.n_sub = g.n_sub;
    e.a_shared = g.a_shared;
}

// ------------------------------------------------------------------ kernel

// GROUPED: one persistent launch over the tiles of several products (the
// descriptors gd[0 .. ng), every product with TA digits of A); each role walks
// its CTA's ascending tiles with a cursor over the descriptors.
template <int TA, int TB, int BN, bool GROUPED>
__global__ void __launch_bounds__(kThreads, 1)
limb_gemm_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, EpiParams ep,
                 const GroupDesc* __restrict__ gd, int ng) {
    using C = Cfg<TA, TB, BN>;
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint64_t* bars = (uint64_t*)(smem + C::STAGES * C::STAGE_BYTES);
    // full[STAGES], empty[STAGES], acc_full[2], acc_empty[2], done; then the TMEM address
    const uint32_t full0 = smem_u32(bars), empty0 = smem_u32(bars + C::STAGES);
    const uint32_t accf0 = smem_u32(bars + 2 * C::STAGES), acce0 = accf0 + 16, done = accf0 + 32;
    uint32_t* tmem_slot = (uint32_t*)(bars + 2 * C::STAGES + 5);

    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    // tile t of this launch: its product's parameters, its index within that
    // product, and the product's tensor maps (for one product: ep and t)
    auto tile_of = [&](int64_t t, int& cur, EpiParams& e, int64_t& lt, const CUtensorMap*& ma,
                       const CUtensorMap*& mb) {
        e = ep;
        lt = t;
        ma = &tmA;
        mb = &tmB;
        if constexpr (GROUPED) {
            cur = cur < 0 ? (int)(group_of(gd, ng, t) - gd) : advance_group(gd, ng, cur, t);
            const GroupDesc* gp = gd + cur;
            set_group(e, *gp);
            lt = t - gp->tile_base;
            ma = &gp->tmA;
            mb = &gp->tmB;
        }
    };

    if (threadIdx.x == 0) {
        for (int s = 0; s < C::STAGES; s++) {
            mbar_init(full0 + 8 * s, 1);
            mbar_init(empty0 + 8 * s, 1);
        }
        for (int b = 0; b < 2; b++) {
            mbar_init(accf0 + 8 * b, 1);
            mbar_init(acce0 + 8 * b, 32 * kEpiWarps);
        }
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
    if (warp >= 2) {  // every MMA accumulates: both accumulator sets start at zero
        const uint32_t tq = tmem + ((uint32_t)((warp % 4) * 32) << 16) + ((warp - 2) / 4) * C::CPE;
        for (int b = 0; b < 2; b++)
            for (int d = 0; d < C::NDIAG; d++)
#pragma unroll
                for (int c = 0; c < C::CPE; c += 8) tmem_st8_zero(tq + b * C::BUF + d * BN + c);
        tmem_st_wait();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();

    if (warp == 0 && lane == 0) {
        // ---------------- TMA producer: a continuous stream of K steps over this CTA's tiles
        uint32_t it = 0;
        bool ok = !(ep.inject & SMF_INJECT_STALL_LOADS);
        int cur = -1;
        for (int64_t t = blockIdx.x; t < ep.tiles && ok; t += gridDim.x) {
            const int prev = cur;
            EpiParams e;
            int64_t lt;
            const CUtensorMap *ma, *mb;
            tile_of(t, cur, e, lt, ma, mb);
            if constexpr (GROUPED) {
                if (cur != prev) {  // maps written before the launch, read through the tensor-map proxy
                    tensormap_acquire(ma);
                    tensormap_acquire(mb);
                }
                const int64_t tn = t + gridDim.x;  // the next tile's maps into the descriptor cache
                if (tn < ep.tiles) {
                    const int nx = advance_group(gd, ng, cur, tn);
                    if (nx != cur) {
                        tensormap_prefetch(&gd[nx].tmA);
                        tensormap_prefetch(&gd[nx].tmB);
                    }
                }
            }
            const int nk = (int)((e.K + BK - 1) / BK);
            int m0, prime_a;
            int64_t c0, c_end;
            tile_coords(e, lt, BN, BM, m0, c0, c_end, prime_a);
            const int planeA = prime_a * TA;
            for (int kt = 0; kt < nk; kt++, it++) {
                const int s = it % C::STAGES;
                if (!(ok = mbar_wait(empty0 + 8 * s, ((it / C::STAGES) & 1) ^ 1, ep.status))) break;
                const uint32_t fb = full0 + 8 * s;
                mbar_expect_tx(fb, C::STAGE_BYTES);
                const uint32_t sa = smem_u32(smem + s * C::STAGE_BYTES);
                const uint32_t sb = sa + TA * C::A_BYTES;
#pragma unroll
                for (int u = 0; u < TA; u++) tma_load_3d(sa + u * C::A_BYTES, ma, fb, kt * BK, m0, planeA + u);
#pragma unroll
                for (int v = 0; v < TB; v++) tma_load_3d(sb + v * C::B_BYTES, mb, fb, kt * BK, (int)c0, v);
            }
        }
        // let copies still in flight land before the block can exit
        for (uint32_t j = it > (uint32_t)C::STAGES ? it - C::STAGES : 0; j < it; j++)
            mbar_wait(full0 + 8 * (j % C::STAGES), (j / C::STAGES) & 1, ep.status);
    } else if (warp == 1 && lane == 0) {
        // ---------------- MMA issuer
        constexpr uint32_t ID_FULL = C::idesc(C::NMMA);
        bool ok = true;
        uint32_t g = 0;
        int s = 0;
        uint32_t ph = 0;  // stage index and its phase bit, advanced incrementally
        bool issued = false;
        // descriptor of stage 0's first A tile; every other operand is a fixed
        // offset from it (start-address field counts 16-byte units and smem
        // addresses stay below 256 KB, so adding offsets never carries out)
        const uint64_t desc0 = sdesc(smem_u32(smem));
        int cur = -1;
        for (int64_t t = blockIdx.x; t < ep.tiles && ok; t += gridDim.x) {
            EpiParams e;
            int64_t lt;
            const CUtensorMap *ma, *mb;
            tile_of(t, cur, e, lt, ma, mb);
            const int nk = (int)((e.K + BK - 1) / BK);
            const int nkb = fold_blocks(nk, e.kblk);
            uint32_t dbase = tmem;
            int kb = 0, kin = 0, bsteps = block_steps(nk, nkb, 0);
            for (int kt = 0; kt < nk; kt++) {
                const bool last_in_block = kin == bsteps - 1;
                if (kin == 0) {
                    const uint32_t buf = g & 1;
                    if (g >= 2 && !(ok = mbar_wait(acce0 + 8 * buf, ((g >> 1) + 1) & 1, ep.status))) break;
                    dbase = tmem + buf * C::BUF;
                }
                if (!(ok = mbar_wait(full0 + 8 * s, ph, ep.status))) break;
                tc_fence_after();
                const uint64_t da = desc0 + (uint64_t)((s * C::STAGE_BYTES) >> 4);
                const uint64_t db = da + (uint64_t)((TA * C::A_BYTES) >> 4);
#pragma unroll
                for (int k16 = 0; k16 < BK / 16; k16++) {
#pragma unroll
                    for (int u = 0; u < TA; u++)
                        mma_bf16(dbase + u * BN, da + (uint64_t)((u * C::A_BYTES + 32 * k16) >> 4),
                                 db + (uint64_t)((32 * k16) >> 4), ID_FULL, 1u);
                }
                issued = true;
                mma_commit(empty0 + 8 * s);
                if (last_in_block) {
                    mma_commit(accf0 + 8 * (g & 1));
                    g++;
                    kin = 0;
                    bsteps = block_steps(nk, nkb, ++kb);
                } else {
                    kin++;
                }
                if (++s == C::STAGES) {
                    s = 0;
                    ph ^= 1u;
                }
            }
        }
        if (issued) {  // all issued MMAs complete before TMEM can be freed
            mma_commit(done);
            mbar_wait(done, 0, ep.status);
        }
    } else if (warp >= 2) {
        // ---------------- drain warps
        const int quad = warp % 4;                 // TMEM lane quadrant this warp may access
        const int half = (warp - 2) / 4;           // which CPE columns of each diagonal (0 with 4 warps)
        const int row = quad * 32 + lane;
        const uint32_t tq = tmem + ((uint32_t)(quad * 32) << 16) + half * C::CPE;
        bool ok = true;
        uint32_t g = 0;
        int cur = -1;
        for (int64_t t = blockIdx.x; t < ep.tiles && ok; t += gridDim.x) {
            EpiParams e;
            int64_t lt;
            const CUtensorMap *ma, *mb;
            tile_of(t, cur, e, lt, ma, mb);
            const int nk = (int)((e.K + BK - 1) / BK);
            const int nkb = fold_blocks(nk, e.kblk);
            int m0, prime_a;
            int64_t c0, c_end;
            tile_coords(e, lt, BN, BM, m0, c0, c_end, prime_a);
            c0 += half * C::CPE;
            // T = sum_s D_s 2^(8s) over the drained blocks: the exact dot product
            // of the centred residues (reduced mod p every kFoldKb blocks)
            int64_t T[C::CPE];
#pragma unroll
            for (int j = 0; j < C::CPE; j++) T[j] = 0;
            const bool folds = nkb > kFoldKb;
            for (int kb = 0; kb < nkb; kb++, g++) {
                const uint32_t buf = g & 1;
                ok = mbar_wait(accf0 + 8 * buf, (g >> 1) & 1, ep.status);
                ok = __all_sync(0xffffffffu, ok);  // tcgen05.ld below is warp-collective
                if (!ok) break;
                tc_fence_after();
#pragma unroll
                for (int d = 0; d < C::NDIAG; d++) {
#pragma unroll
                    for (int c = 0; c < C::CPE; c += 8) {
                        uint32_t r[8];
                        tmem_ld8(tq + buf * C::BUF + d * BN + c, r);
                        tmem_ld_wait();
#pragma unroll
                        for (int j = 0; j < 8; j++)
                            T[c + j] += (int64_t)__float2int_rn(__uint_as_float(r[j])) * ((int64_t)1 << (8 * d));
                        tmem_st8_zero(tq + buf * C::BUF + d * BN + c);  // the next block accumulates from 0
                    }
                }
                tmem_st_wait();
                tc_fence_before();
                mbar_arrive(acce0 + 8 * buf);
                if (folds && (kb % kFoldKb) == kFoldKb - 1 && kb != nkb - 1) {
                    // long K: reduce mod each column's prime to stay far below 2^63
                    int pr = (int)(c0 / e.N);
                    int64_t nn = c0 - (int64_t)pr * e.N;
#pragma unroll
                    for (int j = 0; j < C::CPE; j++) {
                        if (nn == e.N) { nn = 0; pr++; }
                        const int pc = pr < e.L ? pr : e.L - 1;
                        T[j] = mod_p(T[j], e.p[pc], e.mu[pc]);
                        nn++;
                    }
                }
            }
            if (!ok) break;
            const int64_t m = (int64_t)m0 + row;
            if (m < e.M) {
                int pr = (int)(c0 / e.N);
                int64_t nn = c0 - (int64_t)pr * e.N;
                uint32_t p = e.p[pr < e.L ? pr : e.L - 1];
                uint64_t mu = e.mu[pr < e.L ? pr : e.L - 1];
#pragma unroll
                for (int j = 0; j < C::CPE; j += 4) {
                    int32_t v4[4];
                    int prq[4];
                    int64_t nq[4];
                    bool valid[4];
#pragma unroll
                    for (int q = 0; q < 4; q++) {
                        if (nn == e.N) {
                            nn = 0;
                            pr++;
                            const int pc = pr < e.L ? pr : e.L - 1;
                            p = e.p[pc];
                            mu = e.mu[pc];
                        }
                        valid[q] = c0 + j + q < c_end;
                        v4[q] = (int32_t)mod_p(T[j + q], p, mu);
                        prq[q] = pr;
                        nq[q] = nn;
                        nn++;
                    }
                    int32_t* o0 = e.C + ((size_t)prq[0] * e.M + m) * e.N + nq[0];
                    if (valid[3] && prq[3] == prq[0] && (((uintptr_t)o0 & 15) == 0)) {
                        *(int4*)o0 = make_int4(v4[0], v4[1], v4[2], v4[3]);
                    } else {
#pragma unroll
                        for (int q = 0; q < 4; q++)
                            if (valid[q]) e.C[((size_t)prq[q] * e.M + m) * e.N + nq[q]] = v4[q];
                    }
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

// ------------------------------------------------------------------ wide kernel (3x3 digits)
//
// With three digits on each side the MMA N = 3*BN.  BN = 64 makes N = 192,
// which keeps the tensor pipe fed across the issuing thread's barrier waits
// better than N = 144, but five diagonals of 64 columns (320) do not fit twice
// in the 512 TMEM columns.  Consecutive fold blocks therefore alternate
// between two placements that share 128 columns: even blocks use columns
// [0, 320), odd blocks [192, 512).  In each placement one A digit avoids the
// shared part (u = 0 of an even block writes [0, 192); u = 2 of an odd block
// writes [320, 512)).  The hand-over between blocks g and g+1:
//  - the last K step of block g issues the two digits that write the shared
//    columns, commits "shared final", then issues the free digit;
//  - the drain empties block g's shared columns as soon as "shared final"
//    completes and signals "shared free", then drains the rest;
//  - the first K step of block g+1 issues its free digit, waits for "shared
//    free", then issues the other two digits.
// So eight MMAs cover the drain's hand-over latency, and every other K step
// issues its 12 MMAs after a single barrier wait.  Sixteen drain warps (four
// per TMEM lane quadrant, 16 columns each) keep the drain short and its
// registers few.

namespace wide {
constexpr int TA = 3, TB = 3, BN = 64;
constexpr int NDIAG = TA + TB - 1;              // 5
constexpr int NMMA = TB * BN;                   // 192
constexpr int SHIFT = 192;                      // TMEM base of odd blocks
constexpr int kDrainWarps = 16;
constexpr int kThreads = 64 + 32 * kDrainWarps;
constexpr int CPT = BN / 4;                     // columns per drain thread
constexpr int A_BYTES = BM * BK * 2;
constexpr int B_BYTES = BN * BK * 2;
constexpr int STAGE_BYTES = TA * A_BYTES + TB * B_BYTES;
constexpr int STAGES = 3;
constexpr int SMEM = STAGES * STAGE_BYTES + 1024 + 256;
constexpr int kPre = 1;                         // K steps of a block that start with the free digit
constexpr int kSuf = 1;                         // K steps of a block that end with the free digit
constexpr uint32_t IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(NMMA >> 3) << 17) | ((uint32_t)(BM >> 4) << 24);
static_assert(kPre >= 1 && kPre <= STAGES && kSuf >= 1 && kSuf <= STAGES, "held stages must fit the ring");
static_assert(SMEM <= 227 * 1024, "shared memory");
static_assert(SHIFT + NDIAG * BN <= 512, "odd blocks must fit TMEM");
static_assert(NMMA <= SHIFT, "u = 0 of an even block must stay below the odd placement");
static_assert(SHIFT + (TA - 1) * BN >= NDIAG * BN, "u = 2 of an odd block must stay above the even placement");
static_assert(NDIAG * BN - SHIFT == 2 * BN, "the shared columns hold exactly two diagonals");

// One arrival per drain warp, after every lane's TMEM accesses (fenced).
__device__ __forceinline__ void warp_arrive(uint32_t bar, int lane) {
    __syncwarp();
    if (lane == 0) mbar_arrive(bar);
}

// T[j] += D[j] * 2^(8d) for one 16-column slice of diagonal d
template <int D>
__device__ __forceinline__ void add_diag(int64_t* T, const uint32_t* r) {
#pragma unroll
    for (int j = 0; j < CPT; j++) T[j] += (int64_t)__float2int_rn(__uint_as_float(r[j])) * ((int64_t)1 << (8 * D));
}

// Drain one fold block with placement PAR (0: columns [0, 320), 1: [192, 512)):
// the shared columns once `accs` (their last MMA done) completes, the rest once
// `accf` (every MMA of the block done) completes.  Only the block's nd = TA + 2
// lowest diagonals were written; the others are still zero and are skipped.
// False on a timeout.
template <int PAR, int ND>
__device__ __forceinline__ bool drain_block(uint32_t tq, int64_t* T, uint32_t accs, uint32_t accf, uint32_t parity,
                                            uint32_t ovl, uint32_t acce, int lane, int* status) {
    constexpr int D_SHARED = PAR ? 0 : 3;           // diagonals in the shared columns
    constexpr uint32_t REST = PAR ? SHIFT + 2 * BN : 0;
    constexpr int D_REST = PAR ? 2 : 0;
    if (!__all_sync(0xffffffffu, mbar_wait(accs, parity, status))) return false;  // tcgen05.ld is warp-collective
    tc_fence_after();
    {
        uint32_t r0[CPT], r1[CPT];
        constexpr bool s0 = D_SHARED < ND, s1 = D_SHARED + 1 < ND;
        if constexpr (s0) tmem_ld16(tq + SHIFT, r0);
        if constexpr (s1) tmem_ld16(tq + SHIFT + BN, r1);
        tmem_ld_wait();
        if constexpr (s0) tmem_st16_zero(tq + SHIFT);  // the next block accumulates from 0
        if constexpr (s1) tmem_st16_zero(tq + SHIFT + BN);
        tmem_st_wait();
        tc_fence_before();
        warp_arrive(ovl, lane);
        if constexpr (s0) add_diag<D_SHARED>(T, r0);
        if constexpr (s1) add_diag<D_SHARED + 1>(T, r1);
    }
    if (!__all_sync(0xffffffffu, mbar_wait(accf, parity, status))) return false;
    tc_fence_after();
#pragma unroll
    for (int j = 0; j < 3; j++) {
        if (D_REST + j >= ND) break;
        uint32_t r[CPT];
        tmem_ld16(tq + REST + j * BN, r);
        tmem_ld_wait();
        tmem_st16_zero(tq + REST + j * BN);
        if (j == 0) add_diag<D_REST>(T, r);
        else if (j == 1) add_diag<D_REST + 1>(T, r);
        else add_diag<D_REST + 2>(T, r);
    }
    tmem_st_wait();
    tc_fence_before();
    warp_arrive(acce, lane);
    return true;
}
}  // namespace wide


// The CRT fused into the residue product (row a7 of the hot path: one kernel
// for Section 3.1's residue products and their reconstruction).  A CRT unit
// is the block of 128 rows by BN columns of C; its L residue tiles (one per
// prime) are stored by whichever CTAs run them, and each stored tile adds one
// to the unit's counter.  The CTA whose tile brings the counter to L
// reconstructs the unit's entries from the residues (read at L2, where the
// other CTAs' stores are visible after their fences) in its drain warps, while
// its MMA warp already runs the next tile.  No block waits for another.
using FusedCrtQ = CrtConst<24, true, 24>;  // up to 24 primes below 2^24
struct FusedCrt {
    int* count;   // per unit (row tile x column block), zero before the launch
    uint64_t* X;  // output: M x N entries of W words, leading dimension ld (entries)
    int64_t ld;
    int W;
    int nb;       // column blocks per prime: ceil(N / BN)
};

// Named barrier of the 16 drain warps (id 1; __syncthreads uses 0), and the
// same barrier reducing a predicate (true only if every drain thread's is).
__device__ __forceinline__ void drain_bar() { asm volatile("bar.sync 1, %0;" ::"n"(wide::kDrainWarps * 32) : "memory"); }
__device__ __forceinline__ bool drain_bar_and(bool v) {
    uint32_t r;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\tsetp.ne.u32 p, %1, 0;\n\tbar.red.and.pred q, 1, %2, p;\n\t"
        "selp.u32 %0, 1, 0, q;\n\t}"
        : "=r"(r)
        : "r"((uint32_t)v), "n"(wide::kDrainWarps * 32)
        : "memory");
    return r != 0;
}

// MODE 0: one product; 1: a grouped launch over the descriptors gd[0 .. ng);
// 2: one product with the CRT fused into the epilogue (cq, fz).
template <int MODE>
__device__ __forceinline__ void wide_body(const CUtensorMap* tmA, const CUtensorMap* tmB, const EpiParams& ep,
                                          const GroupDesc* __restrict__ gd, int ng, const FusedCrtQ* cq,
                                          const FusedCrt* fz) {
    using namespace wide;
    constexpr bool GROUPED = MODE == 1;
    pdl_wait();  // a no-op unless launched as a programmatic dependent
    pdl_trigger();
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint64_t* bars = (uint64_t*)(smem + STAGES * STAGE_BYTES);
    // full[STAGES], empty[STAGES], acc_full[2], acc_empty[2], done, shared-free, shared-final[2];
    // then the TMEM address.
    const uint32_t full0 = smem_u32(bars), empty0 = smem_u32(bars + STAGES);
    const uint32_t accf0 = smem_u32(bars + 2 * STAGES), acce0 = accf0 + 16, done = accf0 + 32, ovl = accf0 + 40;
    const uint32_t accs0 = accf0 + 48;
    uint32_t* tmem_slot = (uint32_t*)(bars + 2 * STAGES + 8);

    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    const int nk = k_steps(ep.K);

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; s++) {
            mbar_init(full0 + 8 * s, 1);
            mbar_init(empty0 + 8 * s, 1);
        }
        for (int b = 0; b < 2; b++) {
            mbar_init(accf0 + 8 * b, 1);
            mbar_init(acce0 + 8 * b, kDrainWarps);
        }
        mbar_init(done, 1);
        mbar_init(ovl, kDrainWarps);
        mbar_init(accs0, 1);
        mbar_init(accs0 + 8, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(512u));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    const int quad = warp % 4;          // TMEM lane quadrant a warp may access
    const int cgrp = (warp - 2) / 4;    // drain warps: which 16 columns of each diagonal
    if (warp >= 2) {                    // every MMA accumulates: all 512 columns start at zero
        const uint32_t tq = tmem + ((uint32_t)(quad * 32) << 16) + cgrp * CPT;
#pragma unroll
        for (int c = 0; c < 512; c += BN) tmem_st16_zero(tq + c);
        tmem_st_wait();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();

    if (warp == 0 && lane == 0) {
        // ---------------- TMA producer: a continuous stream of K steps over this CTA's tiles
        uint32_t it = 0;
        bool ok = !(ep.inject & SMF_INJECT_STALL_LOADS);
        // nta: A's digits in this product (TA, or fewer in a grouped launch)
        // pf > 0: K step kt + pf of the tile is fetched into L2 while step kt
        // waits for its stage, so that its load later finds it there
        auto load_tile = [&](const EpiParams& e, int64_t lt, int nkt, int nta, const CUtensorMap* ta,
                             const CUtensorMap* tb, int k0, int pf) {
            int m0, prime_a;
            int64_t c0, c_end;
            tile_coords(e, lt, BN, BM, m0, c0, c_end, prime_a);
            const int planeA = prime_a * nta;
            for (int kt = 0; kt < nkt; kt++, it++) {
                if (pf > 0 && kt + pf < nkt) {
                    const int kx = (k0 + kt + pf) * BK;
#pragma unroll
                    for (int u = 0; u < TA; u++)
                        if (u < nta) tma_prefetch_3d(ta, kx, m0, planeA + u);
#pragma unroll
                    for (int v = 0; v < TB; v++) tma_prefetch_3d(tb, kx, (int)c0, v);
                }
                const int s = it % STAGES;
                if (!(ok = mbar_wait(empty0 + 8 * s, ((it / STAGES) & 1) ^ 1, ep.status))) break;
                const uint32_t fb = full0 + 8 * s;
                mbar_expect_tx(fb, nta * A_BYTES + TB * B_BYTES);
                const uint32_t sa = smem_u32(smem + s * STAGE_BYTES);
                const uint32_t sb = sa + TA * A_BYTES;
#pragma unroll
                for (int u = 0; u < TA; u++)
                    if (u < nta) tma_load_3d(sa + u * A_BYTES, ta, fb, (k0 + kt) * BK, m0, planeA + u);
#pragma unroll
                for (int v = 0; v < TB; v++) tma_load_3d(sb + v * B_BYTES, tb, fb, (k0 + kt) * BK, (int)c0, v);
            }
        };
        int cur = -1;
        for (int64_t t = blockIdx.x; t < ep.tiles * ep.split && ok; t += gridDim.x) {
            if constexpr (GROUPED) {
                const int prev = cur;
                cur = cur < 0 ? (int)(group_of(gd, ng, t) - gd) : advance_group(gd, ng, cur, t);
                const GroupDesc* gp = gd + cur;
                if (cur != prev) {  // maps written before the launch, read through the tensor-map proxy
                    tensormap_acquire(&gp->tmA);
                    tensormap_acquire(&gp->tmB);
                }
                const int64_t tn = t + gridDim.x;  // the next tile's maps into the descriptor cache
                if (tn < ep.tiles) {
                    const int nx = advance_group(gd, ng, cur, tn);
                    if (nx != cur) {
                        tensormap_prefetch(&gd[nx].tmA);
                        tensormap_prefetch(&gd[nx].tmB);
                    }
                }
                EpiParams e = ep;
                set_group(e, *gp);
                load_tile(e, t - gp->tile_base, k_steps(gp->K), gp->ta, &gp->tmA, &gp->tmB, 0, gp->pf);
            } else {
                const int sp = (int)(t / ep.tiles), k0 = sp * ep.kchunk;
                load_tile(ep, t - (int64_t)sp * ep.tiles, max(0, min(ep.kchunk, nk - k0)), TA, tmA, tmB, k0, 0);
            }
        }
        // let copies still in flight land before the block can exit: the last
        // stages' MMA commits (empty barriers) follow the completion of their copies
        for (uint32_t j = it > (uint32_t)STAGES ? it - STAGES : 0; j < it; j++)
            mbar_wait(empty0 + 8 * (j % STAGES), (j / STAGES) & 1, ep.status);
    } else if (warp == 1 && lane == 0) {
        // ---------------- MMA issuer
        bool ok = true;
        uint32_t g = 0;   // fold blocks issued so far, over all tiles
        int s = 0;
        uint32_t ph = 0;
        const uint64_t desc0 = sdesc(smem_u32(smem));
        // nta: A's digits in this product (TA, or fewer in a grouped launch); a
        // digit that is absent leaves its diagonals as the drain zeroed them.
        // Placement 0 reaches the shared columns only through diagonals 3 and 4,
        // which a one-digit A never writes: a block then needs no hand-over wait
        // when it, or (placement 1) the block before it, has one digit.
        int prev_ta = TA;
        auto issue_tile = [&](int nkt, int nta, int kblk) {
            const int amask = (1 << nta) - 1;
            for (int kt = 0; kt < nkt && ok; g++) {
                // full blocks first, the remainder last (measured faster here than
                // equal blocks: the hand-over costs the same in every block)
                const int steps = nkt - kt < kblk ? nkt - kt : kblk;
                const uint32_t par = g & 1;
                const bool handover = par ? prev_ta >= 2 : nta >= 2;
                prev_ta = nta;
                const uint32_t dbase = tmem + (par ? SHIFT : 0);
                const int ufree = par ? 2 : 0;   // the digit whose columns avoid the shared part
                // the block that last used this placement has been drained
                if (g >= 2 && !(ok = mbar_wait(acce0 + 8 * par, ((g >> 1) + 1) & 1, ep.status))) break;
                const int m_free = (1 << ufree) & amask, m_rest = amask & ~(1 << ufree);
                // digits u with (mask >> u) & 1 of the K step in stage st, k16-major
                auto issue = [&](int st, int mask) {
                    const uint64_t da = desc0 + (uint64_t)((st * STAGE_BYTES) >> 4);
                    const uint64_t db = da + (uint64_t)((TA * A_BYTES) >> 4);
#pragma unroll
                    for (int k16 = 0; k16 < BK / 16; k16++) {
#pragma unroll
                        for (int u = 0; u < TA; u++)
                            if ((mask >> u) & 1)
                                mma_bf16(dbase + u * BN, da + (uint64_t)((u * A_BYTES + 32 * k16) >> 4),
                                         db + (uint64_t)((32 * k16) >> 4), IDESC, 1u);
                    }
                };
                auto next = [&]() {
                    if (++s == STAGES) { s = 0; ph ^= 1u; }
                };
                const int P = g >= 1 && handover ? (steps < kPre ? steps : kPre) : 0;  // prefix K steps
                const int S0 = steps - kSuf > P ? steps - kSuf : P;          // first suffix K step
                // prefix: the free digit first; the rest once the previous block's shared columns are free
                const int sp = s;
                const uint32_t pp = ph;
                for (int j = 0; j < P; j++) {
                    if (!(ok = mbar_wait(full0 + 8 * s, ph, ep.status))) break;
                    tc_fence_after();
                    issue(s, m_free);
                    next();
                }
                if (!ok) break;
                if (P > 0) {
                    if (!(ok = mbar_wait(ovl, (g - 1) & 1, ep.status))) break;
                    tc_fence_after();
                    s = sp;
                    ph = pp;
                    for (int j = 0; j < P; j++) {
                        issue(s, m_rest);
                        mma_commit(empty0 + 8 * s);
                        next();
                    }
                }
                // middle: every digit
                for (int j = P; j < S0; j++) {
                    if (!(ok = mbar_wait(full0 + 8 * s, ph, ep.status))) break;
                    tc_fence_after();
                    issue(s, amask);
                    mma_commit(empty0 + 8 * s);
                    next();
                }
                if (!ok) break;
                // suffix: the digits that write the shared columns, "shared final", then the free digit
                const int ss = s;
                const uint32_t ps = ph;
                for (int j = S0; j < steps; j++) {
                    if (!(ok = mbar_wait(full0 + 8 * s, ph, ep.status))) break;
                    tc_fence_after();
                    issue(s, m_rest);
                    next();
                }
                if (!ok) break;
                mma_commit(accs0 + 8 * par);
                s = ss;
                ph = ps;
                for (int j = S0; j < steps; j++) {
                    issue(s, m_free);
                    mma_commit(empty0 + 8 * s);
                    next();
                }
                if (!ok) break;
                mma_commit(accf0 + 8 * par);
                kt += steps;
            }
        };
        int cur = -1;
        for (int64_t t = blockIdx.x; t < ep.tiles * ep.split && ok; t += gridDim.x) {
            if constexpr (GROUPED) {
                cur = cur < 0 ? (int)(group_of(gd, ng, t) - gd) : advance_group(gd, ng, cur, t);
                const GroupDesc* gp = gd + cur;
                issue_tile(k_steps(gp->K), gp->ta, gp->kblk);
            } else {
                const int k0 = (int)(t / ep.tiles) * ep.kchunk;
                issue_tile(max(0, min(ep.kchunk, nk - k0)), TA, ep.kblk);
            }
        }
        // every issued MMA completes before TMEM is freed (a commit with nothing
        // outstanding arrives at once)
        mma_commit(done);
        mbar_wait(done, 0, ep.status);
    } else if (warp >= 2) {
        // ---------------- drain warps
        const int row = quad * 32 + lane;
        const uint32_t tq = tmem + ((uint32_t)(quad * 32) << 16) + cgrp * CPT;
        bool ok = true;
        uint32_t g = 0;
        auto drain_tile = [&](const EpiParams& e, int64_t lt, int nkt, int nd) {
            const int nkb = fold_blocks(nkt, e.kblk);
            int m0, prime_a;
            int64_t c0, c_end;
            tile_coords(e, lt, BN, BM, m0, c0, c_end, prime_a);
            const int64_t ct0 = c0;  // the tile's first column
            c0 += cgrp * CPT;
            int64_t T[CPT];
#pragma unroll
            for (int j = 0; j < CPT; j++) T[j] = 0;
            const bool folds = nkb > kFoldKb;
            for (int kb = 0; kb < nkb; kb++, g++) {
                const uint32_t par = g & 1;
                const uint32_t pp = (g >> 1) & 1;
                if (nd == NDIAG) {
                    if (par) ok = drain_block<1, NDIAG>(tq, T, accs0 + 8, accf0 + 8, pp, ovl, acce0 + 8, lane, e.status);
                    else ok = drain_block<0, NDIAG>(tq, T, accs0, accf0, pp, ovl, acce0, lane, e.status);
                } else if constexpr (GROUPED) {  // fewer A digits: only the diagonals they write
                    if (nd == NDIAG - 1) {
                        if (par) ok = drain_block<1, NDIAG - 1>(tq, T, accs0 + 8, accf0 + 8, pp, ovl, acce0 + 8, lane, e.status);
                        else ok = drain_block<0, NDIAG - 1>(tq, T, accs0, accf0, pp, ovl, acce0, lane, e.status);
                    } else {
                        if (par) ok = drain_block<1, NDIAG - 2>(tq, T, accs0 + 8, accf0 + 8, pp, ovl, acce0 + 8, lane, e.status);
                        else ok = drain_block<0, NDIAG - 2>(tq, T, accs0, accf0, pp, ovl, acce0, lane, e.status);
                    }
                }
                if (!ok) break;
                if (folds && (kb % kFoldKb) == kFoldKb - 1 && kb != nkb - 1) {
                    int pr = (int)(c0 / e.N);
                    int64_t nn = c0 - (int64_t)pr * e.N;
#pragma unroll
                    for (int j = 0; j < CPT; j++) {
                        if (nn == e.N) { nn = 0; pr++; }
                        const int pc = pr < e.L ? pr : e.L - 1;
                        T[j] = mod_p(T[j], e.p[pc], e.mu[pc]);
                        nn++;
                    }
                }
            }
            if constexpr (MODE != 2) {
                if (!ok) return;
            }
            const int64_t m = (int64_t)m0 + row;
            if (ok && m < e.M) {
                int pr = (int)(c0 / e.N);
                int64_t nn = c0 - (int64_t)pr * e.N;
                uint32_t p = e.p[pr < e.L ? pr : e.L - 1];
                uint64_t mu = e.mu[pr < e.L ? pr : e.L - 1];
#pragma unroll
                for (int j = 0; j < CPT; j += 4) {
                    int32_t v4[4];
                    int prq[4];
                    int64_t nq[4];
                    bool valid[4];
#pragma unroll
                    for (int q = 0; q < 4; q++) {
                        if (nn == e.N) {
                            nn = 0;
                            pr++;
                            const int pc = pr < e.L ? pr : e.L - 1;
                            p = e.p[pc];
                            mu = e.mu[pc];
                        }
                        valid[q] = c0 + j + q < c_end;
                        v4[q] = (int32_t)mod_p(T[j + q], p, mu);
                        prq[q] = pr;
                        nq[q] = nn;
                        nn++;
                    }
                    int32_t* o0 = e.C + ((size_t)prq[0] * e.M + m) * e.N + nq[0];
                    if (valid[3] && prq[3] == prq[0] && (((uintptr_t)o0 & 15) == 0)) {
                        *(int4*)o0 = make_int4(v4[0], v4[1], v4[2], v4[3]);
                    } else {
#pragma unroll
                        for (int q = 0; q < 4; q++)
                            if (valid[q]) e.C[((size_t)prq[q] * e.M + m) * e.N + nq[q]] = v4[q];
                    }
                }
            }
            if constexpr (MODE == 2) {
                // count the stored tile toward its unit; the tile that completes
                // the unit reconstructs its entries (every drain thread takes
                // part in both barriers, so a timeout ends all of them together)
                __threadfence();  // this thread's residues, visible before the count
                ok = drain_bar_and(ok);
                if (ok) {
                    volatile int* fin = (volatile int*)(bars + 16);
                    const int nb = (int)((ct0 % e.N) / BN);
                    const int unit = (m0 / BM) * fz->nb + nb;
                    if (threadIdx.x == 64) *fin = atomicAdd(fz->count + unit, 1) == e.L - 1 ? 1 : 0;
                    drain_bar();
                    if (*fin) {
                        __threadfence();
                        const int64_t n0 = (int64_t)nb * BN;
                        const int ncols = (int)min((int64_t)BN, e.N - n0);
                        const int rows = (int)min((int64_t)BM, e.M - m0);
                        const int64_t count = e.M * e.N;
                        for (int j = threadIdx.x - 64; j < rows * ncols; j += kDrainWarps * 32) {
                            const int64_t r = m0 + j / ncols, n = n0 + j % ncols;
                            crt_entry<24, true, 24, true>(*cq, e.C, count, e.N, r * e.N + n, fz->X, fz->ld, fz->W);
                        }
                    }
                }
            }
        };
        int cur = -1;
        for (int64_t t = blockIdx.x; t < ep.tiles * ep.split && ok; t += gridDim.x) {
            if constexpr (GROUPED) {
                cur = cur < 0 ? (int)(group_of(gd, ng, t) - gd) : advance_group(gd, ng, cur, t);
                const GroupDesc* gp = gd + cur;
                EpiParams e = ep;
                set_group(e, *gp);
                drain_tile(e, t - gp->tile_base, k_steps(gp->K), gp->ta + TB - 1);
            } else {
                const int sp = (int)(t / ep.tiles), k0 = sp * ep.kchunk;
                EpiParams e = ep;
                e.C += sp * ep.part_stride;
                drain_tile(e, t - (int64_t)sp * ep.tiles, max(0, min(ep.kchunk, nk - k0)), NDIAG);
            }
        }
    }
    __syncwarp();
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512u));
    }
}

template <bool GROUPED>
__global__ void __launch_bounds__(wide::kThreads, 1)
limb_gemm_wide_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, EpiParams ep,
                      const GroupDesc* __restrict__ gd, int ng) {
    wide_body<GROUPED ? 1 : 0>(&tmA, &tmB, ep, gd, ng, nullptr, nullptr);
}

__global__ void __launch_bounds__(wide::kThreads, 1)
limb_gemm_crt_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, EpiParams ep,
                     const __grid_constant__ FusedCrtQ cq, FusedCrt fz) {
    wide_body<2>(&tmA, &tmB, ep, nullptr, 0, &cq, &fz);
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

// Largest |digit u| of values |x| <= h split into t balanced base-2^8 digits:
// 128 below the top; the top digit is what remains, at most
// (h + sum_(i<t-1) 128*256^i) / 256^(t-1).
uint64_t digit_bound(uint64_t h, int t, int u) {
    if (u < t - 1) return 128;
    uint64_t lower = 0, scale = 1;
    for (int i = 0; i < t - 1; i++) {
        lower += 128 * scale;
        scale *= 256;
    }
    return (h + lower) / scale;
}

// 64-wide K steps per fold block: each diagonal s collects, per k, the products
// a_u b_v with u + v = s, so it stays an exact fp32 integer (|.| <= 2^24) for
// 2^24 / max_s sum_(u+v=s) |a_u|max |b_v|max products.
int fold_block_steps(int TA, int TB, uint64_t amax, uint64_t bmax) {
    uint64_t worst = 1;
    for (int d = 0; d < TA + TB - 1; d++) {
        uint64_t w = 0;
        for (int u = 0; u < TA; u++) {
            const int v = d - u;
            if (v >= 0 && v < TB) w += digit_bound(amax, TA, u) * digit_bound(bmax, TB, v);
        }
        worst = w > worst ? w : worst;
    }
    const int64_t steps = (int64_t)(((uint64_t)1 << 24) / worst) / BK;
    return steps < 1 ? 1 : (int)steps;
}

// Tile bookkeeping shared by both kernels.
EpiParams make_epi(const BasisDev& b, const LimbGemmArgs& a, int BN, int tile_m) {
    EpiParams ep;
    ep.C = a.C;
    ep.M = a.M;
    ep.N = a.N;
    ep.K = a.K;
    ep.L = b.L;
    ep.m_tiles = (int)((a.M + tile_m - 1) / tile_m);
    if (a.a_shared) {  // tiles run over the combined (prime, n) columns
        ep.n_sub = 0;
        ep.n_tiles = (int)(((int64_t)b.L * a.N + BN - 1) / BN);
    } else {           // tiles stay within a prime (each prime has its own A)
        ep.n_sub = (int)((a.N + BN - 1) / BN);
        ep.n_tiles = ep.n_sub * b.L;
    }
    ep.tiles = (int64_t)ep.m_tiles * ep.n_tiles;
    ep.a_shared = a.a_shared;
    ep.p = b.p;
    ep.mu = b.mu;
    ep.status = a.d_status;
    ep.inject = a.inject;
    ep.kblk = fold_block_steps(a.TA, a.TB, a.amax, a.bmax);
    ep.split = 1;
    ep.kchunk = (int)((a.K + BK - 1) / BK);
    ep.part_stride = 0;
    return ep;
}

// C = sum_s part[s] mod p over the K splits (every partial canonical, in [0, p)).
__global__ void __launch_bounds__(256) sum_splits_kernel(const int32_t* __restrict__ part, int split, int64_t stride,
                                                         int64_t mn, const uint32_t* __restrict__ p,
                                                         int32_t* __restrict__ C) {
    const int64_t e = (int64_t)blockIdx.x * 256 + threadIdx.x;
    if (e >= stride) return;
    const uint32_t q = p[e / mn];
    uint32_t acc = 0;
    for (int sp = 0; sp < split; sp++) {
        acc += (uint32_t)part[(size_t)sp * stride + e];
        if (acc >= q) acc -= q;
    }
    C[e] = (int32_t)acc;
}

template <int TA, int TB, int BN>
cudaError_t launch_cfg(int num_sms, const BasisDev& b, const LimbGemmArgs& a, cudaStream_t s) {
    using C = Cfg<TA, TB, BN>;
    static std::once_flag once;
    static cudaError_t attr_err = cudaSuccess;
    std::call_once(once, [] {
        attr_err = cudaFuncSetAttribute(limb_gemm_kernel<TA, TB, BN, false>,
                                        cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM);
    });
    if (attr_err != cudaSuccess) return attr_err;
    CUtensorMap tmA, tmB;
    const int64_t planesA = a.a_shared ? TA : (int64_t)TA * b.L;
    if (!encode_planes(&tmA, a.Adig, a.K, a.M, planesA, a.lda, BM)) return cudaErrorInvalidValue;
    // B digit planes [TB][L][N][ldb] seen as TB planes of L*N rows
    if (!encode_planes(&tmB, a.Bdig, a.K, (int64_t)b.L * a.N, TB, a.ldb, BN)) return cudaErrorInvalidValue;
    const EpiParams ep = make_epi(b, a, BN, BM);
    const int grid = (int)(ep.tiles < num_sms ? ep.tiles : num_sms);
    limb_gemm_kernel<TA, TB, BN, false><<<grid, kThreads, C::SMEM, s>>>(tmA, tmB, ep, nullptr, 0);
    return cudaGetLastError();
}

cudaError_t launch_wide(int num_sms, const BasisDev& b, const LimbGemmArgs& a, cudaStream_t s) {
    static std::once_flag once;
    static cudaError_t attr_err = cudaSuccess;
    std::call_once(once, [] {
        attr_err = cudaFuncSetAttribute(limb_gemm_wide_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        wide::SMEM);
    });
    if (attr_err != cudaSuccess) return attr_err;
    CUtensorMap tmA, tmB;
    const int64_t planesA = a.a_shared ? wide::TA : (int64_t)wide::TA * b.L;
    if (!encode_planes(&tmA, a.Adig, a.K, a.M, planesA, a.lda, BM)) return cudaErrorInvalidValue;
    if (!encode_planes(&tmB, a.Bdig, a.K, (int64_t)b.L * a.N, wide::TB, a.ldb, wide::BN)) return cudaErrorInvalidValue;
    EpiParams ep = make_epi(b, a, wide::BN, BM);
    const bool split = a.split > 1 && a.part && a.kchunk > 0;
    if (split) {  // partial residues per K split, then their sum mod p
        ep.C = a.part;
        ep.split = a.split;
        ep.kchunk = a.kchunk;
        ep.part_stride = (int64_t)b.L * a.M * a.N;
    }
    const int64_t units = ep.tiles * ep.split;
    const int grid = (int)(units < num_sms ? units : num_sms);
    cudaError_t e;
    if (a.pdl) {
        e = launch_pdl(limb_gemm_wide_kernel<false>, dim3(grid), dim3(wide::kThreads), wide::SMEM, s, tmA, tmB, ep,
                       (const GroupDesc*)nullptr, 0);
    } else {
        limb_gemm_wide_kernel<false><<<grid, wide::kThreads, wide::SMEM, s>>>(tmA, tmB, ep, nullptr, 0);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess || !split || a.keep_parts) return e;
    const int64_t count = ep.part_stride;
    sum_splits_kernel<<<(unsigned)((count + 255) / 256), 256, 0, s>>>(a.part, a.split, count, a.M * a.N, b.p, a.C);
    return cudaGetLastError();
}

}  // namespace

bool limb_crt_fusable(const CrtHost& h, const LimbGemmArgs& a) {
    return a.TA == wide::TA && a.TB == wide::TB && a.split <= 1 && h.L >= 1 && h.L <= 24 &&
           h.p[0] < (1u << 24) && h.m_limbs <= FusedCrtQ::MLMAX && (!a.a_shared || a.N % wide::BN == 0);
}

int64_t limb_crt_units(int64_t M, int64_t N) { return ((M + BM - 1) / BM) * ((N + wide::BN - 1) / wide::BN); }

cudaError_t launch_gemm_limb_crt(smf_ctx* ctx, const BasisDev& b, const CrtHost& h, const LimbGemmArgs& a,
                                 int* count, uint64_t* X, int64_t ld, int W, cudaStream_t s) {
    if (a.M == 0 || a.N == 0) return cudaSuccess;
    if (!limb_crt_fusable(h, a) || a.K == 0) return cudaErrorNotSupported;
    static std::once_flag once;
    static cudaError_t attr_err = cudaSuccess;
    std::call_once(once, [] {
        attr_err = cudaFuncSetAttribute(limb_gemm_crt_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, wide::SMEM);
    });
    if (attr_err != cudaSuccess) return attr_err;
    CUtensorMap tmA, tmB;
    const int64_t planesA = a.a_shared ? wide::TA : (int64_t)wide::TA * b.L;
    if (!encode_planes(&tmA, a.Adig, a.K, a.M, planesA, a.lda, BM)) return cudaErrorInvalidValue;
    if (!encode_planes(&tmB, a.Bdig, a.K, (int64_t)b.L * a.N, wide::TB, a.ldb, wide::BN)) return cudaErrorInvalidValue;
    const EpiParams ep = make_epi(b, a, wide::BN, BM);
    FusedCrtQ q;
    crt_const(h, q);
    const FusedCrt fz{count, X, ld, W, (int)((a.N + wide::BN - 1) / wide::BN)};
    cudaError_t e = cudaMemsetAsync(count, 0, sizeof(int) * (size_t)limb_crt_units(a.M, a.N), s);
    if (e != cudaSuccess) return e;
    const int sms = ctx && ctx->num_sms > 0 ? ctx->num_sms : 148;
    const int grid = (int)(ep.tiles < sms ? ep.tiles : sms);
    limb_gemm_crt_kernel<<<grid, wide::kThreads, wide::SMEM, s>>>(tmA, tmB, ep, q, fz);
    return cudaGetLastError();
}

size_t limb_group_desc_bytes(int count) { return sizeof(GroupDesc) * (size_t)(count > 0 ? count : 0); }

bool limb_group_supported(const LimbGemmArgs& a) { return a.TA >= 1 && a.TA <= wide::TA && a.TB == wide::TB; }

// A work unit's fixed cost (barriers, pipeline fill, the last drain), in K steps
constexpr int64_t kSplitFill = 2;

void limb_split(int L, int64_t M, int64_t N, int64_t K, bool a_shared, int TA, int TB, int num_sms, int* split,
                int* kchunk) {
    const int nk = (int)((K + BK - 1) / BK);
    *split = 1;
    *kchunk = nk;
    if (num_sms <= 0 || TA != wide::TA || TB != wide::TB || M <= 0 || N <= 0 || nk < 2) return;
    const int64_t m_tiles = (M + BM - 1) / BM;
    const int64_t n_tiles = a_shared ? ((int64_t)L * N + wide::BN - 1) / wide::BN
                                     : ((N + wide::BN - 1) / wide::BN) * L;
    const int64_t tiles = m_tiles * n_tiles;
    if (tiles >= num_sms) return;  // a wave or more of tiles: no split
    // the split count with the fewest waves x (K steps per unit + fill), at most
    // 16 (the step kernels sum the partials in 32-bit words); ties: fewer splits
    int64_t best = -1;
    for (int64_t want = 1; want <= std::min<int64_t>(nk, 16); want++) {
        const int kc = (int)((nk + want - 1) / want);  // K steps per split
        const int sp = (nk + kc - 1) / kc;             // every split non-empty
        const int64_t waves = (tiles * sp + num_sms - 1) / num_sms;
        const int64_t cost = waves * (kc + kSplitFill);
        if (best < 0 || cost < best) {
            best = cost;
            *kchunk = kc;
            *split = sp;
        }
    }
}

int limb_narrow_bn(int L, int64_t M, int64_t N, int64_t K, bool a_shared, int TA, int TB, int num_sms) {
    if (num_sms <= 0 || TB != 3 || (TA != 1 && TA != 2)) return 48;
    auto waves = [&](int bn) {
        const int64_t tiles =
            (M + BM - 1) / BM * (a_shared ? ((int64_t)L * N + bn - 1) / bn : ((N + bn - 1) / bn) * L);
        return (tiles + num_sms - 1) / num_sms;
    };
    (void)K;  // both widths take the same K steps per tile
    return waves(64) * 64 < waves(48) * 48 ? 64 : 48;
}

double limb_cost(int L, int64_t M, int64_t N, int64_t K, bool a_shared, int TA, int TB, int num_sms) {
    const int64_t nk = (K + BK - 1) / BK;
    const int64_t sms = num_sms > 0 ? num_sms : 148;
    if (TA == wide::TA && TB == wide::TB) {
        int split = 1, kchunk = (int)nk;
        limb_split(L, M, N, K, a_shared, TA, TB, num_sms, &split, &kchunk);
        const int64_t tiles = (M + BM - 1) / BM * (a_shared ? ((int64_t)L * N + wide::BN - 1) / wide::BN
                                                            : ((N + wide::BN - 1) / wide::BN) * L);
        const int64_t waves = (tiles * split + sms - 1) / sms;
        return (double)waves * (kchunk + kSplitFill) * (TA * TB * wide::BN);
    }
    const int bn = limb_narrow_bn(L, M, N, K, a_shared, TA, TB, num_sms);  // the narrower kernels: no K split
    const int64_t tiles = (M + BM - 1) / BM * (a_shared ? ((int64_t)L * N + bn - 1) / bn : ((N + bn - 1) / bn) * L);
    const int64_t waves = (tiles + sms - 1) / sms;
    return (double)waves * (nk + kSplitFill) * (TA * TB * bn);
}

cudaError_t limb_group_encode(const BasisDev& b, const LimbGemmArgs* probs, int count, void* host, int tile_order,
                              LimbGroup* out) {
    GroupDesc* gd = (GroupDesc*)host;
    *out = LimbGroup{};
    out->kblk = 1 << 30;
    out->first = -1;
    // longest K first: CTAs take tiles round-robin, so the short tiles of the
    // small products fill the end of the launch instead of leaving a long tail.
    // tile_order 1 weighs K by A's digit count (the MMAs a K step issues).
    std::vector<int> order(count);
    for (int i = 0; i < count; i++) order[i] = i;
    if (tile_order == 1)
        std::stable_sort(order.begin(), order.end(),
                         [&](int x, int y) { return probs[x].K * probs[x].TA > probs[y].K * probs[y].TA; });
    else
        std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return probs[x].K > probs[y].K; });
    for (int oi = 0; oi < count; oi++) {
        const int i = order[oi];
        const LimbGemmArgs& a = probs[i];
        if (!limb_group_supported(a)) return cudaErrorNotSupported;
        if (a.M == 0 || a.N == 0 || a.K == 0) continue;
        GroupDesc& g = gd[out->count];
        const int64_t planesA = a.a_shared ? a.TA : (int64_t)a.TA * b.L;
        if (!encode_planes(&g.tmA, a.Adig, a.K, a.M, planesA, a.lda, BM)) return cudaErrorInvalidValue;
        if (!encode_planes(&g.tmB, a.Bdig, a.K, (int64_t)b.L * a.N, wide::TB, a.ldb, wide::BN))
            return cudaErrorInvalidValue;
        const EpiParams e = make_epi(b, a, wide::BN, BM);
        g.C = a.C;
        g.M = a.M;
        g.N = a.N;
        g.K = a.K;
        g.tile_base = out->tiles;
        g.m_tiles = e.m_tiles;
        g.n_tiles = e.n_tiles;
        g.n_sub = e.n_sub;
        g.a_shared = a.a_shared;
        g.ta = a.TA;
        g.kblk = e.kblk;
        g.pf = a.pf;
        out->tiles += e.tiles;
        out->kblk = e.kblk < out->kblk ? e.kblk : out->kblk;
        if (out->first < 0 || i < out->first) out->first = i;
        out->count++;
    }
    return cudaSuccess;
}

cudaError_t limb_group_launch(smf_ctx* ctx, const BasisDev& b, const LimbGemmArgs* probs, const LimbGroup& g,
                              const void* desc_dev, cudaStream_t s) {
    if (g.count == 0) return cudaSuccess;
    static std::once_flag once;
    static cudaError_t attr_err = cudaSuccess;
    std::call_once(once, [] {
        attr_err = cudaFuncSetAttribute(limb_gemm_wide_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        wide::SMEM);
    });
    if (attr_err != cudaSuccess) return attr_err;
    // the shared parameters (basis, status, injection) from the first product;
    // every product's diagonals stay exact with the smallest fold block
    EpiParams ep = make_epi(b, probs[g.first], wide::BN, BM);
    ep.tiles = g.tiles;
    ep.kblk = g.kblk;
    const int sms = ctx->num_sms > 0 ? ctx->num_sms : 148;
    const int grid = (int)(g.tiles < sms ? g.tiles : sms);
    CUtensorMap unused{};
    limb_gemm_wide_kernel<true><<<grid, wide::kThreads, wide::SMEM, s>>>(unused, unused, ep, (const GroupDesc*)desc_dev,
                                                                        g.count);
    return cudaGetLastError();
}

cudaError_t limb_group_launch_one_digit(smf_ctx* ctx, const BasisDev& b, const LimbGemmArgs* probs,
                                       const LimbGroup& g, const void* desc_dev, cudaStream_t s) {
    using C = Cfg<1, wide::TB, wide::BN>;
    if (g.count == 0) return cudaSuccess;
    static std::once_flag once;
    static cudaError_t attr_err = cudaSuccess;
    std::call_once(once, [] {
        attr_err = cudaFuncSetAttribute(limb_gemm_kernel<1, wide::TB, wide::BN, true>,
                                        cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM);
    });
    if (attr_err != cudaSuccess) return attr_err;
    EpiParams ep = make_epi(b, probs[g.first], wide::BN, BM);
    ep.tiles = g.tiles;
    ep.kblk = g.kblk;
    const int sms = ctx->num_sms > 0 ? ctx->num_sms : 148;
    const int grid = (int)(g.tiles < sms ? g.tiles : sms);
    CUtensorMap unused{};
    limb_gemm_kernel<1, wide::TB, wide::BN, true><<<grid, kThreads, C::SMEM, s>>>(unused, unused, ep,
                                                                                  (const GroupDesc*)desc_dev, g.count);
    return cudaGetLastError();
}

cudaError_t launch_gemm_limb(smf_ctx* ctx, const BasisDev& b, const LimbGemmArgs& a, cudaStream_t s) {
    if (a.M == 0 || a.N == 0) return cudaSuccess;
    const int sms = ctx && ctx->num_sms > 0 ? ctx->num_sms : 148;
    if (a.bn == 64 && a.TB == 3 && a.TA == 1) return launch_cfg<1, 3, 64>(sms, b, a, s);
    if (a.bn == 64 && a.TB == 3 && a.TA == 2) return launch_cfg<2, 3, 64>(sms, b, a, s);
#define SMF_LIMB_CASE(ta, tb, bn) \
    if (a.TA == ta && a.TB == tb) return launch_cfg<ta, tb, bn>(sms, b, a, s);
    SMF_LIMB_CASE(1, 1, 48)
    SMF_LIMB_CASE(2, 1, 48)
    SMF_LIMB_CASE(3, 1, 48)
    SMF_LIMB_CASE(1, 2, 48)
    SMF_LIMB_CASE(2, 2, 48)
    SMF_LIMB_CASE(3, 2, 48)
    SMF_LIMB_CASE(1, 3, 48)
    SMF_LIMB_CASE(2, 3, 48)
#undef SMF_LIMB_CASE
    if (a.TA == 3 && a.TB == 3) return launch_wide(sms, b, a, s);
    return cudaErrorNotSupported;
}

}  // namespace smf
